#!/usr/bin/env python
"""Benchmark of the NFFT hot path: forward + adjoint nodes/s on one GB300 (or N replicas).

One step is one forward NFFT (Algorithm "NFFT") plus one adjoint NFFT (Algorithm "adjoint
NFFT") over the workload's nodes, through the library's C ABI (``nfft_trafo`` /
``nfft_adjoint``), with inputs already resident in HBM. The default workload is the 2-D radial
trajectory: N = (512, 512), n = (1024, 1024), m = 4, M = 512 spokes x 2048 samples
= 1,048,576 nodes, FP32 (complex64). Variants at FP64 and m = 6 are reported beside it.

Printed (rank 0, one JSON line): value = M * K / (sum of the K step times) in nodes/s, the
relative l2 errors of the measured outputs against the FP64 CPU oracle, the roofline of the
dominant kernel (per-stage CUDA events recorded by the library on its stream), the oracle timed
on the host cores (``cpu_baseline``), the end-to-end number through the host-buffer entry points
(``e2e``), the SM clocks sampled during the timed region, and the number of kernel launches.

``--impl reference`` times the CPU oracle instead (the reference arm of this comparison).
Under torchrun each rank runs an independent replica of the workload (weak scaling, no
collective on the data path); the time is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "forward+adjoint NFFT nodes/s, FP32 vs FP64 at stated rel. ℓ2 error; % HBM peak"
UNIT = "nodes/s"


# ------------------------------------------------------------------------------ helpers

def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["radial", "clusters", "batched"], default="radial",
                    help="radial: the 2-D radial benchmark (default); clusters: 3-D clustered "
                         "nodes; batched: 64 uneven 2-D problems in one CUDA graph")
    ap.add_argument("--tune", action="store_true", help="batched: autotune every plan first")
    ap.add_argument("--m", type=int, default=4)
    ap.add_argument("--no-variants", action="store_true", help="skip the FP64 / m=6 variants")
    ap.add_argument("--no-cpu", action="store_true", help="skip the timed CPU oracle")
    ap.add_argument("--no-parity", action="store_true", help="skip the oracle error check")
    ap.add_argument("--no-subrecords", action="store_true",
                    help="skip the clustered 3-D and batched sub-records")
    ap.add_argument("--ncu-step", action="store_true",
                    help="only build the workload's plan and run --steps untimed forward + adjoint "
                         "pairs (a short program for ncu captures of the timed kernels)")
    ap.add_argument("--dtype", choices=["f32", "f64"], default="f32",
                    help="precision used by --ncu-step (the benchmark line itself reports FP32 with FP64 variants)")
    return ap.parse_args(argv)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            pk = json.load(fh)
        return float(pk["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def workload(name: str, m: int, dtype):
    from paper_1810_09891_gb300 import workloads as W
    if name == "clusters":
        return W.config_clusters(dtype=dtype, m=m)
    return W.config_radial(m=m, dtype=dtype)


def algorithmic_bytes(stage: str, d: int, N, n, M: int, p: int) -> float:
    """Bytes each stage must move at least once (per launch of the stage), FP32 p = 4 / FP64 8.

    Per node: d offsets (d p) + cell index and permutation entry (8) + the complex value (2p).
    Grid: |I_n| complex values (2p each); read once by B, read and written by B^H (atomic adds).
    FFT stages: the compact coefficients, the pruned intermediates (written and read once) and the
    full grid (written once by the forward, read once by the adjoint)."""
    c = 2 * p
    G = int(np.prod(n))
    NN = int(np.prod(N))
    node = M * (d * p + 8 + c)
    inter = 0
    if d == 2:
        inter = N[0] * n[1]
    elif d == 3:
        inter = N[0] * N[1] * n[2] + N[0] * n[1] * n[2]
    if stage == "interp":
        return node + G * c
    if stage == "spread":
        return node + 2 * G * c
    if stage in ("fft_forward", "fft_adjoint"):
        return NN * c + G * c + 2 * inter * c
    if stage == "zero_grid":
        return G * c
    return 0.0


def source_sha(files) -> str:
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


STAGE_SOURCES = {
    "spread": ["paper_1810_09891_gb300/csrc/spread_impl.cuh",
               "paper_1810_09891_gb300/csrc/window.cuh"],
    "interp": ["paper_1810_09891_gb300/csrc/interp_impl.cuh",
               "paper_1810_09891_gb300/csrc/window.cuh"],
    "fft_forward": ["paper_1810_09891_gb300/csrc/fft_impl.cuh"],
    "fft_adjoint": ["paper_1810_09891_gb300/csrc/fft_impl.cuh"],
}


def profiled_traffic(stage: str, workload_name: str):
    """DRAM bytes per launch from a committed ncu summary (profiles/<stage>_<workload>.txt), if
    it was taken on the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", f"{stage}_{workload_name}.txt")
    if not os.path.exists(path) or stage not in STAGE_SOURCES:
        return None
    vals = {}
    with open(path) as fh:
        for line in fh:
            if ":" in line:
                k, v = line.split(":", 1)
                vals[k.strip()] = v.strip()
    if vals.get("kernel_source_sha") != source_sha(STAGE_SOURCES[stage]):
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


NUM_SMS = 152  # GB300


def profiled_value(stage: str, workload_name: str, key: str):
    """A counter from a committed ncu summary taken on the current kernel source, else None."""
    path = os.path.join(ROOT, "profiles", f"{stage}_{workload_name}.txt")
    if not os.path.exists(path) or stage not in STAGE_SOURCES:
        return None
    vals = {}
    with open(path) as fh:
        for line in fh:
            if ":" in line:
                k, v = line.split(":", 1)
                vals[k.strip()] = v.strip()
    if vals.get("kernel_source_sha") != source_sha(STAGE_SOURCES[stage]):
        return None
    try:
        return float(vals[key])
    except (KeyError, ValueError):
        return None


def _clock_ghz(clk) -> float:
    mhz = (clk or {}).get("sm_mhz") or (clk or {}).get("sm_max_mhz") or 2070.0
    return float(mhz) / 1000.0


def onchip_roofline(stage, wl, M, m, ms, clk):
    """The spreading kernel against the L1 / shared-memory data pipe, which carries the tile
    read-modify-writes of the shared-memory tile forms: one 128-byte wavefront per cycle per SM.
    The tap floor of those forms is 2 (load and store) x (2m)^d taps x 8 bytes (FP32 complex) /
    128 per node; the measured wavefront and instruction counts come from the committed ncu
    summary when it matches the kernel source."""
    if stage != "spread":
        return None
    d = len(wl["N"])
    peak = NUM_SMS * _clock_ghz(clk) * 1e9  # wavefronts / s
    floor = M * (2 * m) ** d * 2 * 8 / 128.0
    out = {"resource": "L1/shared-memory data pipe (128-byte wavefronts)", "kernel": stage,
           "peak_wavefronts_per_s": peak, "tap_floor_wavefronts": floor,
           "tap_floor_frac": floor / (ms * 1e-3) / peak}
    w = profiled_value(stage, wl["name"], "shared_wavefronts")
    if w is not None:
        out.update({"wavefronts_per_launch": w, "achieved_wavefronts_per_s": w / (ms * 1e-3),
                    "frac": w / (ms * 1e-3) / peak})
    # the register-tile (rows) form moves few wavefronts and is bound by instruction issue
    # instead: warp instructions per launch (ncu) over the event time, against one instruction
    # per cycle per SM sub-partition (4 per SM)
    wi = profiled_value(stage, wl["name"], "warp_instructions")
    if wi is not None:
        ipeak = NUM_SMS * 4 * _clock_ghz(clk) * 1e9
        out["issue"] = {"warp_instructions_per_launch": wi,
                        "achieved_per_s": wi / (ms * 1e-3), "peak_per_s": ipeak,
                        "frac": wi / (ms * 1e-3) / ipeak}
    return out


POLY_DEG = {False: {1: 11, 2: 10, 3: 9}, True: {1: 18, 2: 18, 3: 16, 4: 16, 5: 15}}


def alu_roofline(d, m, fp64, M, stages, clk):
    """B and B^H against the FMA rate: per node, the 2m window values of each of the d axes as m
    mirrored pairs (one even/odd Horner evaluation of degree DEG, DEG + 2 FMAs per pair) and
    (2m)^d taps of 2 FMAs (complex value times real weight); an FMA is 2 flops. Peak: 152 SMs x
    128 FP32 lanes x 2 flops x clock; FP64 at 1/64 of that (GB300)."""
    deg = POLY_DEG[fp64].get(m, 14 if fp64 else 8)
    flops = 2.0 * (d * m * (deg + 2) + 2 * (2 * m) ** d) * M
    peak = NUM_SMS * 128 * 2 * _clock_ghz(clk) * 1e9 / (64.0 if fp64 else 1.0)
    out = {"flops_per_node": flops / M, "peak_tflops": peak / 1e12,
           "peak_kind": "nominal (FMA lanes x clock; FP64 at 1/64 of FP32), not measured"}
    for st in ("interp", "spread"):
        if st in stages:
            t = stages[st]["ms_per_launch"] * 1e-3
            out[st] = {"tflops": flops / t / 1e12, "frac": flops / t / peak}
    return out


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons while the timed region runs."""

    FIELDS = ("timestamp,index,uuid,clocks.sm,clocks.max.sm,power.draw,"
              "clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.uuid = uuid
        self.proc = None
        self.tmp = None

    def start(self):
        try:
            self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                   "-lms", "20"]
            self.proc = subprocess.Popen(cmd, stdout=self.tmp, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self, t0=None, t1=None):
        """Stop sampling; summarise the samples taken between wall-clock times t0 and t1."""
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.tmp.flush()
        rows = []
        with open(self.tmp.name) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 11:
                    continue
                if self.uuid and self.uuid not in parts[2]:
                    continue
                if t0 is not None:
                    try:
                        ts = time.mktime(time.strptime(parts[0].split(".")[0],
                                                       "%Y/%m/%d %H:%M:%S"))
                        ts += float("0." + parts[0].split(".")[1]) if "." in parts[0] else 0.0
                    except (ValueError, IndexError):
                        ts = None
                    if ts is not None and not (t0 - 0.05 <= ts <= t1 + 0.05):
                        continue
                rows.append(parts[1:])
        os.unlink(self.tmp.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = [num(r[2]) for r in rows if num(r[2]) is not None]
        smax = [num(r[3]) for r in rows if num(r[3]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[6 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(rows)}


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a per-rank number over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64,
                     device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(nodes_per_rank: int, steps: int, world: int, total_ms_max: float) -> float:
    """Whole-job nodes/s: every rank processes its own replica of the workload (weak scaling), so
    the job moves world * M * K nodes in the slowest rank's time."""
    return world * nodes_per_rank * steps / (total_ms_max * 1e-3)


def rel_l2(a, b) -> float:
    a = np.asarray(a).reshape(-1)
    b = np.asarray(b).reshape(-1)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


# ------------------------------------------------------------------------------ CPU oracle

def time_oracle(wl, sample_nodes: int, min_seconds: float, max_reps: int, seed: int = 0):
    """Oracle forward + adjoint on a sample of the workload's nodes (all of them if
    sample_nodes >= M), repeated until min_seconds elapsed; returns (nodes/s, reps, seconds)."""
    import oracle
    x = np.asarray(wl["x"], dtype=np.float64)
    M = x.shape[0]
    if sample_nodes < M:
        idx = np.sort(np.random.default_rng(seed).choice(M, sample_nodes, replace=False))
        xs, fs = x[idx], wl["f"][idx]
    else:
        xs, fs = x, wl["f"]
    fh = wl["fhat"].astype(np.complex128)
    reps, t0 = 0, time.perf_counter()
    while True:
        oracle.nfft(xs, fh, n=wl["n"], m=wl["m"])
        oracle.nfft_adjoint(xs, fs, wl["N"], n=wl["n"], m=wl["m"])
        reps += 1
        el = time.perf_counter() - t0
        if el >= min_seconds or reps >= max_reps:
            break
    return xs.shape[0] * reps / el, reps, el


def reference_arm(args):
    """--impl reference: the CPU oracle on the host cores, one step = forward + adjoint on a
    bounded node sample of the same workload."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    wl = workload(args.workload, args.m, np.float32)
    M = wl["x"].shape[0]
    sample = int(max(4096, min(M, (1 << 17) * 60 // max(1, args.steps + args.warmup))))
    for _ in range(args.warmup):
        time_oracle(wl, sample, 0.0, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        time_oracle(wl, sample, 0.0, 1)
    el = time.perf_counter() - t0
    value = sample * args.steps / el
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": wl["name"], "N": list(wl["N"]), "n": list(wl["n"]), "m": wl["m"],
                   "M": M, "sample_nodes": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.max_threads(),
                         "kind": "oracle",
                         "sample": f"{sample} of the {M} nodes (seeded choice), full grid; "
                                   "one forward + one adjoint per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------------------ GPU arm

KERNEL_STAGES = ("fft_forward", "interp", "spread", "fft_adjoint")


def profile_stages(plan, fh, f, steps, flush, torch):
    """Per-stage milliseconds per launch from the library's own CUDA events (nfft_profile) over
    `steps` forward + adjoint steps with the L2 flushed between steps (back to back when `flush`
    is None)."""
    import ctypes

    from paper_1810_09891_gb300 import _lib
    L = _lib.lib()
    L.nfft_profile(plan._h, 1)
    run_variant(plan, fh, f, steps, flush, torch)
    ms = (ctypes.c_double * 7)()
    cnt = (ctypes.c_int64 * 7)()
    L.nfft_profile_read(plan._h, ms, cnt, 7)
    L.nfft_profile(plan._h, 0)
    return {name: {"ms_per_launch": ms[i] / cnt[i], "launches": int(cnt[i])}
            for i, name in enumerate(_lib.STAGES) if cnt[i]}


def roofline_of(stages, wl, M, p, peak, peak_kind, workload_name=None):
    """HBM roofline of the step's dominant kernel: its algorithmic bytes per launch over its
    event time, against the measured copy bandwidth. Adds bytes, GB/s and share to `stages`."""
    d = len(wl["N"])
    ks = {k: v for k, v in stages.items() if k in KERNEL_STAGES}
    step_ms = sum(v["ms_per_launch"] for v in ks.values())
    for k, v in stages.items():
        b = algorithmic_bytes(k, d, wl["N"], wl["n"], M, p)
        v["algorithmic_bytes"] = b
        v["GBps"] = b / (v["ms_per_launch"] * 1e-3) / 1e9 if b else None
        v["share"] = v["ms_per_launch"] / step_ms if k in ks else None
    dom = max(ks, key=lambda k: ks[k]["ms_per_launch"])
    achieved = stages[dom]["GBps"]
    return {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak,
            "traffic": profiled_traffic(dom, workload_name) if workload_name else None,
            "peak_kind": peak_kind}


def fft_vs_cufft(plan, fh, f, n, stages, flush, dev, torch, reps=50):
    """Step F against cuFFT's full (unpruned) forward FFT of the oversampled grid (torch.fft.fftn,
    complex64), both under the same two cache states: with the L2 flushed before every call (the
    state of the timed steps, where the grid, the tables and the kernels' code are fetched from
    HBM) and back to back (all of it resident in L2)."""
    try:
        d = len(n)
        z = torch.randn(tuple(n), dtype=torch.complex64, device=dev)
        dims = tuple(range(d))
        for _ in range(5):
            torch.fft.fftn(z, dim=dims)
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record()
        for _ in range(reps):
            torch.fft.fftn(z, dim=dims)
        a1.record()
        torch.cuda.synchronize()
        warm = a0.elapsed_time(a1) / reps * 1e3
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(reps)]
        for b0, b1 in ev:
            flush.zero_()
            b0.record()
            torch.fft.fftn(z, dim=dims)
            b1.record()
        torch.cuda.synchronize()
        flushed = sum(b0.elapsed_time(b1) for b0, b1 in ev) / reps * 1e3
        del z
        hot = profile_stages(plan, fh, f, reps, None, torch)
        return {"cufft_fftn_us": warm, "cufft_fftn_l2_flushed_us": flushed,
                "ours_fft_forward_us": stages["fft_forward"]["ms_per_launch"] * 1e3,
                "ours_fft_adjoint_us": stages["fft_adjoint"]["ms_per_launch"] * 1e3,
                "ours_fft_forward_back_to_back_us": hot["fft_forward"]["ms_per_launch"] * 1e3,
                "ours_fft_adjoint_back_to_back_us": hot["fft_adjoint"]["ms_per_launch"] * 1e3,
                "note": "cuFFT: full n-point FFT of the grid (torch.fft.fftn, complex64); ours: "
                        "pruned passes with D (or D^H) and zero padding (or cropping) fused. "
                        "cufft_fftn_us and ours_*_back_to_back_us: back-to-back calls (grid, "
                        "tables and code resident in L2); cufft_fftn_l2_flushed_us and "
                        "ours_fft_forward_us / ours_fft_adjoint_us: L2 flushed before every "
                        "call or step, as in the timed steps"}
    except Exception as exc:  # the comparison is optional context
        return {"unavailable": str(exc)[:120]}


def run_variant(plan, fh, f, steps, flush, torch):
    """Times `steps` steps (forward + adjoint) with an L2 flush between steps outside the timed
    events (none when `flush` is None); returns per-step forward / adjoint / total
    milliseconds."""
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    outs = None
    for i in range(steps):
        if flush is not None:
            flush.zero_()
        e0, e1, e2 = ev[i]
        e0.record(stream)
        y = plan.trafo(fh)
        e1.record(stream)
        h = plan.adjoint(f)
        e2.record(stream)
        outs = (y, h)
    torch.cuda.synchronize()
    fwd = [a.elapsed_time(b) for a, b, _ in ev]
    adj = [b.elapsed_time(c) for _, b, c in ev]
    return fwd, adj, outs


_NDFT_CACHE = {}


def parity(wl, y, h, m, n, sample=4096, seed=1, full_adjoint=True):
    """Errors of the GPU outputs on the same (rounded) inputs:
    against the FP64 oracle NFFT (rel. l2; forward on a seeded node sample, adjoint over all
    coefficients, spreading all M nodes), and against the direct NDFT, the exact transform
    (Section 1, eq. NDFT): forward on the node sample, adjoint on a seeded sample of coefficients
    summed over all M nodes, as E_2 (rel. l2) and the paper's E_inf (eq. EI: max error over the
    l1 norm of the input)."""
    import oracle
    x = np.asarray(wl["x"], dtype=np.float64)
    M = x.shape[0]
    g = np.random.default_rng(seed)
    idx = np.sort(g.choice(M, min(sample, M), replace=False))
    nk = int(np.prod(wl["N"]))
    kidx = np.sort(g.choice(nk, min(sample, nk), replace=False))
    ref_f = oracle.nfft(x[idx], wl["fhat_r"], n=n, m=m)
    ref_h = oracle.nfft_adjoint(x, wl["f_r"], wl["N"], n=n, m=m) if full_adjoint else None
    key = (wl["name"], str(wl["x"].dtype), sample, seed)
    if key not in _NDFT_CACHE:  # the exact transform does not depend on m
        _NDFT_CACHE[key] = (oracle.ndft_tab(x[idx], wl["fhat_r"]),
                            oracle.ndft_adjoint_at(x, wl["f_r"], wl["N"], kidx))
    nd_f, nd_h = _NDFT_CACHE[key]
    hs = np.asarray(h).reshape(-1)[kidx]
    return {"fwd_rel_l2_vs_oracle_nfft": rel_l2(y[idx], ref_f),
            "adj_rel_l2_vs_oracle_nfft": rel_l2(h, ref_h) if full_adjoint else None,
            "fwd_rel_l2_vs_ndft": rel_l2(y[idx], nd_f),
            "adj_rel_l2_vs_ndft": rel_l2(hs, nd_h),
            "fwd_einf_vs_ndft": float(np.max(np.abs(y[idx] - nd_f)) /
                                      np.sum(np.abs(wl["fhat_r"]))),
            "adj_einf_vs_ndft": float(np.max(np.abs(hs - nd_h)) / np.sum(np.abs(wl["f_r"]))),
            "sample_nodes": int(idx.size), "sample_coefficients": int(kidx.size)}


def run_concurrent(plan, fh, f, steps, flush, torch):
    """Like run_variant, but each step runs the forward and the adjoint at the same time on two
    streams (the plan keeps separate grids for them), joined before the step's end event;
    returns per-step milliseconds."""
    cur = torch.cuda.current_stream()
    sf, sa = torch.cuda.Stream(), torch.cuda.Stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    for i in range(steps):
        flush.zero_()
        a, b = ev[i]
        a.record(cur)
        sf.wait_stream(cur)
        sa.wait_stream(cur)
        with torch.cuda.stream(sf):
            plan.trafo(fh)
        with torch.cuda.stream(sa):
            plan.adjoint(f)
        cur.wait_stream(sf)
        cur.wait_stream(sa)
        b.record(cur)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def timed_steps(plan, fh, f, steps, warmup, flush, uuid, torch):
    """Warm-up, then `steps` timed forward + adjoint steps with the SM clocks sampled during the
    timed region; returns (forward ms, adjoint ms, outputs, clocks)."""
    run_variant(plan, fh, f, max(3, warmup), flush, torch)
    clocks = ClockSampler(uuid)
    clocks.start()
    run_variant(plan, fh, f, 20, flush, torch)  # keeps the GPU busy while the sampler starts
    torch.cuda.synchronize()
    t0 = time.time()
    fwd, adj, outs = run_variant(plan, fh, f, steps, flush, torch)
    torch.cuda.synchronize()
    t1 = time.time()
    return fwd, adj, outs, clocks.stop(t0, t1)


def clusters_record(args, flush, dev, hbm_peak, peak_kind, uuid, torch):
    """The 3-D clustered workload: N = (128,)*3, n = 2N, m = 4, M = 4,194,304 nodes (half
    uniform, half in 8 Gaussian clusters), FP32; forward + adjoint per step."""
    from paper_1810_09891_gb300.nfft import Plan
    wl = workload("clusters", 4, np.float32)
    wl["fhat_r"] = wl["fhat"].astype(np.complex64).astype(np.complex128)
    wl["f_r"] = wl["f"].astype(np.complex64).astype(np.complex128)
    M = wl["x"].shape[0]
    plan = Plan(wl["N"], M, n=wl["n"], m=4, dtype=torch.float32, device=dev)
    x = torch.tensor(wl["x"], device=dev)
    fh = torch.tensor(wl["fhat"].astype(np.complex64), device=dev)
    f = torch.tensor(wl["f"].astype(np.complex64), device=dev)
    plan.set_nodes(x)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    plan.set_nodes(x)
    e1.record()
    torch.cuda.synchronize()
    set_nodes_ms = e0.elapsed_time(e1)
    steps = max(5, min(args.steps, 20))
    fwd, adj, (y, h), clk = timed_steps(plan, fh, f, steps, args.warmup, flush, uuid, torch)
    if plan.status() != 0:
        raise RuntimeError("device status after the clustered workload")
    stages = profile_stages(plan, fh, f, 5, flush, torch)
    roof = roofline_of(stages, wl, M, 4, hbm_peak, peak_kind, wl["name"])
    total = sum(fwd) + sum(adj)
    rec = {"workload": wl["name"], "N": list(wl["N"]), "n": list(wl["n"]), "m": 4, "M": M,
           "dtype": "f32", "steps": steps, "ms_per_step": total / steps,
           "value": M * steps / (total * 1e-3), "unit": UNIT,
           "fwd_nodes_per_s": M * steps / (sum(fwd) * 1e-3),
           "adj_nodes_per_s": M * steps / (sum(adj) * 1e-3), "set_nodes_ms": set_nodes_ms,
           "roofline": roof, "stages_us": {k: 1e3 * v["ms_per_launch"] for k, v in stages.items()},
           "clocks": clk,
           "l2": "inputs larger than L2 (grid 134 MB, nodes 84 MB); flushed between steps too"}
    run_concurrent(plan, fh, f, 3, flush, torch)
    conc = run_concurrent(plan, fh, f, steps, flush, torch)
    rec["concurrent"] = {"ms_per_step": sum(conc) / len(conc),
                         "nodes_per_s": M * len(conc) / (sum(conc) * 1e-3),
                         "how": "forward and adjoint of each step on two streams at once"}
    rec["fft_vs_cufft"] = fft_vs_cufft(plan, fh, f, wl["n"], stages, flush, dev, torch, reps=10)
    if not args.no_parity:
        rec["errors"] = parity(wl, y.cpu().numpy(), h.cpu().numpy(), 4, plan.n,
                               full_adjoint=False)
    plan.close()
    return rec


def ours(args):
    import torch
    import torch.distributed as dist

    from paper_1810_09891_gb300 import _lib
    from paper_1810_09891_gb300.nfft import Plan

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    hbm_peak, peak_kind = load_peaks()

    # L2 flush buffer: 256 MiB, larger than the 129 MB L2 (the working set of the radial
    # workload, ~60 MB, would otherwise stay resident between steps)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)

    def make(dtype_np, dtype_t, m):
        wl = workload(args.workload, m, dtype_np)
        cdt = np.complex64 if dtype_np == np.float32 else np.complex128
        wl["fhat_r"] = wl["fhat"].astype(cdt).astype(np.complex128)
        wl["f_r"] = wl["f"].astype(cdt).astype(np.complex128)
        plan = Plan(wl["N"], wl["x"].shape[0], n=wl["n"], m=m, dtype=dtype_t, device=dev)
        x = torch.tensor(wl["x"], device=dev)
        fh = torch.tensor(wl["fhat"].astype(cdt), device=dev)
        f = torch.tensor(wl["f"].astype(cdt), device=dev)
        return wl, plan, x, fh, f

    wl, plan, x, fh, f = make(np.float32, torch.float32, args.m)
    M = wl["x"].shape[0]
    d = len(wl["N"])

    # set_nodes (the paper's "precomputation"), timed separately
    plan.set_nodes(x)
    torch.cuda.synchronize()
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sn = []
    for _ in range(5):
        s0.record()
        plan.set_nodes(x)
        s1.record()
        torch.cuda.synchronize()
        sn.append(s0.elapsed_time(s1))
    set_nodes_ms = statistics.median(sn)

    # warm-up, then the timed region: K steps bracketed by barrier + synchronize
    run_variant(plan, fh, f, max(3, args.warmup), flush, torch)
    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    clocks = ClockSampler(uuid)
    clocks.start()
    run_variant(plan, fh, f, 200, flush, torch)  # keeps the GPU busy while the sampler starts
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t_start = time.time()
    fwd, adj, (y, h) = run_variant(plan, fh, f, args.steps, flush, torch)
    torch.cuda.synchronize()
    t_end = time.time()
    if world > 1:
        dist.barrier()
    clk = clocks.stop(t_start, t_end)
    total_ms = max_over_ranks(float(sum(fwd) + sum(adj)), dev)
    ms_per_step = total_ms / args.steps
    value = job_throughput(M, args.steps, world, total_ms)
    st = plan.status()
    if st != 0:
        raise RuntimeError(f"device status {st} after the timed region")

    # per-stage times (library events on the plan's stream) over a second pass of K steps
    stages = profile_stages(plan, fh, f, args.steps, flush, torch)
    kernel_stages = {k: v for k, v in stages.items() if k in KERNEL_STAGES}
    roofline = roofline_of(stages, wl, M, 4, hbm_peak, peak_kind, wl["name"])
    dom = roofline["kernel"]

    # the two further roofline views of the spreading kernel and of the window arithmetic
    onchip = onchip_roofline(dom, wl, M, args.m, kernel_stages[dom]["ms_per_launch"], clk)
    alu = {"f32": alu_roofline(d, args.m, False, M, kernel_stages, clk)}

    # the same steps with the forward and the adjoint running at the same time on two streams
    run_concurrent(plan, fh, f, max(3, args.warmup), flush, torch)
    conc = run_concurrent(plan, fh, f, args.steps, flush, torch)
    concurrent = {"ms_per_step": sum(conc) / len(conc),
                  "nodes_per_s": M * len(conc) / (sum(conc) * 1e-3),
                  "how": "forward and adjoint of each step on two streams at once (separate "
                         "grids per plan), L2 flushed between steps"}

    # cuFFT as a timed comparison for step F only (both cache states)
    cufft = fft_vs_cufft(plan, fh, f, wl["n"], stages, flush, dev, torch)

    # end to end through the host-buffer entry points (pinned host memory)
    pin_fh = torch.tensor(wl["fhat"].astype(np.complex64)).pin_memory()
    pin_f = torch.tensor(wl["f"].astype(np.complex64)).pin_memory()
    out_f = torch.empty(M, dtype=torch.complex64).pin_memory()
    out_h = torch.empty(tuple(wl["N"]), dtype=torch.complex64).pin_memory()
    plan.set_nodes_host(torch.tensor(wl["x"]))
    e2e_steps = max(3, min(args.steps, 50))
    for _ in range(3):
        plan.trafo_host(pin_fh, out_f)
        plan.adjoint_host(pin_f, out_h)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        plan.trafo_host(pin_fh, out_f)
        plan.adjoint_host(pin_f, out_h)
    serial_s = time.perf_counter() - t0
    flushed_s = 0.0
    for _ in range(e2e_steps):
        flush.zero_()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        plan.trafo_host(pin_fh, out_f)
        plan.adjoint_host(pin_f, out_h)
        flushed_s += time.perf_counter() - t1
    plan.set_nodes(x)
    e2e_pipelined(plan, pin_fh, pin_f, out_f, out_h, 3, torch)
    e2e_s = e2e_pipelined(plan, pin_fh, pin_f, out_f, out_h, e2e_steps, torch)
    nn = int(np.prod(wl["N"]))
    e2e = {"value": world * M * e2e_steps / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": 8 * (nn + M), "d2h_bytes_per_step": 8 * (M + nn),
           "steps": e2e_steps,
           "pipeline": "every step copies its inputs from pinned host memory and its results "
                       "back; the input copies of the next step and the result copies of this "
                       "one run on two copy streams beside the kernels (Plan.trafo / "
                       "Plan.adjoint on double-buffered device inputs)",
           "note": "no L2 flush between these steps (the device-timed value flushes L2); the "
                   "copies per step (about 120 us at the ~170 GB/s of pinned copies on this "
                   "machine) hide behind the kernels of the neighbouring step",
           "host_calls_value": world * M * e2e_steps / serial_s,
           "host_calls_l2_flushed_value": world * M * e2e_steps / flushed_s,
           "host_calls": "nfft_trafo_host + nfft_adjoint_host per step (copies, kernels and a "
                         "wait in sequence, through the C ABI); _l2_flushed: a 256 MiB write "
                         "before every step, outside the host timer"}

    line = None
    if rank == 0:
        errors = None
        if not args.no_parity:
            errors = parity(wl, y.cpu().numpy(), h.cpu().numpy(), args.m, plan.n)
        variants = []
        if not args.no_variants:
            for dt_np, dt_t, mm in [(np.float64, torch.float64, args.m),
                                    (np.float32, torch.float32, 6),
                                    (np.float64, torch.float64, 6)]:
                wv, pv, xv, fhv, fv = make(dt_np, dt_t, mm)
                pv.set_nodes(xv)
                run_variant(pv, fhv, fv, 3, flush, torch)
                kv = max(5, min(args.steps, 100))
                fw, ad, (yv, hv) = run_variant(pv, fhv, fv, kv, flush, torch)
                ent = {"dtype": "f64" if dt_t == torch.float64 else "f32", "m": mm,
                       "nodes_per_s": M * kv / ((sum(fw) + sum(ad)) * 1e-3),
                       "fwd_nodes_per_s": M * kv / (sum(fw) * 1e-3),
                       "adj_nodes_per_s": M * kv / (sum(ad) * 1e-3),
                       "ms_per_step": (sum(fw) + sum(ad)) / kv}
                stv = profile_stages(pv, fhv, fv, 10, flush, torch)
                pbytes = 8 if dt_t == torch.float64 else 4
                ent["roofline"] = roofline_of(stv, wv, M, pbytes, hbm_peak, peak_kind)
                ent["stages_us"] = {k: 1e3 * v["ms_per_launch"] for k, v in stv.items()}
                if dt_t == torch.float64 and mm == args.m:
                    # FP64 window and tap arithmetic against the nominal FP64 FMA rate
                    alu["f64"] = alu_roofline(d, mm, True, M, stv, clk)
                if not args.no_parity:
                    ent.update(parity(wv, yv.cpu().numpy(), hv.cpu().numpy(), mm, pv.n))
                variants.append(ent)
                pv.close()
        cpu = None
        if not args.no_cpu:
            import oracle
            oracle.build()
            v, reps, el = time_oracle(wl, M, 10.0, 3)
            cpu = {"value": v, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
                   "sample": f"the full workload ({M} nodes) x {reps} forward+adjoint, "
                             f"{el:.1f} s"}
        sub = {}
        if not args.no_subrecords:
            sub["clusters"] = clusters_record(args, flush, dev, hbm_peak, peak_kind, uuid, torch)
            sub["batched"] = batched_record(args, dev, uuid, flush, torch)
        launches_per_step = 2 * d + 2
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": wl["name"], "N": list(wl["N"]), "n": list(wl["n"]),
                       "m": args.m, "M": M, "precision": "FP32 data, FP64 phihat and offsets",
                       "l2": "flushed (256 MiB write) between timed steps, outside the events",
                       "parallelism": f"{world} independent replica(s)"},
            "ms_per_step_median": statistics.median([a + b for a, b in zip(fwd, adj)]),
            "fwd_nodes_per_s": M * args.steps / (sum(fwd) * 1e-3),
            "adj_nodes_per_s": M * args.steps / (sum(adj) * 1e-3),
            "set_nodes_ms": set_nodes_ms,
            "concurrent": concurrent,
            "errors": errors,
            "roofline": roofline,
            "onchip": onchip,
            "alu": alu,
            "fft_vs_cufft": cufft,
            "stages": stages,
            "variants": variants,
            "cpu_baseline": cpu,
            "subrecords": sub or None,
            "e2e": e2e,
            "gpu_launches": launches_per_step * args.steps,
            "clocks": clk,
        }
    plan.close()
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if line is not None:
        print(json.dumps(line))
    return 0


def ncu_step(args):
    """The timed kernels of the workload, untimed: set_nodes once, then --steps forward +
    adjoint pairs on the same plan and inputs as the benchmark."""
    import torch

    from paper_1810_09891_gb300.nfft import Plan
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    if args.workload == "batched":
        return ncu_step_batched(args, dev, torch)
    npdt, tdt, cdt = ((np.float32, torch.float32, np.complex64) if args.dtype == "f32" else
                      (np.float64, torch.float64, np.complex128))
    wl = workload(args.workload, args.m, npdt)
    plan = Plan(wl["N"], wl["x"].shape[0], n=wl["n"], m=args.m, dtype=tdt, device=dev)
    plan.set_nodes(torch.tensor(wl["x"], device=dev))
    fh = torch.tensor(wl["fhat"].astype(cdt), device=dev)
    f = torch.tensor(wl["f"].astype(cdt), device=dev)
    for _ in range(max(1, args.steps)):
        plan.trafo(fh)
        plan.adjoint(f)
    torch.cuda.synchronize()
    st = plan.status()
    plan.close()
    if st != 0:
        raise RuntimeError(f"device status {st}")
    return 0


def ncu_step_batched(args, dev, torch):
    """The batched workload's kernels, untimed and without a graph: the 64-problem batch with the
    benchmark's inputs, set_nodes once, then --steps forward + adjoint steps of the batch (fused
    where the batch qualifies)."""
    from paper_1810_09891_gb300 import workloads as W
    from paper_1810_09891_gb300.batch import PlanBatch, batched_specs
    specs = batched_specs()
    b = PlanBatch(specs, dtype=torch.float32, device=dev)
    xs = [torch.tensor(W.round_nodes(W.uniform_nodes(s["M"], 2, seed_offset=1000 + i),
                                     np.float32), device=dev) for i, s in enumerate(specs)]
    fhs = [torch.tensor(W.gaussian_fhat(s["N"], 2000 + i).astype(np.complex64), device=dev)
           for i, s in enumerate(specs)]
    fs = [torch.tensor(W.gaussian_values(s["M"], 3000 + i).astype(np.complex64), device=dev)
          for i, s in enumerate(specs)]
    b.set_nodes(xs)
    for _ in range(max(1, args.steps)):
        b.trafo(fhs)
        b.adjoint(fs)
    torch.cuda.synchronize()
    b.close()
    return 0


def e2e_pipelined(plan, pin_fh, pin_f, out_f, out_h, steps, torch):
    """Seconds (host clock) for `steps` forward + adjoint steps through host buffers: each step
    copies fhat and f from pinned host memory to the device and f and hhat back. The input
    copies run on one copy stream, double-buffered so that step k + 1's copies overlap step k's
    kernels; the result copies run on another stream as soon as each result exists."""
    dev = plan.device
    comp = torch.cuda.current_stream(dev)
    cin, cout = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    d_fh = [torch.empty(pin_fh.shape, dtype=pin_fh.dtype, device=dev) for _ in range(2)]
    d_f = [torch.empty(pin_f.shape, dtype=pin_f.dtype, device=dev) for _ in range(2)]
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_free = [torch.cuda.Event() for _ in range(2)]
    ev_y, ev_h = torch.cuda.Event(), torch.cuda.Event()
    for e in ev_free:
        e.record(comp)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(steps):
        j = k & 1
        with torch.cuda.stream(cin):
            cin.wait_event(ev_free[j])
            d_fh[j].copy_(pin_fh, non_blocking=True)
            d_f[j].copy_(pin_f, non_blocking=True)
            ev_in[j].record(cin)
        comp.wait_event(ev_in[j])
        y = plan.trafo(d_fh[j])
        ev_y.record(comp)
        h = plan.adjoint(d_f[j])
        ev_h.record(comp)
        ev_free[j].record(comp)
        with torch.cuda.stream(cout):
            cout.wait_event(ev_y)
            out_f.copy_(y, non_blocking=True)
            cout.wait_event(ev_h)
            out_h.copy_(h.reshape(out_h.shape), non_blocking=True)
        y.record_stream(cout)
        h.record_stream(cout)
    torch.cuda.synchronize()
    return time.perf_counter() - t0


def batched_record(args, dev, uuid, flush, torch):
    """64 independent 2-D problems (N_i per axis from {64, ..., 512}, M_i log-uniform in
    [1e4, 1e6], uniform nodes, FP32, m = 4): forward + adjoint of the whole batch captured in one
    CUDA graph; value = sum of M_i per step / step time. ``with_backward`` times a second graph
    that also holds the backward of the forward transform."""
    from paper_1810_09891_gb300 import workloads as W
    from paper_1810_09891_gb300.batch import PlanBatch, batched_specs
    specs = batched_specs()
    b = PlanBatch(specs, dtype=torch.float32, device=dev)
    xs = [torch.tensor(W.round_nodes(W.uniform_nodes(s["M"], 2, seed_offset=1000 + i),
                                     np.float32), device=dev) for i, s in enumerate(specs)]
    fhs = [torch.tensor(W.gaussian_fhat(s["N"], 2000 + i).astype(np.complex64), device=dev)
           for i, s in enumerate(specs)]
    fs = [torch.tensor(W.gaussian_values(s["M"], 3000 + i).astype(np.complex64), device=dev)
          for i, s in enumerate(specs)]
    gs = [torch.tensor(W.gaussian_values(s["M"], 4000 + i).astype(np.complex64), device=dev)
          for i, s in enumerate(specs)]
    b.set_nodes(xs)
    tuned = b.tune(fhs, fs) if getattr(args, "tune", False) else None
    steps = max(5, min(args.steps, 50))

    def timed_replays(sample_clocks=False):
        for _ in range(max(3, args.warmup)):
            b.replay()
        torch.cuda.synchronize()
        clocks = ClockSampler(uuid) if sample_clocks else None
        if clocks:
            clocks.start()
            for _ in range(20):
                b.replay()
            torch.cuda.synchronize()
        t0 = time.time()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        for a, c in ev:
            flush.zero_()
            a.record()
            b.replay()
            c.record()
        torch.cuda.synchronize()
        t1 = time.time()
        clk = clocks.stop(t0, t1) if clocks else None
        return sum(a.elapsed_time(c) for a, c in ev), clk

    fused = b.fused
    b.capture(fhs, fs)
    total_ms, clk = timed_replays(True)
    # the same step with the forward and the adjoint on two streams at once
    b.capture(fhs, fs, concurrent=True)
    conc_ms, _ = timed_replays()
    # the same step plus the backward of the forward transform (grad fhat and grad x for an
    # output gradient per problem) in one graph
    b.capture(fhs, fs, grad_fs=gs)
    bwd_ms, _ = timed_replays()
    # the same batch plan by plan (per-plan launches on eight side streams, parallel branches of
    # the graph), for comparison
    plan_by_plan = None
    if fused:
        b.set_fused(False)
        b.capture(fhs, fs)
        pbp_ms, _ = timed_replays()
        b.capture(fhs, fs, concurrent=True)
        pbpc_ms, _ = timed_replays()
        plan_by_plan = {"ms_per_step": pbp_ms / steps,
                        "nodes_per_s": sum(s["M"] for s in specs) * steps / (pbp_ms * 1e-3),
                        "how": "per-plan launches on 8 side streams, one CUDA graph",
                        "concurrent": {"ms_per_step": pbpc_ms / steps,
                                       "nodes_per_s": sum(s["M"] for s in specs) * steps /
                                       (pbpc_ms * 1e-3)}}
        b.set_fused(True)
    nodes = sum(s["M"] for s in specs)
    # whole-step HBM view: the algorithmic bytes of every plan's four kernel stages over the
    # step time
    alg = 0.0
    for s in specs:
        n = tuple(2 * v for v in s["N"])
        for st in KERNEL_STAGES:
            alg += algorithmic_bytes(st, 2, s["N"], n, s["M"], 4)
    hbm_peak, peak_kind = load_peaks()
    step_s = total_ms / steps * 1e-3
    rec = {"workload": "batched_64x2d_uneven", "problems": len(specs), "nodes_per_step": nodes,
           "m": 4, "dtype": "f32", "steps": steps, "ms_per_step": total_ms / steps,
           "value": nodes * steps / (total_ms * 1e-3), "unit": UNIT,
           "graph": "one CUDA graph per step",
           "fused": fused, "plan_by_plan": plan_by_plan,
           "concurrent": {"ms_per_step": conc_ms / steps,
                          "nodes_per_s": nodes * steps / (conc_ms * 1e-3),
                          "how": "the forward and the adjoint of the batch on two streams at once "
                                 "in the graph"},
           "roofline": {"bound": "hbm", "kernel": "whole step (all plans, all stages)",
                        "achieved": alg / step_s / 1e9, "peak": hbm_peak, "unit": "GB/s",
                        "frac": alg / step_s / 1e9 / hbm_peak, "traffic": None,
                        "peak_kind": peak_kind},
           "clocks": clk, "tuned": bool(tuned),
           "l2": "flushed (256 MiB write) between timed steps",
           "with_backward": {"ms_per_step": bwd_ms / steps,
                             "nodes_per_s": nodes * steps / (bwd_ms * 1e-3),
                             "step": "forward + adjoint + backward of the forward "
                                     "(adjoint for grad fhat, node-gradient kernel for grad x)"},
           "tuning": [{"N": list(s["N"]), "M": s["M"], "spread": t["spread_method"],
                       "bins": t["bins"]} for s, t in zip(specs, tuned)] if tuned else None}
    b.close()
    return rec


def batched(args):
    """--workload batched: the batched record alone, as a bench line."""
    import torch
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    r = batched_record(args, dev, uuid, flush, torch)
    line = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": 1,
            "steps": r["steps"], "warmup": args.warmup, "ms_per_step": r["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": r["workload"], "problems": r["problems"],
                       "nodes_per_step": r["nodes_per_step"], "m": 4, "graph": r["graph"],
                       "fused": r["fused"], "tuned": r["tuned"], "l2": r["l2"]},
            "plan_by_plan": r["plan_by_plan"],
            "roofline": r["roofline"], "clocks": r["clocks"],
            "with_backward": r["with_backward"], "tuning": r["tuning"]}
    print(json.dumps(line))
    return 0


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        return reference_arm(args)
    if args.ncu_step:
        return ncu_step(args)
    if args.workload == "batched":
        return batched(args)
    return ours(args)


if __name__ == "__main__":
    sys.exit(main())
