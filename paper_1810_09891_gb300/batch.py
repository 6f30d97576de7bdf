"""Many NFFTs of uneven size at once: a batch of plans, run fused (one launch per stage over all
plans) or plan by plan on side streams, captured in one CUDA graph, with per-plan tuning by
measurement.

``PlanBatch`` owns one ``Plan`` per problem (its own N, M, n, m, precision) and one library
batch over them (``nfft_batch_*`` of the C ABI: the plans run concurrently on side streams
forked from and joined into the current stream). ``trafo`` / ``adjoint`` / ``backward`` call the
library batch; ``capture`` records the forward and the adjoint of the whole batch into one CUDA
graph over static input and output buffers, and ``replay`` launches the batch with a single
graph launch (no per-kernel host overhead).
``autotune`` chooses, per plan, the spreading method, bin sizes and subproblem size, then the
interpolation form (threads per node), by timing candidates on the plan's own nodes (the measured counterpart of the plan search the paper's FFTW flags select,
Section 3.1, Table tab:fttwflags). Every candidate computes the same transform up to rounding.
"""
from __future__ import annotations

import ctypes
import json
import os
import statistics

import torch

from . import _lib
from ._lib import check
from .nfft import Plan


def _prod(v) -> int:
    r = 1
    for x in v:
        r *= int(x)
    return r

# Candidate options per dimension: (spread_method, bins, nodes per spreading work item)
CANDIDATES = {
    1: [(s, (b,), w) for s in ("warp_private", "warp_atomic") for b in (256, 1024, 4096)
        for w in (256, 1024)],
    2: [("rows", (4, 8), 32), ("rows", (4, 8), 64), ("rows", (4, 8), 128), ("rows", (8, 8), 64),
        ("rows", (8, 16), 128), ("half", (8, 16), 128), ("half", (8, 16), 256),
        ("half", (16, 16), 128), ("octet", (8, 16), 256), ("warp_private", (16, 16), 256),
        ("warp_atomic", (16, 16), 256)],
    3: [("plane", b, w) for b in ((8, 8, 16), (4, 16, 16), (8, 8, 8)) for w in (512, 1024)] +
       [(s, b, w) for s in ("warp_atomic", "thread") for b in ((8, 8, 8), (8, 8, 16))
        for w in (256, 1024)],
}

# Interpolation forms, by threads per node: one thread per node, a warp per node, a CTA per
# subproblem tile, eight lanes per node
INTERP_CANDIDATES = ("thread", "warp", "tile", "octet")


def _apply(plan: Plan, spread: str, bins, sub: int = 0) -> None:
    plan.set_option("spread_method", spread)
    for t, b in enumerate(bins):
        plan.set_option(f"bin{t}", int(b))
    plan.set_option("subproblem", int(sub))


def _timed(run, steps: int) -> float:
    """Median milliseconds of `run()` over `steps` calls on the current stream (CUDA events)."""
    run()
    times = []
    for _ in range(steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        run()
        b.record()
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    return statistics.median(times)


def time_step(plan: Plan, x: torch.Tensor, fhat: torch.Tensor, f: torch.Tensor,
              steps: int = 5) -> float:
    """Median milliseconds of one forward + one adjoint on the plan's stream (CUDA events)."""
    plan.set_nodes(x)

    def step():
        plan.trafo(fhat)
        plan.adjoint(f)
    return _timed(step, steps)


def autotune(plan: Plan, x: torch.Tensor, fhat: torch.Tensor, f: torch.Tensor,
             candidates=None, interp_candidates=INTERP_CANDIDATES, steps: int = 5) -> dict:
    """Measured plan search. First every candidate (spread_method, bins, subproblem) on this
    plan and these inputs, timing one forward + adjoint step (interpolation form automatic);
    then, with the fastest of them, every interpolation form (threads per node), timing the
    forward alone. The plan ends configured with the winners, nodes set. Returns
    {"spread_method", "bins", "subproblem", "interp_method", "ms", "tried": [(spread, bins,
    subproblem, ms), ...], "tried_interp": [(interp, ms), ...]}; "ms" is the step time with
    both choices. Candidates that do not fit the hardware are skipped."""
    cands = candidates if candidates is not None else CANDIDATES[plan.d]
    plan.set_option("interp_method", "auto")
    tried = []
    for spread, bins, sub in cands:
        bins = tuple(min(int(b), nn) for b, nn in zip(bins, plan.n))
        try:
            _apply(plan, spread, bins, sub)
            ms = time_step(plan, x, fhat, f, steps)
        except RuntimeError:
            continue
        tried.append((spread, bins, sub, ms))
    if not tried:
        raise RuntimeError("autotune: no candidate ran")
    spread, bins, sub, _ = min(tried, key=lambda t: t[3])
    _apply(plan, spread, bins, sub)
    plan.set_nodes(x)
    tried_interp = []
    for form in interp_candidates:
        try:
            plan.set_option("interp_method", form)
            tried_interp.append((form, _timed(lambda: plan.trafo(fhat), steps)))
        except RuntimeError:
            continue
    interp = min(tried_interp, key=lambda t: t[1])[0] if tried_interp else "auto"
    plan.set_option("interp_method", interp)
    ms = time_step(plan, x, fhat, f, steps)
    return {"spread_method": spread, "bins": list(bins), "subproblem": sub,
            "interp_method": interp, "ms": ms, "tried": tried, "tried_interp": tried_interp}


class TuningCache:
    """Chosen options keyed by (d, N, n, m, precision, M), optionally persisted as JSON."""

    def __init__(self, path: str | None = None):
        self.path = path
        self.table = {}
        if path and os.path.exists(path):
            with open(path) as fh:
                self.table = json.load(fh)

    @staticmethod
    def key(plan: Plan) -> str:
        return json.dumps([plan.d, list(plan.N), list(plan.n), plan.m, str(plan.dtype), plan.M])

    def get(self, plan: Plan):
        return self.table.get(self.key(plan))

    def put(self, plan: Plan, choice: dict) -> None:
        self.table[self.key(plan)] = {"spread_method": choice["spread_method"],
                                      "bins": list(choice["bins"]),
                                      "subproblem": int(choice.get("subproblem", 0)),
                                      "interp_method": choice.get("interp_method", "auto"),
                                      "ms": choice["ms"]}
        if self.path:
            with open(self.path, "w") as fh:
                json.dump(self.table, fh, indent=1)


class PlanBatch:
    """A batch of independent NFFT problems (uneven N and M) on one device.

    The plans run on ``streams`` side streams of the library batch, forked from and joined
    back into the caller's stream, so that small problems execute concurrently (in a captured
    graph they become parallel branches). The library assigns plans to side streams largest
    first, each to the stream with the least work so far (work ~ M + |I_n|)."""

    def __init__(self, specs, dtype=torch.float32, device=None, streams: int = 8):
        """specs: iterable of dicts with keys N, M and optionally n, m (default 4)."""
        specs = list(specs)
        if not specs:
            raise ValueError("a batch needs at least one problem")
        self.plans = [Plan(s["N"], s["M"], n=s.get("n"), m=s.get("m", 4), dtype=dtype,
                           device=device) for s in specs]
        self.device = self.plans[0].device
        self.dtype = dtype
        self.graph = None
        k = len(self.plans)
        L = _lib.lib()
        handles = (ctypes.c_void_p * k)(*[p._h.value for p in self.plans])
        self._b = ctypes.c_void_p()
        check(L.nfft_batch_create(ctypes.byref(self._b), ctypes.cast(handles, ctypes.c_void_p),
                                  k, int(streams)), "nfft_batch_create")
        cnt, ns = ctypes.c_int(), ctypes.c_int()
        check(L.nfft_batch_size(self._b, ctypes.byref(cnt), ctypes.byref(ns)), "nfft_batch_size")
        self.n_streams = ns.value
        self.lane = [L.nfft_batch_lane(self._b, i) for i in range(k)]

    @property
    def fused(self) -> bool:
        """Whether the next call runs every stage of all plans in one launch (nfft_batch_*
        fused execution: 2-D FP32 plans with one m and window; see include/gbnfft.h)."""
        v = ctypes.c_int()
        check(_lib.lib().nfft_batch_get_fused(self._b, ctypes.byref(v)), "nfft_batch_get_fused")
        return bool(v.value)

    def set_fused(self, enable: bool) -> None:
        """Turn fused execution on (NFFT_EUNSUPPORTED if the plans do not qualify) or off (plan
        by plan on the side streams)."""
        check(_lib.lib().nfft_batch_set_fused(self._b, int(bool(enable))), "nfft_batch_set_fused")

    def close(self):
        b = getattr(self, "_b", None)
        if b is not None and b.value:
            _lib.lib().nfft_batch_destroy(b)
            self._b = ctypes.c_void_p()
        for p in getattr(self, "plans", []):
            p.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _call(self, name: str, *arrays) -> None:
        """One library batch call on the current stream; each argument is a list of tensors
        (one per plan) passed as an array of device pointers."""
        L = _lib.lib()
        stream = torch.cuda.current_stream(self.device)
        check(L.nfft_batch_set_stream(self._b, ctypes.c_void_p(stream.cuda_stream)),
              "nfft_batch_set_stream")
        k = len(self.plans)
        ptrs = [ctypes.cast((ctypes.c_void_p * k)(*[t.data_ptr() for t in a]), ctypes.c_void_p)
                for a in arrays]
        check(getattr(L, name)(self._b, *ptrs), name)

    def _fhats(self, fhats, name="fhat") -> list:
        if len(fhats) != len(self.plans):
            raise ValueError(f"one {name} per plan")
        return [p._complex_in(t, _prod(p.N), name) for p, t in zip(self.plans, fhats)]

    def _fs(self, fs, name="f") -> list:
        if len(fs) != len(self.plans):
            raise ValueError(f"one {name} per plan")
        return [p._complex_in(t, p.M, name) for p, t in zip(self.plans, fs)]

    def __len__(self):
        return len(self.plans)

    def set_nodes(self, xs) -> None:
        for p, x in zip(self.plans, xs):
            p.set_nodes(x)
        self._x = list(xs)

    def tune(self, fhats, fs, cache: TuningCache | None = None, steps: int = 3) -> list:
        """Autotune every plan (or reuse a cached choice for its signature)."""
        out = []
        for p, x, fh, f in zip(self.plans, self._x, fhats, fs):
            choice = cache.get(p) if cache is not None else None
            if choice is None:
                choice = autotune(p, x, fh, f, steps=steps)
                if cache is not None:
                    cache.put(p, choice)
            else:
                _apply(p, choice["spread_method"], choice["bins"], choice.get("subproblem", 0))
                p.set_option("interp_method", choice.get("interp_method", "auto"))
                p.set_nodes(x)
            out.append(choice)
        return out

    def trafo(self, fhats) -> list:
        """Forward NFFT of every problem (Algorithm "NFFT"); returns the list of f_i."""
        ins = self._fhats(fhats)
        outs = [torch.empty(p.M, dtype=p.cdtype, device=p.device) for p in self.plans]
        self._call("nfft_batch_trafo", ins, outs)
        return outs

    def adjoint(self, fs) -> list:
        """Adjoint NFFT of every problem (Algorithm "adjoint NFFT"); returns the hhat_i."""
        ins = self._fs(fs)
        outs = [torch.empty(p.N, dtype=p.cdtype, device=p.device) for p in self.plans]
        self._call("nfft_batch_adjoint", ins, outs)
        return outs

    def backward(self, grad_fs, fhats, want_fhat: bool = True, want_x: bool = True) -> tuple:
        """Backward of the batched forward transform f_i = A_i fhat_i for output gradients
        grad_f_i: per plan, grad fhat_i = A_i^H grad_f_i (the adjoint kernels) and grad x_i =
        Re(conj(grad_f_i) d(A_i fhat_i)/dx) (the node-gradient kernel), both on the plan's side
        stream. Returns (grad_fhats, grad_xs); a list not asked for is all None."""
        k = len(self.plans)
        g_fhat, g_x = [None] * k, [None] * k
        if want_fhat:
            g_fhat = self.adjoint(grad_fs)
        if want_x:
            coef = self._fhats(fhats)
            w = self._fs(grad_fs, "grad_f")
            g_x = [torch.empty((p.M, p.d), dtype=p.dtype, device=p.device) for p in self.plans]
            self._call("nfft_batch_grad_x", coef, w, g_x)
        return g_fhat, g_x

    def capture(self, fhats, fs, grad_fs=None, concurrent: bool = False) -> None:
        """Record forward(fhats) and adjoint(fs) of the whole batch into one CUDA graph. The
        graph reads the given input tensors and writes ``self.out_f`` / ``self.out_h``; copy new
        inputs into ``fhats`` / ``fs`` before each ``replay``. Nodes must be set beforehand.
        With ``grad_fs`` the graph also holds the backward of the forward transform for those
        output gradients (read from ``self.in_grad_f``), written to ``self.out_grad_fhat`` and
        ``self.out_grad_x``. With ``concurrent`` the forward and the adjoint run on two streams
        at the same time (a plan's forward and adjoint use separate grids); the backward, if
        any, follows both."""
        self.in_fhat = list(fhats)
        self.in_f = list(fs)
        self.in_grad_f = list(grad_fs) if grad_fs is not None else None
        if concurrent and not hasattr(self, "_pair"):
            self._pair = (torch.cuda.Stream(self.device), torch.cuda.Stream(self.device))

        def step():
            if concurrent:
                cur = torch.cuda.current_stream(self.device)
                sf, sa = self._pair
                sf.wait_stream(cur)
                sa.wait_stream(cur)
                with torch.cuda.stream(sf):
                    yf = self.trafo(self.in_fhat)
                with torch.cuda.stream(sa):
                    yh = self.adjoint(self.in_f)
                cur.wait_stream(sf)
                cur.wait_stream(sa)
                out = (yf, yh)
            else:
                out = (self.trafo(self.in_fhat), self.adjoint(self.in_f))
            if self.in_grad_f is not None:
                out += self.backward(self.in_grad_f, self.in_fhat)
            return out

        s = torch.cuda.Stream(self.device)
        s.wait_stream(torch.cuda.current_stream(self.device))
        with torch.cuda.stream(s):  # warm-up outside the capture (kernel attributes, caches)
            step()
        torch.cuda.current_stream(self.device).wait_stream(s)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            out = step()
        self.out_f, self.out_h = out[0], out[1]
        self.out_grad_fhat, self.out_grad_x = (out[2], out[3]) if len(out) > 2 else (None, None)
        self.graph = g

    def replay(self):
        if self.graph is None:
            raise RuntimeError("capture() first")
        self.graph.replay()
        return self.out_f, self.out_h


class _BatchNFFTFunction(torch.autograd.Function):
    """[f_i] = [A_i fhat_i] for every plan of a PlanBatch, differentiable in every fhat_i and
    every node set x_i; forward and backward run the plans on the batch's side streams."""

    @staticmethod
    def forward(ctx, batch, *args):
        k = len(batch.plans)
        fhats, xs = args[:k], args[k:]
        for p, x in zip(batch.plans, xs):
            p.ensure_nodes(x)
        outs = batch.trafo(fhats)
        ctx.save_for_backward(*fhats, *xs)
        ctx.batch = batch
        return tuple(outs)

    @staticmethod
    def backward(ctx, *grad_fs):
        batch = ctx.batch
        k = len(batch.plans)
        saved = ctx.saved_tensors
        fhats, xs = saved[:k], saved[k:]
        for p, x in zip(batch.plans, xs):
            p.ensure_nodes(x)
        gs = [g.contiguous() if g is not None else
              torch.zeros(p.M, dtype=p.cdtype, device=p.device)
              for p, g in zip(batch.plans, grad_fs)]
        g_fhat, g_x = batch.backward(gs, fhats, want_fhat=any(ctx.needs_input_grad[1:1 + k]),
                                     want_x=any(ctx.needs_input_grad[1 + k:]))
        return (None, *g_fhat, *g_x)


def batch_nfft(fhats, xs, batch: PlanBatch) -> list:
    """Differentiable forward NFFT of every problem of ``batch`` (with respect to each fhat_i
    and each node set x_i); returns the list of f_i."""
    if len(fhats) != len(batch.plans) or len(xs) != len(batch.plans):
        raise ValueError("one fhat and one node set per plan")
    return list(_BatchNFFTFunction.apply(batch, *fhats, *xs))


def batched_specs(count: int = 64, seed_offset: int = 40, sizes=(64, 128, 256, 512),
                  log_m=(4.0, 6.0)):
    """Problem sizes of the batched workload: N_i per axis drawn from `sizes` independently,
    M_i log-uniform in [10^log_m[0], 10^log_m[1]] (seeded)."""
    from .workloads import rng

    g = rng(seed_offset)
    specs = []
    for _ in range(count):
        N = tuple(int(g.choice(sizes)) for _ in range(2))
        M = int(10 ** g.uniform(*log_m))
        specs.append({"N": N, "M": M, "m": 4})
    return specs
