"""Batched NFFTs of uneven size: every plan of a batch against the oracle, one CUDA graph for
the forward and adjoint of the whole batch (replayed with new inputs), and the autotuner."""
import numpy as np
import pytest
import torch

import oracle
from paper_1810_09891_gb300 import workloads as W
from paper_1810_09891_gb300.batch import PlanBatch, TuningCache, autotune, batched_specs
from paper_1810_09891_gb300.nfft import Plan

from gpu_helpers import DEV, TOL, rel_l2, rounded, to_dev

pytestmark = pytest.mark.gpu

SPECS = [{"N": (64, 32), "M": 3000}, {"N": (16, 128), "M": 777}, {"N": (32, 32), "M": 12000},
         {"N": (128, 64), "M": 5001}, {"N": (8, 8), "M": 50}, {"N": (96, 48), "M": 20000}]


def _inputs(specs, dtype, salt):
    npdt = np.float32 if dtype == torch.float32 else np.float64
    xs = [W.round_nodes(W.uniform_nodes(s["M"], 2, seed_offset=salt + i), npdt)
          for i, s in enumerate(specs)]
    fhs = [W.gaussian_fhat(s["N"], seed_offset=salt + 100 + i) for i, s in enumerate(specs)]
    fs = [W.gaussian_values(s["M"], seed_offset=salt + 200 + i) for i, s in enumerate(specs)]
    return xs, fhs, fs


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_batch_matches_oracle_and_graph_replay(dtype):
    b = PlanBatch(SPECS, dtype=dtype, device=DEV)
    xs, fhs, fs = _inputs(SPECS, dtype, 800)
    b.set_nodes([to_dev(x, dtype) for x in xs])
    fh_t = [to_dev(v, dtype) for v in fhs]
    f_t = [to_dev(v, dtype) for v in fs]
    outs_f = [o.cpu().numpy() for o in b.trafo(fh_t)]
    outs_h = [o.cpu().numpy() for o in b.adjoint(f_t)]
    for i, s in enumerate(SPECS):
        n = b.plans[i].n
        xr, fhr, fr = rounded(xs[i], dtype), rounded(fhs[i], dtype), rounded(fs[i], dtype)
        assert rel_l2(outs_f[i], oracle.nfft(xr, fhr, n=n, m=4)) <= TOL[dtype]
        assert rel_l2(outs_h[i], oracle.nfft_adjoint(xr, fr, s["N"], n=n, m=4)) <= TOL[dtype]
    # one graph for the whole batch; same results on replay
    b.capture(fh_t, f_t)
    gf, gh = b.replay()
    torch.cuda.synchronize()
    tol = 1e-13 if dtype == torch.float64 else 1e-6
    for i in range(len(SPECS)):
        assert rel_l2(gf[i].cpu().numpy(), outs_f[i]) <= tol
        assert rel_l2(gh[i].cpu().numpy(), outs_h[i]) <= tol
    # new inputs copied into the captured buffers
    _, fhs2, fs2 = _inputs(SPECS, dtype, 900)
    for i in range(len(SPECS)):
        b.in_fhat[i].copy_(to_dev(fhs2[i], dtype))
        b.in_f[i].copy_(to_dev(fs2[i], dtype))
    gf, gh = b.replay()
    torch.cuda.synchronize()
    for i, s in enumerate(SPECS):
        n = b.plans[i].n
        xr = rounded(xs[i], dtype)
        assert rel_l2(gf[i].cpu().numpy(),
                      oracle.nfft(xr, rounded(fhs2[i], dtype), n=n, m=4)) <= TOL[dtype]
        assert rel_l2(gh[i].cpu().numpy(), oracle.nfft_adjoint(
            xr, rounded(fs2[i], dtype), s["N"], n=n, m=4)) <= TOL[dtype]


@pytest.mark.parametrize("d", [1, 2, 3])
def test_autotune_keeps_the_transform(d, tmp_path):
    N = {1: (200,), 2: (64, 48), 3: (16, 16, 16)}[d]
    M = 30000
    x = W.uniform_nodes(M, d, seed_offset=810)
    fh = W.gaussian_fhat(N, 811)
    f = W.gaussian_values(M, 812)
    plan = Plan(N, M, m=4, dtype=torch.float64, device=DEV)
    xt, fht, ft = to_dev(x, torch.float64), to_dev(fh, torch.float64), to_dev(f, torch.float64)
    choice = autotune(plan, xt, fht, ft, steps=2)
    assert choice["ms"] > 0 and len(choice["tried"]) >= 2
    assert len(choice["tried_interp"]) >= 2  # the interpolation forms were timed too
    assert choice["interp_method"] in [t[0] for t in choice["tried_interp"]]
    assert tuple(plan.bin) == tuple(choice["bins"])
    assert rel_l2(plan.trafo(fht).cpu().numpy(), oracle.nfft(x, fh, n=plan.n, m=4)) <= 1e-12
    assert rel_l2(plan.adjoint(ft).cpu().numpy(),
                  oracle.nfft_adjoint(x, f, N, n=plan.n, m=4)) <= 1e-12
    cache = TuningCache(str(tmp_path / "tune.json"))
    cache.put(plan, choice)
    back = TuningCache(str(tmp_path / "tune.json")).get(plan)
    assert back["bins"] == list(choice["bins"])
    assert back["interp_method"] == choice["interp_method"]


def test_batched_workload_specs():
    specs = batched_specs()
    assert len(specs) == 64
    assert all(s["N"][t] in (64, 128, 256, 512) for s in specs for t in range(2))
    assert all(10 ** 4 <= s["M"] <= 10 ** 6 for s in specs)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_batch_backward_matches_oracle_and_graph_replay(dtype):
    """Backward of the batched forward transform: grad fhat_i = A_i^H g_i and grad x_i from the
    node-gradient kernel, per problem against the oracle, eagerly and captured in the graph
    together with the forward and adjoint."""
    b = PlanBatch(SPECS, dtype=dtype, device=DEV)
    xs, fhs, fs = _inputs(SPECS, dtype, 1000)
    _, _, gs = _inputs(SPECS, dtype, 1300)
    b.set_nodes([to_dev(x, dtype) for x in xs])
    fh_t = [to_dev(v, dtype) for v in fhs]
    f_t = [to_dev(v, dtype) for v in fs]
    g_t = [to_dev(v, dtype) for v in gs]
    g_fhat, g_x = b.backward(g_t, fh_t)
    g_fhat = [t.cpu().numpy() for t in g_fhat]
    g_x = [t.cpu().numpy() for t in g_x]
    tol_x = 1e-11 if dtype == torch.float64 else 1e-5
    for i, s in enumerate(SPECS):
        n = b.plans[i].n
        xr, fhr, gr = rounded(xs[i], dtype), rounded(fhs[i], dtype), rounded(gs[i], dtype)
        assert rel_l2(g_fhat[i], oracle.nfft_adjoint(xr, gr, s["N"], n=n, m=4)) <= TOL[dtype]
        assert rel_l2(g_x[i], oracle.nfft_grad_x(xr, fhr, gr, n=n, m=4)) <= tol_x
    b.capture(fh_t, f_t, grad_fs=g_t)
    b.replay()
    torch.cuda.synchronize()
    tol = 1e-13 if dtype == torch.float64 else 1e-6
    for i in range(len(SPECS)):
        assert rel_l2(b.out_grad_fhat[i].cpu().numpy(), g_fhat[i]) <= tol
        assert rel_l2(b.out_grad_x[i].cpu().numpy(), g_x[i]) <= tol


def test_batch_autograd_equals_per_plan_autograd():
    """batch_nfft through torch.autograd: the gradients of a loss over every problem equal
    those of the single-plan autograd function, problem by problem (FP64)."""
    from paper_1810_09891_gb300.batch import batch_nfft
    from paper_1810_09891_gb300.nfft import nfft

    dtype = torch.float64
    b = PlanBatch(SPECS, dtype=dtype, device=DEV)
    xs, fhs, _ = _inputs(SPECS, dtype, 1100)
    _, _, ws = _inputs(SPECS, dtype, 1200)
    xt = [to_dev(x, dtype).requires_grad_() for x in xs]
    fht = [to_dev(v, dtype).requires_grad_() for v in fhs]
    wt = [to_dev(v, dtype) for v in ws]
    outs = batch_nfft(fht, xt, b)
    loss = sum((torch.conj(w) * o).real.sum() for w, o in zip(wt, outs))
    loss.backward()
    for i, s in enumerate(SPECS):
        x1 = to_dev(xs[i], dtype).requires_grad_()
        f1 = to_dev(fhs[i], dtype).requires_grad_()
        plan = Plan(s["N"], s["M"], m=4, dtype=dtype, device=DEV)
        (torch.conj(wt[i]) * nfft(f1, x1, plan)).real.sum().backward()
        assert rel_l2(outs[i].detach().cpu().numpy(),
                      nfft(f1.detach(), x1.detach(), plan).cpu().numpy()) <= 1e-14
        assert rel_l2(fht[i].grad.cpu().numpy(), f1.grad.cpu().numpy()) <= 1e-14
        assert rel_l2(xt[i].grad.cpu().numpy(), x1.grad.cpu().numpy()) <= 1e-14
        plan.close()


def test_batch_autograd_only_fhat():
    """Nodes without requires_grad: only the adjoint runs in the backward, grad fhat_i equals
    the oracle adjoint of the output gradient."""
    from paper_1810_09891_gb300.batch import batch_nfft

    dtype = torch.float64
    specs = SPECS[:3]
    b = PlanBatch(specs, dtype=dtype, device=DEV)
    xs, fhs, _ = _inputs(specs, dtype, 1400)
    fht = [to_dev(v, dtype).requires_grad_() for v in fhs]
    outs = batch_nfft(fht, [to_dev(x, dtype) for x in xs], b)
    sum(o.abs().square().sum() for o in outs).backward()
    for i, s in enumerate(specs):
        f = oracle.nfft(xs[i], fhs[i], n=b.plans[i].n, m=4)
        ref = 2 * oracle.nfft_adjoint(xs[i], f, s["N"], n=b.plans[i].n, m=4)
        assert rel_l2(fht[i].grad.cpu().numpy(), ref) <= 1e-12


def _lib_batch(plans, streams=0):
    import ctypes

    from paper_1810_09891_gb300 import _lib
    L = _lib.lib()
    arr = (ctypes.c_void_p * len(plans))(*[p._h.value for p in plans])
    b = ctypes.c_void_p()
    assert L.nfft_batch_create(ctypes.byref(b), ctypes.cast(arr, ctypes.c_void_p), len(plans),
                               streams) == 0
    return L, b


def _ptr_array(ts):
    import ctypes
    return ctypes.cast((ctypes.c_void_p * len(ts))(*[t.data_ptr() for t in ts]), ctypes.c_void_p)


def test_library_batch_mixed_dimensions_and_precisions():
    """The C-ABI batch over plans of different d and precision: every forward, adjoint and node
    gradient equals the oracle's, and the lanes balance the work."""
    import ctypes
    cases = [((40,), 900, torch.float64), ((32, 24), 3000, torch.float32),
             ((8, 12, 10), 2500, torch.float32), ((8, 8, 8), 1200, torch.float64),
             ((64, 64), 20000, torch.float32)]
    plans, xs, fhs, fs = [], [], [], []
    for i, (N, M, dt) in enumerate(cases):
        p = Plan(N, M, m=4, dtype=dt, device=DEV)
        x = W.round_nodes(W.uniform_nodes(M, len(N), seed_offset=1500 + i),
                          np.float32 if dt == torch.float32 else np.float64)
        p.set_nodes(to_dev(x, dt))
        plans.append(p)
        xs.append(x)
        fhs.append(W.gaussian_fhat(N, 1510 + i))
        fs.append(W.gaussian_values(M, 1520 + i))
    L, b = _lib_batch(plans, streams=3)
    cnt, ns = ctypes.c_int(), ctypes.c_int()
    assert L.nfft_batch_size(b, ctypes.byref(cnt), ctypes.byref(ns)) == 0
    assert (cnt.value, ns.value) == (len(cases), 3)
    lanes = [L.nfft_batch_lane(b, i) for i in range(len(cases))]
    assert all(0 <= v < 3 for v in lanes) and L.nfft_batch_lane(b, len(cases)) == -1
    work = [p.M + int(np.prod(p.n)) for p in plans]
    load = [sum(w for w, v in zip(work, lanes) if v == j) for j in range(3)]
    assert max(load) - min(load) <= max(work)
    stream = torch.cuda.current_stream(DEV)
    assert L.nfft_batch_set_stream(b, ctypes.c_void_p(stream.cuda_stream)) == 0
    fht = [to_dev(v, p.dtype) for v, p in zip(fhs, plans)]
    ft = [to_dev(v, p.dtype) for v, p in zip(fs, plans)]
    out_f = [torch.empty(p.M, dtype=p.cdtype, device=DEV) for p in plans]
    out_h = [torch.empty(p.N, dtype=p.cdtype, device=DEV) for p in plans]
    out_g = [torch.empty((p.M, p.d), dtype=p.dtype, device=DEV) for p in plans]
    assert L.nfft_batch_trafo(b, _ptr_array(fht), _ptr_array(out_f)) == 0
    assert L.nfft_batch_adjoint(b, _ptr_array(ft), _ptr_array(out_h)) == 0
    assert L.nfft_batch_grad_x(b, _ptr_array(fht), _ptr_array(ft), _ptr_array(out_g)) == 0
    torch.cuda.synchronize()
    for i, (N, M, dt) in enumerate(cases):
        n = plans[i].n
        xr, fhr, fr = rounded(xs[i], dt), rounded(fhs[i], dt), rounded(fs[i], dt)
        assert rel_l2(out_f[i].cpu().numpy(), oracle.nfft(xr, fhr, n=n, m=4)) <= TOL[dt]
        assert rel_l2(out_h[i].cpu().numpy(), oracle.nfft_adjoint(xr, fr, N, n=n, m=4)) <= TOL[dt]
        tol_x = 1e-11 if dt == torch.float64 else 1e-5
        assert rel_l2(out_g[i].cpu().numpy(), oracle.nfft_grad_x(xr, fhr, fr, n=n, m=4)) <= tol_x
    assert L.nfft_batch_destroy(b) == 0


def test_library_batch_checks_every_plan_before_enqueuing():
    """A plan without nodes or a null pointer in the arrays fails the whole call with nothing
    enqueued: the outputs of the other plans keep their previous contents."""
    import ctypes
    specs = [((32, 32), 2000), ((16, 48), 1000), ((24, 24), 500)]
    plans = [Plan(N, M, m=4, dtype=torch.float64, device=DEV) for N, M in specs]
    for i, p in enumerate(plans[:2]):
        p.set_nodes(to_dev(W.uniform_nodes(p.M, 2, seed_offset=1530 + i), torch.float64))
    L, b = _lib_batch(plans)
    stream = torch.cuda.current_stream(DEV)
    assert L.nfft_batch_set_stream(b, ctypes.c_void_p(stream.cuda_stream)) == 0
    fht = [to_dev(W.gaussian_fhat(p.N, 1540), torch.float64) for p in plans]
    outs = [torch.full((p.M,), 7.0 + 0j, dtype=p.cdtype, device=DEV) for p in plans]
    assert L.nfft_batch_trafo(b, _ptr_array(fht), _ptr_array(outs)) == 4  # NFFT_ENOTREADY
    plans[2].set_nodes(to_dev(W.uniform_nodes(plans[2].M, 2, seed_offset=1532), torch.float64))
    bad = ctypes.cast((ctypes.c_void_p * 3)(outs[0].data_ptr(), None, outs[2].data_ptr()),
                      ctypes.c_void_p)
    assert L.nfft_batch_trafo(b, _ptr_array(fht), bad) == 1  # NFFT_EINVAL
    torch.cuda.synchronize()
    for o in outs:
        assert bool((o == 7.0).all())
    assert L.nfft_batch_trafo(b, _ptr_array(fht), _ptr_array(outs)) == 0
    torch.cuda.synchronize()
    for p, fh, o in zip(plans, fht, outs):
        assert rel_l2(o.cpu().numpy(), p.trafo(fh).cpu().numpy()) <= 1e-14
        assert p.status() == 0
    assert L.nfft_batch_destroy(b) == 0


# ------------------------------------------------------------------ fused execution

def _check_batch(b, xs, fhs, fs, gs, dtype=torch.float32, tol_x=1e-5):
    fh_t = [to_dev(v, dtype) for v in fhs]
    f_t = [to_dev(v, dtype) for v in fs]
    g_t = [to_dev(v, dtype) for v in gs]
    outs_f = [o.cpu().numpy() for o in b.trafo(fh_t)]
    outs_h = [o.cpu().numpy() for o in b.adjoint(f_t)]
    _, g_x = b.backward(g_t, fh_t, want_fhat=False)
    g_x = [t.cpu().numpy() for t in g_x]
    for i, p in enumerate(b.plans):
        xr, fhr, fr, gr = (rounded(xs[i], dtype), rounded(fhs[i], dtype), rounded(fs[i], dtype),
                           rounded(gs[i], dtype))
        assert rel_l2(outs_f[i], oracle.nfft(xr, fhr, n=p.n, m=p.m)) <= TOL[dtype], i
        assert rel_l2(outs_h[i], oracle.nfft_adjoint(xr, fr, p.N, n=p.n, m=p.m)) <= TOL[dtype], i
        if p.M:
            assert rel_l2(g_x[i], oracle.nfft_grad_x(xr, fhr, gr, n=p.n, m=p.m)) <= tol_x, i
    return outs_f, outs_h, g_x


def test_fused_batch_matches_oracle_and_plan_by_plan():
    """2-D FP32 plans with one m run fused (one launch per stage over all plans): forward,
    adjoint and node gradient of every plan against the oracle, and against the same batch run
    plan by plan on side streams."""
    specs = SPECS + [{"N": (256, 16), "M": 0}, {"N": (2048, 32), "M": 4000}]
    b = PlanBatch(specs, dtype=torch.float32, device=DEV)
    assert b.fused
    xs, fhs, fs = _inputs(specs, torch.float32, 1500)
    _, _, gs = _inputs(specs, torch.float32, 1600)
    b.set_nodes([to_dev(x, torch.float32) for x in xs])
    ff, fh, fx = _check_batch(b, xs, fhs, fs, gs)
    b.set_fused(False)
    assert not b.fused
    sf, sh, sx = _check_batch(b, xs, fhs, fs, gs)
    for i in range(len(specs)):
        assert rel_l2(ff[i], sf[i]) <= 1e-6
        assert rel_l2(fh[i], sh[i]) <= 1e-6
        if specs[i]["M"]:
            assert rel_l2(fx[i], sx[i]) <= 1e-6
    b.set_fused(True)
    assert b.fused
    b.close()


def test_fused_batch_follows_plan_changes_and_graph_replay():
    """A plan retuned after the fused tables were built (new bins, nodes set again) is picked
    up by the next call; a captured graph of the fused batch replays with new inputs."""
    b = PlanBatch(SPECS, dtype=torch.float32, device=DEV)
    xs, fhs, fs = _inputs(SPECS, torch.float32, 1700)
    _, _, gs = _inputs(SPECS, torch.float32, 1750)
    b.set_nodes([to_dev(x, torch.float32) for x in xs])
    _check_batch(b, xs, fhs, fs, gs)
    b.plans[3].set_option("bin0", 16)
    b.plans[3].set_option("bin1", 32)
    b.set_nodes([to_dev(x, torch.float32) for x in xs])
    assert b.fused
    _check_batch(b, xs, fhs, fs, gs)
    fh_t = [to_dev(v, torch.float32) for v in fhs]
    f_t = [to_dev(v, torch.float32) for v in fs]
    b.capture(fh_t, f_t)
    _, fhs2, fs2 = _inputs(SPECS, torch.float32, 1800)
    for i in range(len(SPECS)):
        b.in_fhat[i].copy_(to_dev(fhs2[i], torch.float32))
        b.in_f[i].copy_(to_dev(fs2[i], torch.float32))
    gf, gh = b.replay()
    torch.cuda.synchronize()
    for i, p in enumerate(b.plans):
        xr = rounded(xs[i], torch.float32)
        assert rel_l2(gf[i].cpu().numpy(), oracle.nfft(
            xr, rounded(fhs2[i], torch.float32), n=p.n, m=4)) <= TOL[torch.float32]
        assert rel_l2(gh[i].cpu().numpy(), oracle.nfft_adjoint(
            xr, rounded(fs2[i], torch.float32), p.N, n=p.n, m=4)) <= TOL[torch.float32]
    b.close()


def test_batches_that_do_not_qualify_run_plan_by_plan():
    from paper_1810_09891_gb300._lib import NfftError
    mixed = [dict(SPECS[0]), dict(SPECS[1], m=3)]  # two window cutoffs
    b = PlanBatch(mixed, dtype=torch.float32, device=DEV)
    assert not b.fused
    with pytest.raises(NfftError, match="NFFT_EUNSUPPORTED"):
        b.set_fused(True)
    xs, fhs, fs = _inputs(mixed, torch.float32, 1900)
    _, _, gs = _inputs(mixed, torch.float32, 1950)
    b.set_nodes([to_dev(x, torch.float32) for x in xs])
    _check_batch(b, xs, fhs, fs, gs)
    b.close()
    b64 = PlanBatch(SPECS, dtype=torch.float64, device=DEV)
    assert not b64.fused  # FP64 batches run plan by plan
    b64.close()
    odd = PlanBatch([{"N": (60, 60), "M": 100, "n": (130, 128)}], dtype=torch.float32,
                    device=DEV)
    assert not odd.fused  # a length that is not a power of two
    odd.close()
    spread = PlanBatch(SPECS[:2], dtype=torch.float32, device=DEV)
    spread.plans[0].set_option("spread_method", "octet")
    assert not spread.fused  # the fused spreading is the half-warp form
    spread.close()


def test_fused_batched_workload_full_size():
    """The 64-problem batched workload (N_i per axis in {64, ..., 512}, M_i up to 1e6), fused:
    the forward on 2048 sampled nodes and the adjoint of every coefficient against the oracle
    for the largest problem and three others."""
    specs = batched_specs()
    b = PlanBatch(specs, dtype=torch.float32, device=DEV)
    assert b.fused
    xs = [W.round_nodes(W.uniform_nodes(s["M"], 2, seed_offset=1000 + i), np.float32)
          for i, s in enumerate(specs)]
    fhs = [W.gaussian_fhat(s["N"], 2000 + i) for i, s in enumerate(specs)]
    fs = [W.gaussian_values(s["M"], 3000 + i) for i, s in enumerate(specs)]
    b.set_nodes([to_dev(x, torch.float32) for x in xs])
    yf = b.trafo([to_dev(v, torch.float32) for v in fhs])
    yh = b.adjoint([to_dev(v, torch.float32) for v in fs])
    torch.cuda.synchronize()
    big = int(np.argmax([s["M"] for s in specs]))
    for i in (big, 0, 17, 63):
        p = b.plans[i]
        xr, fhr, fr = (rounded(xs[i], torch.float32), rounded(fhs[i], torch.float32),
                       rounded(fs[i], torch.float32))
        idx = np.sort(np.random.default_rng(i).choice(p.M, min(2048, p.M), replace=False))
        assert rel_l2(yf[i].cpu().numpy()[idx], oracle.nfft(xr[idx], fhr, n=p.n, m=4)) <= \
            TOL[torch.float32], i
        assert rel_l2(yh[i].cpu().numpy(), oracle.nfft_adjoint(xr, fr, p.N, n=p.n, m=4)) <= \
            TOL[torch.float32], i
    b.close()
