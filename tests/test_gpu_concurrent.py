"""A forward and an adjoint of the same plan running at the same time on two streams (the plan
keeps separate grids for the two), checked against the FP64 oracle: single plans of every d,
and batches (fused and plan by plan) captured in a CUDA graph with the two transforms on two
streams, replayed with new inputs; and calls whose inputs are copied on another stream just
before them."""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import DEV, TOL, rel_l2, rounded, to_dev
from paper_1810_09891_gb300 import workloads as W
from paper_1810_09891_gb300.batch import PlanBatch
from paper_1810_09891_gb300.nfft import Plan

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("N", [(96,), (64, 48), (16, 24, 16)])
def test_forward_and_adjoint_on_two_streams(N, dtype):
    torch.cuda.set_device(DEV)
    M = 20000 if len(N) < 3 else 6000
    npdt = np.float32 if dtype == torch.float32 else np.float64
    x = W.round_nodes(W.uniform_nodes(M, len(N), seed_offset=960 + len(N)), npdt)
    plan = Plan(N, M, m=4, dtype=dtype, device=DEV)
    plan.set_nodes(to_dev(x, dtype))
    xr = rounded(x, dtype)
    sf, sa = torch.cuda.Stream(DEV), torch.cuda.Stream(DEV)
    cur = torch.cuda.current_stream(DEV)
    for k in range(3):
        fh = W.gaussian_fhat(N, 970 + k)
        f = W.gaussian_values(M, 980 + k)
        fh_d, f_d = to_dev(fh, dtype), to_dev(f, dtype)
        sf.wait_stream(cur)
        sa.wait_stream(cur)
        with torch.cuda.stream(sf):
            y = plan.trafo(fh_d)
        with torch.cuda.stream(sa):
            h = plan.adjoint(f_d)
        cur.wait_stream(sf)
        cur.wait_stream(sa)
        torch.cuda.synchronize()
        assert rel_l2(y.cpu().numpy(), oracle.nfft(xr, rounded(fh, dtype), n=plan.n, m=4)) \
            <= TOL[dtype]
        assert rel_l2(h.cpu().numpy(), oracle.nfft_adjoint(xr, rounded(f, dtype), N, n=plan.n,
                                                           m=4)) <= TOL[dtype]
    assert plan.status() == 0
    plan.close()


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_inputs_copied_on_a_copy_stream_just_before_each_call(dtype):
    """Each step's inputs arrive by copies from pinned host memory on a copy stream, into one of
    two device buffers, and the compute stream waits for them by an event just before the
    calls (the pipelined host-buffer pattern). Every result matches the oracle of its own step's
    inputs: no kernel of a call (the FFT passes start as programmatic dependents of the previous
    kernel) reads its input before the copies it waits for have landed."""
    torch.cuda.set_device(DEV)
    N, M, K, steps = (512, 512), 50000, 4, 24
    npdt = np.float32 if dtype == torch.float32 else np.float64
    cnp = np.complex64 if dtype == torch.float32 else np.complex128
    cdt = torch.complex64 if dtype == torch.float32 else torch.complex128
    x = W.round_nodes(W.uniform_nodes(M, 2, seed_offset=1100), npdt)
    plan = Plan(N, M, m=4, dtype=dtype, device=DEV)
    plan.set_nodes(to_dev(x, dtype))
    xr = rounded(x, dtype)
    fhs = [W.gaussian_fhat(N, 1110 + k) for k in range(K)]
    fs = [W.gaussian_values(M, 1120 + k) for k in range(K)]
    pin_fh = [torch.tensor(a.astype(cnp)).pin_memory() for a in fhs]
    pin_f = [torch.tensor(a.astype(cnp)).pin_memory() for a in fs]
    comp = torch.cuda.current_stream(DEV)
    cin = torch.cuda.Stream(DEV)
    d_fh = [torch.empty(N, dtype=cdt, device=DEV) for _ in range(2)]
    d_f = [torch.empty(M, dtype=cdt, device=DEV) for _ in range(2)]
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_free = [torch.cuda.Event() for _ in range(2)]
    for e in ev_free:
        e.record(comp)
    ys, hs, which = [], [], []
    for s in range(steps):
        j, k = s & 1, (s * 3) % K  # buffer j, input set k (consecutive steps differ)
        with torch.cuda.stream(cin):
            cin.wait_event(ev_free[j])
            d_fh[j].copy_(pin_fh[k], non_blocking=True)
            d_f[j].copy_(pin_f[k], non_blocking=True)
            ev_in[j].record(cin)
        comp.wait_event(ev_in[j])
        ys.append(plan.trafo(d_fh[j]))
        hs.append(plan.adjoint(d_f[j]))
        ev_free[j].record(comp)
        which.append(k)
    torch.cuda.synchronize()
    ref_y = [oracle.nfft(xr, rounded(fhs[k], dtype), n=plan.n, m=4) for k in range(K)]
    ref_h = [oracle.nfft_adjoint(xr, rounded(fs[k], dtype), N, n=plan.n, m=4) for k in range(K)]
    for y, h, k in zip(ys, hs, which):
        assert rel_l2(y.cpu().numpy(), ref_y[k]) <= TOL[dtype]
        assert rel_l2(h.cpu().numpy(), ref_h[k]) <= TOL[dtype]
    assert plan.status() == 0
    plan.close()


@pytest.mark.parametrize("fused", [True, False])
def test_batch_graph_with_concurrent_forward_and_adjoint(fused):
    torch.cuda.set_device(DEV)
    specs = [{"N": (64, 32), "M": 5000}, {"N": (128, 64), "M": 20000},
             {"N": (32, 32), "M": 300}]
    dtype = torch.float32
    b = PlanBatch(specs, dtype=dtype, device=DEV)
    if not fused:
        b.set_fused(False)
    xs = [W.round_nodes(W.uniform_nodes(s["M"], 2, seed_offset=990 + i), np.float32)
          for i, s in enumerate(specs)]
    b.set_nodes([to_dev(x, dtype) for x in xs])
    assert b.fused == fused
    fhs = [to_dev(W.gaussian_fhat(s["N"], 1000 + i), dtype) for i, s in enumerate(specs)]
    fs = [to_dev(W.gaussian_values(s["M"], 1010 + i), dtype) for i, s in enumerate(specs)]
    b.capture(fhs, fs, concurrent=True)
    for k in range(2):
        new_fh = [W.gaussian_fhat(s["N"], 1020 + 10 * k + i) for i, s in enumerate(specs)]
        new_f = [W.gaussian_values(s["M"], 1040 + 10 * k + i) for i, s in enumerate(specs)]
        for i in range(len(specs)):
            fhs[i].copy_(to_dev(new_fh[i], dtype))
            fs[i].copy_(to_dev(new_f[i], dtype))
        yf, yh = b.replay()
        torch.cuda.synchronize()
        for i, s in enumerate(specs):
            xr = rounded(xs[i], dtype)
            n = b.plans[i].n
            assert rel_l2(yf[i].cpu().numpy(),
                          oracle.nfft(xr, rounded(new_fh[i], dtype), n=n, m=4)) <= TOL[dtype]
            assert rel_l2(yh[i].cpu().numpy(),
                          oracle.nfft_adjoint(xr, rounded(new_f[i], dtype), s["N"], n=n, m=4)) \
                <= TOL[dtype]
    b.close()
