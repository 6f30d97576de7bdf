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
    assert tuple(plan.bin) == tuple(choice["bins"])
    assert rel_l2(plan.trafo(fht).cpu().numpy(), oracle.nfft(x, fh, n=plan.n, m=4)) <= 1e-12
    assert rel_l2(plan.adjoint(ft).cpu().numpy(),
                  oracle.nfft_adjoint(x, f, N, n=plan.n, m=4)) <= 1e-12
    cache = TuningCache(str(tmp_path / "tune.json"))
    cache.put(plan, choice)
    assert TuningCache(str(tmp_path / "tune.json")).get(plan)["bins"] == list(choice["bins"])


def test_batched_workload_specs():
    specs = batched_specs()
    assert len(specs) == 64
    assert all(s["N"][t] in (64, 128, 256, 512) for s in specs for t in range(2))
    assert all(10 ** 4 <= s["M"] <= 10 ** 6 for s in specs)
