"""The rows form of the adjoint's spreading step (d = 2): a half-warp (tiles at most 16 cells
wide) or a warp holds a subproblem's whole tile in registers, each lane all rows of one tile
column, the nodes' row weights staged at their tile rows. Checked against the FP64 oracle
adjoint NFFT element by element over every window cutoff, both precisions, both window
evaluations, both bin heights (4 and 8 rows) with half-warp and warp tiles, work items from 32
nodes to 1024, a grid with partial last bins, and nodes on grid points (one axis or both),
coincident and clustered; and the same form inside fused batches, where the two half-warps of
a warp may work on different plans."""
import numpy as np
import pytest
import torch

import oracle
from paper_1810_09891_gb300 import workloads as W
from paper_1810_09891_gb300.batch import PlanBatch
from paper_1810_09891_gb300.nfft import Plan

from gpu_helpers import DEV, TOL, rel_l2, rounded, to_dev

pytestmark = pytest.mark.gpu


def nodes(M, seed, n):
    """Uniform nodes, one cluster, nodes on grid points of one or both axes (some coincident)
    and nodes at -1/2."""
    x = W.uniform_nodes(M, 2, seed_offset=seed)
    g = np.random.default_rng(seed)
    k = M // 5
    x[:k] = W.wrap(g.normal(0.1, 0.02, size=(k, 2)))
    q = M // 10
    x[k:k + q, 0] = np.round(x[k:k + q, 0] * n[0]) / n[0]
    x[k + q:k + 2 * q, 1] = np.round(x[k + q:k + 2 * q, 1] * n[1]) / n[1]
    x[k + 2 * q:k + 2 * q + 20] = 0.0
    x[k + 2 * q + 20:k + 2 * q + 30] = -0.5
    return x


def run_adjoint(N, n, m, x, f, dtype, opts, window_table=0):
    plan = Plan(N, x.shape[0], n=n, m=m, dtype=dtype, device=DEV)
    plan.set_option("spread_method", "rows")
    for k, v in opts.items():
        plan.set_option(k, v)
    if window_table:
        plan.set_option("window_table", window_table)
    plan.set_nodes(to_dev(x, dtype))
    h1 = plan.adjoint(to_dev(f, dtype)).cpu().numpy()
    h2 = plan.adjoint(to_dev(f, dtype)).cpu().numpy()  # the work counters reset after a launch
    st = plan.status()
    plan.close()
    assert st == 0
    return h1, h2


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("m", [1, 2, 3, 4, 5, 6, 7, 8])
def test_every_window_cutoff(m, dtype):
    """Half-warp tiles (last-axis bin + 2m <= 16) where they fit, warp tiles otherwise."""
    N, n = (40, 48), (96, 112)  # 112 / 8 = 14 bins, 112 / 16 = 7 (a partial 2 x 2 block)
    bins = {"bin0": 4, "bin1": 8 if 2 * m <= 8 else 16}
    x = W.round_nodes(nodes(5000, 700 + m, n), np.float32 if dtype == torch.float32
                      else np.float64)
    f = W.gaussian_values(x.shape[0], 701 + m)
    h1, h2 = run_adjoint(N, n, m, x, f, dtype, bins)
    ref = oracle.nfft_adjoint(rounded(x, dtype), rounded(f, dtype), N, n=n, m=m)
    tol = TOL[dtype] if (dtype == torch.float64 or m <= 6) else 3e-5
    assert rel_l2(h1, ref) <= tol
    assert rel_l2(h2, ref) <= tol


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("bins,sub", [((4, 8), 32), ((4, 8), 1024), ((8, 8), 64),
                                      ((8, 16), 128), ((4, 16), 256), ((8, 4), 32),
                                      ((4, 2), 64)])
def test_bins_and_items(bins, sub, dtype):
    """Bin heights 4 and 8, tiles 10 to 24 cells wide (half-warp and warp groups), work items
    of 32 ... 1024 nodes (heavy clustered bins cut into many)."""
    N, n, m = (96, 160), (256, 320), 4
    x = W.round_nodes(nodes(30000, 710, n), np.float32 if dtype == torch.float32 else np.float64)
    f = W.gaussian_values(x.shape[0], 711)
    h1, _ = run_adjoint(N, n, m, x, f, dtype, {"bin0": bins[0], "bin1": bins[1],
                                               "subproblem": sub})
    ref = oracle.nfft_adjoint(rounded(x, dtype), rounded(f, dtype), N, n=n, m=m)
    assert rel_l2(h1, ref) <= TOL[dtype]


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_lookup_table_window(dtype):
    N, n, m, K = (48, 100), (96, 256), 4, 4096
    x = W.round_nodes(nodes(8000, 720, n), np.float32 if dtype == torch.float32 else np.float64)
    f = W.gaussian_values(x.shape[0], 721)
    h1, _ = run_adjoint(N, n, m, x, f, dtype, {"bin0": 4, "bin1": 8}, window_table=K)
    ref = oracle.nfft_adjoint(rounded(x, dtype), rounded(f, dtype), N, n=n, m=m, lin_psi=K)
    assert rel_l2(h1, ref) <= TOL[dtype]


def test_non_power_of_two_grid():
    """n = (90, 300) (Bluestein FFTs): the last bins of both axes are partial."""
    N, n, m = (40, 120), (90, 300), 4
    x = W.round_nodes(nodes(12000, 730, n), np.float32)
    f = W.gaussian_values(x.shape[0], 731)
    h1, _ = run_adjoint(N, n, m, x, f, torch.float32, {})
    ref = oracle.nfft_adjoint(rounded(x, torch.float32), rounded(f, torch.float32), N, n=n, m=m)
    assert rel_l2(h1, ref) <= TOL[torch.float32]


def test_falls_back_where_tiles_do_not_fit():
    """A tile wider than a warp (last-axis bin + 2m > 32) or a bin height other than 4 or 8
    runs the half-warp form: same result."""
    N, n, m = (24, 40), (64, 128), 4
    x = W.round_nodes(nodes(3000, 740, n), np.float32)
    f = W.gaussian_values(x.shape[0], 741)
    ref = oracle.nfft_adjoint(rounded(x, torch.float32), rounded(f, torch.float32), N, n=n, m=m)
    for bins in ((8, 32), (16, 8), (2, 8)):
        h1, _ = run_adjoint(N, n, m, x, f, torch.float32, {"bin0": bins[0], "bin1": bins[1]})
        assert rel_l2(h1, ref) <= TOL[torch.float32]


def test_default_2d_fp32_plan_spreads_in_rows_form():
    plan = Plan((64, 64), 100, m=4, dtype=torch.float32, device=DEV)
    assert tuple(plan.bin) == (4, 8)
    plan.close()
    plan = Plan((64, 64), 100, m=6, dtype=torch.float32, device=DEV)
    assert tuple(plan.bin) == (8, 16)
    plan.close()


@pytest.mark.parametrize("m", [3, 4, 6])
def test_fused_batch_rows_form(m):
    """Fused batches spread in the rows form (default bins: half-warp tiles for m <= 4, warp
    tiles for m = 6); plans of very different sizes, so that the two half-warps of a warp often
    hold entries of different plans."""
    torch.cuda.set_device(DEV)
    specs = [{"N": (64, 32), "M": 300, "m": m}, {"N": (128, 128), "M": 40000, "m": m},
             {"N": (32, 64), "M": 17, "m": m}, {"N": (256, 64), "M": 9000, "m": m},
             {"N": (16, 16), "M": 1, "m": m}]
    dtype = torch.float32
    b = PlanBatch(specs, dtype=dtype, device=DEV)
    xs = [W.round_nodes(nodes(s["M"], 750 + i, tuple(2 * v for v in s["N"])), np.float32)
          if s["M"] >= 20 else W.round_nodes(W.uniform_nodes(s["M"], 2, seed_offset=750 + i),
                                               np.float32) for i, s in enumerate(specs)]
    fs = [W.gaussian_values(s["M"], 760 + i) for i, s in enumerate(specs)]
    b.set_nodes([to_dev(x, dtype) for x in xs])
    assert b.fused
    for _ in range(2):
        hs = b.adjoint([to_dev(f, dtype) for f in fs])
        for i, s in enumerate(specs):
            ref = oracle.nfft_adjoint(rounded(xs[i], dtype), rounded(fs[i], dtype), s["N"],
                                      n=b.plans[i].n, m=m)
            assert rel_l2(hs[i].cpu().numpy(), ref) <= TOL[dtype]
    b.close()
