"""The stripe form of the adjoint's spreading step (d = 2): one shared tile per CTA over a
super-bin of 16 stripes of whole sort bins, each at least 2m cells wide; half-warps add the even
stripes together, then the odd ones. Checked against the FP64 oracle adjoint NFFT element by
element over every window cutoff, both precisions, both window evaluations, sort-bin shapes that
make a stripe of one or several bins, work items from 8 nodes per stripe (heavy super-bins cut into
many parts) to one item per super-bin, a last super-bin that is only partly inside the grid, and nodes
on grid points, coincident and clustered."""
import numpy as np
import pytest
import torch

import oracle
from paper_1810_09891_gb300 import workloads as W
from paper_1810_09891_gb300.nfft import Plan

from gpu_helpers import DEV, TOL, rel_l2, rounded, to_dev

pytestmark = pytest.mark.gpu


def stripe_width(m):
    return 2 if 2 * m <= 2 else 4 if 2 * m <= 4 else 8 if 2 * m <= 8 else 16


def nodes(M, seed, n):
    """Uniform nodes, one cluster, nodes on grid points (some coincident) and nodes at -1/2."""
    x = W.uniform_nodes(M, 2, seed_offset=seed)
    g = np.random.default_rng(seed)
    k = M // 5
    x[:k] = W.wrap(g.normal(0.1, 0.02, size=(k, 2)))
    q = M // 10
    x[k:k + q, 0] = np.round(x[k:k + q, 0] * n[0]) / n[0]
    x[k:k + q, 1] = np.round(x[k:k + q, 1] * n[1]) / n[1]
    x[k + q:k + q + 20] = 0.0
    x[k + q + 20:k + q + 30] = -0.5
    return x


def run_adjoint(N, n, m, x, f, dtype, opts, window_table=0):
    plan = Plan(N, x.shape[0], n=n, m=m, dtype=dtype, device=DEV)
    plan.set_option("spread_method", "stripe")
    for k, v in opts.items():
        plan.set_option(k, v)
    if window_table:
        plan.set_option("window_table", window_table)
    plan.set_nodes(to_dev(x, dtype))
    h1 = plan.adjoint(to_dev(f, dtype)).cpu().numpy()
    h2 = plan.adjoint(to_dev(f, dtype)).cpu().numpy()  # the tile is clean again after a launch
    st = plan.status()
    plan.close()
    assert st == 0
    return h1, h2


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("m", [1, 2, 3, 4, 5, 6, 7, 8])
def test_every_window_cutoff(m, dtype):
    w = stripe_width(m)
    n = (64, 16 * w + 2 * m + 2 * w)  # wide enough for a super-bin, with a partial last one
    N = (40, 2 * (n[1] // 4))
    x = W.round_nodes(nodes(4000, 800 + m, n), np.float32 if dtype == torch.float32
                      else np.float64)
    f = W.gaussian_values(x.shape[0], 801 + m)
    h1, h2 = run_adjoint(N, n, m, x, f, dtype, {"bin1": min(w, 8), "stripe_item": 256})
    ref = oracle.nfft_adjoint(rounded(x, dtype), rounded(f, dtype), N, n=n, m=m)
    tol = TOL[dtype] if (dtype == torch.float64 or m <= 6) else 3e-5
    assert rel_l2(h1, ref) <= tol
    assert np.array_equal(h1, h2) or rel_l2(h2, ref) <= tol


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("bins,item", [((8, 8), 64), ((1, 8), 8), ((4, 4), 128),
                                       ((16, 2), 4096), ((32, 1), 65536), ((2, 8), 16)])
def test_bins_and_items(bins, item, dtype):
    N, n, m = (96, 160), (256, 320), 4  # n_1 = 320: three super-bins, the last one partial
    x = W.round_nodes(nodes(30000, 810, n), np.float32 if dtype == torch.float32 else np.float64)
    f = W.gaussian_values(x.shape[0], 811)
    h1, _ = run_adjoint(N, n, m, x, f, dtype, {"bin0": bins[0], "bin1": bins[1],
                                               "stripe_item": item})
    ref = oracle.nfft_adjoint(rounded(x, dtype), rounded(f, dtype), N, n=n, m=m)
    assert rel_l2(h1, ref) <= TOL[dtype]


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_lookup_table_window(dtype):
    N, n, m, K = (48, 100), (96, 256), 4, 4096
    x = W.round_nodes(nodes(8000, 820, n), np.float32 if dtype == torch.float32 else np.float64)
    f = W.gaussian_values(x.shape[0], 821)
    h1, _ = run_adjoint(N, n, m, x, f, dtype, {}, window_table=K)
    ref = oracle.nfft_adjoint(rounded(x, dtype), rounded(f, dtype), N, n=n, m=m, lin_psi=K)
    assert rel_l2(h1, ref) <= TOL[dtype]


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_radial_reduced_every_window(dtype):
    """Golden-angle radial nodes (every spoke through the origin, a grid point) with each window
    of the library."""
    N, n, m = (128, 128), (256, 256), 4
    x = W.round_nodes(W.radial_nodes(64, 512), np.float32 if dtype == torch.float32
                      else np.float64)
    f = W.gaussian_values(x.shape[0], 830)
    for window in ("kaiser_bessel", "gaussian", "bspline", "sinc"):
        plan = Plan(N, x.shape[0], n=n, m=m, dtype=dtype, device=DEV, window=window)
        plan.set_option("spread_method", "stripe")
        plan.set_nodes(to_dev(x, dtype))
        h = plan.adjoint(to_dev(f, dtype)).cpu().numpy()
        assert plan.status() == 0
        plan.close()
        ref = oracle.nfft_adjoint(rounded(x, dtype), rounded(f, dtype), N, n=n, m=m,
                                  window=window)
        assert rel_l2(h, ref) <= TOL[dtype], window


def test_non_power_of_two_grid():
    """n_1 = 300 (Bluestein FFT): sort bins of an axis that is not a power of two end in a
    partial bin, and the last super-bin lies partly outside the grid."""
    N, n, m = (64, 120), (128, 300), 4
    x = W.round_nodes(nodes(12000, 840, n), np.float32)
    f = W.gaussian_values(x.shape[0], 841)
    h1, _ = run_adjoint(N, n, m, x, f, torch.float32, {"stripe_item": 512})
    ref = oracle.nfft_adjoint(rounded(x, torch.float32), rounded(f, torch.float32), N, n=n, m=m)
    assert rel_l2(h1, ref) <= TOL[torch.float32]


def test_falls_back_where_stripes_do_not_fit():
    """A grid narrower than one super-bin (n_1 < 16 stripes + 2m) or a sort bin wider than a
    stripe runs the half-warp form: same result."""
    N, m = (24, 40), 4
    for n, bins in (((64, 96), (8, 8)), ((64, 256), (8, 16))):
        x = W.round_nodes(nodes(3000, 850, n), np.float32)
        f = W.gaussian_values(x.shape[0], 851)
        h1, _ = run_adjoint(N, n, m, x, f, torch.float32, {"bin0": bins[0], "bin1": bins[1]})
        ref = oracle.nfft_adjoint(rounded(x, torch.float32), rounded(f, torch.float32), N, n=n,
                                  m=m)
        assert rel_l2(h1, ref) <= TOL[torch.float32]


def test_item_option_range():
    from paper_1810_09891_gb300._lib import NfftError
    plan = Plan((32, 32), 10, m=4, dtype=torch.float32, device=DEV)
    for bad in (4, 100, 131072, -1):
        with pytest.raises(NfftError, match="NFFT_EINVAL"):
            plan.set_option("stripe_item", bad)
    for good in (0, 8, 64, 65536):
        plan.set_option("stripe_item", good)
    plan.close()
