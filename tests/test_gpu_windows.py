"""GPU parity for the four windows (Kaiser-Bessel, Gaussian, B-spline, sinc; Section 4.1): the
CUDA forward, adjoint and node gradient against the FP64 oracle with the same window, element
by element, in 1-D, 2-D and 3-D with ragged tails, and switching the window of a plan whose
nodes are already set."""
import numpy as np
import pytest
import torch

import oracle
from paper_1810_09891_gb300 import workloads as W
from paper_1810_09891_gb300.nfft import Plan

from gpu_helpers import DEV, TOL, rel_l2, rounded, to_dev

pytestmark = pytest.mark.gpu

WINDOWS = ["kaiser_bessel", "gaussian", "bspline", "sinc"]
CASES = [
    ((200,), (512,), 4, 3001),
    ((64, 48), (128, 128), 4, 5003),
    ((30, 62), (64, 128), 7, 2049),
    ((10, 14, 6), (32, 32, 16), 2, 3333),
    ((16, 16, 16), (32, 32, 32), 5, 4097),
]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("N,n,m,M", CASES)
@pytest.mark.parametrize("window", WINDOWS)
def test_window_parity(window, N, n, m, M, dtype):
    d = len(N)
    x = W.uniform_nodes(M, d, seed_offset=900 + M)
    fh = W.gaussian_fhat(N, seed_offset=901 + M)
    f = W.gaussian_values(M, seed_offset=902 + M)
    plan = Plan(N, M, n=n, m=m, dtype=dtype, device=DEV, window=window)
    assert plan.info()["window"] == window
    plan.set_nodes(to_dev(x, dtype))
    out_f = plan.trafo(to_dev(fh, dtype)).cpu().numpy()
    out_h = plan.adjoint(to_dev(f, dtype)).cpu().numpy()
    assert plan.status() == 0
    xr, fhr, fr = rounded(x, dtype), rounded(fh, dtype), rounded(f, dtype)
    ref_f = oracle.nfft(xr, fhr, n=n, m=m, window=window)
    ref_h = oracle.nfft_adjoint(xr, fr, N, n=n, m=m, window=window)
    assert rel_l2(out_f, ref_f) <= TOL[dtype]
    assert rel_l2(out_h, ref_h) <= TOL[dtype]


@pytest.mark.parametrize("N,m,M", [((64,), 6, 700), ((24, 20), 4, 3000), ((12, 10, 8), 3, 2500)])
@pytest.mark.parametrize("window", WINDOWS)
def test_window_grad_x(window, N, m, M):
    d = len(N)
    x = W.uniform_nodes(M, d, seed_offset=910 + M)
    c = W.gaussian_fhat(N, seed_offset=911)
    w = W.gaussian_values(M, seed_offset=912)
    plan = Plan(N, M, m=m, dtype=torch.float64, device=DEV, window=window)
    plan.set_nodes(to_dev(x, torch.float64))
    gx = plan.grad_x(to_dev(c, torch.float64), to_dev(w, torch.float64)).cpu().numpy()
    ref = oracle.nfft_grad_x(x, c, w, n=plan.n, m=m, window=window)
    assert rel_l2(gx, ref) <= 1e-11


def test_grid_point_nodes_every_window():
    """Nodes on grid points take the extra edge tap psibar(m) (zero for the B-spline)."""
    N, n, m = (32, 16), (64, 32), 4
    g = np.random.default_rng(920)
    x = np.stack([g.integers(-32, 32, 600) / 64.0, g.integers(-16, 16, 600) / 32.0], axis=1)
    fh = W.gaussian_fhat(N, 921)
    f = W.gaussian_values(600, 922)
    for window in WINDOWS:
        plan = Plan(N, 600, n=n, m=m, dtype=torch.float64, device=DEV, window=window)
        plan.set_nodes(to_dev(x, torch.float64))
        out_f = plan.trafo(to_dev(fh, torch.float64)).cpu().numpy()
        out_h = plan.adjoint(to_dev(f, torch.float64)).cpu().numpy()
        assert rel_l2(out_f, oracle.nfft(x, fh, n=n, m=m, window=window)) <= 1e-12
        assert rel_l2(out_h, oracle.nfft_adjoint(x, f, N, n=n, m=m, window=window)) <= 1e-12


def test_switch_window_keeps_nodes():
    """set_option("window") rewrites the tables in place; the node precomputation stays valid."""
    N, n, m, M = (48, 40), (128, 64), 5, 4000
    x = W.uniform_nodes(M, 2, seed_offset=930)
    fh = W.gaussian_fhat(N, 931)
    plan = Plan(N, M, n=n, m=m, dtype=torch.float64, device=DEV)
    plan.set_nodes(to_dev(x, torch.float64))
    fht = to_dev(fh, torch.float64)
    for window in ["gaussian", "sinc", "kaiser_bessel", "bspline"]:
        plan.set_option("window", window)
        assert plan.info()["window"] == window
        out = plan.trafo(fht).cpu().numpy()
        assert rel_l2(out, oracle.nfft(x, fh, n=n, m=m, window=window)) <= 1e-12
    with pytest.raises(Exception):
        plan.set_option("window", "hann")


@pytest.mark.parametrize("window", WINDOWS)
def test_window_error_against_ndft(window):
    """The GPU NFFT with each window reaches the window's own approximation error against the
    exact NDFT (FP64, sigma = 2, m = 6; Kaiser-Bessel is the most accurate, Section 4.1)."""
    N, m, M = (64, 64), 6, 2000
    x = W.uniform_nodes(M, 2, seed_offset=940)
    fh = W.gaussian_fhat(N, 941)
    plan = Plan(N, M, m=m, dtype=torch.float64, device=DEV, window=window)
    plan.set_nodes(to_dev(x, torch.float64))
    out = plan.trafo(to_dev(fh, torch.float64)).cpu().numpy()
    exact = oracle.ndft(x, fh)
    e = oracle.error_Einf(exact, out, fh)
    e_oracle = oracle.error_Einf(exact, oracle.nfft(x, fh, n=plan.n, m=m, window=window), fh)
    assert e <= 1.01 * e_oracle + 1e-15
    assert e <= (3e-12 if window == "kaiser_bessel" else 1e-6)
