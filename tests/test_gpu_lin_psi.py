"""GPU parity of the lookup-table window (PRE_LIN_PSI, NFFT_OPT_WINDOW_TABLE = K) against the
oracle NFFT with the same table: forward, adjoint and node gradient in 1-D, 2-D and 3-D, every
spreading form, every window, nodes on grid points (kinks of the interpolated window), and
switching the table on and off on a plan whose nodes are set."""
import numpy as np
import pytest
import torch

import oracle
from paper_1810_09891_gb300 import workloads as W
from paper_1810_09891_gb300.nfft import Plan

from gpu_helpers import DEV, TOL, rel_l2, rounded, to_dev

pytestmark = pytest.mark.gpu

CASES = [((200,), (512,), 4, 3001), ((64, 48), (128, 128), 4, 5003),
         ((30, 62), (50, 128), 3, 2049), ((16, 16, 16), (32, 32, 32), 5, 4097)]


def _run(N, n, m, K, x, fh, f, dtype, window="kaiser_bessel", spread=None):
    plan = Plan(N, x.shape[0], n=n, m=m, dtype=dtype, device=DEV, window=window)
    plan.set_option("window_table", K)
    if spread:
        plan.set_option("spread_method", spread)
    assert plan.info()["window_table"] == K
    plan.set_nodes(to_dev(x, dtype))
    yf = plan.trafo(to_dev(fh, dtype)).cpu().numpy()
    yh = plan.adjoint(to_dev(f, dtype)).cpu().numpy()
    assert plan.status() == 0
    plan.close()
    xr, fhr, fr = rounded(x, dtype), rounded(fh, dtype), rounded(f, dtype)
    return (yf, oracle.nfft(xr, fhr, n=n, m=m, window=window, lin_psi=K),
            yh, oracle.nfft_adjoint(xr, fr, N, n=n, m=m, window=window, lin_psi=K))


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("K", [64, 1024])
@pytest.mark.parametrize("N,n,m,M", CASES)
def test_table_window_parity(N, n, m, M, K, dtype):
    d = len(N)
    x = W.uniform_nodes(M, d, seed_offset=1200 + M)
    fh = W.gaussian_fhat(N, 1201 + M)
    f = W.gaussian_values(M, 1202 + M)
    yf, rf, yh, rh = _run(N, n, m, K, x, fh, f, dtype)
    assert rel_l2(yf, rf) <= TOL[dtype]
    assert rel_l2(yh, rh) <= TOL[dtype]


@pytest.mark.parametrize("spread", ["thread", "warp_atomic", "warp_private", "octet", "half", "plane",
                                    "rows"])
@pytest.mark.parametrize("window", ["kaiser_bessel", "gaussian", "bspline", "sinc"])
def test_table_window_every_form(spread, window):
    N, n, m, K = (48, 40), (96, 80), 4, 128
    x = W.round_nodes(W.radial_nodes(32, 256), np.float64)
    fh = W.gaussian_fhat(N, 1210)
    f = W.gaussian_values(x.shape[0], 1211)
    yf, rf, yh, rh = _run(N, n, m, K, x, fh, f, torch.float64, window, spread)
    assert rel_l2(yf, rf) <= 1e-12
    assert rel_l2(yh, rh) <= 1e-12


@pytest.mark.parametrize("d", [1, 2, 3])
def test_table_window_grad_x_with_grid_points(d):
    """Node gradient with the interpolated window, including nodes on grid points, where the
    window has kinks and the derivative is taken from larger t (from inside at t = +m)."""
    N = {1: (40,), 2: (20, 18), 3: (8, 10, 6)}[d]
    n = {1: (96,), 2: (48, 40), 3: (16, 20, 16)}[d]
    m, K = 3, 32
    g = np.random.default_rng(1220)
    k = np.stack([g.integers(-n[t] // 2, n[t] // 2, 100) for t in range(d)], axis=1)
    x = np.concatenate([k / np.array(n, dtype=float), W.uniform_nodes(700, d, 1221)])
    M = x.shape[0]
    c = W.gaussian_fhat(N, 1222)
    w = W.gaussian_values(M, 1223)
    plan = Plan(N, M, n=n, m=m, dtype=torch.float64, device=DEV)
    plan.set_option("window_table", K)
    plan.set_nodes(to_dev(x, torch.float64))
    gx = plan.grad_x(to_dev(c, torch.float64), to_dev(w, torch.float64)).cpu().numpy()
    ref = oracle.nfft_grad_x(x, c, w, n=n, m=m, lin_psi=K)
    assert rel_l2(gx, ref) <= 1e-11


def test_table_switch_on_and_off():
    N, n, m, M = (48, 40), (96, 80), 5, 4000
    x = W.uniform_nodes(M, 2, 1230)
    fh = W.gaussian_fhat(N, 1231)
    plan = Plan(N, M, n=n, m=m, dtype=torch.float64, device=DEV)
    plan.set_nodes(to_dev(x, torch.float64))
    fht = to_dev(fh, torch.float64)
    for K, window in [(256, "kaiser_bessel"), (256, "gaussian"), (0, "gaussian"),
                      (512, "kaiser_bessel"), (0, "kaiser_bessel")]:
        plan.set_option("window", window)
        plan.set_option("window_table", K)
        out = plan.trafo(fht).cpu().numpy()
        assert rel_l2(out, oracle.nfft(x, fh, n=n, m=m, window=window, lin_psi=K)) <= 1e-12
    from paper_1810_09891_gb300._lib import NfftError
    for bad in (1, -3, 70000):
        with pytest.raises(NfftError, match="NFFT_EINVAL"):
            plan.set_option("window_table", bad)


def test_table_error_converges_on_gpu():
    """The GPU NFFT with the table approaches the exact window as K grows (about 4x per
    doubling of K while the table error dominates)."""
    N, m, M = (64, 64), 6, 2000
    x = W.uniform_nodes(M, 2, 1240)
    fh = W.gaussian_fhat(N, 1241)
    exact = oracle.ndft(x, fh)
    plan = Plan(N, M, m=m, dtype=torch.float64, device=DEV)
    plan.set_nodes(to_dev(x, torch.float64))
    errs = []
    for K in (64, 128, 256, 512):
        plan.set_option("window_table", K)
        errs.append(oracle.error_E2(exact, plan.trafo(to_dev(fh, torch.float64)).cpu().numpy()))
    for a, b in zip(errs, errs[1:]):
        assert 3.0 <= a / b <= 5.0, errs


@pytest.mark.parametrize("interp", ["thread", "warp", "tile", "octet"])
@pytest.mark.parametrize("d", [2, 3])
def test_table_window_interp_forms(interp, d):
    N = {2: (40, 36), 3: (12, 10, 8)}[d]
    n = {2: (80, 72), 3: (24, 20, 16)}[d]
    m, K, M = 4, 64, 2500
    x = W.uniform_nodes(M, d, 1250 + d)
    fh = W.gaussian_fhat(N, 1251)
    plan = Plan(N, M, n=n, m=m, dtype=torch.float64, device=DEV)
    plan.set_option("window_table", K)
    plan.set_option("interp_method", interp)
    plan.set_nodes(to_dev(x, torch.float64))
    out = plan.trafo(to_dev(fh, torch.float64)).cpu().numpy()
    assert rel_l2(out, oracle.nfft(x, fh, n=n, m=m, lin_psi=K)) <= 1e-12
