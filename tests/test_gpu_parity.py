"""GPU parity: the CUDA path (through the C ABI binding) against the FP64 oracle NFFT, element
by element, on seeded inputs spanning several tiles with ragged tails, plus the edge cases of the
method (nodes on grid points, coincident nodes, nodes outside [-1/2, 1/2), M = 0, tiny grids,
every window cutoff m)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1810_09891_gb300 import workloads as W
from paper_1810_09891_gb300.nfft import Plan

from gpu_helpers import DEV, TOL, rel_l2, rounded, to_dev

pytestmark = pytest.mark.gpu

DTYPES = [torch.float64, torch.float32]


def _run(N, n, m, x, fh, f, dtype, interp=None, spread=None):
    M = x.shape[0]
    plan = Plan(N, M, n=n, m=m, dtype=dtype, device=DEV)
    if interp:
        plan.set_option("interp_method", interp)
    if spread:
        plan.set_option("spread_method", spread)
    plan.set_nodes(to_dev(x, dtype))
    out_f = plan.trafo(to_dev(fh, dtype)).cpu().numpy()
    out_h = plan.adjoint(to_dev(f, dtype)).cpu().numpy()
    st = plan.status()
    n_used = plan.n
    plan.close()
    assert st == 0
    xr, fhr, fr = rounded(x, dtype), rounded(fh, dtype), rounded(f, dtype)
    ref_f = oracle.nfft(xr, fhr, n=n_used, m=m)
    ref_h = oracle.nfft_adjoint(xr, fr, N, n=n_used, m=m)
    return out_f, ref_f, out_h, ref_h, xr, fhr, fr


@pytest.mark.parametrize("dtype", DTYPES)
def test_config_1d_full(dtype):
    """1-D, N = 256, n = 512, m = 6, M = 512 uniform nodes: against the oracle NFFT and the
    direct NDFT."""
    c = W.config_1d(np.float32 if dtype == torch.float32 else np.float64)
    out_f, ref_f, out_h, ref_h, xr, fhr, fr = _run(c["N"], c["n"], c["m"], c["x"], c["fhat"],
                                                  c["f"], dtype)
    assert rel_l2(out_f, ref_f) <= TOL[dtype]
    assert rel_l2(out_h.reshape(-1), ref_h.reshape(-1)) <= TOL[dtype]
    # against the NDFT: the window error of m = 6, sigma = 2 (~2e-12 for the paper's f_1)
    nd_f = oracle.ndft(xr, fhr)
    nd_h = oracle.ndft_adjoint(xr, fr, c["N"])
    bound = 1e-10 if dtype == torch.float64 else 1e-5
    assert rel_l2(out_f, nd_f) <= bound
    assert rel_l2(out_h, nd_h) <= bound


CASES = [
    # (N, n, m, M)  several bins, ragged tails, non-square, non-power-of-two N
    ((200,), (512,), 4, 3001),
    ((6,), (16,), 3, 77),
    ((64, 48), (128, 128), 4, 5003),
    ((30, 62), (64, 128), 3, 2049),
    ((16, 16, 16), (32, 32, 32), 4, 4097),
    ((10, 14, 6), (32, 32, 16), 2, 3333),
    ((32, 24, 20), (64, 64, 64), 5, 20000),
]


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("N,n,m,M", CASES)
def test_uniform_nodes(N, n, m, M, dtype):
    d = len(N)
    x = W.uniform_nodes(M, d, seed_offset=300 + M)
    fh = W.gaussian_fhat(N, seed_offset=301 + M)
    f = W.gaussian_values(M, seed_offset=302 + M)
    out_f, ref_f, out_h, ref_h, *_ = _run(N, n, m, x, fh, f, dtype)
    assert rel_l2(out_f, ref_f) <= TOL[dtype]
    assert rel_l2(out_h, ref_h) <= TOL[dtype]


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("d", [1, 2, 3])
@pytest.mark.parametrize("m", [1, 2, 3, 4, 5, 6, 7, 8])
@pytest.mark.parametrize("forms", [("thread", "thread"), ("warp", "warp_atomic"),
                                   ("tile", "warp_private"), ("thread", "octet"),
                                   ("thread", "half"), ("thread", "plane"),
                                   ("octet", "half"), ("octet", "plane"), ("thread", "rows")])
def test_every_window_cutoff(d, m, dtype, forms):
    N = {1: (40,), 2: (20, 24), 3: (12, 8, 10)}[d]
    n = {1: (128,), 2: (64, 64), 3: (32, 32, 32)}[d]
    M = 1500
    x = W.uniform_nodes(M, d, seed_offset=400 + m)
    fh = W.gaussian_fhat(N, seed_offset=401 + m)
    f = W.gaussian_values(M, seed_offset=402 + m)
    out_f, ref_f, out_h, ref_h, *_ = _run(N, n, m, x, fh, f, dtype, *forms)
    tol = TOL[dtype] if (dtype == torch.float64 or m <= 6) else 3e-5
    assert rel_l2(out_f, ref_f) <= tol
    assert rel_l2(out_h, ref_h) <= tol


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("d", [1, 2, 3])
@pytest.mark.parametrize("forms", [("thread", "thread"), ("warp", "warp_atomic"),
                                   ("tile", "warp_private"), ("thread", "octet"),
                                   ("thread", "half"), ("thread", "plane"),
                                   ("octet", "half"), ("octet", "plane"), ("thread", "rows")])
def test_nodes_on_grid_points_and_edges(d, dtype, forms):
    """Nodes exactly on grid points (2m+1 taps), at -1/2, coincident nodes, and nodes outside
    the torus (any real is taken modulo 1)."""
    N = {1: (32,), 2: (16, 24), 3: (8, 12, 8)}[d]
    n = {1: (64,), 2: (32, 64), 3: (16, 32, 16)}[d]
    m = 3
    g = np.random.default_rng(7)
    k = g.integers(-n[0] // 2, n[0] // 2, size=(200, d))
    x_grid = k / np.array(n, dtype=float)  # exactly representable
    x = np.concatenate([
        x_grid,
        np.full((50, d), -0.5),
        np.zeros((60, d)),
        W.uniform_nodes(100, d, seed_offset=9) + g.integers(-3, 4, size=(100, d)),
        W.uniform_nodes(300, d, seed_offset=10),
    ])
    fh = W.gaussian_fhat(N, seed_offset=11)
    f = W.gaussian_values(x.shape[0], seed_offset=12)
    out_f, ref_f, out_h, ref_h, *_ = _run(N, n, m, x, fh, f, dtype, *forms)
    assert rel_l2(out_f, ref_f) <= TOL[dtype]
    assert rel_l2(out_h, ref_h) <= TOL[dtype]


@pytest.mark.parametrize("dtype", DTYPES)
def test_smallest_grid(dtype):
    """N = 2, n = 4, m = 1 (2m + 2 = n): the tile wraps onto itself."""
    for d in (1, 2, 3):
        N, n, m, M = (2,) * d, (4,) * d, 1, 37
        x = W.uniform_nodes(M, d, seed_offset=13)
        fh = W.gaussian_fhat(N, seed_offset=14)
        f = W.gaussian_values(M, seed_offset=15)
        out_f, ref_f, out_h, ref_h, *_ = _run(N, n, m, x, fh, f, dtype)
        assert rel_l2(out_f, ref_f) <= TOL[dtype]
        assert rel_l2(out_h, ref_h) <= TOL[dtype]


@pytest.mark.parametrize("dtype", DTYPES)
def test_zero_nodes(dtype):
    N = (16, 16)
    plan = Plan(N, 0, m=4, dtype=dtype, device=DEV)
    plan.set_nodes(torch.zeros((0, 2), dtype=dtype, device=DEV))
    f = plan.trafo(to_dev(W.gaussian_fhat(N, 16), dtype))
    assert f.numel() == 0
    h = plan.adjoint(torch.zeros(0, dtype=plan.cdtype, device=DEV))
    assert torch.count_nonzero(h).item() == 0
    assert plan.status() == 0


@pytest.mark.parametrize("dtype", DTYPES)
def test_adjoint_identity(dtype):
    """<A fhat, f> = <fhat, A^H f> for the CUDA path itself (same nodes, same plan)."""
    N, M, m = (48, 40), 9000, 4
    x = W.uniform_nodes(M, 2, seed_offset=17)
    plan = Plan(N, M, m=m, dtype=dtype, device=DEV)
    plan.set_nodes(to_dev(x, dtype))
    fh = to_dev(W.gaussian_fhat(N, 18), dtype)
    f = to_dev(W.gaussian_values(M, 19), dtype)
    lhs = torch.vdot(plan.trafo(fh), f).item()
    rhs = torch.vdot(fh.reshape(-1), plan.adjoint(f).reshape(-1)).item()
    tol = 1e-13 if dtype == torch.float64 else 2e-6
    assert abs(lhs - rhs) <= tol * abs(lhs)


def test_bad_node_sets_status():
    N, M = (16, 16), 64
    x = W.uniform_nodes(M, 2, seed_offset=20)
    x[5, 1] = np.nan
    x[9, 0] = np.inf
    plan = Plan(N, M, m=3, dtype=torch.float64, device=DEV)
    plan.set_nodes(to_dev(x, torch.float64))
    plan.trafo(to_dev(W.gaussian_fhat(N, 21), torch.float64))
    assert plan.status() == 5  # NFFT_EBADNODE
    assert plan.status() == 0  # cleared by the read


def test_trafo_before_nodes_is_refused():
    from paper_1810_09891_gb300._lib import NfftError
    plan = Plan((8,), 10, m=2, dtype=torch.float64, device=DEV)
    with pytest.raises(NfftError, match="NFFT_ENOTREADY"):
        plan.trafo(torch.zeros(8, dtype=torch.complex128, device=DEV))


def test_repeatable_within_rounding():
    """Spreading adds with atomics, so two adjoints differ only by rounding order."""
    N, M = (32, 32, 32), 200000
    x = W.clustered_nodes(M, 3, seed_offset=22)
    plan = Plan(N, M, m=4, dtype=torch.float32, device=DEV)
    plan.set_nodes(to_dev(x, torch.float32))
    f = to_dev(W.gaussian_values(M, 23), torch.float32)
    a = plan.adjoint(f).cpu().numpy()
    b = plan.adjoint(f).cpu().numpy()
    assert rel_l2(a, b) <= 1e-6
