"""GPU parity on the workloads the benchmark times: the 2-D golden-angle radial trajectory
(coincident nodes at the origin, density ~ 1/r) and the 3-D clustered node set, at reduced sizes
element by element for every spreading method, and at full size on sampled outputs."""
import numpy as np
import pytest
import torch

import oracle
from paper_1810_09891_gb300 import workloads as W
from paper_1810_09891_gb300.nfft import Plan

from gpu_helpers import DEV, TOL, rel_l2, rounded, to_dev

pytestmark = pytest.mark.gpu

METHODS = ["thread", "warp_atomic", "warp_private"]
METHODS_2D = METHODS + ["octet", "half", "rows"]  # the group forms exist for d = 2 only
METHODS_3D = METHODS + ["plane"]  # the plane form exists for d = 3 only
INTERP = ["thread", "warp", "tile", "octet"]


def _plan(N, n, m, M, dtype, method=None, bins=None, interp=None):
    plan = Plan(N, M, n=n, m=m, dtype=dtype, device=DEV)
    if method:
        plan.set_option("spread_method", method)
    if interp:
        plan.set_option("interp_method", interp)
    for t, b in enumerate(bins or ()):
        plan.set_option(f"bin{t}", b)
    return plan


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("method", METHODS_2D)
@pytest.mark.parametrize("interp", INTERP)
@pytest.mark.parametrize("m", [4, 6])
def test_radial_reduced(dtype, method, interp, m):
    N = (128, 128)
    n = (256, 256)
    x = W.round_nodes(W.radial_nodes(64, 512), np.float32 if dtype == torch.float32 else
                      np.float64)
    M = x.shape[0]
    fh = W.gaussian_fhat(N, 600)
    f = W.gaussian_values(M, 601)
    plan = _plan(N, n, m, M, dtype, method, interp=interp)
    plan.set_nodes(to_dev(x, dtype))
    yf = plan.trafo(to_dev(fh, dtype)).cpu().numpy()
    yh = plan.adjoint(to_dev(f, dtype)).cpu().numpy()
    assert plan.status() == 0
    xr, fhr, fr = rounded(x, dtype), rounded(fh, dtype), rounded(f, dtype)
    assert rel_l2(yf, oracle.nfft(xr, fhr, n=n, m=m)) <= TOL[dtype]
    assert rel_l2(yh, oracle.nfft_adjoint(xr, fr, N, n=n, m=m)) <= TOL[dtype]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("method", METHODS_3D)
@pytest.mark.parametrize("interp", INTERP)
def test_clusters_reduced(dtype, method, interp):
    N = (32, 32, 32)
    n = (64, 64, 64)
    m = 4
    x = W.round_nodes(W.clustered_nodes(120000, 3, seed_offset=602),
                      np.float32 if dtype == torch.float32 else np.float64)
    M = x.shape[0]
    fh = W.gaussian_fhat(N, 603)
    f = W.gaussian_values(M, 604)
    plan = _plan(N, n, m, M, dtype, method, interp=interp)
    plan.set_nodes(to_dev(x, dtype))
    yf = plan.trafo(to_dev(fh, dtype)).cpu().numpy()
    yh = plan.adjoint(to_dev(f, dtype)).cpu().numpy()
    assert plan.status() == 0
    xr, fhr, fr = rounded(x, dtype), rounded(fh, dtype), rounded(f, dtype)
    idx = np.arange(0, M, 7)
    assert rel_l2(yf[idx], oracle.nfft(xr[idx], fhr, n=n, m=m)) <= TOL[dtype]
    assert rel_l2(yh, oracle.nfft_adjoint(xr, fr, N, n=n, m=m)) <= TOL[dtype]


def test_bin_size_too_large_for_shared_memory_is_rejected():
    from paper_1810_09891_gb300._lib import NfftError
    plan = Plan((64, 64), 10, n=(128, 128), m=4, dtype=torch.float64, device=DEV)
    plan.set_option("bin0", 128)
    with pytest.raises(NfftError, match="NFFT_EINVAL"):
        plan.set_option("bin1", 128)  # (128 + 8)^2 complex128 > 227 KB


@pytest.mark.parametrize("bins", [(4, 64), (64, 8), (32, 64), (1, 1)])
def test_bin_sizes(bins):
    """Any power-of-two bin size gives the same transform (only the work split changes)."""
    N, n, m = (64, 64), (128, 128), 4
    x = W.radial_nodes(32, 256)
    M = x.shape[0]
    fh = W.gaussian_fhat(N, 605)
    f = W.gaussian_values(M, 606)
    for method in METHODS_2D:
        plan = _plan(N, n, m, M, torch.float64, method, bins)
        assert plan.bin == tuple(min(b, v) for b, v in zip(bins, n))
        plan.set_nodes(to_dev(x, torch.float64))
        yf = plan.trafo(to_dev(fh, torch.float64)).cpu().numpy()
        yh = plan.adjoint(to_dev(f, torch.float64)).cpu().numpy()
        assert rel_l2(yf, oracle.nfft(x, fh, n=n, m=m)) <= 1e-12
        assert rel_l2(yh, oracle.nfft_adjoint(x, f, N, n=n, m=m)) <= 1e-12


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("bins,sub", [((8, 8, 8), 1024), ((16, 16, 8), 256), ((4, 4, 8), 32),
                                      ((2, 32, 4), 128), ((8, 16, 16), 1024)])
def test_plane_form_bins_and_subproblems(dtype, bins, sub):
    """The d = 3 plane form over tile shapes (padded and unpadded row pitch), subproblem sizes
    below and above one staged chunk of nodes, and clustered nodes (bins split into many
    subproblems): the same transform as the oracle."""
    N, n, m = (24, 32, 16), (48, 64, 32), 4
    x = W.round_nodes(W.clustered_nodes(40000, 3, seed_offset=607),
                      np.float32 if dtype == torch.float32 else np.float64)
    M = x.shape[0]
    f = W.gaussian_values(M, 608)
    plan = _plan(N, n, m, M, dtype, "plane", bins)
    plan.set_option("subproblem", sub)
    plan.set_nodes(to_dev(x, dtype))
    yh = plan.adjoint(to_dev(f, dtype)).cpu().numpy()
    assert plan.status() == 0
    xr, fr = rounded(x, dtype), rounded(f, dtype)
    assert rel_l2(yh, oracle.nfft_adjoint(xr, fr, N, n=n, m=m)) <= TOL[dtype]


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_radial_full_size(dtype):
    """N = (512, 512), n = (1024, 1024), m = 4, M = 1,048,576 radial nodes, the benchmark's
    launch configuration: forward on 4096 sampled nodes, adjoint on every coefficient."""
    c = W.config_radial(m=4, dtype=np.float32 if dtype == torch.float32 else np.float64)
    M = c["x"].shape[0]
    plan = Plan(c["N"], M, n=c["n"], m=4, dtype=dtype, device=DEV)
    plan.set_nodes(to_dev(c["x"], dtype))
    yf = plan.trafo(to_dev(c["fhat"], dtype)).cpu().numpy()
    yh = plan.adjoint(to_dev(c["f"], dtype)).cpu().numpy()
    assert plan.status() == 0
    xr, fhr, fr = rounded(c["x"], dtype), rounded(c["fhat"], dtype), rounded(c["f"], dtype)
    idx = np.sort(np.random.default_rng(1).choice(M, 4096, replace=False))
    idx[0] = 1024  # spoke 0, sample 1024: the origin, shared by every spoke
    assert rel_l2(yf[idx], oracle.nfft(xr[idx], fhr, n=c["n"], m=4)) <= TOL[dtype]
    assert rel_l2(yh, oracle.nfft_adjoint(xr, fr, c["N"], n=c["n"], m=4)) <= TOL[dtype]


def test_clusters_full_size_fp32():
    """N = (128,)*3, n = 2N, m = 4, M = 4,194,304 clustered nodes, FP32: forward on sampled nodes;
    adjoint of a vector that is zero except on a 20000-node sample (the full plan spreads all
    M nodes), against the oracle adjoint of the sample."""
    c = W.config_clusters(dtype=np.float32)
    M = c["x"].shape[0]
    plan = Plan(c["N"], M, n=c["n"], m=4, dtype=torch.float32, device=DEV)
    plan.set_nodes(to_dev(c["x"], torch.float32))
    yf = plan.trafo(to_dev(c["fhat"], torch.float32)).cpu().numpy()
    rng = np.random.default_rng(2)
    idx = np.sort(rng.choice(M, 20000, replace=False))
    fz = np.zeros(M, dtype=np.complex128)
    fz[idx] = c["f"][idx]
    yh = plan.adjoint(to_dev(fz, torch.float32)).cpu().numpy()
    assert plan.status() == 0
    xr = rounded(c["x"], torch.float32)
    fhr = rounded(c["fhat"], torch.float32)
    fr = rounded(fz, torch.float32)
    s = idx[:4096]
    assert rel_l2(yf[s], oracle.nfft(xr[s], fhr, n=c["n"], m=4)) <= TOL[torch.float32]
    assert rel_l2(yh, oracle.nfft_adjoint(xr[idx], fr[idx], c["N"], n=c["n"], m=4)) <= \
        TOL[torch.float32]


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_subproblem_sizes(dtype):
    """Cutting the bins' sorted nodes into work items of 32 ... 1024 nodes changes only the work
    split; sizes that are not powers of two in that range are rejected."""
    from paper_1810_09891_gb300._lib import NfftError
    N, n, m = (64, 64), (128, 128), 4
    npdt = np.float32 if dtype == torch.float32 else np.float64
    x = W.round_nodes(W.radial_nodes(48, 512), npdt)
    M = x.shape[0]
    fh = W.gaussian_fhat(N, 607)
    f = W.gaussian_values(M, 608)
    xr, fhr, fr = rounded(x, dtype), rounded(fh, dtype), rounded(f, dtype)
    ref_f = oracle.nfft(xr, fhr, n=n, m=m)
    ref_h = oracle.nfft_adjoint(xr, fr, N, n=n, m=m)
    for method in METHODS_2D:
        for sub in (32, 128, 1024, 0):
            plan = _plan(N, n, m, M, dtype, method)
            plan.set_option("subproblem", sub)
            plan.set_nodes(to_dev(x, dtype))
            yf = plan.trafo(to_dev(fh, dtype)).cpu().numpy()
            yh = plan.adjoint(to_dev(f, dtype)).cpu().numpy()
            assert plan.status() == 0
            assert rel_l2(yf, ref_f) <= TOL[dtype]
            assert rel_l2(yh, ref_h) <= TOL[dtype]
    plan = _plan(N, n, m, M, dtype)
    for bad in (16, 33, 2048, -1):
        with pytest.raises(NfftError, match="NFFT_EINVAL"):
            plan.set_option("subproblem", bad)


def test_method_option_ranges():
    """NFFT_OPT_SPREAD_METHOD takes 0..8 and NFFT_OPT_INTERP_METHOD 0..4; other values are
    rejected with NFFT_EINVAL and leave the plan usable."""
    from paper_1810_09891_gb300 import _lib

    L = _lib.lib()
    plan = Plan((16, 16, 16), 100, m=4, dtype=torch.float32, device=DEV)
    for v in range(0, 9):
        assert L.nfft_set_option(plan._h, _lib.OPT_SPREAD_METHOD, v) == 0
    for v in range(0, 5):
        assert L.nfft_set_option(plan._h, _lib.OPT_INTERP_METHOD, v) == 0
    einval = L.nfft_set_option(plan._h, _lib.OPT_SPREAD_METHOD, 9)
    assert einval != 0
    assert L.nfft_set_option(plan._h, _lib.OPT_SPREAD_METHOD, -1) == einval
    assert L.nfft_set_option(plan._h, _lib.OPT_INTERP_METHOD, 5) == einval
    assert _lib.SPREAD_METHODS["rows"] == 8 and _lib.INTERP_METHODS["octet"] == 4
    x = W.uniform_nodes(100, 3, seed_offset=609)
    fh = W.gaussian_fhat((16, 16, 16), 610)
    plan.set_nodes(to_dev(x, torch.float32))
    y = plan.trafo(to_dev(fh, torch.float32)).cpu().numpy()
    assert rel_l2(y, oracle.nfft(rounded(x, torch.float32), rounded(fh, torch.float32),
                                 n=plan.n, m=4)) <= TOL[torch.float32]
