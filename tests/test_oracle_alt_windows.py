"""Pins for the oracle's Gaussian, B-spline and sinc windows (Section 4.1 names them as the
alternatives to Kaiser-Bessel; the pairs are the standard ones of the NFFT literature).

Each reading is tied to something outside the oracle: the cardinal B-spline to scipy's B-spline
basis and to its partition of unity; every phihat to a numerical Fourier transform of psi
(exact for the compactly supported B-spline, within the truncation tail for the Gaussian, and
over the untruncated sinc power with scipy's Fourier-integral quadrature); psi' to central
differences; and the full NFFT with each window to the exact NDFT within the published error
bounds (Steidl 1998: Gaussian 4 exp(-m pi (1 - 1/(2 sigma - 1))), B-spline 4 (2 sigma - 1)^(-2m);
the sinc window has the B-spline's rate). A dropped term, a wrong parameter or a transposed pair
breaks at least one of them.
"""
import numpy as np
import pytest
from scipy import integrate, interpolate, special

import oracle
from paper_1810_09891_gb300 import workloads as W

ALT = ("gaussian", "bspline", "sinc")


def _scipy_bspline(p, t):
    knots = np.arange(p + 1, dtype=np.float64) - 0.5 * p
    v = interpolate.BSpline.basis_element(knots, extrapolate=False)(np.asarray(t, np.float64))
    return np.nan_to_num(v, nan=0.0)


@pytest.mark.parametrize("p", [2, 3, 4, 6, 8, 11, 12, 16])
def test_bspline_matches_scipy_basis(p):
    t = np.linspace(-0.5 * p - 0.3, 0.5 * p + 0.3, 257)
    t = np.concatenate([t, np.arange(-p, p + 1) * 0.5])  # knots and half-knots
    ours = np.array([oracle.bspline(p, float(u)) for u in t])
    ref = _scipy_bspline(p, t)
    assert np.max(np.abs(ours - ref)) <= 1e-14


def test_bspline_known_values():
    # cubic: M_4(0) = 2/3, M_4(+-1) = 1/6; order 8: M_8(0) = 151/315, M_8(3) = 1/5040
    assert oracle.bspline(4, 0.0) == pytest.approx(2.0 / 3.0, rel=1e-15)
    assert oracle.bspline(4, 1.0) == pytest.approx(1.0 / 6.0, rel=1e-15)
    assert oracle.bspline(4, -1.0) == pytest.approx(1.0 / 6.0, rel=1e-15)
    assert oracle.bspline(8, 0.0) == pytest.approx(151.0 / 315.0, rel=1e-15)
    assert oracle.bspline(8, 3.0) == pytest.approx(1.0 / 5040.0, rel=1e-13)
    assert oracle.bspline(8, 4.0) == 0.0
    assert oracle.bspline(1, -0.5) == 1.0 and oracle.bspline(1, 0.5) == 0.0


@pytest.mark.parametrize("p", [2, 4, 8, 16])
def test_bspline_partition_of_unity(p):
    g = np.random.default_rng(11)
    for t in g.uniform(-1.0, 1.0, 20):
        s = sum(oracle.bspline(p, float(t - k)) for k in range(-p, p + 1))
        assert s == pytest.approx(1.0, abs=1e-14)


@pytest.mark.parametrize("m", [1, 2, 4, 8])
@pytest.mark.parametrize("n,N", [(128, 64), (96, 64)])
def test_window_parameters_give_stated_shapes(m, n, N):
    """The Gaussian's variance parameter b sets psi(t) = e^{-1} at t = sqrt(b); the sinc's a
    puts the first zero of psi at t = 1/a, and 1/a > m for every sigma > 1 (the first zero lies
    outside the cut-off support)."""
    b = oracle.window_param("gaussian", n, N, m)
    assert oracle.window_psi("gaussian", np.sqrt(b), m, b) == pytest.approx(np.exp(-1.0))
    a = oracle.window_param("sinc", n, N, m)
    sigma = n / N
    assert 1.0 / a == pytest.approx(2.0 * m * sigma / (2.0 * sigma - 1.0), rel=1e-15)
    assert 1.0 / a > m
    t = np.linspace(-m, m, 41)
    ours = np.array([oracle.window_psi("sinc", float(u), m, a) for u in t])
    assert np.allclose(ours, np.sinc(a * t) ** (2 * m), rtol=1e-14, atol=0)
    assert oracle.window_psi("bspline", 0.0, m, 0.0) == pytest.approx(oracle.bspline(2 * m, 0.0))
    for w in ALT:
        prm = oracle.window_param(w, n, N, m)
        assert oracle.window_psi(w, m + 1e-9, m, prm) == 0.0  # cut off to |t| <= m


@pytest.mark.parametrize("m", [2, 4, 8])
@pytest.mark.parametrize("k", [0, 7, 31])
def test_bspline_phihat_is_fourier_transform(m, k):
    """psi = M_2m has support [-m, m], so the transform over the support is exact."""
    n = 128
    f = lambda t: oracle.window_psi("bspline", t, m, 0.0) * np.cos(2 * np.pi * k * t / n)
    v, _ = integrate.quad(f, -m, m, points=list(range(-m + 1, m)), limit=200, epsabs=1e-15,
                          epsrel=1e-13)
    assert n * oracle.window_phihat("bspline", k, n, m, 0.0) == pytest.approx(v, rel=1e-11)


@pytest.mark.parametrize("m", [2, 4, 8])
@pytest.mark.parametrize("k", [0, 7, 31])
def test_gaussian_phihat_is_fourier_transform(m, k):
    """Transform of the cut-off psi over [-m, m]; it differs from phihat (the transform of the
    untruncated Gaussian) by at most the tail mass sqrt(pi b) erfc(m / sqrt(b))."""
    n, N = 128, 64
    b = oracle.window_param("gaussian", n, N, m)
    f = lambda t: oracle.window_psi("gaussian", t, m, b) * np.cos(2 * np.pi * k * t / n)
    v, _ = integrate.quad(f, -m, m, limit=200, epsabs=1e-15, epsrel=1e-13)
    tail = np.sqrt(np.pi * b) * special.erfc(m / np.sqrt(b))
    ph = n * oracle.window_phihat("gaussian", k, n, m, b)
    assert abs(ph - v) <= tail + 1e-12 * abs(v)


@pytest.mark.parametrize("m", [2, 4, 8])
@pytest.mark.parametrize("k", [0, 5, 31])
def test_sinc_phihat_is_fourier_transform(m, k):
    """The untruncated sinc^2m(pi a t) transformed with scipy's Fourier-integral quadrature over
    [0, inf) (QAWF; plain quadrature at k = 0)."""
    n, N = 128, 64
    a = oracle.window_param("sinc", n, N, m)
    f = lambda t: np.sinc(a * t) ** (2 * m)
    if k == 0:
        v, _ = integrate.quad(f, 0.0, np.inf, limit=500)
    else:
        v, _ = integrate.quad(f, 0.0, np.inf, weight="cos", wvar=2 * np.pi * k / n)
    assert n * oracle.window_phihat("sinc", k, n, m, a) == pytest.approx(2.0 * v, rel=1e-8)


@pytest.mark.parametrize("window", ALT)
@pytest.mark.parametrize("m", [1, 3, 6])
def test_window_derivative_matches_central_difference(window, m):
    n, N = 128, 64
    prm = oracle.window_param(window, n, N, m)
    h = 1e-6
    g = np.random.default_rng(12)
    scale = oracle.window_psi(window, 0.0, m, prm)
    for t in g.uniform(-m + 2e-3, m - 2e-3, 25):
        fd = (oracle.window_psi(window, t + h, m, prm) -
              oracle.window_psi(window, t - h, m, prm)) / (2 * h)
        assert oracle.window_dpsi(window, t, m, prm) == pytest.approx(fd, abs=1e-7 * scale)


def _bound(window, m, sigma):
    if window == "gaussian":
        return 4.0 * np.exp(-m * np.pi * (1.0 - 1.0 / (2.0 * sigma - 1.0)))
    return 4.0 * (2.0 * sigma - 1.0) ** (-2 * m)


@pytest.mark.parametrize("window", ALT)
@pytest.mark.parametrize("d,N,n", [(1, (64,), (128,)), (1, (64,), (96,)),
                                   (2, (16, 12), (32, 24))])
def test_nfft_error_within_published_bound(window, d, N, n):
    """E_inf (Section 2, eq. EI) of the NFFT with the window against the exact NDFT: below the
    bound for m = 1..8 wherever the bound is above rounding, and decreasing in m."""
    M = 200
    x = W.uniform_nodes(M, d, 30 + d)
    fh = W.gaussian_fhat(N, 31)
    exact = oracle.ndft(x, fh)
    sigma = min(n[t] / N[t] for t in range(d))
    errs = []
    for m in range(1, 9):
        e = oracle.error_Einf(exact, oracle.nfft(x, fh, n=n, m=m, window=window), fh)
        errs.append(e)
        assert e <= max(_bound(window, m, sigma), 1e-14), (m, e)
    assert all(errs[i + 1] < errs[i] for i in range(4)), errs


@pytest.mark.parametrize("window", ALT)
def test_adjoint_identity(window):
    """<A fhat, f> = <fhat, A^H f>: B^H and D^H are the adjoints of B and D for every window."""
    N, n, m = (16, 12), (32, 24), 4
    M = 150
    x = W.uniform_nodes(M, 2, 40)
    fh = W.gaussian_fhat(N, 41)
    f = W.gaussian_values(M, 42)
    lhs = np.vdot(f, oracle.nfft(x, fh, n=n, m=m, window=window))
    rhs = np.vdot(oracle.nfft_adjoint(x, f, N, n=n, m=m, window=window), fh)
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


@pytest.mark.parametrize("window", ALT)
def test_node_gradient_matches_finite_difference(window):
    """Re(conj(w_j) d/dx f_j) of the windowed NFFT against central differences of the oracle's
    own NFFT (1-D, nodes kept away from support-box changes)."""
    N, n, m = (32,), (64,), 5
    M = 40
    x = W.uniform_nodes(M, 1, 50)
    c = W.gaussian_fhat(N, 51)
    w = W.gaussian_values(M, 52)
    gx = oracle.nfft_grad_x(x, c, w, n=n, m=m, window=window)
    h = 1e-7
    fp = oracle.nfft(x + h, c, n=n, m=m, window=window)
    fm = oracle.nfft(x - h, c, n=n, m=m, window=window)
    fd = np.real(np.conj(w) * (fp - fm) / (2 * h))
    keep = (np.floor(n[0] * (x[:, 0] + h) + m) == np.floor(n[0] * (x[:, 0] - h) + m)) & \
           (np.ceil(n[0] * (x[:, 0] + h) - m) == np.ceil(n[0] * (x[:, 0] - h) - m))
    assert keep.sum() > M // 2
    scale = np.max(np.abs(gx[keep, 0]))
    assert np.max(np.abs(gx[keep, 0] - fd[keep])) <= 1e-6 * scale
