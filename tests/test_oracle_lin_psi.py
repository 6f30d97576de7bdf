"""Pins for the oracle's lookup-table window (PRE_LIN_PSI, Section 3.1, Table tab:nfftflags:
the window read from a table of its values and linearly interpolated; K samples per unit of the
grid-scaled argument t = n x).

Checked against facts that do not reuse the interpolation code: exactness at the samples,
collinearity inside a segment, the linear-interpolation error bound h^2 max|psi''| / 8 (psi''
by central differences of the exact window), the derivative as a difference quotient inside a
segment, K^-2 convergence of the NFFT error, and the adjoint identity of the windowed B / B^H.
"""
import numpy as np
import pytest

import oracle
from paper_1810_09891_gb300 import workloads as W

WINDOWS = ("kaiser_bessel", "gaussian", "bspline", "sinc")


def _prm(window, m, n=128, N=64):
    return oracle.window_param(window, n, N, m)


@pytest.mark.parametrize("window", WINDOWS)
@pytest.mark.parametrize("K", [16, 256])
def test_exact_at_the_samples(window, K):
    m = 4
    prm = _prm(window, m)
    for j in range(0, m * K + 1, 7):
        for t in (j / K, -j / K):
            assert oracle.window_psi_eval(window, t, m, prm, lin_psi=K) == pytest.approx(
                oracle.window_psi(window, t, m, prm), rel=1e-14, abs=1e-300)


@pytest.mark.parametrize("window", WINDOWS)
def test_linear_inside_a_segment(window):
    m, K = 3, 64
    prm = _prm(window, m)
    g = np.random.default_rng(21)
    for j in g.integers(0, m * K, 25):
        t = (j + np.array([0.1, 0.45, 0.9])) / K
        v = [oracle.window_psi_eval(window, float(u), m, prm, lin_psi=K) for u in t]
        slope1 = (v[1] - v[0]) / (t[1] - t[0])
        slope2 = (v[2] - v[1]) / (t[2] - t[1])
        scale = oracle.window_psi(window, 0.0, m, prm)
        assert slope1 == pytest.approx(slope2, abs=1e-6 * scale * K)


@pytest.mark.parametrize("window", WINDOWS)
@pytest.mark.parametrize("K", [32, 512])
def test_interpolation_error_bound(window, K):
    """|psi_lin - psi| <= h^2 / 8 max|psi''| on each segment (h = 1/K); psi'' from central
    differences of the exact window over the segment's neighbourhood (plus rounding slack)."""
    m = 4
    prm = _prm(window, m)
    g = np.random.default_rng(22)
    h = 1.0 / K
    scale = oracle.window_psi(window, 0.0, m, prm)
    for t in g.uniform(-m + 2 * h, m - 2 * h, 200):
        j = np.floor(abs(t) * K)
        a = j / K
        e = 1e-4
        d2 = max(abs((oracle.window_psi(window, u + e, m, prm) - 2 * oracle.window_psi(window, u, m, prm)
                      + oracle.window_psi(window, u - e, m, prm)) / e**2)
                 for u in np.linspace(a, a + h, 5))
        err = abs(oracle.window_psi_eval(window, float(t), m, prm, lin_psi=K)
                  - oracle.window_psi(window, float(t), m, prm))
        assert err <= 1.2 * h * h / 8 * d2 + 1e-12 * scale


@pytest.mark.parametrize("window", ["kaiser_bessel", "gaussian"])
def test_derivative_is_the_segment_slope(window):
    m, K = 4, 128
    prm = _prm(window, m)
    g = np.random.default_rng(23)
    for t in g.uniform(-m + 0.01, m - 0.01, 40):
        u = abs(t) * K
        if abs(u - np.round(u)) < 0.05:
            continue  # keep the difference quotient inside one segment
        e = 1e-3 / K
        fd = (oracle.window_psi_eval(window, t + e, m, prm, lin_psi=K)
              - oracle.window_psi_eval(window, t - e, m, prm, lin_psi=K)) / (2 * e)
        got = oracle.window_dpsi_eval(window, t, m, prm, lin_psi=K)
        assert got == pytest.approx(fd, rel=1e-6, abs=1e-9 * oracle.window_psi(window, 0, m, prm))


@pytest.mark.parametrize("d,N,n", [(1, (64,), (128,)), (2, (16, 12), (32, 24))])
def test_nfft_error_converges_like_k_minus_2(d, N, n):
    """m = 6 (window error ~1e-11): E_2 of the table-driven NFFT against the NDFT falls by about
    4 per doubling of K and approaches the exact-window error."""
    M = 300
    x = W.uniform_nodes(M, d, seed_offset=24 + d)
    fh = W.gaussian_fhat(N, 25)
    exact = oracle.ndft(x, fh)
    e = [oracle.error_E2(exact, oracle.nfft(x, fh, n=n, m=6, lin_psi=K)) for K in (64, 128, 256, 512)]
    for a, b in zip(e, e[1:]):
        assert 3.0 <= a / b <= 5.0, e
    e0 = oracle.error_E2(exact, oracle.nfft(x, fh, n=n, m=6))
    assert e0 < e[-1] / 10


@pytest.mark.parametrize("window", WINDOWS)
def test_adjoint_identity_with_table(window):
    N, n, m, M = (16, 12), (32, 24), 4, 150
    x = W.uniform_nodes(M, 2, 26)
    fh = W.gaussian_fhat(N, 27)
    f = W.gaussian_values(M, 28)
    lhs = np.vdot(f, oracle.nfft(x, fh, n=n, m=m, window=window, lin_psi=100))
    rhs = np.vdot(oracle.nfft_adjoint(x, f, N, n=n, m=m, window=window, lin_psi=100), fh)
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


@pytest.mark.parametrize("window", ["kaiser_bessel", "sinc"])
def test_derivative_at_a_sample_is_the_right_derivative(window):
    """At a kink of the interpolant (t = j/K, e.g. a node on a grid point) the derivative is the
    one from larger t: the forward difference quotient, on both sides of 0 and at t = -m; at
    t = +m, where the cut-off window jumps to 0, the backward one (from inside the support)."""
    m, K = 3, 32
    prm = _prm(window, m)
    e = 1e-4 / K
    for j in (-m * K, -m * K + 1, -17, -1, 0, 1, 40, m * K - 1, m * K):
        t = j / K
        s = -1.0 if j == m * K else 1.0
        fwd = s * (oracle.window_psi_eval(window, t + s * e, m, prm, lin_psi=K)
                   - oracle.window_psi_eval(window, t, m, prm, lin_psi=K)) / e
        got = oracle.window_dpsi_eval(window, t, m, prm, lin_psi=K)
        assert got == pytest.approx(fwd, rel=1e-6, abs=1e-9 * oracle.window_psi(window, 0, m, prm)), j
