"""Pins for the oracle's Kaiser-Bessel window (Section 2, eq. window and eq. window_cutoff).

The window pair is not printed in the paper (it defers to Plonka-Potts-Steidl-Tasche, Ch. 7.2);
the oracle's reading is checked here against facts fixed by mathematics and by scipy:
I0 against scipy.special.i0, the pair against a numerical inverse Fourier transform of phihat,
psi' against a finite difference, and the shape parameter against the closed form.
"""
import numpy as np
import pytest
from scipy import integrate, special

import oracle


@pytest.mark.parametrize("z", [0.0, 1e-3, 0.5, 1.0, 3.7, 10.0, 18.85, 30.0, 47.1])
def test_bessel_i0_matches_scipy(z):
    # scipy evaluates I0 by Chebyshev expansions accurate to a few ulp
    assert oracle.bessel_i0(z) == pytest.approx(special.i0(z), rel=5e-15)


def test_bessel_i0_known_values():
    # I0(0) = 1; I0(1) = 1.2660658777520083... (Abramowitz-Stegun Table 9.8).
    assert oracle.bessel_i0(0.0) == 1.0
    assert oracle.bessel_i0(1.0) == pytest.approx(1.2660658777520083, rel=1e-15)


@pytest.mark.parametrize("n,N", [(512, 256), (1024, 512), (48, 32), (100, 64)])
def test_shape_parameter(n, N):
    sigma = n / N
    assert oracle.kb_b(n, N) == pytest.approx(np.pi * (2.0 - 1.0 / sigma), rel=1e-15)


@pytest.mark.parametrize("m", [2, 4, 6, 8])
@pytest.mark.parametrize("n,N", [(64, 32), (96, 64)])
def test_kb_pair_inverse_fourier(m, n, N):
    """phi(x) = int phihat(xi) e^{2 pi i xi x} d xi over the compact band |2 pi xi / n| <= b.
    phihat is evaluated at real xi by the same closed form as at integers (kb_phihat is only
    defined at integers, so the band integral is done with scipy on the formula's I0 factor,
    cross-checked against kb_phihat at the integer points)."""
    b = oracle.kb_b(n, N)

    def phihat_real(xi):
        s = b * b - (2 * np.pi * xi / n) ** 2
        return special.i0(m * np.sqrt(max(s, 0.0))) / n

    for k in range(-N // 2, N // 2, 7):
        assert oracle.kb_phihat(k, n, m, b) == pytest.approx(phihat_real(k), rel=1e-13)

    xi_max = b * n / (2 * np.pi)
    for t in [0.0, 0.3, 1.0, m - 1.5, m - 0.2, m - 1e-9]:
        x = t / n
        val, _ = integrate.quad(lambda xi: phihat_real(xi) * np.cos(2 * np.pi * xi * x),
                                -xi_max, xi_max, limit=400, epsabs=0, epsrel=1e-13)
        # quadrature of an integrand of size ~psi(0) leaves an absolute error ~1e-13 psi(0)
        peak = oracle.kb_psi(0.0, m, b)
        assert oracle.kb_psi(t, m, b) == pytest.approx(val, rel=1e-9, abs=1e-12 * peak), (t, m)
        assert oracle.kb_psi(-t, m, b) == oracle.kb_psi(t, m, b)


@pytest.mark.parametrize("m", [2, 4, 8])
def test_kb_truncation_and_edge(m):
    b = oracle.kb_b(1024, 512)
    assert oracle.kb_psi(m + 1e-12, m, b) == 0.0
    assert oracle.kb_psi(-m - 1e-9, m, b) == 0.0
    # limit of sinh(b u)/(pi u) as u -> 0 is b/pi
    assert oracle.kb_psi(float(m), m, b) == pytest.approx(b / np.pi, rel=1e-15)
    assert oracle.kb_psi(m - 1e-12, m, b) == pytest.approx(b / np.pi, rel=1e-9)


@pytest.mark.parametrize("m", [2, 4, 6])
def test_kb_derivative_matches_finite_difference(m):
    b = oracle.kb_b(512, 256)
    h = 1e-6
    for t in np.linspace(-m + 1e-3, m - 1e-3, 37):
        fd = (oracle.kb_psi(t + h, m, b) - oracle.kb_psi(t - h, m, b)) / (2 * h)
        scale = oracle.kb_psi(0.0, m, b)
        assert abs(oracle.kb_dpsi(t, m, b) - fd) <= 1e-7 * scale, t
    # the Taylor branch near the edge agrees with the direct formula where both are accurate
    t_edge = m - 1e-7
    t_mid = m - 1e-3
    assert oracle.kb_dpsi(0.0, m, b) == 0.0
    assert np.sign(oracle.kb_dpsi(t_edge, m, b)) == -1
    assert np.sign(oracle.kb_dpsi(-t_mid, m, b)) == 1
    assert oracle.kb_dpsi(m + 0.1, m, b) == 0.0


def test_kb_dpsi_taylor_branch_continuity():
    m, b = 4, oracle.kb_b(1024, 512)
    # u = sqrt(m^2 - t^2) crosses b u = 1e-2 at u = 1e-2/b; compare both sides
    u0 = 1e-2 / b
    for eps in [-1e-7, 1e-7]:
        u = u0 * (1 + eps)
        t = np.sqrt(m * m - u * u)
        z = b * u
        direct = -t * (z * np.cosh(z) - np.sinh(z)) / (u ** 3) / np.pi
        assert oracle.kb_dpsi(t, m, b) == pytest.approx(direct, rel=1e-6)
