"""Pins for the oracle's FFT and direct transforms (Section 1, eq. NDFT and its adjoint).

Checked against numpy.fft (a library routine the oracle does not call), closed forms, a value
worked out by hand, the equispaced special case and the adjoint identity.
"""
import numpy as np
import pytest

import oracle
from paper_1810_09891_gb300 import workloads as W


@pytest.mark.parametrize("shape", [(8,), (12,), (30,), (64,), (6, 10), (16, 8), (4, 6, 8),
                                   (8, 8, 16)])
@pytest.mark.parametrize("sign", [-1, 1])
def test_fft_matches_numpy(shape, sign):
    g = np.random.default_rng(3)
    a = g.standard_normal(shape) + 1j * g.standard_normal(shape)
    ref = np.fft.fftn(a) if sign == -1 else np.fft.ifftn(a) * a.size
    out = oracle.fft(a, sign)
    assert np.max(np.abs(out - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_ndft_hand_values():
    # N = 2: f(x) = fhat_{-1} e^{+2 pi i x} + fhat_0.
    fh = np.array([1 + 2j, 3 - 1j])
    x = np.array([0.25, -0.5, 0.0])
    want = np.array([(1 + 2j) * 1j + (3 - 1j), (1 + 2j) * (-1) + (3 - 1j), (1 + 2j) + (3 - 1j)])
    assert np.allclose(oracle.ndft(x, fh), want, atol=1e-15, rtol=0)
    # N = 4, x = 1/8: e^{-2 pi i k/8} for k = -2..1 is (i, e^{i pi/4}, 1, e^{-i pi/4}).
    fh = np.array([1.0, 2.0, 3.0, 4.0], dtype=complex)
    r = np.sqrt(0.5)
    want = 1 * 1j + 2 * (r + 1j * r) + 3 + 4 * (r - 1j * r)
    assert oracle.ndft(np.array([0.125]), fh)[0] == pytest.approx(want, abs=1e-14)
    # d = 2, N = (2, 2), x = (1/4, 1/2): f = sum fhat_k e^{-2 pi i (k0/4 + k1/2)}.
    fh = np.array([[1, 2], [3, 4]], dtype=complex)  # k0 in {-1, 0}, k1 in {-1, 0}
    # (k0,k1) = (-1,-1): e^{+2pi i (1/4 + 1/2)} = e^{i 3pi/2} = -i ; (-1,0): e^{i pi/2} = i
    # (0,-1): e^{i pi} = -1 ; (0,0): 1
    want = 1 * (-1j) + 2 * 1j + 3 * (-1) + 4
    assert oracle.ndft(np.array([[0.25, 0.5]]), fh)[0] == pytest.approx(want, abs=1e-14)


@pytest.mark.parametrize("N", [(16,), (8, 6), (4, 6, 8)])
def test_ndft_single_coefficient_closed_form(N):
    d = len(N)
    x = W.uniform_nodes(40, d, 11)
    g = np.random.default_rng(5)
    for _ in range(3):
        k = [int(g.integers(-v // 2, v // 2)) for v in N]
        fh = np.zeros(N, dtype=complex)
        fh[tuple(kk + v // 2 for kk, v in zip(k, N))] = 1.0
        want = np.exp(-2j * np.pi * (x @ np.array(k, dtype=float)))
        assert np.max(np.abs(oracle.ndft(x, fh) - want)) < 1e-14


@pytest.mark.parametrize("N", [(16,), (8, 6), (4, 6, 8)])
def test_ndft_adjoint_single_node_closed_form(N):
    d = len(N)
    x = W.uniform_nodes(1, d, 12)
    fj = 0.7 - 0.2j
    got = oracle.ndft_adjoint(x, np.array([fj]), N)
    ks = np.meshgrid(*W.centred_k(N), indexing="ij")
    phase = sum(kk * x[0, t] for t, kk in enumerate(ks))
    assert np.max(np.abs(got - fj * np.exp(2j * np.pi * phase))) < 1e-14


def test_ndft_at_origin_sums_coefficients():
    for N in [(10,), (4, 8), (2, 4, 6)]:
        fh = np.ones(N, dtype=complex)
        assert oracle.ndft(np.zeros((1, len(N))), fh)[0] == pytest.approx(np.prod(N), abs=1e-12)


@pytest.mark.parametrize("Nv", [8, 16, 64])
def test_ndft_equispaced_nodes_reduce_to_fft(Nv):
    """x_j = j/N - 1/2 gives f_j = sum_k fhat_k (-1)^k e^{-2 pi i k j / N}, i.e. numpy's FFT of
    the coefficients multiplied by (-1)^k and moved to natural order."""
    g = np.random.default_rng(2)
    fh = g.standard_normal(Nv) + 1j * g.standard_normal(Nv)
    k = np.arange(-Nv // 2, Nv // 2)
    x = np.arange(Nv) / Nv - 0.5
    nat = np.zeros(Nv, dtype=complex)
    nat[k % Nv] = fh * (-1.0) ** k
    want = np.fft.fft(nat)
    assert np.max(np.abs(oracle.ndft(x, fh) - want)) < 1e-12
    # the 2-D version: tensor product of the 1-D mapping
    fh2 = g.standard_normal((Nv, 8)) + 1j * g.standard_normal((Nv, 8))
    k0 = np.arange(-Nv // 2, Nv // 2)[:, None]
    k1 = np.arange(-4, 4)[None, :]
    nat2 = np.zeros((Nv, 8), dtype=complex)
    nat2[np.ix_(np.arange(-Nv // 2, Nv // 2) % Nv, np.arange(-4, 4) % 8)] = fh2 * (-1.0) ** (k0 + k1)
    want2 = np.fft.fft2(nat2)
    xx = np.stack(np.meshgrid(np.arange(Nv) / Nv - 0.5, np.arange(8) / 8 - 0.5, indexing="ij"),
                  axis=-1).reshape(-1, 2)
    assert np.max(np.abs(oracle.ndft(xx, fh2) - want2.reshape(-1))) < 1e-11


@pytest.mark.parametrize("N", [(12,), (6, 8), (4, 4, 6)])
def test_ndft_adjoint_identity(N):
    d = len(N)
    g = np.random.default_rng(9)
    x = W.uniform_nodes(30, d, 13)
    fh = g.standard_normal(N) + 1j * g.standard_normal(N)
    f = g.standard_normal(30) + 1j * g.standard_normal(30)
    lhs = np.vdot(oracle.ndft(x, fh), f)
    rhs = np.vdot(fh.reshape(-1), oracle.ndft_adjoint(x, f, N).reshape(-1))
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


def test_ndft_periodic_in_nodes():
    N = (8, 6)
    x = W.uniform_nodes(20, 2, 14)
    fh = W.gaussian_fhat(N, 3)
    assert np.max(np.abs(oracle.ndft(x + np.array([1.0, -2.0]), fh) - oracle.ndft(x, fh))) < 1e-12


@pytest.mark.parametrize("N", [(16,), (6, 8), (4, 4, 6)])
def test_ndft_grad_matches_finite_difference(N):
    d = len(N)
    x = W.uniform_nodes(12, d, 15)
    fh = W.gaussian_fhat(N, 4)
    df = oracle.ndft_grad(x, fh)
    h = 1e-6
    for t in range(d):
        e = np.zeros(d)
        e[t] = h
        fd = (oracle.ndft(x + e, fh) - oracle.ndft(x - e, fh)) / (2 * h)
        assert np.max(np.abs(df[:, t] - fd)) <= 1e-7 * np.max(np.abs(df[:, t]))


# ---------------------------------------------------------------- the faster direct sums
# ndft_tab and ndft_adjoint_at evaluate the same sums as ndft / ndft_adjoint with each term's
# exponential built from per-axis factors; they are what the GPU is checked against at full size.

@pytest.mark.parametrize("N", [(2,), (16,), (30,), (8, 6), (12, 10), (4, 6, 8), (6, 4, 10)])
def test_ndft_tab_closed_forms_and_direct_sum(N):
    d = len(N)
    x = W.uniform_nodes(60, d, 40) * 7.0  # nodes far outside the torus too
    g = np.random.default_rng(41)
    # single coefficient: a pure exponential
    k = [int(g.integers(-v // 2, v // 2)) for v in N]
    fh = np.zeros(N, dtype=complex)
    fh[tuple(kk + v // 2 for kk, v in zip(k, N))] = 1.0
    want = np.exp(-2j * np.pi * (x @ np.array(k, dtype=float)))
    assert np.max(np.abs(oracle.ndft_tab(x, fh) - want)) < 1e-13
    # x = 0 with fhat = 1 sums to |I_N|
    assert abs(oracle.ndft_tab(np.zeros((1, d)), np.ones(N))[0] - np.prod(N)) < 1e-12
    # a random polynomial: the plain direct sum
    fh = g.standard_normal(N) + 1j * g.standard_normal(N)
    ref = oracle.ndft(x, fh)
    assert np.max(np.abs(oracle.ndft_tab(x, fh) - ref)) <= 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("N", [(16,), (10, 8), (4, 6, 8)])
def test_ndft_adjoint_at_closed_form_and_direct_sum(N):
    d = len(N)
    g = np.random.default_rng(42)
    nk = int(np.prod(N))
    kidx = np.concatenate([[0, nk - 1], g.choice(nk, 9, replace=False)])
    # one node: hhat_k = f_j e^{+2 pi i k.x_j}
    x1 = W.uniform_nodes(1, d, 43)
    ks = np.stack(np.unravel_index(kidx, N), axis=1) - np.array(N) // 2
    want = (0.3 + 0.9j) * np.exp(2j * np.pi * (ks @ x1[0]))
    got = oracle.ndft_adjoint_at(x1, np.array([0.3 + 0.9j]), N, kidx)
    assert np.max(np.abs(got - want)) < 1e-14
    # many nodes (more than threads, ragged split): the plain adjoint sum at those indices
    x = W.uniform_nodes(1003, d, 44)
    f = g.standard_normal(1003) + 1j * g.standard_normal(1003)
    ref = oracle.ndft_adjoint(x, f, N).reshape(-1)[kidx]
    got = oracle.ndft_adjoint_at(x, f, N, kidx)
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))
    with pytest.raises(ValueError):
        oracle.ndft_adjoint_at(x, f, N, [nk])


@pytest.mark.parametrize("N,n,m", [((16, 12), (32, 32), 3), ((8, 6, 10), (16, 16, 32), 2),
                                   ((40,), (128,), 5)])
def test_spreading_is_the_same_with_any_thread_count(N, n, m):
    """The oracle's B^H splits the grid into per-thread slabs; every grid value still receives
    its terms in node order, so any thread count gives the same bits."""
    d = len(N)
    x = W.uniform_nodes(3001, d, 45)
    x[:40] = 0.0  # coincident nodes on a grid point
    f = W.gaussian_values(3001, 46)
    keep = oracle.max_threads()
    try:
        oracle.set_threads(1)
        one = oracle.nfft_BH(x, f, N, n, m)
        oracle.set_threads(5)
        five = oracle.nfft_BH(x, f, N, n, m)
    finally:
        oracle.set_threads(keep)
    assert np.array_equal(one, five)
