"""GPU node gradients and autograd: the derivative-of-window kernel against the oracle's node
gradient, against central finite differences of the CUDA forward itself (FP64), and the FP32
gradients against FP64 analytic gradients."""
import numpy as np
import pytest
import torch

import oracle
from paper_1810_09891_gb300 import workloads as W
from paper_1810_09891_gb300.nfft import Plan, nfft, nfft_adjoint

from gpu_helpers import DEV, rel_l2, rounded, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N,m,M", [((64,), 6, 700), ((24, 20), 4, 3000), ((12, 10, 8), 3, 2500),
                                   ((16, 16, 16), 8, 600)])
def test_grad_x_matches_oracle(N, m, M):
    d = len(N)
    x = W.uniform_nodes(M, d, seed_offset=500 + M)
    c = W.gaussian_fhat(N, seed_offset=501)
    w = W.gaussian_values(M, seed_offset=502)
    plan = Plan(N, M, m=m, dtype=torch.float64, device=DEV)
    plan.set_nodes(to_dev(x, torch.float64))
    gx = plan.grad_x(to_dev(c, torch.float64), to_dev(w, torch.float64)).cpu().numpy()
    ref = oracle.nfft_grad_x(x, c, w, n=plan.n, m=m)
    assert rel_l2(gx, ref) <= 1e-11


@pytest.mark.parametrize("N,m", [((32,), 6), ((16, 12), 4), ((8, 6, 8), 3)])
def test_autograd_forward_finite_difference(N, m):
    """L = Re(<w, NFFT(fhat; x)>): dL/dx by autograd vs central differences of the CUDA forward
    (FP64, h = 1e-7, nodes whose support box changes under +-h are excluded)."""
    d = len(N)
    M = 300
    n = oracle.default_n(N)
    x = W.uniform_nodes(M, d, seed_offset=503)
    fh = W.gaussian_fhat(N, 504)
    w = W.gaussian_values(M, 505)
    plan = Plan(N, M, m=m, dtype=torch.float64, device=DEV)
    xt = to_dev(x, torch.float64).requires_grad_(True)
    fht = to_dev(fh, torch.float64).requires_grad_(True)
    wt = to_dev(w, torch.float64)
    loss = torch.real(torch.vdot(wt, nfft(fht, xt, plan)))
    loss.backward()
    gx = xt.grad.cpu().numpy()
    h = 1e-7
    with torch.no_grad():
        for t in range(d):
            e = np.zeros(d)
            e[t] = h
            fp = nfft(fht, to_dev(x + e, torch.float64), plan).cpu().numpy()
            fm = nfft(fht, to_dev(x - e, torch.float64), plan).cpu().numpy()
            fd = np.real(np.conj(w) * (fp - fm)) / (2 * h)
            ok = np.ones(M, dtype=bool)
            for y in (x + e, x - e):
                ok &= np.ceil(n[t] * y[:, t] - m) == np.ceil(n[t] * x[:, t] - m)
                ok &= np.floor(n[t] * y[:, t] + m) == np.floor(n[t] * x[:, t] + m)
            assert ok.sum() > M // 2
            err = np.abs(gx[ok, t] - fd[ok])
            assert np.max(err) <= 1e-6 * np.max(np.abs(gx[:, t]))
    # gradient with respect to fhat is the adjoint applied to w
    plan.set_nodes(to_dev(x, torch.float64))
    ref = plan.adjoint(wt).cpu().numpy()
    assert rel_l2(fht.grad.cpu().numpy(), ref) <= 1e-14


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_autograd_adjoint(dtype):
    """L = Re(<G, NFFT^H(f; x)>): grad f = NFFT(G), grad x = Re(conj(f) d s_G / dx)."""
    N, M, m = (20, 16), 2000, 4
    x = W.uniform_nodes(M, 2, seed_offset=506)
    f = W.gaussian_values(M, 507)
    G = W.gaussian_fhat(N, 508)
    plan = Plan(N, M, m=m, dtype=dtype, device=DEV)
    xt = to_dev(x, dtype).requires_grad_(True)
    ft = to_dev(f, dtype).requires_grad_(True)
    Gt = to_dev(G, dtype)
    loss = torch.real(torch.vdot(Gt.reshape(-1), nfft_adjoint(ft, xt, plan).reshape(-1)))
    loss.backward()
    xr, fr, Gr = rounded(x, dtype), rounded(f, dtype), rounded(G, dtype)
    ref_gf = oracle.nfft(xr, Gr, n=plan.n, m=m)
    ref_gx = oracle.nfft_grad_x(xr, Gr, fr, n=plan.n, m=m)
    tol = 1e-11 if dtype == torch.float64 else 1e-5
    assert rel_l2(ft.grad.cpu().numpy(), ref_gf) <= tol
    assert rel_l2(xt.grad.cpu().numpy(), ref_gx) <= tol


def test_fp32_gradients_against_fp64_analytic():
    """FP32 node and coefficient gradients vs the FP64 oracle on the same (rounded) inputs."""
    N, M, m = (32, 32, 32), 20000, 4
    x = W.round_nodes(W.clustered_nodes(M, 3, seed_offset=509), np.float32)
    fh = W.gaussian_fhat(N, 510)
    w = W.gaussian_values(M, 511)
    plan = Plan(N, M, m=m, dtype=torch.float32, device=DEV)
    xt = to_dev(x, torch.float32).requires_grad_(True)
    fht = to_dev(fh, torch.float32).requires_grad_(True)
    loss = torch.real(torch.vdot(to_dev(w, torch.float32), nfft(fht, xt, plan)))
    loss.backward()
    xr, fhr, wr = rounded(x, torch.float32), rounded(fh, torch.float32), rounded(w, torch.float32)
    ref_gx = oracle.nfft_grad_x(xr, fhr, wr, n=plan.n, m=m)
    ref_gf = oracle.nfft_adjoint(xr, wr, N, n=plan.n, m=m)
    assert rel_l2(xt.grad.cpu().numpy(), ref_gx) <= 1e-5
    assert rel_l2(fht.grad.cpu().numpy(), ref_gf) <= 1e-5


def test_node_gradient_against_ndft_derivative():
    """At m = 8 the NFFT derivative approaches the NDFT's analytic derivative
    d f/d x_t = sum_k (-2 pi i k_t) fhat_k e^{-2 pi i k.x} (window error times ~pi N)."""
    N, M, m = (32, 32), 400, 8
    x = W.uniform_nodes(M, 2, seed_offset=512)
    fh = W.gaussian_fhat(N, 513)
    w = W.gaussian_values(M, 514)
    plan = Plan(N, M, m=m, dtype=torch.float64, device=DEV)
    plan.set_nodes(to_dev(x, torch.float64))
    gx = plan.grad_x(to_dev(fh, torch.float64), to_dev(w, torch.float64)).cpu().numpy()
    ref = np.real(np.conj(w)[:, None] * oracle.ndft_grad(x, fh))
    assert rel_l2(gx, ref) <= 1e-10


def test_autograd_3d_clusters_finite_difference():
    """The 3-D clustered node distribution (half uniform, half in 8 Gaussian clusters): dL/dx by
    autograd against central differences of the CUDA forward in FP64, and dL/dfhat against the
    adjoint, for L = Re(<w, NFFT(fhat; x)>) (N = 16^3, m = 4)."""
    N, m, M = (16, 16, 16), 4, 3000
    n = oracle.default_n(N)
    x = W.clustered_nodes(M, 3, seed_offset=515)
    fh = W.gaussian_fhat(N, 516)
    w = W.gaussian_values(M, 517)
    plan = Plan(N, M, m=m, dtype=torch.float64, device=DEV)
    xt = to_dev(x, torch.float64).requires_grad_(True)
    fht = to_dev(fh, torch.float64).requires_grad_(True)
    wt = to_dev(w, torch.float64)
    torch.real(torch.vdot(wt, nfft(fht, xt, plan))).backward()
    gx = xt.grad.cpu().numpy()
    h = 1e-7
    with torch.no_grad():
        for t in range(3):
            e = np.zeros(3)
            e[t] = h
            fp = nfft(fht, to_dev(x + e, torch.float64), plan).cpu().numpy()
            fm = nfft(fht, to_dev(x - e, torch.float64), plan).cpu().numpy()
            fd = np.real(np.conj(w) * (fp - fm)) / (2 * h)
            ok = np.ones(M, dtype=bool)
            for y in (x + e, x - e):
                ok &= np.ceil(n[t] * y[:, t] - m) == np.ceil(n[t] * x[:, t] - m)
                ok &= np.floor(n[t] * y[:, t] + m) == np.floor(n[t] * x[:, t] + m)
            assert ok.sum() > M // 2
            assert np.max(np.abs(gx[ok, t] - fd[ok])) <= 1e-6 * np.max(np.abs(gx[:, t]))
    plan.set_nodes(to_dev(x, torch.float64))
    assert rel_l2(fht.grad.cpu().numpy(), plan.adjoint(wt).cpu().numpy()) <= 1e-14
