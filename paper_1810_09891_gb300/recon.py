"""Differentiable reconstruction with the NFFT: conjugate gradients on the normal equations.

Given samples y_j ~ f(x_j) of a trigonometric polynomial at nonequispaced nodes, the
least-squares coefficients solve A^H A fhat = A^H y, where A is the NFFT (Algorithm "NFFT") and
A^H its adjoint (Algorithm "adjoint NFFT"). ``cg_normal`` runs a fixed number of CG iterations
from fhat = 0. Every application of A and A^H goes through the autograd functions
``nfft`` / ``nfft_adjoint``, so the iterate is differentiable with respect to y and to the
node coordinates x (the node gradient uses the derivative-of-window kernel in both directions).
The vector arithmetic of CG (dot products, updates) is plain PyTorch on the plan's device.
"""
from __future__ import annotations

import torch

from .nfft import Plan, nfft, nfft_adjoint


def _dot(a: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
    """<a, b> = sum conj(a) b (complex scalar, differentiable)."""
    return torch.sum(torch.conj(a) * b)


def normal_op(v: torch.Tensor, x: torch.Tensor, plan: Plan) -> torch.Tensor:
    """A^H A v with the nodes x (both factors differentiable in v and x)."""
    return nfft_adjoint(nfft(v, x, plan), x, plan)


def cg_normal(y: torch.Tensor, x: torch.Tensor, plan: Plan, iters: int = 20,
              return_history: bool = False):
    """``iters`` conjugate-gradient iterations on A^H A fhat = A^H y from fhat = 0.

    y: (M,) complex samples; x: (M, d) nodes (may require grad); plan: an NFFT plan of matching
    N, M and precision. Returns fhat (shape N), and the list of residual norms ||r_k|| if
    ``return_history``. The iteration is the textbook one for a Hermitian positive
    semi-definite operator: alpha = <r, r> / <p, A^H A p>, beta = <r', r'> / <r, r>."""
    b = nfft_adjoint(y, x, plan)
    z = torch.zeros_like(b)
    r = b
    p = r
    rr = torch.real(_dot(r, r))
    hist = [float(torch.sqrt(rr).detach())] if return_history else None
    for _ in range(int(iters)):
        q = normal_op(p, x, plan)
        alpha = rr / torch.real(_dot(p, q))
        z = z + alpha * p
        r = r - alpha * q
        rr_new = torch.real(_dot(r, r))
        beta = rr_new / rr
        p = r + beta * p
        rr = rr_new
        if return_history:
            hist.append(float(torch.sqrt(rr).detach()))
    return (z, hist) if return_history else z
