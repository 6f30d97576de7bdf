"""gbnfft: a nonequispaced fast Fourier transform for one NVIDIA GB300 GPU (sm_103a).

Implements the NFFT of Schmischke, "NFFT Interface for Julia" (arXiv 1810.09891), Section 2:
the forward transform f = B F D fhat (Algorithm "NFFT") and its adjoint D^H F^H B^H f
(Algorithm "adjoint NFFT") for d = 1, 2, 3 with the Kaiser-Bessel window, in FP32 and FP64,
behind the C ABI of ``include/gbnfft.h``. The modules:

* ``nfft``: ``Plan`` and the autograd functions ``nfft`` / ``nfft_adjoint``;
* ``_lib``: the ctypes loader of ``libgbnfft.so``;
* ``build_lib``: builds ``libgbnfft.so`` with nvcc;
* ``workloads``: seeded synthetic inputs shaped like the paper's workloads.

Importing the package does not load the CUDA library; the first ``Plan`` does, and raises if
it is missing.
"""
from __future__ import annotations

__all__ = ["Plan", "nfft", "nfft_adjoint"]


def __getattr__(name):
    if name in __all__:
        from . import nfft as _m
        return getattr(_m, name)
    raise AttributeError(name)
