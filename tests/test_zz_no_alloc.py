"""The no-allocation entry point nfft_trafo_1d_noalloc, called through the C ABI.

It is meant for callers that cannot allocate device memory where they transform: their device
memory belongs to another allocator, or they run latency-bound loops that cannot take the
synchronisation of cudaMalloc / cudaFree. This test checks that it gives the same result as the
planned nfft_trafo, within the FP64 tolerance of the other parity tests, on calls in a row with
different sizes (the largest size its scratch allows first, so that the later calls run on scratch
an earlier call left behind), and that sizes beyond its fixed scratch are refused. This file is
collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1810_09891_gb300 import _lib
from paper_1810_09891_gb300 import workloads as W
from paper_1810_09891_gb300.nfft import Plan

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda", 0)
TOL_FP64 = 1e-12  # the FP64 parity tolerance used by the other GPU tests


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _noalloc(lib, N, x, fh, m, n=None):
    M = x.numel()
    out = torch.full((M,), complex("nan"), dtype=torch.complex128, device=DEV)
    nptr = None if n is None else ctypes.byref(ctypes.c_int64(n))
    stream = ctypes.c_void_p(torch.cuda.current_stream(DEV).cuda_stream)
    rc = lib.nfft_trafo_1d_noalloc(N, M, nptr, m, _p(x), _p(fh), _p(out), stream)
    return rc, out


def test_noalloc_matches_planned_forward_on_two_calls():
    torch.cuda.set_device(DEV)
    lib = _lib.lib()
    # the largest size the scratch holds (n = 8192, N = 4096) first, then smaller ones
    cases = [(4096, 2000, 8, 8192, 69), (512, 5000, 8, None, 70), (96, 1234, 4, 256, 71)]
    for N, M, m, n, seed in cases:
        x = torch.tensor(W.uniform_nodes(M, 1, seed_offset=seed).reshape(-1), device=DEV)
        fh = torch.tensor(W.gaussian_fhat((N,), seed_offset=seed + 1), device=DEV)
        rc, out = _noalloc(lib, N, x, fh, m, n)
        assert rc == 0, _lib.STATUS.get(rc, rc)
        plan = Plan((N,), M, n=None if n is None else (n,), m=m, dtype=torch.float64, device=DEV)
        plan.set_nodes(x.reshape(M, 1))
        ref = plan.trafo(fh)
        torch.cuda.synchronize()
        got, want = out.cpu().numpy(), ref.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.linalg.norm(got - want) / np.linalg.norm(want) <= TOL_FP64
        plan.close()


def test_noalloc_refuses_sizes_beyond_its_scratch():
    torch.cuda.set_device(DEV)
    lib = _lib.lib()
    x = torch.zeros(4, dtype=torch.float64, device=DEV)
    fh = torch.zeros(8192, dtype=torch.complex128, device=DEV)
    rc, _ = _noalloc(lib, 8192, x, fh, 4)  # default n = 16384 > 8192
    assert rc == 8  # NFFT_ESCRATCH
    assert b"fixed scratch" in lib.nfft_strerror(rc)
