"""Failure paths of the C ABI that need a device to reach (the host-side argument checks without
one are in test_abi.py): a caller workspace that is too small, device allocations that fail
(injected on the host with GBNFFT_FAIL_ALLOC, nothing faulty reaches the GPU), a plan listed twice
in a batch, and a plan that keeps working after each refusal."""
import ctypes
import os

import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import DEV, TOL, rel_l2
from paper_1810_09891_gb300 import _lib
from paper_1810_09891_gb300 import workloads as W
from paper_1810_09891_gb300.nfft import Plan

pytestmark = pytest.mark.gpu

ENOMEM, EINVAL, ENOTREADY = 2, 1, 4


@pytest.fixture
def fail_alloc():
    """Set GBNFFT_FAIL_ALLOC for the duration of one test."""
    old = os.environ.get("GBNFFT_FAIL_ALLOC")

    def set_sites(v):
        if v is None:
            os.environ.pop("GBNFFT_FAIL_ALLOC", None)
        else:
            os.environ["GBNFFT_FAIL_ALLOC"] = v
    yield set_sites
    set_sites(old)


def _raw_plan(lib, N, M, m=4, dtype=_lib.NFFT_FP64):
    h = ctypes.c_void_p()
    Nv = (ctypes.c_int64 * 3)(*(list(N) + [0] * (3 - len(N))))
    rc = lib.nfft_plan_create(ctypes.byref(h), len(N), Nv, M, None, m, dtype)
    return rc, h


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _inputs(N, M, seed):
    x = W.uniform_nodes(M, len(N), seed_offset=seed)
    fh = W.gaussian_fhat(N, seed_offset=seed + 1)
    return x, fh


def test_workspace_too_small_is_refused_and_plan_recovers():
    torch.cuda.set_device(DEV)
    lib = _lib.lib()
    N, M = (32, 48), 900
    rc, h = _raw_plan(lib, N, M)
    assert rc == 0
    need = ctypes.c_size_t()
    assert lib.nfft_workspace_size(h, ctypes.byref(need)) == 0
    ws = torch.empty(need.value, dtype=torch.uint8, device=DEV)
    # one byte short: refused, and the plan has no nodes yet
    assert lib.nfft_set_workspace(h, _p(ws), need.value - 1) == ENOMEM
    x, fh = _inputs(N, M, 300)
    xt = torch.tensor(x, device=DEV)
    fht = torch.tensor(fh, device=DEV)
    f = torch.empty(M, dtype=torch.complex128, device=DEV)
    assert lib.nfft_trafo(h, _p(fht), _p(f)) == ENOTREADY
    # the exact size works
    assert lib.nfft_set_workspace(h, _p(ws), need.value) == 0
    assert lib.nfft_set_nodes(h, _p(xt)) == 0
    assert lib.nfft_trafo(h, _p(fht), _p(f)) == 0
    assert lib.nfft_status(h) == 0
    ref = oracle.nfft(x, fh, n=(64, 128), m=4)  # default n_t = 2^(ceil(log2 N_t) + 1)
    assert rel_l2(f.cpu().numpy(), ref) <= TOL[torch.float64]
    # a larger bin grows the workspace past the caller's buffer: set_nodes reports it
    assert lib.nfft_set_option(h, _lib.OPT_BIN[0], 64) == 0
    need2 = ctypes.c_size_t()
    assert lib.nfft_workspace_size(h, ctypes.byref(need2)) == 0
    if need2.value > need.value:
        assert lib.nfft_set_nodes(h, _p(xt)) == ENOMEM
        assert lib.nfft_trafo(h, _p(fht), _p(f)) == ENOTREADY
    assert lib.nfft_destroy(h) == 0


def test_plan_tables_allocation_failure(fail_alloc):
    torch.cuda.set_device(DEV)
    lib = _lib.lib()
    fail_alloc("tables")
    rc, h = _raw_plan(lib, (16,), 10)
    assert rc == ENOMEM
    assert not h.value  # no plan handed out
    fail_alloc("workspace,stage")  # other sites do not affect plan creation
    rc, h = _raw_plan(lib, (16,), 10)
    assert rc == 0 and h.value
    assert lib.nfft_destroy(h) == 0


def test_own_workspace_allocation_failure(fail_alloc):
    torch.cuda.set_device(DEV)
    lib = _lib.lib()
    N, M = (24, 16, 8), 700
    rc, h = _raw_plan(lib, N, M)
    assert rc == 0
    x, fh = _inputs(N, M, 310)
    xt = torch.tensor(x, device=DEV)
    fht = torch.tensor(fh, device=DEV)
    f = torch.empty(M, dtype=torch.complex128, device=DEV)
    fail_alloc("workspace")  # no caller workspace: set_nodes allocates one itself
    assert lib.nfft_set_nodes(h, _p(xt)) == ENOMEM
    assert lib.nfft_trafo(h, _p(fht), _p(f)) == ENOTREADY
    fail_alloc(None)
    assert lib.nfft_set_nodes(h, _p(xt)) == 0
    assert lib.nfft_trafo(h, _p(fht), _p(f)) == 0
    assert lib.nfft_status(h) == 0
    n = (64, 32, 16)  # default n_t = 2^(ceil(log2 N_t) + 1)
    assert rel_l2(f.cpu().numpy(), oracle.nfft(x, fh, n=n, m=4)) <= TOL[torch.float64]
    assert lib.nfft_destroy(h) == 0


def test_host_staging_allocation_failure(fail_alloc):
    torch.cuda.set_device(DEV)
    N, M = (40,), 300
    x, fh = _inputs(N, M, 320)
    plan = Plan(N, M, m=5, dtype=torch.float64, device=DEV)
    fail_alloc("stage")
    with pytest.raises(_lib.NfftError, match="NFFT_ENOMEM"):
        plan.set_nodes_host(torch.tensor(x))
    fail_alloc(None)
    plan.set_nodes_host(torch.tensor(x))
    out = torch.empty(M, dtype=torch.complex128)
    plan.trafo_host(torch.tensor(fh), out)
    assert rel_l2(out.numpy(), oracle.nfft(x, fh, n=plan.n, m=5)) <= TOL[torch.float64]
    plan.close()


def test_window_table_allocation_failure_keeps_polynomial_window(fail_alloc):
    torch.cuda.set_device(DEV)
    N, M = (20, 20), 500
    x, fh = _inputs(N, M, 330)
    plan = Plan(N, M, m=4, dtype=torch.float64, device=DEV)
    plan.set_nodes(torch.tensor(x, device=DEV))
    fail_alloc("lin")
    with pytest.raises(_lib.NfftError, match="NFFT_ENOMEM"):
        plan.set_option("window_table", 4096)
    fail_alloc(None)
    assert plan.info()["window_table"] == 0
    f = plan.trafo(torch.tensor(fh, device=DEV)).cpu().numpy()
    assert rel_l2(f, oracle.nfft(x, fh, n=plan.n, m=4)) <= TOL[torch.float64]
    plan.close()


def test_batch_rejects_a_plan_listed_twice():
    torch.cuda.set_device(DEV)
    lib = _lib.lib()
    plans = [Plan((16, 16), 100, m=3, dtype=torch.float32, device=DEV) for _ in range(2)]
    arr = (ctypes.c_void_p * 3)(plans[0]._h, plans[1]._h, plans[0]._h)
    b = ctypes.c_void_p()
    assert lib.nfft_batch_create(ctypes.byref(b), ctypes.cast(arr, ctypes.c_void_p), 3, 0) \
        == EINVAL
    assert not b.value
    assert lib.nfft_batch_create(ctypes.byref(b), ctypes.cast(arr, ctypes.c_void_p), 2, 0) == 0
    assert lib.nfft_batch_destroy(b) == 0
    for p in plans:
        p.close()
