"""Host-side checks of the C ABI (no GPU needed): the library builds and loads, exports every
function include/gbnfft.h declares, and rejects invalid plans before touching the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gbnfft.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1810_09891_gb300 import _lib, build_lib
    build_lib.build()
    return _lib.lib()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(nfft_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["nfft_plan_create", "nfft_set_nodes", "nfft_trafo", "nfft_adjoint",
                 "nfft_destroy", "nfft_grad_x", "nfft_status", "nfft_workspace_size",
                 "nfft_set_workspace", "nfft_set_stream", "nfft_strerror",
                 "nfft_batch_create", "nfft_batch_trafo", "nfft_batch_adjoint",
                 "nfft_batch_destroy"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1810_09891_gb300._lib import SIGNATURES
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in SIGNATURES, name


def test_strerror(lib):
    for code in range(8):
        assert len(lib.nfft_strerror(code)) > 0
    assert lib.nfft_strerror(99) == b"unknown error"


def _create(lib, d, N, M, n=None, m=4, dtype=0):
    h = ctypes.c_void_p()
    Nv = (ctypes.c_int64 * 3)(*(list(N) + [0] * (3 - len(N))))
    nv = None if n is None else (ctypes.c_int64 * 3)(*(list(n) + [0] * (3 - len(n))))
    return lib.nfft_plan_create(ctypes.byref(h), d, Nv, M, nv, m, dtype)


@pytest.mark.parametrize("args,code", [
    (dict(d=0, N=(8,), M=1), 1),             # d out of range
    (dict(d=4, N=(8, 8, 8), M=1), 1),
    (dict(d=1, N=(7,), M=1), 1),             # odd N
    (dict(d=1, N=(0,), M=1), 1),
    (dict(d=1, N=(8,), M=-1), 1),            # negative M
    (dict(d=1, N=(8,), M=1, n=(8,)), 1),     # n <= N
    (dict(d=1, N=(8,), M=1, n=(15,)), 1),    # odd n
    (dict(d=1, N=(8,), M=1, n=(16,), m=8), 1),   # 2m + 2 > n
    (dict(d=1, N=(8,), M=1, dtype=2), 1),    # bad dtype
    (dict(d=1, N=(8,), M=1, n=(4098,)), 7),  # even n, not a power of two, beyond 4096 (FP32)
    (dict(d=1, N=(8,), M=1, n=(2050,), dtype=1), 7),  # ... beyond 2048 (FP64)
    (dict(d=1, N=(8,), M=1, n=(64,), m=9), 7),   # m > 8
    (dict(d=1, N=(8192,), M=1, n=(32768,)), 7),  # n beyond the in-shared-memory FFT
])
def test_plan_validation(lib, args, code):
    a = dict(n=None, m=4, dtype=0)
    a.update(args)
    assert _create(lib, a["d"], a["N"], a["M"], a["n"], a["m"], a["dtype"]) == code


def test_null_arguments(lib):
    assert lib.nfft_plan_create(None, 1, None, 1, None, 4, 0) == 1
    assert lib.nfft_destroy(None) == 0
    assert lib.nfft_trafo(None, None, None) == 1
    assert lib.nfft_adjoint(None, None, None) == 1
    assert lib.nfft_set_nodes(None, None) == 1
    assert lib.nfft_status(None) == 1
    # batches: argument checks come before any CUDA call
    b = ctypes.c_void_p()
    nulls = (ctypes.c_void_p * 2)(None, None)
    assert lib.nfft_batch_create(None, None, 1, 0) == 1
    assert lib.nfft_batch_create(ctypes.byref(b), None, 1, 0) == 1
    assert lib.nfft_batch_create(ctypes.byref(b), ctypes.cast(nulls, ctypes.c_void_p), 0, 0) == 1
    assert lib.nfft_batch_create(ctypes.byref(b), ctypes.cast(nulls, ctypes.c_void_p), 2, 0) == 1
    assert not b.value
    assert lib.nfft_batch_destroy(None) == 1
    assert lib.nfft_batch_set_stream(None, None) == 1
    assert lib.nfft_batch_size(None, None, None) == 1
    assert lib.nfft_batch_lane(None, 0) == -1
    assert lib.nfft_batch_trafo(None, None, None) == 1
    assert lib.nfft_batch_adjoint(None, None, None) == 1
    assert lib.nfft_batch_grad_x(None, None, None, None) == 1


def test_plain_c_consumer_compiles_and_links(tmp_path):
    """include/gbnfft.h is plain C: a C11 program using it compiles and links against the
    library (running it needs a GPU: tests/test_gpu_c_consumer.py)."""
    import shutil
    import subprocess
    from paper_1810_09891_gb300 import _lib
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None or not os.path.exists(_lib.LIB_PATH):
        pytest.skip("no C compiler or library not built")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    exe = str(tmp_path / "abi_consumer")
    subprocess.run([cc, "-O2", "-std=c11", "-Wall", "-Werror",
                    os.path.join(root, "tests", "c", "abi_consumer.c"),
                    "-I", os.path.join(root, "include"), _lib.LIB_PATH, "-lm", "-o", exe],
                   check=True)
    assert os.path.exists(exe)
