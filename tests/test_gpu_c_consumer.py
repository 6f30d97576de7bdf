"""The C ABI used from plain C: tests/c/abi_consumer.c is compiled with gcc against
include/gbnfft.h and libgbnfft.so and run; it checks a 2-D FP64 forward and adjoint NFFT
(host-buffer entry points) against a direct NDFT it computes itself."""
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_plain_c_consumer(tmp_path):
    from paper_1810_09891_gb300 import _lib
    lib = _lib.LIB_PATH
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    exe = str(tmp_path / "abi_consumer")
    subprocess.run([cc, "-O2", "-std=c11", os.path.join(ROOT, "tests", "c", "abi_consumer.c"),
                    "-I", os.path.join(ROOT, "include"), lib, "-Wl,-rpath," + os.path.dirname(lib),
                    "-lm", "-o", exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    rf, rh = (float(v) for v in r.stdout.split())
    assert rf < 1e-9 and rh < 1e-9
