"""FP64 CPU oracle for the NFFT (arXiv 1810.09891, Sections 1-2).

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline leg (``bench.py``, ``cpu_baseline`` and ``--impl reference``) may import this
package. The CUDA library never calls it, and it shares no code with the CUDA library.

Two independent references live here:

* O-direct: the NDFT of Section 1 (eq. NDFT) and its adjoint, summed term by term.
* O-nfft: Algorithm "NFFT" and Algorithm "adjoint NFFT" of Section 2, step by step (D, FFT, B
  and B^H, inverse FFT, D^H) with the Kaiser-Bessel window.

The arithmetic is plain C (``nfft_oracle.c``) compiled with gcc; this module only marshals numpy
arrays. All arrays are FP64 / complex128. Layouts:

* ``x``: (M, d) nodes; ``fhat``: shape N (row-major, index k_t + N_t/2 on axis t);
* ``g``: shape n (row-major, natural FFT order, index l_t mod n_t).

Every function listed here is pinned by a ``-m "not gpu"`` test in ``tests/test_oracle_*.py``
against something other than itself (closed forms, numpy/scipy, the paper's printed errors,
finite differences, dense matrices).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nfft_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``nfft_oracle.c`` into ``liboracle.so`` (gcc, OpenMP, no FP contraction)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        I64 = ctypes.c_int64
        D = ctypes.c_double
        Int = ctypes.c_int
        sigs = {
            "ora_version": ([], Int),
            "ora_max_threads": ([], Int),
            "ora_set_threads": ([Int], Int),
            "ora_ndft_tab": ([Int, P, I64, P, P, P], None),
            "ora_ndft_adjoint_at": ([Int, P, I64, P, P, I64, P, P], None),
            "ora_ndft": ([Int, P, I64, P, P, P], None),
            "ora_ndft_adjoint": ([Int, P, I64, P, P, P], None),
            "ora_ndft_grad": ([Int, P, I64, P, P, P], None),
            "ora_bessel_i0": ([D], D),
            "ora_kb_b": ([I64, I64], D),
            "ora_kb_psi": ([D, Int, D], D),
            "ora_kb_dpsi": ([D, Int, D], D),
            "ora_kb_phihat": ([I64, I64, Int, D], D),
            "ora_fft": ([Int, P, P, Int], None),
            "ora_nfft_D": ([Int, P, P, Int, P, P], None),
            "ora_nfft_DH": ([Int, P, P, Int, P, P], None),
            "ora_nfft_B": ([Int, P, P, Int, I64, P, P, P], None),
            "ora_nfft_BH": ([Int, P, P, Int, I64, P, P, P], None),
            "ora_nfft_dB": ([Int, P, P, Int, I64, P, P, P], None),
            "ora_nfft": ([Int, P, P, Int, I64, P, P, P], Int),
            "ora_nfft_adjoint": ([Int, P, P, Int, I64, P, P, P], Int),
            "ora_nfft_grad_x": ([Int, P, P, Int, I64, P, P, P, P], Int),
            "ora_bspline": ([Int, D], D),
            "ora_window_param": ([Int, I64, I64, Int], D),
            "ora_window_psi": ([Int, D, Int, D], D),
            "ora_window_dpsi": ([Int, D, Int, D], D),
            "ora_window_psi_eval": ([Int, D, Int, D], D),
            "ora_window_dpsi_eval": ([Int, D, Int, D], D),
            "ora_window_phihat": ([Int, I64, I64, Int, D], D),
            "ora_nfft_D_w": ([Int, Int, P, P, Int, P, P], None),
            "ora_nfft_DH_w": ([Int, Int, P, P, Int, P, P], None),
            "ora_nfft_B_w": ([Int, Int, P, P, Int, I64, P, P, P], None),
            "ora_nfft_BH_w": ([Int, Int, P, P, Int, I64, P, P, P], None),
            "ora_nfft_dB_w": ([Int, Int, P, P, Int, I64, P, P, P], None),
            "ora_nfft_w": ([Int, Int, P, P, Int, I64, P, P, P], Int),
            "ora_nfft_adjoint_w": ([Int, Int, P, P, Int, I64, P, P, P], Int),
            "ora_nfft_grad_x_w": ([Int, Int, P, P, Int, I64, P, P, P, P], Int),
        }
        for name, (argt, rest) in sigs.items():
            fn = getattr(lib, name)
            fn.argtypes = argt
            fn.restype = rest
        _lib = lib
        return lib


WINDOWS = {"kaiser_bessel": 0, "gaussian": 1, "bspline": 2, "sinc": 3}


def _win(window, lin_psi: int = 0) -> int:
    """Window spec of the C oracle: the window kind in the low 8 bits, the lookup-table size K
    (samples per unit of t, 0 = the exact window) above them."""
    kind = window if isinstance(window, int) else WINDOWS[window]
    K = int(lin_psi)
    if K < 0 or K >= (1 << 22):
        raise ValueError("lin_psi must be in [0, 2^22)")
    return int(kind) | (K << 8)


def _i64(v) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(v, dtype=np.int64).reshape(-1))


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.complex128))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _nodes(x, d: int) -> np.ndarray:
    x = _f64(x).reshape(-1, d)
    return x


def default_n(N) -> tuple:
    """Default oversampled FFT length n_t = 2^(ceil(log2 N_t) + 1) (Section 2, after eq. gl)."""
    return tuple(int(2 ** (int(np.ceil(np.log2(int(v)))) + 1)) for v in N)


def max_threads() -> int:
    return int(_load().ora_max_threads())


# ------------------------------------------------------------------------------------ window

def bessel_i0(z: float) -> float:
    return float(_load().ora_bessel_i0(float(z)))


def kb_b(n: int, N: int) -> float:
    return float(_load().ora_kb_b(int(n), int(N)))


def kb_psi(t: float, m: int, b: float) -> float:
    return float(_load().ora_kb_psi(float(t), int(m), float(b)))


def kb_dpsi(t: float, m: int, b: float) -> float:
    return float(_load().ora_kb_dpsi(float(t), int(m), float(b)))


def kb_phihat(k: int, n: int, m: int, b: float) -> float:
    return float(_load().ora_kb_phihat(int(k), int(n), int(m), float(b)))


def bspline(p: int, t: float) -> float:
    """Centred cardinal B-spline of order p."""
    return float(_load().ora_bspline(int(p), float(t)))


def window_param(window, n: int, N: int, m: int) -> float:
    return float(_load().ora_window_param(_win(window), int(n), int(N), int(m)))


def window_psi(window, t: float, m: int, prm: float) -> float:
    return float(_load().ora_window_psi(_win(window), float(t), int(m), float(prm)))


def window_dpsi(window, t: float, m: int, prm: float) -> float:
    return float(_load().ora_window_dpsi(_win(window), float(t), int(m), float(prm)))


def window_psi_eval(window, t: float, m: int, prm: float, lin_psi: int = 0) -> float:
    """psi(t) as steps B, B^H use it: exact, or from the K-point lookup table (lin_psi = K)."""
    return float(_load().ora_window_psi_eval(_win(window, lin_psi), float(t), int(m), float(prm)))


def window_dpsi_eval(window, t: float, m: int, prm: float, lin_psi: int = 0) -> float:
    return float(_load().ora_window_dpsi_eval(_win(window, lin_psi), float(t), int(m), float(prm)))


def window_phihat(window, k: int, n: int, m: int, prm: float) -> float:
    return float(_load().ora_window_phihat(_win(window), int(k), int(n), int(m), float(prm)))


# ------------------------------------------------------------------------------------ direct

def ndft(x, fhat) -> np.ndarray:
    """f_j = sum_{k in I_N} fhat_k exp(-2 pi i k.x_j) (Section 1, eq. NDFT)."""
    fhat = _c128(fhat)
    d = fhat.ndim
    N = _i64(fhat.shape)
    x = _nodes(x, d)
    M = x.shape[0]
    f = np.zeros(M, dtype=np.complex128)
    _load().ora_ndft(d, _p(N), M, _p(x), _p(fhat), _p(f))
    return f


def ndft_adjoint(x, f, N) -> np.ndarray:
    """hhat_k = sum_j f_j exp(+2 pi i k.x_j), k in I_N (Section 1)."""
    N = tuple(int(v) for v in N)
    d = len(N)
    x = _nodes(x, d)
    f = _c128(f).reshape(-1)
    out = np.zeros(N, dtype=np.complex128)
    _load().ora_ndft_adjoint(d, _p(_i64(N)), x.shape[0], _p(x), _p(f), _p(out))
    return out


def ndft_tab(x, fhat) -> np.ndarray:
    """The NDFT of Section 1 (eq. NDFT) with every term's exponential formed from its per-axis
    factors e^{-2 pi i k_t x_t} (a node's factors are computed once): the same sum as ``ndft``,
    much faster for large |I_N|."""
    fhat = _c128(fhat)
    d = fhat.ndim
    N = _i64(fhat.shape)
    x = _nodes(x, d)
    M = x.shape[0]
    f = np.zeros(M, dtype=np.complex128)
    _load().ora_ndft_tab(d, _p(N), M, _p(x), _p(fhat), _p(f))
    return f


def ndft_adjoint_at(x, f, N, kidx) -> np.ndarray:
    """The adjoint NDFT (Section 1) at selected coefficients: sum_j f_j exp(+2 pi i k.x_j) for
    the multi-indices k at row-major positions ``kidx`` of I_N (axis t at k_t + N_t/2)."""
    N = tuple(int(v) for v in N)
    d = len(N)
    x = _nodes(x, d)
    f = _c128(f).reshape(-1)
    kidx = _i64(kidx)
    if kidx.size and (kidx.min() < 0 or kidx.max() >= int(np.prod(N))):
        raise ValueError("kidx outside I_N")
    out = np.zeros(kidx.size, dtype=np.complex128)
    _load().ora_ndft_adjoint_at(d, _p(_i64(N)), x.shape[0], _p(x), _p(f), kidx.size, _p(kidx),
                                _p(out))
    return out


def set_threads(n: int) -> int:
    """OpenMP threads of later oracle calls; returns the number in effect."""
    return int(_load().ora_set_threads(int(n)))


def ndft_grad(x, fhat) -> np.ndarray:
    """(M, d) complex: d f / d x_t at x_j = sum_k (-2 pi i k_t) fhat_k exp(-2 pi i k.x_j)."""
    fhat = _c128(fhat)
    d = fhat.ndim
    x = _nodes(x, d)
    df = np.zeros((x.shape[0], d), dtype=np.complex128)
    _load().ora_ndft_grad(d, _p(_i64(fhat.shape)), x.shape[0], _p(x), _p(fhat), _p(df))
    return df


# ------------------------------------------------------------------------------------ FFT

def fft(a, sign: int = -1) -> np.ndarray:
    """Unnormalised d-variate DFT, sum_k a_k exp(sign 2 pi i k.l/n)."""
    a = _c128(a).copy()
    _load().ora_fft(a.ndim, _p(_i64(a.shape)), _p(a), int(sign))
    return a


# ------------------------------------------------------------------------------------ NFFT steps

def nfft_D(fhat, n, m: int, window="kaiser_bessel") -> np.ndarray:
    fhat = _c128(fhat)
    n = tuple(int(v) for v in n)
    g = np.zeros(n, dtype=np.complex128)
    _load().ora_nfft_D_w(_win(window), fhat.ndim, _p(_i64(fhat.shape)), _p(_i64(n)), int(m),
                         _p(fhat), _p(g))
    return g


def nfft_DH(ghat, N, m: int, window="kaiser_bessel") -> np.ndarray:
    ghat = _c128(ghat)
    N = tuple(int(v) for v in N)
    out = np.zeros(N, dtype=np.complex128)
    _load().ora_nfft_DH_w(_win(window), ghat.ndim, _p(_i64(N)), _p(_i64(ghat.shape)), int(m),
                          _p(ghat), _p(out))
    return out


def nfft_B(x, g, N, m: int, window="kaiser_bessel", lin_psi: int = 0) -> np.ndarray:
    g = _c128(g)
    d = g.ndim
    x = _nodes(x, d)
    f = np.zeros(x.shape[0], dtype=np.complex128)
    _load().ora_nfft_B_w(_win(window, lin_psi), d, _p(_i64(N)), _p(_i64(g.shape)), int(m), x.shape[0],
                         _p(x), _p(g), _p(f))
    return f


def nfft_BH(x, f, N, n, m: int, window="kaiser_bessel", lin_psi: int = 0) -> np.ndarray:
    n = tuple(int(v) for v in n)
    d = len(n)
    x = _nodes(x, d)
    f = _c128(f).reshape(-1)
    g = np.zeros(n, dtype=np.complex128)
    _load().ora_nfft_BH_w(_win(window, lin_psi), d, _p(_i64(N)), _p(_i64(n)), int(m), x.shape[0], _p(x),
                          _p(f), _p(g))
    return g


def nfft_dB(x, g, N, m: int, window="kaiser_bessel", lin_psi: int = 0) -> np.ndarray:
    g = _c128(g)
    d = g.ndim
    x = _nodes(x, d)
    ds = np.zeros((x.shape[0], d), dtype=np.complex128)
    _load().ora_nfft_dB_w(_win(window, lin_psi), d, _p(_i64(N)), _p(_i64(g.shape)), int(m), x.shape[0],
                          _p(x), _p(g), _p(ds))
    return ds


# ------------------------------------------------------------------------------------ NFFT

def nfft(x, fhat, n=None, m: int = 8, window="kaiser_bessel", lin_psi: int = 0) -> np.ndarray:
    """Algorithm "NFFT" (Section 2): f = B F D fhat."""
    fhat = _c128(fhat)
    d = fhat.ndim
    n = default_n(fhat.shape) if n is None else tuple(int(v) for v in n)
    x = _nodes(x, d)
    f = np.zeros(x.shape[0], dtype=np.complex128)
    rc = _load().ora_nfft_w(_win(window, lin_psi), d, _p(_i64(fhat.shape)), _p(_i64(n)), int(m),
                            x.shape[0], _p(x), _p(fhat), _p(f))
    if rc:
        raise MemoryError("oracle nfft: allocation failed")
    return f


def nfft_adjoint(x, f, N, n=None, m: int = 8, window="kaiser_bessel", lin_psi: int = 0) -> np.ndarray:
    """Algorithm "adjoint NFFT" (Section 2): hhat = D^H F^H B^H f."""
    N = tuple(int(v) for v in N)
    d = len(N)
    n = default_n(N) if n is None else tuple(int(v) for v in n)
    x = _nodes(x, d)
    f = _c128(f).reshape(-1)
    out = np.zeros(N, dtype=np.complex128)
    rc = _load().ora_nfft_adjoint_w(_win(window, lin_psi), d, _p(_i64(N)), _p(_i64(n)), int(m),
                                    x.shape[0], _p(x), _p(f), _p(out))
    if rc:
        raise MemoryError("oracle nfft_adjoint: allocation failed")
    return out


def nfft_grad_x(x, c, w, n=None, m: int = 8, window="kaiser_bessel", lin_psi: int = 0) -> np.ndarray:
    """(M, d) real: Re(conj(w_j) d s_c/d x_t (x_j)), s_c the NFFT approximation built from c."""
    c = _c128(c)
    d = c.ndim
    n = default_n(c.shape) if n is None else tuple(int(v) for v in n)
    x = _nodes(x, d)
    w = _c128(w).reshape(-1)
    gx = np.zeros((x.shape[0], d), dtype=np.float64)
    rc = _load().ora_nfft_grad_x_w(_win(window, lin_psi), d, _p(_i64(c.shape)), _p(_i64(n)), int(m),
                                   x.shape[0], _p(x), _p(c), _p(w), _p(gx))
    if rc:
        raise MemoryError("oracle nfft_grad_x: allocation failed")
    return gx


# ------------------------------------------------------------------------------------ errors

def error_E2(f_exact, f_approx) -> float:
    """Relative l2 error E_2 = ||f - f~||_2 / ||f||_2 (Section 2, eq. E2)."""
    f_exact = np.asarray(f_exact).reshape(-1)
    f_approx = np.asarray(f_approx).reshape(-1)
    return float(np.linalg.norm(f_exact - f_approx) / np.linalg.norm(f_exact))


def error_Einf(f_exact, f_approx, fhat) -> float:
    """E_inf = ||f - f~||_inf / ||fhat||_1 (Section 2, eq. EI)."""
    f_exact = np.asarray(f_exact).reshape(-1)
    f_approx = np.asarray(f_approx).reshape(-1)
    return float(np.max(np.abs(f_exact - f_approx)) / np.sum(np.abs(np.asarray(fhat))))
