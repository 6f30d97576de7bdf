"""Python binding of the gbnfft C ABI: ``Plan`` plus ``torch.autograd`` functions.

Everything here is argument marshalling: tensors are checked, outputs are allocated with torch on
the plan's device, and the pointers plus the current CUDA stream are handed to ``libgbnfft.so``.
Every step of the transform runs in the library's CUDA kernels.

Conventions (Section 1 and 2 of the paper):

* forward  ``f = plan.trafo(fhat)``:    f_j ~ sum_{k in I_N} fhat_k exp(-2 pi i k.x_j)
* adjoint  ``h = plan.adjoint(f)``:     h_k ~ sum_j f_j exp(+2 pi i k.x_j)
* ``fhat`` has shape N (axis t indexed by k_t + N_t/2); ``x`` has shape (M, d); ``f`` shape (M,).
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib
from ._lib import NFFT_FP32, NFFT_FP64, check

_REAL = {torch.float32: NFFT_FP32, torch.float64: NFFT_FP64}
_COMPLEX = {torch.float32: torch.complex64, torch.float64: torch.complex128}


def _ptr(t: torch.Tensor):
    return ctypes.c_void_p(t.data_ptr()) if t.numel() else ctypes.c_void_p(0)


class Plan:
    """An NFFT plan on one CUDA device (Section 3.1, Table tab:params: N, M, n, m).

    Parameters
    ----------
    N : tuple of d even ints (d = 1, 2, 3)
    M : number of nodes
    n : FFT lengths (default 2^(ceil(log2 N_t) + 1), i.e. 2N for power-of-two N)
    m : window cutoff (default 8, the paper's standard choice)
    dtype : torch.float32 or torch.float64 (precision of x, fhat, f and the grid)
    device : CUDA device (default: the current one)
    window : "kaiser_bessel" (default), "gaussian", "bspline" or "sinc" (Section 4.1)
    """

    def __init__(self, N, M: int, n=None, m: int = 8, dtype=torch.float32, device=None,
                 window: str = "kaiser_bessel"):
        if window not in _lib.WINDOWS:
            raise ValueError(f"window must be one of {sorted(_lib.WINDOWS)}")
        if dtype not in _REAL:
            raise TypeError("dtype must be torch.float32 or torch.float64")
        if not torch.cuda.is_available():
            raise RuntimeError("gbnfft needs a CUDA device; there is no CPU implementation")
        self.N = tuple(int(v) for v in N)
        self.d = len(self.N)
        self.M = int(M)
        self.dtype = dtype
        self.cdtype = _COMPLEX[dtype]
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None \
            else torch.device(device)
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        L = _lib.lib()
        check(L.nfft_use_device(self.device.index), "nfft_use_device")
        Nv = (ctypes.c_int64 * 3)(*(list(self.N) + [0] * (3 - self.d)))
        nv = None
        if n is not None:
            n = tuple(int(v) for v in n)
            nv = (ctypes.c_int64 * 3)(*(list(n) + [0] * (3 - len(n))))
        h = ctypes.c_void_p()
        check(L.nfft_plan_create(ctypes.byref(h), self.d, Nv, self.M, nv, int(m), _REAL[dtype]),
              "nfft_plan_create")
        self._h = h
        info = _lib.NfftInfo()
        check(L.nfft_get_info(h, ctypes.byref(info)), "nfft_get_info")
        self.n = tuple(int(info.n[t]) for t in range(self.d))
        self.m = int(info.m)
        self.bin = tuple(int(info.bin[t]) for t in range(self.d))
        self.workspace_bytes = int(info.workspace_bytes)
        self._ws = torch.empty(max(self.workspace_bytes, 256), dtype=torch.uint8,
                               device=self.device)
        check(L.nfft_set_workspace(h, _ptr(self._ws), self._ws.numel()), "nfft_set_workspace")
        self._nodes_key = None
        self.window = "kaiser_bessel"
        if window != self.window:
            self.set_option("window", window)

    # ------------------------------------------------------------------ plumbing
    def _bind(self):
        stream = torch.cuda.current_stream(self.device)
        check(_lib.lib().nfft_set_stream(self._h, ctypes.c_void_p(stream.cuda_stream)),
              "nfft_set_stream")

    def _complex_in(self, t: torch.Tensor, count: int, name: str) -> torch.Tensor:
        if not isinstance(t, torch.Tensor):
            raise TypeError(f"{name} must be a torch.Tensor")
        if t.device != self.device:
            raise ValueError(f"{name} is on {t.device}, the plan on {self.device}")
        if t.dtype != self.cdtype:
            raise TypeError(f"{name} must be {self.cdtype}, got {t.dtype}")
        if t.numel() != count:
            raise ValueError(f"{name} must have {count} elements, got {t.numel()}")
        return t.contiguous()

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            _lib.lib().nfft_destroy(h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ API
    def set_option(self, key: str, value) -> None:
        """``window`` in {kaiser_bessel, gaussian, bspline, sinc} and ``window_table`` (K > 0:
        the window from a K-point-per-cell lookup table, PRE_LIN_PSI; 0: polynomials) change the
        approximation (they wait for the device to go idle); tuning: ``spread_method`` in {auto, thread,
        warp_atomic, warp_private, octet, half, plane, stripe}, ``interp_method`` in {auto, thread,
        warp, tile, octet}, or ``bin0`` / ``bin1`` / ``bin2`` (power-of-two bin sizes),
        ``subproblem`` (nodes per spreading work item, a power of two in 32..1024),
        ``stripe_item`` (nodes per work item of the stripe form, a power of two in 64..65536).
        Changing a bin, subproblem or item size discards the node precomputation; set the nodes
        again afterwards."""
        L = _lib.lib()
        if key == "window_table":
            check(L.nfft_set_option(self._h, _lib.OPT_WINDOW_TABLE, int(value)),
                  "nfft_set_option")
            return
        if key == "window":
            if value not in _lib.WINDOWS:
                raise ValueError(f"window must be one of {sorted(_lib.WINDOWS)}")
            check(L.nfft_set_option(self._h, _lib.OPT_WINDOW, _lib.WINDOWS[value]),
                  "nfft_set_option")
            self.window = value
            return
        if key == "spread_method":
            check(L.nfft_set_option(self._h, _lib.OPT_SPREAD_METHOD,
                                    _lib.SPREAD_METHODS[value]), "nfft_set_option")
            return
        if key == "interp_method":
            check(L.nfft_set_option(self._h, _lib.OPT_INTERP_METHOD,
                                    _lib.INTERP_METHODS[value]), "nfft_set_option")
            return
        if key in ("bin0", "bin1", "bin2", "subproblem", "stripe_item"):
            opt = {"subproblem": _lib.OPT_SUBPROBLEM, "stripe_item": _lib.OPT_STRIPE_ITEM}.get(
                key) or _lib.OPT_BIN[int(key[-1])]
            check(L.nfft_set_option(self._h, opt, int(value)), "nfft_set_option")
            info = _lib.NfftInfo()
            check(L.nfft_get_info(self._h, ctypes.byref(info)), "nfft_get_info")
            self.bin = tuple(int(info.bin[u]) for u in range(self.d))
            self.workspace_bytes = int(info.workspace_bytes)
            if self.workspace_bytes > self._ws.numel():
                torch.cuda.current_stream(self.device).synchronize()
                self._ws = torch.empty(self.workspace_bytes, dtype=torch.uint8,
                                       device=self.device)
                check(L.nfft_set_workspace(self._h, _ptr(self._ws), self._ws.numel()),
                      "nfft_set_workspace")
            self._nodes_key = None
            return
        raise KeyError(key)

    def set_nodes(self, x: torch.Tensor) -> None:
        """Precompute for the nodes x (shape (M, d), plan dtype, on the plan's device)."""
        if x.device != self.device or x.dtype != self.dtype:
            raise TypeError(f"x must be a {self.dtype} tensor on {self.device}")
        if x.numel() != self.M * self.d:
            raise ValueError(f"x must have shape ({self.M}, {self.d})")
        xc = x.detach().contiguous()
        self._bind()
        check(_lib.lib().nfft_set_nodes(self._h, _ptr(xc)), "nfft_set_nodes")
        self._x_keep = xc  # keep alive until the stream has consumed it
        self._nodes_key = (x.data_ptr(), x._version, tuple(x.shape))

    def ensure_nodes(self, x: torch.Tensor) -> None:
        key = (x.data_ptr(), x._version, tuple(x.shape))
        if key != self._nodes_key:
            self.set_nodes(x)

    def trafo(self, fhat: torch.Tensor) -> torch.Tensor:
        """Forward NFFT (Algorithm "NFFT"): returns f of shape (M,)."""
        fhat = self._complex_in(fhat, _prod(self.N), "fhat")
        f = torch.empty(self.M, dtype=self.cdtype, device=self.device)
        self._bind()
        check(_lib.lib().nfft_trafo(self._h, _ptr(fhat), _ptr(f)), "nfft_trafo")
        return f

    def adjoint(self, f: torch.Tensor) -> torch.Tensor:
        """Adjoint NFFT (Algorithm "adjoint NFFT"): returns hhat of shape N."""
        f = self._complex_in(f, self.M, "f")
        out = torch.empty(self.N, dtype=self.cdtype, device=self.device)
        self._bind()
        check(_lib.lib().nfft_adjoint(self._h, _ptr(f), _ptr(out)), "nfft_adjoint")
        return out

    def grad_x(self, coef: torch.Tensor, w: torch.Tensor) -> torch.Tensor:
        """(M, d) real: Re(conj(w_j) d s_coef / d x_t (x_j))."""
        coef = self._complex_in(coef, _prod(self.N), "coef")
        w = self._complex_in(w, self.M, "w")
        gx = torch.empty((self.M, self.d), dtype=self.dtype, device=self.device)
        self._bind()
        check(_lib.lib().nfft_grad_x(self._h, _ptr(coef), _ptr(w), _ptr(gx)), "nfft_grad_x")
        return gx

    def info(self) -> dict:
        """Plan parameters after defaults (nfft_get_info)."""
        i = _lib.NfftInfo()
        check(_lib.lib().nfft_get_info(self._h, ctypes.byref(i)), "nfft_get_info")
        inv = {v: k for k, v in _lib.WINDOWS.items()}
        return dict(d=i.d, m=i.m, dtype=i.dtype, M=int(i.M),
                    N=tuple(int(i.N[t]) for t in range(i.d)),
                    n=tuple(int(i.n[t]) for t in range(i.d)),
                    bin=tuple(int(i.bin[t]) for t in range(i.d)),
                    workspace_bytes=int(i.workspace_bytes), window=inv[int(i.window)],
                    window_table=int(i.window_table))

    def status(self) -> int:
        """Wait for the stream; return (and clear) the device-side error code."""
        self._bind()
        return int(_lib.lib().nfft_status(self._h))

    # host-buffer entry points (copies inside the library, synchronous)
    def set_nodes_host(self, x: torch.Tensor) -> None:
        x = x.contiguous()
        assert x.device.type == "cpu" and x.dtype == self.dtype
        self._bind()
        check(_lib.lib().nfft_set_nodes_host(self._h, _ptr(x)), "nfft_set_nodes_host")
        self._nodes_key = None

    def trafo_host(self, fhat: torch.Tensor, out: torch.Tensor) -> torch.Tensor:
        assert fhat.device.type == "cpu" and out.device.type == "cpu"
        self._bind()
        check(_lib.lib().nfft_trafo_host(self._h, _ptr(fhat), _ptr(out)), "nfft_trafo_host")
        return out

    def adjoint_host(self, f: torch.Tensor, out: torch.Tensor) -> torch.Tensor:
        assert f.device.type == "cpu" and out.device.type == "cpu"
        self._bind()
        check(_lib.lib().nfft_adjoint_host(self._h, _ptr(f), _ptr(out)), "nfft_adjoint_host")
        return out


def _prod(v) -> int:
    p = 1
    for a in v:
        p *= int(a)
    return p


class _NFFTFunction(torch.autograd.Function):
    """f = NFFT(fhat; x). Backward: grad fhat = NFFT^H grad f; grad x = Re(conj(grad f) ds/dx)."""

    @staticmethod
    def forward(ctx, fhat, x, plan):
        plan.ensure_nodes(x)
        f = plan.trafo(fhat)
        ctx.save_for_backward(fhat, x)
        ctx.plan = plan
        return f

    @staticmethod
    def backward(ctx, grad_f):
        fhat, x = ctx.saved_tensors
        plan = ctx.plan
        plan.ensure_nodes(x)
        grad_f = grad_f.contiguous()
        g_fhat = plan.adjoint(grad_f) if ctx.needs_input_grad[0] else None
        g_x = plan.grad_x(fhat, grad_f) if ctx.needs_input_grad[1] else None
        return g_fhat, g_x, None


class _NFFTAdjointFunction(torch.autograd.Function):
    """hhat = NFFT^H(f; x). Backward: grad f = NFFT grad hhat; grad x = Re(conj(f) ds_G/dx)."""

    @staticmethod
    def forward(ctx, f, x, plan):
        plan.ensure_nodes(x)
        h = plan.adjoint(f)
        ctx.save_for_backward(f, x)
        ctx.plan = plan
        return h

    @staticmethod
    def backward(ctx, grad_h):
        f, x = ctx.saved_tensors
        plan = ctx.plan
        plan.ensure_nodes(x)
        grad_h = grad_h.contiguous()
        g_f = plan.trafo(grad_h) if ctx.needs_input_grad[0] else None
        g_x = plan.grad_x(grad_h, f) if ctx.needs_input_grad[1] else None
        return g_f, g_x, None


def nfft(fhat: torch.Tensor, x: torch.Tensor, plan: Plan) -> torch.Tensor:
    """Differentiable forward NFFT (with respect to fhat and to the nodes x)."""
    return _NFFTFunction.apply(fhat, x, plan)


def nfft_adjoint(f: torch.Tensor, x: torch.Tensor, plan: Plan) -> torch.Tensor:
    """Differentiable adjoint NFFT (with respect to f and to the nodes x)."""
    return _NFFTAdjointFunction.apply(f, x, plan)
