"""Helpers shared by the GPU tests: run the CUDA path through the C ABI binding and compare
with the FP64 oracle element by element."""
import numpy as np
import torch

DEV = torch.device("cuda", 0)


def rel_l2(a, b) -> float:
    a = np.asarray(a).reshape(-1)
    b = np.asarray(b).reshape(-1)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def to_dev(a, dtype):
    """numpy -> device tensor in the run's precision (complex stays complex)."""
    a = np.asarray(a)
    if np.iscomplexobj(a):
        t = torch.tensor(a.astype(np.complex64 if dtype == torch.float32 else np.complex128))
    else:
        t = torch.tensor(a.astype(np.float32 if dtype == torch.float32 else np.float64))
    return t.to(DEV)


def rounded(a, dtype):
    """The values the GPU actually receives, converted exactly to FP64 / complex128 for the
    oracle (FP32 inputs are rounded first)."""
    a = np.asarray(a)
    if dtype == torch.float32:
        if np.iscomplexobj(a):
            return a.astype(np.complex64).astype(np.complex128)
        return a.astype(np.float32).astype(np.float64)
    return a.astype(np.complex128) if np.iscomplexobj(a) else a.astype(np.float64)


# Tolerances of the CUDA path against the FP64 oracle NFFT (rel. l2):
#   FP64 path: 1e-12 (the target of the build);
#   FP32 path: 1e-5 (the target at m = 4, sigma = 2; the FP32 rounding of the grid values and
#   weights gives ~1e-6 in practice).
TOL = {torch.float64: 1e-12, torch.float32: 1e-5}
