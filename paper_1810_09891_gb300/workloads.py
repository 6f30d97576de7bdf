"""Seeded synthetic inputs shaped like the paper's NFFT workloads.

This module only draws inputs: it holds none of the transform's arithmetic, and both the CUDA
path and the CPU oracle consume what it returns. Every generator takes an explicit seed and
uses numpy's PCG64, so the same call gives the same arrays on any machine.

Workloads:

* ``paper_fhat(N)``: the coefficients fhat_k = 1 / (1 + ||k||_2) of the paper's test
  polynomials (Section 4, eq. trigpolys), with uniform random nodes (Section 4).
* ``config_1d``: d = 1, N = 256, n = 512, m = 6, M = 512 uniform nodes.
* ``config_radial``: d = 2, N = (512, 512), n = (1024, 1024), M = 512 spokes x 2048 samples on
  a golden-angle radial trajectory (radius in [-1/2, 1/2)).
* ``config_clusters``: d = 3, N = (128, 128, 128), n = 2N, M = 4,194,304 nodes, half uniform,
  half in 8 Gaussian clusters of standard deviation 0.05 wrapped to the torus.

Nodes are drawn in FP64, wrapped into [-1/2, 1/2), then rounded to the run's precision; the
rounded values are what every consumer (GPU and oracle) receives.
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 1_810_09891


def rng(seed_offset: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(BASE_SEED + int(seed_offset)))


def wrap(x: np.ndarray) -> np.ndarray:
    """Wrap real coordinates into [-1/2, 1/2) (the torus T identified with [-1/2, 1/2))."""
    y = np.mod(np.asarray(x, dtype=np.float64) + 0.5, 1.0) - 0.5
    y = np.where(y >= 0.5, y - 1.0, y)
    return y


def round_nodes(x: np.ndarray, dtype) -> np.ndarray:
    """Round wrapped FP64 nodes to ``dtype`` and keep them inside [-1/2, 1/2)."""
    y = np.asarray(x, dtype=np.float64).astype(dtype)
    y = np.where(y >= dtype(0.5), y - dtype(1.0), y).astype(dtype)
    return np.ascontiguousarray(y)


def centred_k(N) -> list:
    """Frequency index vectors k_t = -N_t/2 .. N_t/2 - 1 for each axis (eq. index_set)."""
    return [np.arange(-int(v) // 2, int(v) // 2) for v in N]


def paper_fhat(N) -> np.ndarray:
    """fhat_k = 1 / (1 + ||k||_2) on I_N (Section 4, eq. trigpolys), complex128, shape N."""
    grids = np.meshgrid(*centred_k(N), indexing="ij")
    r = np.sqrt(sum(g.astype(np.float64) ** 2 for g in grids))
    return (1.0 / (1.0 + r)).astype(np.complex128)


def gaussian_fhat(N, seed_offset: int = 0) -> np.ndarray:
    """fhat_k with real and imaginary parts iid N(0, 1), complex128, shape N."""
    g = rng(seed_offset)
    shape = tuple(int(v) for v in N)
    return (g.standard_normal(shape) + 1j * g.standard_normal(shape)).astype(np.complex128)


def gaussian_values(M: int, seed_offset: int = 0) -> np.ndarray:
    """M complex values with real and imaginary parts iid N(0, 1)."""
    g = rng(seed_offset)
    return (g.standard_normal(M) + 1j * g.standard_normal(M)).astype(np.complex128)


def uniform_nodes(M: int, d: int, seed_offset: int = 0) -> np.ndarray:
    """M nodes iid uniform on [-1/2, 1/2)^d, FP64, shape (M, d)."""
    g = rng(seed_offset)
    return wrap(g.random((int(M), int(d))) - 0.5)


GOLDEN_ANGLE = np.pi * (np.sqrt(5.0) - 1.0) / 2.0  # ~111.25 degrees


def radial_nodes(spokes: int = 512, samples: int = 2048) -> np.ndarray:
    """Radial trajectory: spoke s at angle s * golden angle, sample i at radius
    -1/2 + i / samples; spoke-major order, FP64, shape (spokes * samples, 2).

    The centre sample (i = samples / 2) of every spoke lies exactly at x = 0, so all spokes share
    one node position (coincident nodes on a grid point)."""
    s = np.arange(spokes, dtype=np.float64)
    theta = np.mod(s * GOLDEN_ANGLE, 2.0 * np.pi)
    r = -0.5 + np.arange(samples, dtype=np.float64) / samples
    x0 = (r[None, :] * np.cos(theta)[:, None]).reshape(-1)
    x1 = (r[None, :] * np.sin(theta)[:, None]).reshape(-1)
    return wrap(np.stack([x0, x1], axis=1))


def clustered_nodes(M: int = 4_194_304, d: int = 3, clusters: int = 8, std: float = 0.05,
                    seed_offset: int = 2) -> np.ndarray:
    """Half of the nodes iid uniform, half split evenly over ``clusters`` Gaussian clusters
    (centres uniform, isotropic standard deviation ``std``), wrapped to the torus."""
    g = rng(seed_offset)
    mu = M // 2
    per = (M - mu) // clusters
    parts = [g.random((mu, d)) - 0.5]
    centres = g.random((clusters, d)) - 0.5
    for c in range(clusters):
        cnt = per if c < clusters - 1 else (M - mu) - per * (clusters - 1)
        parts.append(centres[c][None, :] + std * g.standard_normal((cnt, d)))
    return wrap(np.concatenate(parts, axis=0))


def config_1d(dtype=np.float64):
    """1-D workload: N = 256, n = 512, m = 6, M = 512 uniform nodes, Gaussian fhat."""
    N, n, m, M = (256,), (512,), 6, 512
    x = round_nodes(uniform_nodes(M, 1, seed_offset=0), dtype)
    fhat = gaussian_fhat(N, seed_offset=100)
    f = gaussian_values(M, seed_offset=200)
    return dict(name="1d_N256_M512", N=N, n=n, m=m, x=x, fhat=fhat, f=f)


def config_radial(m: int = 4, dtype=np.float32, spokes: int = 512, samples: int = 2048,
                  N=(512, 512)):
    """2-D radial workload: N = (512, 512), n = 2N, 512 golden-angle spokes x 2048 samples."""
    N = tuple(int(v) for v in N)
    n = tuple(2 * v for v in N)
    x = round_nodes(radial_nodes(spokes, samples), dtype)
    fhat = gaussian_fhat(N, seed_offset=101)
    f = gaussian_values(x.shape[0], seed_offset=201)
    return dict(name=f"2d_radial_N{N[0]}_M{x.shape[0]}_m{m}", N=N, n=n, m=m, x=x, fhat=fhat, f=f)


def config_clusters(M: int = 4_194_304, dtype=np.float32, N=(128, 128, 128), m: int = 4):
    """3-D workload: N = (128,)*3, n = 2N, m = 4, half uniform, half in 8 Gaussian clusters."""
    N = tuple(int(v) for v in N)
    n = tuple(2 * v for v in N)
    x = round_nodes(clustered_nodes(M, 3), dtype)
    fhat = gaussian_fhat(N, seed_offset=102)
    f = gaussian_values(x.shape[0], seed_offset=202)
    return dict(name=f"3d_clusters_N{N[0]}_M{M}", N=N, n=n, m=m, x=x, fhat=fhat, f=f)


def spiral_nodes(arms: int = 32, samples: int = 8192, turns: float = 4.0) -> np.ndarray:
    """Interleaved Archimedean spiral: arm a, sample s at radius 0.5 s / samples and angle
    2 pi turns s / samples + 2 pi a / arms; arm-major order, FP64, shape (arms * samples, 2)."""
    s = np.arange(samples, dtype=np.float64)
    r = 0.5 * s / samples
    th = 2.0 * np.pi * turns * s / samples
    a = np.arange(arms, dtype=np.float64)[:, None]
    ang = th[None, :] + 2.0 * np.pi * a / arms
    x0 = (r[None, :] * np.cos(ang)).reshape(-1)
    x1 = (r[None, :] * np.sin(ang)).reshape(-1)
    return wrap(np.stack([x0, x1], axis=1))


def ellipse_phantom_fhat(N, count: int = 20, seed_offset: int = 5) -> np.ndarray:
    """Fourier coefficients fhat_k = int f(x) e^{+2 pi i k.x} dx of a sum of `count` random
    ellipse indicators f = sum_e rho_e 1_{E_e} on [-1/2, 1/2)^2 (so that
    f(x) = sum_k fhat_k e^{-2 pi i k.x}). Ellipse e: density rho ~ U[0.1, 1], semi-axes
    a, b ~ U[0.05, 0.3], centre c ~ U[-0.3, 0.3]^2, rotation ~ U[0, pi). For the unit disc the
    transform is J1(2 pi |k|) / |k|; an ellipse scales and rotates k and adds the phase of c."""
    from scipy.special import j1

    g = rng(seed_offset)
    k0, k1 = np.meshgrid(*centred_k(N), indexing="ij")
    k0 = k0.astype(np.float64)
    k1 = k1.astype(np.float64)
    out = np.zeros(tuple(int(v) for v in N), dtype=np.complex128)
    for _ in range(count):
        rho = g.uniform(0.1, 1.0)
        a, b = g.uniform(0.05, 0.3, size=2)
        c = g.uniform(-0.3, 0.3, size=2)
        al = g.uniform(0.0, np.pi)
        u = a * (np.cos(al) * k0 + np.sin(al) * k1)
        v = b * (-np.sin(al) * k0 + np.cos(al) * k1)
        q = np.sqrt(u * u + v * v)
        with np.errstate(invalid="ignore", divide="ignore"):
            disc = np.where(q > 0, j1(2.0 * np.pi * q) / np.where(q > 0, q, 1.0), np.pi)
        out += rho * a * b * disc * np.exp(2j * np.pi * (k0 * c[0] + k1 * c[1]))
    return out


def config_spiral(dtype=np.float32, N=(256, 256), m: int = 4, arms: int = 32,
                  samples: int = 8192):
    """2-D reconstruction workload: N = (256, 256), n = 2N, m = 4, M = 32 x 8192 spiral nodes,
    fhat_true an ellipse phantom."""
    N = tuple(int(v) for v in N)
    n = tuple(2 * v for v in N)
    x = round_nodes(spiral_nodes(arms, samples), dtype)
    return dict(name=f"2d_spiral_N{N[0]}_M{x.shape[0]}_m{m}", N=N, n=n, m=m, x=x,
                fhat_true=ellipse_phantom_fhat(N))
