"""Seeded synthetic workloads shaped like the paper's experiments.

The paper's synthetic data are uniform[0,1] matrices drawn with Matlab
``rand`` (Section 5, experiments) and its real data are image and text
matrices (MNIST, 20News, UMist, YaleB); none of those streams or files is
available, so every workload here is a seeded, counter-based stand-in (see
``synth.rng``).  Index conventions, shared with the device generator:

* planted basis ``B0[i, k]`` is word ``k*M + i`` of its stream (column-major),
* planted coordinates ``C0[k, j]`` is word ``k*N + j`` (row-major),
* per-entry noise and masks on ``X[i, j]`` use word ``j*M + i``
  (column-major, samples are columns),
* solver initialisation ``B[i, k]`` / ``C[k, j]`` use the same indices as
  ``B0`` / ``C0`` on their own streams.

All matrices are returned as NumPy arrays of shape ``(rows, cols)``; ``X`` is
float32 and Fortran-ordered, so column ``j`` (sample ``j``) is contiguous,
which is the layout the C-ABI expects.
"""

import math

import numpy as np

from . import rng


def _idx_colmajor(M, N):
    # word index j*M + i laid out as an (M, N) array
    return (np.arange(N, dtype=np.uint64)[None, :] * np.uint64(M)
            + np.arange(M, dtype=np.uint64)[:, None])


def _idx_rowmajor(R, Ccols):
    return (np.arange(R, dtype=np.uint64)[:, None] * np.uint64(Ccols)
            + np.arange(Ccols, dtype=np.uint64)[None, :])


def uniform_basis(M, K, seed, stream=rng.STREAM_B0):
    """(M, K) float32 uniform[0,1) with word index k*M + i."""
    idx = _idx_rowmajor(K, M).T          # [i, k] -> k*M + i
    return rng.uniform_f32(seed, stream, idx)


def uniform_coords(K, N, seed, stream=rng.STREAM_C0):
    """(K, N) float32 uniform[0,1) with word index k*N + j."""
    return rng.uniform_f32(seed, stream, _idx_rowmajor(K, N))


def exp_coords(K, N, seed, zero_frac):
    """(K, N) exponential(1) coordinates with a Bernoulli(zero_frac) share zeroed."""
    idx = _idx_rowmajor(K, N)
    c = rng.exponential_f64(seed, rng.STREAM_C0, idx).astype(np.float32)
    if zero_frac > 0:
        c[rng.bernoulli(seed, rng.STREAM_MASK, idx, zero_frac)] = 0.0
    return c


def init_factors(M, N, K, seed):
    """Solver start point: B, C uniform[0,1) from the init streams."""
    B = uniform_basis(M, K, seed, rng.STREAM_INIT_B)
    C = uniform_coords(K, N, seed, rng.STREAM_INIT_C)
    return B, C


def planted(M, N, K, seed, coords="uniform", zero_frac=0.0, sigma=0.0,
            salt_frac=0.0, salt_value=5.0):
    """X = B0 C0 (+ |N(0, sigma^2)| noise) (with salt entries set to salt_value).

    The product is formed in float64 and rounded once to float32.
    Returns (X, B0, C0).
    """
    B0 = uniform_basis(M, K, seed)
    if coords == "uniform":
        C0 = uniform_coords(K, N, seed)
    elif coords == "exp":
        C0 = exp_coords(K, N, seed, zero_frac)
    else:
        raise ValueError(coords)
    X = B0.astype(np.float64) @ C0.astype(np.float64)
    if sigma > 0:
        X += sigma * np.abs(rng.normal_f64(seed, rng.STREAM_NOISE, _idx_colmajor(M, N)))
    if salt_frac > 0:
        X[rng.bernoulli(seed, rng.STREAM_MASK, _idx_colmajor(M, N), salt_frac)] = salt_value
    return np.asfortranarray(X.astype(np.float32)), B0, C0


def image_like(M, N, seed, zero_frac=0.8):
    """Entries in [0,1]: a Bernoulli(zero_frac) share exact zeros, the rest Beta(2,2)."""
    idx = _idx_colmajor(M, N)
    X = rng.beta22_f32(seed, rng.STREAM_BETA, idx)
    X[rng.bernoulli(seed, rng.STREAM_MASK, idx, zero_frac)] = 0.0
    return np.asfortranarray(X.astype(np.float32))


# Workload recipes.  ``scale`` shrinks M and N (not K) for oracle-sized cases.
CONFIGS = {
    # M=200, N=1000, K=10; X = B0 C0 + |N(0, 0.01^2)|, B0, C0 ~ U[0,1]
    "planted_uniform_200x1000_k10": dict(M=200, N=1000, K=10, kind="planted",
                                         coords="uniform", sigma=0.01),
    # tall-and-wide: M=5000, N=200000, K=50; C0 ~ Exp(1) with 30% zeros
    "planted_exp_5000x200000_k50": dict(M=5000, N=200000, K=50, kind="planted",
                                        coords="exp", zero_frac=0.3, sigma=0.05),
    # image-like stand-in for MNIST: M=784, N=70000, K=16
    "image_like_784x70000_k16": dict(M=784, N=70000, K=16, kind="image"),
    # precision workload: M=10000, N=500000, K=100, 1% salt set to 5.0
    "salt_10000x500000_k100": dict(M=10000, N=500000, K=100, kind="planted",
                                   coords="uniform", salt_frac=0.01),
}


def make(name, seed=0, M=None, N=None, K=None):
    """Generate X for a named recipe, optionally at other sizes (same generator)."""
    cfg = dict(CONFIGS[name])
    M = cfg["M"] if M is None else M
    N = cfg["N"] if N is None else N
    K = cfg["K"] if K is None else K
    if cfg["kind"] == "planted":
        X, _, _ = planted(M, N, K, seed, coords=cfg.get("coords", "uniform"),
                          zero_frac=cfg.get("zero_frac", 0.0), sigma=cfg.get("sigma", 0.0),
                          salt_frac=cfg.get("salt_frac", 0.0))
    else:
        X = image_like(M, N, seed)
    return X, M, N, K


# ---------------------------------------------------------------- serving
SERVE_K_CHOICES = (8, 16, 32, 64)


def log_uniform_int(u, lo, hi):
    return int(round(math.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))))


def request_shape(base_seed, r):
    """(M, N, K) of request r: M ~ logU[64,4096], N ~ logU[256,65536], K in {8,16,32,64}."""
    um = float(rng.uniform_f64(base_seed, rng.STREAM_SIZE_M, [r])[0])
    un = float(rng.uniform_f64(base_seed, rng.STREAM_SIZE_N, [r])[0])
    uk = float(rng.uniform_f64(base_seed, rng.STREAM_SIZE_K, [r])[0])
    return (log_uniform_int(um, 64, 4096), log_uniform_int(un, 256, 65536),
            SERVE_K_CHOICES[min(3, int(uk * 4))])


def request_seed(base_seed, r):
    """Seed of request r's own matrices (B0, C0, noise, init)."""
    return (int(base_seed) << 32) + int(r)


def arrival_times(base_seed, n, rate_per_s):
    """Poisson arrivals: cumulative exponential gaps of mean 1/rate (seconds)."""
    gaps = rng.exponential_f64(base_seed, rng.STREAM_ARRIVAL, np.arange(n, dtype=np.uint64))
    return np.cumsum(gaps / rate_per_s)
