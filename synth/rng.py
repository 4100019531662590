"""Counter-based random numbers for the synthetic NMF workloads.

This module holds no arithmetic of the factorisation method.  It defines one
counter-based generator and the distributions the workloads draw from; the
CUDA library carries its own, separately written implementation of the same
definition (``paper_1802_08938_gb300/csrc/did_internal.cuh`` for the
generator, ``paper_1802_08938_gb300/csrc/did_dense.cu`` for the device
workload kernels) so that very large inputs can be generated on the device.

Definition (the contract both implementations follow):

* ``mix64(z)`` is the SplitMix64 output function (Steele, Lea and Flood,
  "Fast splittable pseudorandom number generators", OOPSLA 2014):
  ``z ^= z >> 30; z *= 0xBF58476D1CE4E5B9; z ^= z >> 27;
  z *= 0x94D049BB133111EB; z ^= z >> 31`` (all mod 2**64).
* ``key(seed, stream) = mix64(seed + (stream + 1) * G)`` with
  ``G = 0x9E3779B97F4A7C15`` (the golden-ratio increment of SplitMix64).
* ``draw(seed, stream, i) = mix64(key(seed, stream) + (i + 1) * G)`` is the
  i-th 64-bit word of the stream, so any element can be drawn on its own.
* ``u24 = draw >> 40``; ``uniform_f32 = u24 * 2**-24`` (exact in float32, in
  [0, 1)); ``uniform_f64 = (draw >> 11) * 2**-53``.
* normal: Box-Muller on words 2i and 2i+1 of the stream, in float64:
  ``sqrt(-2 ln(1 - u1)) * cos(2 pi u2)``.
* exponential(1): ``-ln(1 - u)`` in float64.
* Beta(2, 2): the median of three float32 uniforms drawn at words 3i, 3i+1,
  3i+2 (the second order statistic of three uniforms has density 6x(1-x)).
* Bernoulli(p): ``uniform_f64 < p``.
"""

import numpy as np

G = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Stream identifiers shared with the device generator.
STREAM_B0 = 0       # planted basis B0
STREAM_C0 = 1       # planted coordinates C0
STREAM_NOISE = 2    # additive |N(0, sigma^2)| noise on X
STREAM_MASK = 3     # Bernoulli masks (zeroed C0 entries, zero pixels, salt)
STREAM_INIT_B = 4   # initial B of the solver
STREAM_INIT_C = 5   # initial C of the solver
STREAM_BETA = 6     # Beta(2,2) pixel values
STREAM_SIZE_M = 7   # serving: request row count
STREAM_SIZE_N = 8   # serving: request column count
STREAM_SIZE_K = 9   # serving: request rank
STREAM_ARRIVAL = 10  # serving: inter-arrival gaps

TWO_M24 = np.float32(2.0 ** -24)
TWO_M53 = 2.0 ** -53


def mix64(z):
    """SplitMix64 output function on a uint64 array (wrapping arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def key(seed, stream):
    with np.errstate(over="ignore"):
        s = np.uint64(seed % (1 << 64)) + np.uint64(stream + 1) * G
    return mix64(np.array([s], dtype=np.uint64))[0]


def draw(seed, stream, idx):
    """64-bit words ``idx`` (an integer array) of ``stream``."""
    k = key(seed, stream)
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return mix64(k + (idx + np.uint64(1)) * G)


def uniform_f32(seed, stream, idx):
    w = draw(seed, stream, idx)
    return (w >> np.uint64(40)).astype(np.float32) * TWO_M24


def uniform_f64(seed, stream, idx):
    w = draw(seed, stream, idx)
    return (w >> np.uint64(11)).astype(np.float64) * TWO_M53


def normal_f64(seed, stream, idx):
    idx = np.asarray(idx, dtype=np.uint64)
    u1 = uniform_f64(seed, stream, np.uint64(2) * idx)
    u2 = uniform_f64(seed, stream, np.uint64(2) * idx + np.uint64(1))
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)


def exponential_f64(seed, stream, idx):
    return -np.log1p(-uniform_f64(seed, stream, idx))


def beta22_f32(seed, stream, idx):
    idx = np.asarray(idx, dtype=np.uint64)
    three = np.uint64(3)
    a = uniform_f32(seed, stream, three * idx)
    b = uniform_f32(seed, stream, three * idx + np.uint64(1))
    c = uniform_f32(seed, stream, three * idx + np.uint64(2))
    return np.maximum(np.minimum(a, b), np.minimum(np.maximum(a, b), c))


def bernoulli(seed, stream, idx, p):
    return uniform_f64(seed, stream, idx) < p
