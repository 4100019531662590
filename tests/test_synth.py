"""The seeded input generators: published SplitMix64 values and distribution moments."""

import json
import os

import numpy as np

from synth import rng
from synth import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_mix64_published_values():
    g = json.load(open(os.path.join(GOLDEN, "splitmix64_state0.json")))
    z = np.array([1, 2, 3], dtype=np.uint64)
    with np.errstate(over="ignore"):
        out = rng.mix64(z * rng.G)
    assert [int(v) for v in out] == [int(h, 16) for h in g["outputs_hex"]]


def test_counter_streams_are_random_access():
    a = rng.draw(5, rng.STREAM_B0, np.arange(100))
    b = rng.draw(5, rng.STREAM_B0, np.array([37]))
    assert a[37] == b[0]
    assert not np.array_equal(a, rng.draw(5, rng.STREAM_C0, np.arange(100)))
    assert not np.array_equal(a, rng.draw(6, rng.STREAM_B0, np.arange(100)))


def test_distribution_moments():
    n = 400000
    idx = np.arange(n, dtype=np.uint64)
    u = rng.uniform_f32(1, 0, idx)
    assert u.dtype == np.float32 and u.min() >= 0 and u.max() < 1
    assert abs(u.mean() - 0.5) < 3e-3 and abs(u.var() - 1 / 12) < 2e-3
    z = rng.normal_f64(1, 2, idx)
    assert abs(z.mean()) < 1e-2 and abs(z.var() - 1) < 1e-2
    e = rng.exponential_f64(1, 3, idx)
    assert e.min() >= 0 and abs(e.mean() - 1) < 1e-2 and abs(e.var() - 1) < 3e-2
    bt = rng.beta22_f32(1, 6, idx)          # Beta(2,2): mean 1/2, variance 1/20
    assert abs(bt.mean() - 0.5) < 3e-3 and abs(bt.var() - 0.05) < 2e-3
    m = rng.bernoulli(1, 4, idx, 0.3)
    assert abs(m.mean() - 0.3) < 3e-3


def test_workload_shapes_and_layout():
    X, M, N, K = W.make("planted_exp_5000x200000_k50", seed=0, M=50, N=300, K=5)
    assert X.shape == (50, 300) and X.dtype == np.float32 and X.flags.f_contiguous
    assert X.min() >= 0
    X2 = W.image_like(40, 500, 3)
    frac0 = np.mean(X2 == 0)
    assert 0.75 < frac0 < 0.85 and X2.max() <= 1.0
    X3, _, _ = W.planted(60, 400, 4, 1, salt_frac=0.01)
    assert 0.005 < np.mean(X3 == 5.0) < 0.02
    B, C = W.init_factors(7, 9, 3, 4)
    # index convention: B[i,k] is word k*M + i of the init-B stream
    assert B[2, 1] == rng.uniform_f32(4, rng.STREAM_INIT_B, np.array([1 * 7 + 2]))[0]
    assert C[1, 5] == rng.uniform_f32(4, rng.STREAM_INIT_C, np.array([1 * 9 + 5]))[0]


def test_request_stream():
    shapes = [W.request_shape(0, r) for r in range(2000)]
    Ms = np.array([s[0] for s in shapes])
    Ns = np.array([s[1] for s in shapes])
    Ks = np.array([s[2] for s in shapes])
    assert Ms.min() >= 64 and Ms.max() <= 4096 and Ns.min() >= 256 and Ns.max() <= 65536
    assert set(Ks.tolist()) == {8, 16, 32, 64}
    # log-uniform: the median of M is near sqrt(64*4096) = 512
    assert 400 < np.median(Ms) < 650
    t = W.arrival_times(0, 4096, 200.0)
    assert abs(t[-1] / 4096 - 1 / 200) < 5e-4
