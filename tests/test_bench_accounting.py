"""The byte and flop counts the benchmark's roofline rests on, checked against
counts made by hand from the kernels' passes (CPU only).

The interleaved sweep reads R once per k and writes it once per k, except
that with deferred write-back a pair (k, k+1) shares one write; the batched
order (Algorithm 3) moves R three times per sweep: the g pass reads it, the
update pass reads and writes it.
"""

import json
import os

import pytest

bench = pytest.importorskip("bench")


def passes_by_hand(K, lazy):
    """Walk the k-steps: a deferred step (k even with a partner k+1) only
    reads R; every other step reads and writes it."""
    reads = writes = 0
    for k in range(K):
        deferred = lazy and k % 2 == 0 and k + 1 < K
        reads += 1
        writes += 0 if deferred else 1
    return reads + writes


@pytest.mark.parametrize("K", [1, 2, 3, 5, 16, 50, 63, 100])
@pytest.mark.parametrize("lazy", [False, True])
def test_sweep_passes_match_the_pass_walk(K, lazy):
    assert bench.sweep_passes(K, lazy) == passes_by_hand(K, lazy)


def test_default_workload_bytes():
    # 5000 x 200000, K = 50, float32: 75 passes of 4 GB with deferred
    # write-back, 100 without
    M, N, K = 5000, 200000, 50
    assert bench.sweep_passes(K, True) * M * N * 4 == 300e9
    assert bench.sweep_passes(K, False) * M * N * 4 == 400e9


def test_batched_roofline_counts_three_passes():
    M, N, K = 5000, 200000, 50
    ms = 5.0
    r = bench.batched_roofline(M, N, K, ms)
    assert r["passes_of_R"] == 3
    assert r["alg_bytes_per_sweep"] == 3 * M * N * 4
    assert r["achieved"] == pytest.approx(3 * M * N * 4 / (ms / 1e3) / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    # six bfloat16 products per float32 product of the three contractions
    assert r["tensor_tflops_bf16x6"] == pytest.approx(6 * r["flops_per_sweep_f32"] / (ms / 1e3) / 1e12)


def test_batched_flops_lead_term():
    # g (2KMN), the rank-2K update (4KMN) and W (2KMN) dominate; the K x K
    # products and the solves add O(K^2 (M + N))
    M, N, K = 5000, 200000, 50
    f = bench.batched_flops(M, N, K)
    assert 8 * K * M * N <= f <= 8 * K * M * N * 1.05


def test_peaks_are_the_measured_file():
    p = os.path.join(os.path.dirname(bench.__file__), "MEASURED_PEAKS.json")
    peak, kind = bench.measured_peaks()
    if os.path.exists(p):
        with open(p) as fh:
            assert peak == float(json.load(fh)["hbm_gbs"])
        assert kind == "measured"
    else:
        assert kind == "fallback"
