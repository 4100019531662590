"""Pins of the oracle's inner repeats (Algorithm 3 with its C and B steps run
several times per iteration, in the manner of accelerated HALS).

With one factor fixed, NMF is a convex nonnegative least-squares problem, and
each repeat of a block step is one cyclic pass of exact coordinate
minimisation on it.  Many repeats must therefore reach the NNLS solution that
an independent active-set solver (scipy's Lawson-Hanson ``nnls``) finds, column
by column for C and row by row for B.  Dropping the residual update between B
repeats, a wrong sign in the delta-b rule, or a wrong Gram entry all move the
limit away from it.
"""

import numpy as np
import pytest
from scipy.optimize import nnls

from oracle import did_oracle as O


def _problem(seed, M, N, K):
    rs = np.random.default_rng(seed)
    X = rs.uniform(0, 1, (M, N))
    B = rs.uniform(0, 1, (M, K)) + 0.5 * np.eye(M, K)     # well conditioned Gram
    C = rs.uniform(0, 1, (K, N)) + 0.5 * np.eye(K, N)
    return X, B, C


@pytest.mark.parametrize("seed", range(3))
def test_c_repeats_reach_nnls(seed):
    X, B, C = _problem(seed, 14, 9, 4)
    B1, C1, _ = O.sweep_did(X, B, C, inner_c=3000, inner_b=0)
    assert np.array_equal(B1, B)                          # B step skipped
    for j in range(X.shape[1]):
        ref, _ = nnls(B, X[:, j])
        assert np.max(np.abs(C1[:, j] - ref)) <= 1e-9 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("seed", range(3))
def test_b_repeats_reach_nnls(seed):
    X, B, C = _problem(10 + seed, 9, 15, 4)
    B1, C1, _ = O.sweep_did(X, B, C, inner_c=0, inner_b=3000)
    assert np.array_equal(C1, C)                          # C step skipped
    for m in range(X.shape[0]):
        ref, _ = nnls(C.T, X[m, :])
        assert np.max(np.abs(B1[m, :] - ref)) <= 1e-9 * max(1.0, np.abs(ref).max())


def test_each_repeat_is_monotone():
    X, B, C = _problem(7, 20, 30, 5)
    prev = O.objective(X, B, C)
    for r in range(1, 8):                                 # more C repeats, same start
        _, C1, _ = O.sweep_did(X, B, C, inner_c=r, inner_b=0)
        f = O.objective(X, B, C1)
        assert f <= prev * (1 + 1e-14)
        prev = f
    prev = O.objective(X, B, C)
    for r in range(1, 8):
        B1, _, _ = O.sweep_did(X, B, C, inner_c=0, inner_b=r)
        f = O.objective(X, B1, C)
        assert f <= prev * (1 + 1e-14)
        prev = f


def test_repeats_trace_monotone_and_nonnegative():
    X, B, C = _problem(3, 30, 40, 6)
    r = O.factor(X, B, C, order="did", max_iter=15, stop="none", inner_c=3, inner_b=4)
    t = r["trace"]
    assert np.all(np.diff(t) <= 1e-12 * t[0])
    assert r["B"].min() >= 0 and r["C"].min() >= 0


def test_one_repeat_is_the_plain_iteration():
    X, B, C = _problem(5, 12, 17, 3)
    a = O.sweep_did(X, B, C)
    b = O.sweep_did(X, B, C, inner_c=1, inner_b=1)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    # two C steps are one sweep of Algorithm 2 with its B step replaced by a second C step
    _, C2, _ = O.sweep_did(X, B, C, inner_c=2, inner_b=0)
    E = O.residual(X, B, C)
    Cs = C.copy()
    for _ in range(2):
        for i in range(3):
            b = B[:, i]
            E += np.outer(b, Cs[i])
            Cs[i] = np.maximum(b @ E / (b @ b), 0.0)
            E -= np.outer(b, Cs[i])
    assert np.max(np.abs(C2 - Cs)) <= 1e-13


def test_repeats_rejected_for_other_orders():
    X, B, C = _problem(1, 5, 6, 2)
    with pytest.raises(ValueError):
        O.factor(X, B, C, order="hals", max_iter=1, inner_c=2)
