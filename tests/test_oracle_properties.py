"""Property-based pins of the oracle on random tiny problems.

Across shapes M, N in 1..7 and K in 1..min(M, N, 4), nonnegative X with exact
zeros, and start points with exact-zero rows of C or columns of B (so that the
zero-norm rule is reached), the oracle must satisfy what the mathematics fixes,
whatever the input:
  * every block step of a sweep is the exact minimiser of its block: per entry
    of b_k (or of c_k) the one-variable NNLS problem that scipy solves (Section
    2, HALS closed forms; Section 4.1 for the C-first order);
  * a block whose partner has zero norm is left unchanged;
  * the objective never rises, and the kept residual equals X - B C;
  * Algorithm 3 (W, V, delta b) gives the same B and C as Algorithm 2 with a
    kept residual (Section 5, "Correctness");
  * inner repeats of Algorithm 3's steps never raise the objective.
The cases are drawn by hypothesis (CPU only; skipped where it is missing).
"""

import numpy as np
import pytest
from scipy.optimize import nnls

from oracle import did_oracle as O

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402


@st.composite
def problems(draw):
    M = draw(st.integers(1, 7))
    N = draw(st.integers(1, 7))
    K = draw(st.integers(1, min(M, N, 4)))
    seed = draw(st.integers(0, 2 ** 32 - 1))
    zero_frac = draw(st.sampled_from([0.0, 0.3, 0.8]))
    rs = np.random.default_rng(seed)
    X = rs.uniform(0, 1, (M, N)) * (rs.uniform(0, 1, (M, N)) >= zero_frac)
    B = rs.uniform(0, 1, (M, K))
    C = rs.uniform(0, 1, (K, N))
    if draw(st.booleans()):
        C[rs.integers(K), :] = 0.0
    if draw(st.booleans()):
        B[:, rs.integers(K)] = 0.0
    return X, B, C


def _nnls_1d(a, y):
    """argmin_{x >= 0} ||y - a x||, by scipy's active-set NNLS."""
    return nnls(a[:, None], y)[0][0]


def _block_checker(X, B0, C0, order_kinds):
    """on_block callback: residual identity, monotone objective, block optimality."""
    scale = max(1.0, float(np.abs(X).max()), float(np.abs(B0).max()) * float(np.abs(C0).max()))
    state = {"B": np.array(B0, np.float64), "C": np.array(C0, np.float64), "f": O.objective(X, B0, C0),
             "steps": 0}

    def on_block(kind, k, B, C, R):
        assert kind in order_kinds
        assert np.all(B >= 0) and np.all(C >= 0)
        assert np.max(np.abs(R - (X - B @ C))) <= 1e-12 * scale * max(1, B.shape[1])
        f = 0.5 * float(np.sum(R ** 2))
        assert f <= state["f"] + 1e-12 * (state["f"] + scale ** 2 * 1e-6)
        state["f"] = f
        A = R + np.outer(B[:, k], C[k, :])          # residual without block k
        if kind == "b":
            c = C[k, :]
            if float(c @ c) == 0.0:
                assert np.array_equal(B[:, k], state["B"][:, k])
            else:
                for i in range(B.shape[0]):
                    x = _nnls_1d(c, A[i, :])
                    assert abs(B[i, k] - x) <= 1e-10 * max(1.0, abs(x))
        else:
            b = B[:, k]
            if float(b @ b) == 0.0:
                assert np.array_equal(C[k, :], state["C"][k, :])
            else:
                for j in range(C.shape[1]):
                    x = _nnls_1d(b, A[:, j])
                    assert abs(C[k, j] - x) <= 1e-10 * max(1.0, abs(x))
        state["B"] = B.copy()
        state["C"] = C.copy()
        state["steps"] += 1

    return on_block, state


@settings(max_examples=80, deadline=None)
@given(problems())
def test_interleaved_block_steps_are_exact_minimisers(p):
    X, B0, C0 = p
    on_block, state = _block_checker(X, B0, C0, ("b", "c"))
    B, C, R, _ = O.sweep_hals(X, B0, C0, on_block=on_block)
    assert state["steps"] == 2 * B0.shape[1]
    assert np.max(np.abs(R - (X - B @ C))) <= 1e-12 * max(1.0, float(np.abs(X).max())) * B0.shape[1]


@settings(max_examples=80, deadline=None)
@given(problems())
def test_c_first_block_steps_are_exact_minimisers(p):
    X, B0, C0 = p
    on_block, state = _block_checker(X, B0, C0, ("b", "c"))
    O.sweep_dbcd(X, B0, C0, on_block=on_block)
    assert state["steps"] == 2 * B0.shape[1]


@settings(max_examples=80, deadline=None)
@given(problems())
def test_algorithm_3_equals_algorithm_2(p):
    X, B0, C0 = p
    Bd, Cd, deg_d = O.sweep_did(X, B0, C0)
    Bb, Cb, _, deg_b = O.sweep_dbcd(X, B0, C0)
    np.testing.assert_array_equal(Cd, Cb)           # the same C step
    # The B steps differ only in rounding order: b_i from b_i + (w_i - sum_k
    # v_ik db_k) / v_ii against y / z on the kept residual; the error is
    # measured against the size of the terms that are added.
    V = Cd @ Cd.T
    W = (X - Bd @ Cd + (Bd - B0) @ Cd) @ Cd.T        # E' C^T with the C step's E'
    for i in range(B0.shape[1]):
        if V[i, i] == 0.0:
            np.testing.assert_array_equal(Bd[:, i], B0[:, i])
            np.testing.assert_array_equal(Bb[:, i], B0[:, i])
            continue
        terms = np.abs(B0[:, i]) + np.abs(W[:, i]) / V[i, i] + np.abs(Bd - B0) @ (np.abs(V[i, :]) / V[i, i])
        assert np.all(np.abs(Bd[:, i] - Bb[:, i]) <= 1e-12 * (1.0 + terms))
    assert deg_d == deg_b


@settings(max_examples=60, deadline=None)
@given(problems(), st.integers(1, 3), st.integers(1, 3))
def test_inner_repeats_never_raise_the_objective(p, inner_c, inner_b):
    X, B0, C0 = p
    f0 = O.objective(X, B0, C0)
    f1 = O.objective(X, *O.sweep_did(X, B0, C0)[:2])
    fr = O.objective(X, *O.sweep_did(X, B0, C0, inner_c=inner_c, inner_b=inner_b)[:2])
    tol = 1e-12 * (f0 + 1e-6)
    assert f1 <= f0 + tol and fr <= f0 + tol
