"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: hand-derived
worked examples (tests/golden), a library NNLS solver, brute-force search,
invariants (monotone objective, R == X - BC), the paper's own correctness
claim (DID, DBCD and BCD take the same number of iterations, Section 5),
special cases with known answers, and equivariances.
"""

import json
import os
from fractions import Fraction

import numpy as np
import pytest
from scipy.optimize import nnls

from oracle import did_oracle as O
from synth import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _frac_matrix(rows):
    return np.array([[float(Fraction(v)) for v in r] for r in rows], dtype=np.float64)


def _rand_problem(rs, M, N, K, low_rank=False):
    if low_rank:
        X = rs.uniform(0, 1, (M, K)) @ rs.uniform(0, 1, (K, N))
    else:
        X = rs.uniform(0, 1, (M, N))
    B = rs.uniform(0, 1, (M, K))
    C = rs.uniform(0, 1, (K, N))
    return X, B, C


# --------------------------------------------------------------- golden cases
def test_golden_rank1_hals_and_c_first():
    g = json.load(open(os.path.join(GOLDEN, "hals_2x2_rank1.json")))
    X = np.array(g["X"], float)
    B0 = np.array(g["B_init"], float)
    C0 = np.array(g["C_init"], float)
    B, C, R, _ = O.sweep_hals(X, B0, C0)
    np.testing.assert_allclose(B, _frac_matrix(g["hals"]["B"]), rtol=0, atol=1e-15)
    np.testing.assert_allclose(C, _frac_matrix(g["hals"]["C"]), rtol=0, atol=1e-15)
    assert abs(0.5 * np.sum(R * R) - float(Fraction(g["hals"]["f"]))) < 1e-15
    for sweep in (lambda: O.sweep_dbcd(X, B0, C0)[:2], lambda: O.sweep_did(X, B0, C0)[:2]):
        B, C = sweep()
        np.testing.assert_allclose(B, _frac_matrix(g["c_first"]["B"]), rtol=0, atol=1e-15)
        np.testing.assert_allclose(C, _frac_matrix(g["c_first"]["C"]), rtol=0, atol=1e-15)
        assert abs(O.objective(X, B, C) - float(Fraction(g["c_first"]["f"]))) < 1e-15


def test_golden_projection_clips():
    g = json.load(open(os.path.join(GOLDEN, "hals_projection_2x2_rank2.json")))
    X = np.array(g["X"], float)
    B, C, R, _ = O.sweep_hals(X, np.array(g["B_init"], float), np.array(g["C_init"], float))
    np.testing.assert_allclose(B, _frac_matrix(g["hals"]["B"]), atol=1e-15)
    np.testing.assert_allclose(C, _frac_matrix(g["hals"]["C"]), atol=1e-15)
    assert np.max(np.abs(R)) < 1e-15


def test_projection_signs():
    z = np.array([-1.0, -0.0, 0.0, 2.5, np.nan, -np.inf, np.inf])
    p = O.project(z)
    assert np.all(p[:3] == 0.0) and not np.any(np.signbit(p))
    assert p[3] == 2.5 and p[4] == 0.0 and p[5] == 0.0 and p[6] == np.inf


# ----------------------------------------------- closed forms vs library NNLS
@pytest.mark.parametrize("seed", range(6))
def test_closed_forms_equal_nnls(seed):
    """Each rank-one block problem is an NNLS problem; scipy's NNLS solves it."""
    rs = np.random.default_rng(seed)
    M, N = rs.integers(1, 7), rs.integers(1, 7)
    A = rs.normal(0, 1, (M, N))          # A = X - sum_{i != k} b_i c_i may be negative
    c = np.abs(rs.normal(0, 1, N))
    b = np.abs(rs.normal(0, 1, M))
    b_new, ok = O.update_b_hals(A, c, b)
    assert ok
    for i in range(M):                    # min_{b_i >= 0} || A[i,:] - b_i c ||
        x, _ = nnls(c[:, None], A[i, :])
        assert abs(b_new[i] - x[0]) <= 1e-12 * max(1.0, abs(x[0]))
    c_new, ok = O.update_c_hals(A, b, c)
    assert ok
    for j in range(N):                    # min_{c_j >= 0} || A[:,j] - b c_j ||
        x, _ = nnls(b[:, None], A[:, j])
        assert abs(c_new[j] - x[0]) <= 1e-12 * max(1.0, abs(x[0]))


def _golden_section(f, lo, hi, iters=200):
    g = (np.sqrt(5.0) - 1.0) / 2.0
    a, b = lo, hi
    c, d = b - g * (b - a), a + g * (b - a)
    for _ in range(iters):
        if f(c) < f(d):
            b = d
        else:
            a = c
        c, d = b - g * (b - a), a + g * (b - a)
    return 0.5 * (a + b)


@pytest.mark.parametrize("seed", range(4))
def test_closed_forms_vs_brute_force(seed):
    """Brute-force projected minimisation of the full objective over one block."""
    rs = np.random.default_rng(100 + seed)
    M, N, K = 5, 6, 3
    X, B, C = _rand_problem(rs, M, N, K)
    k = int(rs.integers(0, K))
    A = X - B @ C + np.outer(B[:, k], C[k, :])
    b_cf, _ = O.update_b_hals(A, C[k, :], B[:, k])
    for i in range(M):
        def f_i(v, i=i):
            Bt = B.copy()
            Bt[:, k] = b_cf
            Bt[i, k] = v
            return O.objective(X, Bt, C)
        hi = 4.0 + 4.0 * abs(b_cf[i])
        grid = np.linspace(0.0, hi, 4001)
        vals = np.array([f_i(v) for v in grid])
        j = int(np.argmin(vals))
        lo_, hi_ = grid[max(j - 1, 0)], grid[min(j + 1, len(grid) - 1)]
        v = _golden_section(f_i, lo_, hi_)
        if f_i(0.0) <= f_i(v):
            v = 0.0
        assert abs(v - b_cf[i]) < 1e-7, (i, v, b_cf[i])
        assert f_i(b_cf[i]) <= f_i(v) + 1e-12
    c_cf, _ = O.update_c_hals(A, b_cf, C[k, :])
    Bt = B.copy()
    Bt[:, k] = b_cf
    for j in range(N):
        def g_j(v, j=j):
            Ct = C.copy()
            Ct[k, :] = c_cf
            Ct[k, j] = v
            return O.objective(X, Bt, Ct)
        hi = 4.0 + 4.0 * abs(c_cf[j])
        grid = np.linspace(0.0, hi, 4001)
        vals = np.array([g_j(v) for v in grid])
        jj = int(np.argmin(vals))
        v = _golden_section(g_j, grid[max(jj - 1, 0)], grid[min(jj + 1, len(grid) - 1)])
        if g_j(0.0) <= g_j(v):
            v = 0.0
        assert abs(v - c_cf[j]) < 1e-7


@pytest.mark.parametrize("seed", range(4))
def test_kkt_after_block_update(seed):
    """Projected gradient conditions: x > 0 => df/dx = 0 ; x = 0 => df/dx >= 0."""
    rs = np.random.default_rng(200 + seed)
    X, B, C = _rand_problem(rs, 7, 9, 3)
    R = X - B @ C
    for k in range(3):
        A = R + np.outer(B[:, k], C[k, :])
        B[:, k], _ = O.update_b_hals(A, C[k, :], B[:, k])
        grad_b = -(A - np.outer(B[:, k], C[k, :])) @ C[k, :]
        assert np.all(np.abs(grad_b[B[:, k] > 0]) < 1e-10)
        assert np.all(grad_b[B[:, k] == 0] >= -1e-10)
        C[k, :], _ = O.update_c_hals(A, B[:, k], C[k, :])
        grad_c = -B[:, k] @ (A - np.outer(B[:, k], C[k, :]))
        assert np.all(np.abs(grad_c[C[k, :] > 0]) < 1e-10)
        assert np.all(grad_c[C[k, :] == 0] >= -1e-10)
        R = A - np.outer(B[:, k], C[k, :])


# ----------------------------------------------------------------- invariants
@pytest.mark.parametrize("order", ["hals", "dbcd"])
def test_monotone_and_residual_invariant(order):
    """Monotone: f never increases after a block step.  Kept residual: R == X - BC."""
    rs = np.random.default_rng(7)
    X, B, C = _rand_problem(rs, 30, 40, 5)
    fs = [O.objective(X, B, C)]

    def on_block(kind, k, Bc, Cc, R):
        f = O.objective(X, Bc, Cc)
        assert f <= fs[-1] * (1 + 1e-12) + 1e-300
        fs.append(f)
        assert np.max(np.abs(R - (X - Bc @ Cc))) <= 1e-12 * max(1.0, np.max(np.abs(X)))

    sweep = O.sweep_hals if order == "hals" else O.sweep_dbcd
    R = None
    for _ in range(8):
        B, C, R, _ = sweep(X, B, C, R, on_block=on_block)
        assert B.min() >= 0 and C.min() >= 0
        assert not np.any(np.signbit(B)) and not np.any(np.signbit(C))
    assert fs[-1] < fs[0]


def test_did_equals_dbcd_literal_form():
    """Incremental form: Algorithm 3 (W, V, delta b) equals DBCD with a kept residual."""
    rs = np.random.default_rng(11)
    X, B, C = _rand_problem(rs, 25, 60, 6)
    B1, C1, R1 = B.copy(), C.copy(), None
    B2, C2 = B.copy(), C.copy()
    for _ in range(10):
        B1, C1, R1, _ = O.sweep_dbcd(X, B1, C1, R1)
        B2, C2, _ = O.sweep_did(X, B2, C2)
        assert np.max(np.abs(B1 - B2)) <= 1e-12 * max(1.0, np.max(np.abs(B1)))
        assert np.max(np.abs(C1 - C2)) <= 1e-12 * max(1.0, np.max(np.abs(C1)))


def test_same_iteration_count_did_dbcd():
    """Section 5: DID takes exactly as many iterations as DBCD/BCD (paper rule)."""
    rs = np.random.default_rng(3)
    X, B, C = _rand_problem(rs, 12, 50, 3, low_rank=True)
    r_did = O.factor(X, B, C, order="did", max_iter=2000, tol=1e-6, stop="paper_eps")
    r_dbcd = O.factor(X, B, C, order="dbcd", max_iter=2000, tol=1e-6, stop="paper_eps")
    assert r_did["iters"] == r_dbcd["iters"] < 2000
    assert r_did["trace"][-1] <= 1e-6 * r_did["trace"][0]


# -------------------------------------------------------------- special cases
@pytest.mark.parametrize("seed", range(3))
def test_rank_one_recovered_in_one_sweep(seed):
    """Exact rank-one recovery: K = 1, X = u v^T with u, v > 0: one HALS sweep reaches f = 0."""
    rs = np.random.default_rng(seed)
    u, v = rs.uniform(0.1, 1, 17), rs.uniform(0.1, 1, 23)
    X = np.outer(u, v)
    B, C, R, _ = O.sweep_hals(X, rs.uniform(0.1, 1, (17, 1)), rs.uniform(0.1, 1, (1, 23)))
    assert 0.5 * np.sum(R * R) <= 1e-24 * np.sum(X * X)
    assert O.objective(X, B, C) <= 1e-24 * np.sum(X * X)


@pytest.mark.parametrize("order", ["hals", "dbcd", "did"])
def test_exact_factorisation_is_fixed_point(order):
    """Fixed point: with X = B0 C0 and start (B0, C0), a sweep changes nothing."""
    rs = np.random.default_rng(5)
    B0, C0 = rs.uniform(0, 1, (9, 4)), rs.uniform(0, 1, (4, 13))
    X = B0 @ C0
    r = O.factor(X, B0, C0, order=order, max_iter=1, stop="none")
    np.testing.assert_allclose(r["B"], B0, rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(r["C"], C0, rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("order", ["hals", "dbcd", "did"])
def test_equivariance(order):
    """Equivariance: permuting columns of X permutes C; permuting rows permutes B;
    scaling X and the start of B by a scales B only."""
    rs = np.random.default_rng(9)
    X, B, C = _rand_problem(rs, 11, 14, 3)
    base = O.factor(X, B, C, order=order, max_iter=3, stop="none")
    pc = rs.permutation(14)
    r = O.factor(X[:, pc], B, C[:, pc], order=order, max_iter=3, stop="none")
    np.testing.assert_allclose(r["C"], base["C"][:, pc], rtol=1e-11, atol=1e-13)
    np.testing.assert_allclose(r["B"], base["B"], rtol=1e-11, atol=1e-13)
    pr = rs.permutation(11)
    r = O.factor(X[pr, :], B[pr, :], C, order=order, max_iter=3, stop="none")
    np.testing.assert_allclose(r["B"], base["B"][pr, :], rtol=1e-11, atol=1e-13)
    np.testing.assert_allclose(r["C"], base["C"], rtol=1e-11, atol=1e-13)
    a = 3.0
    r = O.factor(a * X, a * B, C, order=order, max_iter=3, stop="none")
    np.testing.assert_allclose(r["B"], a * base["B"], rtol=1e-11, atol=1e-13)
    np.testing.assert_allclose(r["C"], base["C"], rtol=1e-11, atol=1e-13)


def test_degenerate_blocks_left_unchanged():
    """Zero-norm rule: a zero row of C keeps b_k; a b_k projected to zero keeps c_k."""
    rs = np.random.default_rng(4)
    X, B, C = _rand_problem(rs, 6, 8, 3)
    C[1, :] = 0.0
    B2, C2, R, d = O.sweep_hals(X, B, C)
    np.testing.assert_array_equal(B2[:, 1], B[:, 1])
    assert d >= 1
    assert np.max(np.abs(R - (X - B2 @ C2))) < 1e-12
    # a block whose optimal b is zero: X = 0 forces b' = 0, then c is kept
    Z = np.zeros((4, 5))
    B3, C3, R3, d3 = O.sweep_hals(Z, np.ones((4, 1)), np.ones((1, 5)))
    assert np.all(B3 == 0) and np.all(C3 == 1.0) and d3 == 1


def test_init_scale_is_least_squares_scale():
    """Initial scaling: alpha = <X,BC>/||BC||^2 is the least-squares scale (library lstsq)."""
    rs = np.random.default_rng(2)
    X, B, C = _rand_problem(rs, 8, 10, 3)
    Bs, Cs = O.init_scale(X, B, C)
    alpha = np.linalg.lstsq((B @ C).reshape(-1, 1), X.reshape(-1), rcond=None)[0][0]
    np.testing.assert_allclose(Bs @ Cs, alpha * (B @ C), rtol=1e-12)
    np.testing.assert_allclose(Bs / B, np.sqrt(alpha), rtol=1e-12)


def test_stopping_rules():
    rs = np.random.default_rng(8)
    X, B, C = _rand_problem(rs, 10, 30, 2)
    r = O.factor(X, B, C, order="hals", max_iter=500, tol=1e-4, stop="relchange")
    t = r["trace"]
    assert r["iters"] < 500
    assert abs(t[-2] - t[-1]) / t[-2] < 1e-4
    for i in range(1, len(t) - 1):
        assert abs(t[i - 1] - t[i]) / t[i - 1] >= 1e-4
    r = O.factor(X, B, C, order="hals", max_iter=7, stop="none")
    assert r["iters"] == 7 and len(r["trace"]) == 8


def test_workload_sweep_decreases_objective():
    """The 200x1000 K=10 planted workload: objective trace non-increasing."""
    X, M, N, K = W.make("planted_uniform_200x1000_k10", seed=0)
    B, C = W.init_factors(M, N, K, 0)
    r = O.factor(X, B, C, order="hals", max_iter=10, stop="none")
    t = r["trace"]
    assert np.all(np.diff(t) <= 1e-12 * t[:-1])
    assert r["B"].min() >= 0 and r["C"].min() >= 0
