"""FP64 CPU oracle for DID / DBCD / HALS nonnegative matrix factorisation.

TEST INFRASTRUCTURE ONLY.  This module is the plain, slow, obviously correct
statement of what the GPU library computes.  Only the tests, the smoke check
and the benchmark's CPU-baseline leg may import it; the product path never
does.  It shares no code with the CUDA library and imports nothing from it.

Problem (Section 1, the optimisation problem ``opt:nmf``):
    minimise f(B, C) = 1/2 ||X - B C||_F^2  subject to  B >= 0, C >= 0,
with X (M x N, one sample per column), B (M x K), C (K x N).  ``b_k`` is
column k of B, ``c_k`` is row k of C (the paper's c_k^r).

Everything is float64 NumPy; a matrix product or a vector dot from NumPy is
the only library step.  Sums follow NumPy's order (the result is exact up to
rounding order).

Readings of the paper taken here (each is a choice the paper leaves open):
* Zero denominator (the zero-norm rule): when ||c_k||^2 == 0 (resp.
  ||b_k||^2 == 0) the block b_k (resp. c_k) is left unchanged.  The paper only says the methods can fail
  when a norm is near zero (Section 5); keeping the block is a valid exact
  minimiser because every value of the block gives the same objective.
* Projection: [z]_+ = z if z > 0 else +0.0 (so -0.0 and NaN map to +0.0).
* Block orders: ``sweep_hals`` takes b_1 c_1 b_2 c_2 ... (Section 2, HALS);
  ``sweep_dbcd`` takes c_1..c_K then b_1..b_K (Algorithm 2); ``sweep_did``
  is the incremental form with one reduction (Algorithm 3).  The paper states
  that HALS, (D)BCD and DID share their update rules and differ only in the
  order (Section 5, "Correctness").
* Initial scaling (optional): B and C are both multiplied by sqrt(alpha),
  alpha = <X, BC> / ||BC||_F^2, the least-squares scale of BC onto X; the
  paper asks for "well scaled initial points" without a formula (Section 5).
* Stopping: relative change |f_{t-1} - f_t| / f_{t-1} < tol, or f_t == 0;
  the paper's own rule ||E^t||^2 <= eps ||E^0||^2 (Section 5) is ``paper_eps``.
* Inner repeats (the acceleration the paper leaves to future work, Section 6,
  in the manner of Gillis & Glineur's accelerated HALS, Neural Computation
  24(4), 2012): ``sweep_did(..., inner_c, inner_b)`` runs Algorithm 3's C step
  inner_c times and then its B step inner_b times per iteration, a fixed count
  each (their relative-change exit of the inner loop is not taken).  Every
  repeat is the same exact block minimisation, applied to the current residual.
"""

import numpy as np

__all__ = [
    "project", "residual", "objective", "update_b_hals", "update_c_hals",
    "sweep_hals", "sweep_dbcd", "sweep_did", "init_scale", "factor",
]


def project(z):
    """[z]_+ = max{0, z} (Section 2, HALS closed forms), -0 and NaN -> +0."""
    z = np.asarray(z, dtype=np.float64)
    return np.where(z > 0.0, z, 0.0)


def residual(X, B, C):
    """E = X - B C (Section 4.2: the residual matrix)."""
    return np.asarray(X, np.float64) - np.asarray(B, np.float64) @ np.asarray(C, np.float64)


def objective(X, B, C):
    """f(B, C) = 1/2 ||X - B C||_F^2 (Section 1, problem opt:nmf)."""
    E = residual(X, B, C)
    return 0.5 * float(np.sum(E * E))


# ---------------------------------------------------------------------------
# Rank-one closed forms (Section 2, HALS): with A = X - sum_{i != k} b_i c_i,
#   b_k := [(c_k c_k^T)^{-1} (A c_k^T)]_+ ,  c_k := [(b_k^T b_k)^{-1} (A^T b_k)]_+
# ---------------------------------------------------------------------------

def update_b_hals(A, c, b_old):
    """Minimiser of ||A - b c||_F^2 over b >= 0 (HALS b_k closed form)."""
    cc = float(c @ c)
    if cc == 0.0:                       # zero-norm rule: block left unchanged
        return np.array(b_old, dtype=np.float64), False
    return project((A @ c) / cc), True


def update_c_hals(A, b, c_old):
    """Minimiser of ||A - b c||_F^2 over c >= 0 (HALS c_k closed form)."""
    bb = float(b @ b)
    if bb == 0.0:                       # zero-norm rule
        return np.array(c_old, dtype=np.float64), False
    return project((b @ A) / bb), True


def sweep_hals(X, B, C, R=None, on_block=None):
    """One sweep in the order b_1, c_1, b_2, c_2, ..., b_K, c_K.

    For each k the residual without block k, A = R + b_k c_k, is formed; b_k and
    then c_k take their closed forms; the residual becomes R = A - b_k c_k.
    ``R`` is the kept residual X - BC (recomputed densely when None).
    ``on_block(kind, k, B, C, R)`` is called after every block step (tests).
    Returns (B, C, R, degenerate_events).
    """
    B = np.array(B, dtype=np.float64)
    C = np.array(C, dtype=np.float64)
    R = residual(X, B, C) if R is None else np.array(R, dtype=np.float64)
    K = B.shape[1]
    degenerate = 0
    for k in range(K):
        A = R + np.outer(B[:, k], C[k, :])
        B[:, k], ok = update_b_hals(A, C[k, :], B[:, k])
        degenerate += not ok
        R = A - np.outer(B[:, k], C[k, :])
        if on_block is not None:
            on_block("b", k, B, C, R)
        C[k, :], ok = update_c_hals(A, B[:, k], C[k, :])
        degenerate += not ok
        R = A - np.outer(B[:, k], C[k, :])
        if on_block is not None:
            on_block("c", k, B, C, R)
    return B, C, R, degenerate


def _c_step(B, C, E, on_block=None):
    """C update of Algorithms 2 and 3, all columns at once.

    Per column j and i = 1..K, equations up:c (Section 4.1):
        e_j := e_j + b_i c_ij ;  c_ij := [b_i^T e_j / b_i^T b_i]_+ ;  e_j := e_j - b_i c_ij
    The columns are independent, so the j loop is a vector operation.
    """
    degenerate = 0
    for i in range(B.shape[1]):
        b = B[:, i]
        bb = float(b @ b)
        E += np.outer(b, C[i, :])
        if bb == 0.0:                   # zero-norm rule
            degenerate += 1
        else:
            C[i, :] = project((b @ E) / bb)
        E -= np.outer(b, C[i, :])
        if on_block is not None:
            on_block("c", i, B, C, E)
    return degenerate


def sweep_dbcd(X, B, C, R=None, on_block=None):
    """One iteration of DBCD (Algorithm 2): C update, then B column by column.

    B step, per i (Section 4.1, messages y_j, z_j):
        e_j := e_j + b_i c_ij ; y = sum_j e_j c_ij ; z = sum_j c_ij^2 ;
        b_i := [y / z]_+ ;  e_j := e_j - b_i c_ij
    The residual is the kept ``R`` (Algorithm 2 sets e_j := x_j - B c_j at the
    top of each iteration; with R == X - BC that is the same vector).
    """
    B = np.array(B, dtype=np.float64)
    C = np.array(C, dtype=np.float64)
    E = residual(X, B, C) if R is None else np.array(R, dtype=np.float64)
    degenerate = _c_step(B, C, E, on_block)
    for i in range(B.shape[1]):
        c = C[i, :]
        E += np.outer(B[:, i], c)
        y = E @ c
        z = float(c @ c)
        if z == 0.0:                    # zero-norm rule
            degenerate += 1
        else:
            B[:, i] = project(y / z)
        E -= np.outer(B[:, i], c)
        if on_block is not None:
            on_block("b", i, B, C, E)
    return B, C, E, degenerate


def sweep_did(X, B, C, inner_c=1, inner_b=1):
    """One iteration of DID (Algorithm 3): what it computes, in its order.

    - The residual E := X - B C, every column recomputed from X.
    - The C step: the updates of equations up:c.
    - The one reduction: W := E C^T (M x K; column i is sum_j e_j c_ij, the
      matrices W_j summed over j) and V := lower triangle of C C^T (the V_j
      summed over j).
    - The B step, for i = 1..K:
          b_i^{t+1} := [b_i^t + w_i / v_ii - sum_{k<i} (v_ik / v_ii) delta b_k]_+
          delta b_i := b_i^{t+1} - b_i^t
    With inner repeats, the C step runs inner_c times on the kept residual,
    and the reduction with the B step runs inner_b times; before each further
    B repeat the residual takes the paper's incremental rule
    E := E - delta b_i c_i for every i.
    inner_c = 0 (or inner_b = 0) leaves C (or B) fixed.
    Returns (B, C, degenerate_events).
    """
    B = np.array(B, dtype=np.float64)
    C = np.array(C, dtype=np.float64)
    E = residual(X, B, C)
    degenerate = 0
    for _ in range(inner_c):
        degenerate += _c_step(B, C, E)
    K = B.shape[1]
    for rep in range(inner_b):
        W = E @ C.T
        V = np.tril(C @ C.T)
        dB = np.zeros_like(B)
        for i in range(K):
            vii = V[i, i]
            if vii == 0.0:                  # zero-norm rule: b_i unchanged, delta b_i = 0
                degenerate += 1
                continue
            s = B[:, i] + W[:, i] / vii
            for k in range(i):
                s = s - (V[i, k] / vii) * dB[:, k]
            b_new = project(s)
            dB[:, i] = b_new - B[:, i]
            B[:, i] = b_new
        if rep + 1 < inner_b:
            E -= dB @ C                     # E := E - sum_i delta b_i c_i
    return B, C, degenerate


def init_scale(X, B, C):
    """Initial scaling: B and C times sqrt(alpha), alpha = <X, BC> / ||BC||_F^2."""
    B = np.asarray(B, np.float64)
    C = np.asarray(C, np.float64)
    P = B @ C
    den = float(np.sum(P * P))
    if den == 0.0:
        return B.copy(), C.copy()
    alpha = float(np.sum(np.asarray(X, np.float64) * P)) / den
    if alpha <= 0.0:
        return B.copy(), C.copy()
    s = np.sqrt(alpha)
    return B * s, C * s


def factor(X, B, C, order="hals", max_iter=100, tol=0.0, stop="relchange", inner_c=1, inner_b=1):
    """Run sweeps until a stopping rule holds.

    order: "hals" (b_k then c_k per k), "dbcd" (Algorithm 2, kept residual) or
    "did" (Algorithm 3 as written).  Returns dict with B, C, the objective
    trace (f_0 at the start point, then f after each sweep) and the count of
    sweeps done.  The trace value after a sweep is 1/2 ||R||^2 of the kept
    residual for "hals"/"dbcd" and 1/2 ||X - BC||^2 for "did".
    inner_c, inner_b: repeats of the C and B steps per iteration ("did" only).
    stop: "relchange" -> |f_{t-1} - f_t| / f_{t-1} < tol or f_t == 0;
          "paper_eps" -> f_t <= tol * f_0 (Section 5, with eps = tol);
          "none"      -> exactly max_iter sweeps.
    """
    if order != "did" and (inner_c, inner_b) != (1, 1):
        raise ValueError("inner repeats are defined for the did order only")
    B = np.array(B, dtype=np.float64)
    C = np.array(C, dtype=np.float64)
    R = residual(X, B, C)
    trace = [0.5 * float(np.sum(R * R))]
    degenerate = 0
    it = 0
    while it < max_iter:
        if order == "hals":
            B, C, R, d = sweep_hals(X, B, C, R)
            f = 0.5 * float(np.sum(R * R))
        elif order == "dbcd":
            B, C, R, d = sweep_dbcd(X, B, C, R)
            f = 0.5 * float(np.sum(R * R))
        elif order == "did":
            B, C, d = sweep_did(X, B, C, inner_c, inner_b)
            f = objective(X, B, C)
        else:
            raise ValueError(order)
        degenerate += d
        it += 1
        trace.append(f)
        prev = trace[-2]
        if stop == "relchange":
            if f == 0.0 or (prev > 0.0 and abs(prev - f) / prev < tol):
                break
        elif stop == "paper_eps":
            if f <= tol * trace[0]:
                break
        elif stop != "none":
            raise ValueError(stop)
    return dict(B=B, C=C, trace=np.array(trace), iters=it, degenerate=degenerate)
