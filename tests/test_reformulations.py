"""The algebra the GPU kernels use in place of the paper's plain forms, checked
in float64 against the oracle (no GPU needed).

1. Deferred write-back (interleaved order).  For a pair (k, k+1) the pass for
   k updates c_k but stores nothing; R_s stays stale by the pending change
   P_k = b_k c_k - b_k' c_k'.  The b-update for k+1 takes
   R' c_{k+1}^T = R_s c_{k+1}^T + b_k (c_k . c_{k+1}) - b_k' (c_k' . c_{k+1}),
   the pass for k+1 takes b_{k+1}'^T R' = b_{k+1}'^T R_s + beta_o c_k -
   beta_n c_k' (beta_o = b_{k+1}' . b_k, beta_n = b_{k+1}' . b_k'), and then
   writes R_s + P_k + P_{k+1} once.  Exactly the HALS sweep of Section 2.
2. Batched Algorithm 3.  The stored R_s carries the last B step's change
   D = delta B pending, E = R_s - D C.  The C step takes g = B^T R_s -
   (B^T D) C and G = B^T B, per column the K updates of equations up:c with
   t_i = g_i - sum_l G_il Delta_l; then R_s -= [D B][C_old; Delta] (one
   rank-2K product), after which R_s holds E' = E - B Delta exactly; the B
   step takes W = E' C'^T, V = C' C'^T and the delta-b rule of Section 4.2,
   and leaves D := delta B pending; the objective after it is
   ||E''||^2 = ||E'||^2 - 2 sum(delta B o W) + sum((delta B^T delta B) o V).
   Exactly the oracle's Algorithm 3.
These are models of the reformulations written from the formulas above, in
plain NumPy; they share nothing with the CUDA sources.
"""

import numpy as np
import pytest

from oracle import did_oracle as O


def _problem(seed, M, N, K, zero_row=False):
    rs = np.random.default_rng(seed)
    X = rs.uniform(0, 1, (M, N)) * (rs.uniform(0, 1, (M, N)) > 0.3)
    B = rs.uniform(0, 1, (M, K))
    C = rs.uniform(0, 1, (K, N))
    if zero_row:
        C[K // 2, :] = 0.0
    return X, B, C


def _proj(z):
    return np.where(z > 0, z, 0.0)


def deferred_sweep(X, B, C, R):
    """One interleaved sweep in the deferred form (pairs (0,1), (2,3), ...)."""
    B = B.copy()
    C = C.copy()
    Rs = R.copy()
    K = B.shape[1]
    # partials for b_1 from the stored residual (the prologue or the refresh)
    s = Rs @ C[0]
    pending = None                       # (b_old, b_new, c_old, c_new) of a deferred k
    for k in range(K):
        ck = C[k].copy()
        cc = float(ck @ ck)
        b_old = B[:, k].copy()
        b_new = b_old if cc == 0.0 else _proj(b_old + s / cc)
        B[:, k] = b_new
        bb = float(b_new @ b_new)
        # b_k'^T R' for every column, with the pending change of k-1 if any
        dot = b_new @ Rs
        if pending is not None:
            pbo, pbn, pco, pcn = pending
            dot = dot + float(b_new @ pbo) * pco - float(b_new @ pbn) * pcn
        c_new = ck if bb == 0.0 else _proj((dot + float(b_new @ b_old) * ck) / bb)
        C[k] = c_new
        deferred = pending is None and k % 2 == 0 and k + 1 < K
        knext = k + 1 if k + 1 < K else 0
        if deferred:
            # no store: the partials for k+1 come from R_s plus the pending change
            pending = (b_old, b_new, ck, c_new)
            cn = C[knext]
            s = Rs @ cn + b_old * float(ck @ cn) - b_new * float(c_new @ cn)
        else:
            if pending is not None:
                pbo, pbn, pco, pcn = pending
                Rs = Rs + np.outer(pbo, pco) - np.outer(pbn, pcn)
                pending = None
            Rs = Rs + np.outer(b_old, ck) - np.outer(b_new, c_new)
            s = Rs @ C[knext]
    return B, C, Rs


@pytest.mark.parametrize("M,N,K", [(7, 9, 1), (7, 9, 2), (6, 11, 3), (10, 8, 5), (12, 15, 6), (9, 20, 7)])
@pytest.mark.parametrize("zero_row", [False, True])
def test_deferred_write_back_is_the_hals_sweep(M, N, K, zero_row):
    X, B, C = _problem(M * 100 + N * 10 + K, M, N, K, zero_row)
    R = X - B @ C
    for sweep in range(3):
        Bo, Co, Ro, _ = O.sweep_hals(X, B, C, R=R)
        Bd, Cd, Rd = deferred_sweep(X, B, C, R)
        scale = 1.0 + np.abs(X).max()
        assert np.max(np.abs(Bd - Bo)) <= 1e-12 * scale * (1 + np.abs(Bo).max())
        assert np.max(np.abs(Cd - Co)) <= 1e-12 * scale * (1 + np.abs(Co).max())
        assert np.max(np.abs(Rd - Ro)) <= 1e-12 * scale * K
        B, C, R = Bo, Co, Ro


def batched_sweep(X, B, C, Rs, D):
    """One sweep of Algorithm 3 on a stored residual with a pending D = delta B."""
    B = B.copy()
    C = C.copy()
    K = B.shape[1]
    N = C.shape[1]
    # C step: g = B^T E = B^T R_s - (B^T D) C, G = B^T B
    g = B.T @ Rs - (B.T @ D) @ C
    G = B.T @ B
    C_old = C.copy()
    Delta = np.zeros_like(C)
    for j in range(N):
        for i in range(K):
            gii = G[i, i]
            if gii == 0.0:
                continue
            t = g[i, j] - G[i, :] @ Delta[:, j]        # b_i^T e_j on the current residual
            c_new = _proj(C[i, j] + t / gii)
            Delta[i, j] = c_new - C[i, j]
            C[i, j] = c_new
    # R_s -= [D B][C_old; Delta]: E' = R_s - D C_old - B Delta is now stored exactly
    Rs = Rs - D @ C_old - B @ Delta
    E1 = Rs                                              # E' (D applied)
    f1 = 0.5 * float(np.sum(E1 ** 2))
    # B step: W = E' C'^T, V = C' C'^T, delta-b rule
    W = E1 @ C.T
    Vf = C @ C.T
    dB = np.zeros_like(B)
    for i in range(K):
        vii = Vf[i, i]
        if vii == 0.0:
            continue
        s = B[:, i] + (W[:, i] - dB[:, :i] @ Vf[i, :i]) / vii
        b_new = _proj(s)
        dB[:, i] = b_new - B[:, i]
        B[:, i] = b_new
    # objective after the B step from W, V and delta B (no pass over R)
    f2 = f1 - float(np.sum(dB * W)) + 0.5 * float(np.sum((dB.T @ dB) * Vf))
    return B, C, Rs, dB, f2


@pytest.mark.parametrize("M,N,K", [(7, 9, 1), (6, 11, 3), (10, 8, 5), (12, 15, 6)])
@pytest.mark.parametrize("zero_row", [False, True])
def test_batched_form_is_algorithm_3(M, N, K, zero_row):
    X, B, C = _problem(M * 7 + N * 3 + K, M, N, K, zero_row)
    Rs = X - B @ C
    D = np.zeros_like(B)
    for sweep in range(3):
        Bo, Co, _ = O.sweep_did(X, B, C)
        Bb, Cb, Rs, D, f2 = batched_sweep(X, B, C, Rs, D)
        scale = 1.0 + np.abs(X).max()
        assert np.max(np.abs(Bb - Bo)) <= 1e-11 * scale * (1 + np.abs(Bo).max())
        assert np.max(np.abs(Cb - Co)) <= 1e-11 * scale * (1 + np.abs(Co).max())
        # the stored residual with its pending D is the true residual
        np.testing.assert_allclose(Rs - D @ Cb, X - Bb @ Cb, rtol=0, atol=1e-11 * scale * K)
        f_true = O.objective(X, Bo, Co)
        assert abs(f2 - f_true) <= 1e-11 * (f_true + scale ** 2)
        B, C = Bb, Cb
