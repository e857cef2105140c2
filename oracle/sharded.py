"""FP64 CPU oracle of one sWLR iteration (Algorithm 1) split by rows, for the sharding
identity: the per-row steps of Section 3 are local to a block of rows, and every
cross-row quantity is a sum over rows, so a rank that owns rows [r0, r1) needs only
summed partials from the other ranks.

TEST INFRASTRUCTURE ONLY, under the same rules as fp64.py: only the test suite may import
it, and it imports nothing from the product package.  Plain float64 NumPy; library steps:
``numpy.linalg.cholesky``, ``numpy.linalg.eigh``, ``numpy.linalg.solve``,
``scipy.linalg.solve_triangular``.

The iteration, written so that each line is either row-local or a sum over rows:
  * setup (once):   K = A2^T A2 = sum over rows,  ||A2||_F^2 = sum over rows;
  * exchange 1:     S1 = X1^T X1 (sum over rows) -> X1 = Q1 R1 with R1^T R1 = S1
                    (the triangular factor of a thin QR of a full-rank X1 is the
                    Cholesky factor of its Gram, unique with a positive diagonal);
  * exchange 2:     [S2 | T] = Q1^T [Q1 A2] (sum over rows), Q1 = X1 R1^{-1} row-local;
                    S2 = R2^T R2, Q = Q1 R2^{-1}, R = R2 R1 (CholeskyQR2), so
                    B = Q^T A2 = R2^{-T} T and C = R^{-1} B (Section 3: C = R^{-1} Q^T A2);
  * no exchange:    G2 = (P_perp A2)^T (P_perp A2) = K - B^T B (Q has orthonormal columns),
                    its s = r - k leading eigenpairs (sigma_j^2, V_s) give
                    D = (P_perp A2) V_s V_s^T = H_s(P_perp A2) (Eq. 2); every rank forms
                    the same C and V_s from the same sums;
  * row-local:      P_perp A2 (rows) = A2 - X1 C (since X1 C = Q Q^T A2),
                    E = A1 o W1 o W1 + (A2 - D) C^T,
                    X1_{p+1}(i,:) = E(i,:) (diag(W1(i,:)^2) + C C^T)^{-1};
  * exchange 3:     F_p = sum over rows of ||(A1 - X1) o W1||^2 + ||P_perp A2 - D||^2
                    (scalars; they can travel with the next iteration's exchange 1).

Pinned by tests/test_sharding.py against fp64.swlr_step on the whole problem (Householder
QR and a dense SVD, a different route to the same step).
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import solve_triangular

__all__ = ["setup_partials", "gram_x1", "qr_factor", "coef_partials", "global_factors",
           "rows_update"]


def setup_partials(A_rows: np.ndarray, k: int):
    """(K, ||A2||^2) of a block of rows: A2(rows)^T A2(rows) and its squared norm."""
    A2 = np.asarray(A_rows, dtype=np.float64)[:, k:]
    return A2.T @ A2, float(np.sum(A2 * A2))


def gram_x1(X1_rows: np.ndarray) -> np.ndarray:
    """S1 partial: X1(rows)^T X1(rows)."""
    X1 = np.asarray(X1_rows, dtype=np.float64)
    return X1.T @ X1


def qr_factor(S: np.ndarray) -> np.ndarray:
    """Upper triangular R with R^T R = S (S = Y^T Y of a full-rank Y, so Y = (Y R^{-1}) R
    is the thin QR of Y with a positive diagonal)."""
    return np.linalg.cholesky(S).T


def coef_partials(A_rows: np.ndarray, X1_rows: np.ndarray, R1: np.ndarray, k: int):
    """Exchange-2 partial: Q1(rows)^T [Q1(rows) A2(rows)] with Q1 = X1 R1^{-1}."""
    X1 = np.asarray(X1_rows, dtype=np.float64)
    Q1 = solve_triangular(R1, X1.T, trans="T", lower=False).T     # X1 R1^{-1}
    A2 = np.asarray(A_rows, dtype=np.float64)[:, k:]
    return Q1.T @ np.hstack([Q1, A2])


def global_factors(R1: np.ndarray, Q1tQ1A2: np.ndarray, K: np.ndarray, s: int):
    """C, V_s and the s leading sigma_j^2 of P_perp A2 from the summed partials.
    Q1tQ1A2 = [S2 | T] (k x (k + n2)); K = A2^T A2."""
    k = R1.shape[0]
    S2, T = Q1tQ1A2[:, :k], Q1tQ1A2[:, k:]
    R2 = qr_factor(S2)
    B = solve_triangular(R2, T, trans="T", lower=False)          # R2^{-T} T = Q^T A2
    R = R2 @ R1
    C = solve_triangular(R, B, lower=False)                       # R^{-1} B
    n2 = K.shape[0]
    if s <= 0 or n2 == 0:
        return C, np.zeros((n2, 0)), np.zeros(0)
    G2 = K - B.T @ B
    lam, V = np.linalg.eigh(G2)
    order = np.argsort(lam)[::-1][:s]
    return C, V[:, order], np.maximum(lam[order], 0.0)


def rows_update(A_rows: np.ndarray, W1_rows: np.ndarray, X1_rows: np.ndarray, C: np.ndarray,
                Vs: np.ndarray):
    """Row-local part of the loop body for a block of rows: X1_{p+1}(rows) and the block's
    objective partials (||(A1 - X1) o W1||^2, ||P_perp A2 - D||^2)."""
    k = C.shape[0]
    A = np.asarray(A_rows, dtype=np.float64)
    W1 = np.asarray(W1_rows, dtype=np.float64)
    X1 = np.asarray(X1_rows, dtype=np.float64)
    A1, A2 = A[:, :k], A[:, k:]
    P = A2 - X1 @ C
    D = (P @ Vs) @ Vs.T
    E = A1 * W1 * W1 + (A2 - D) @ C.T
    G = C @ C.T
    M = np.repeat(G[None, :, :], A.shape[0], axis=0)
    idx = np.arange(k)
    M[:, idx, idx] += W1 ** 2
    X1n = np.linalg.solve(M, E[:, :, None])[:, :, 0]
    wterm = float(np.sum(((A1 - X1) * W1) ** 2))
    rterm = float(np.sum((P - D) ** 2))
    return X1n, wterm, rterm
