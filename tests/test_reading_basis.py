"""Pins for the reading that step a1 may use any orthonormal basis of range(X1).

Algorithm 1 writes X1 = QR; the FP32 path's steady state takes the symmetric second factor
(I + F)^{1/2} of Q1^T Q1 = I + F (Q1 = X1 R_p^{-1}, R_p the previous iteration's factor)
and sums its inverse as a binomial series.  These tests check, against the oracle's
Householder route, that what the step uses does not depend on that choice (C, the
projector Q Q^T, so B^T B and ||B||^2, and D), and that the series with its term rule
leaves Q orthonormal to about float precision for ||F||_F <= 0.06."""
import numpy as np
import pytest

import oracle


def _problem(seed, m=60, n=26, k=5):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, 4)) @ rng.standard_normal((4, n)) + 0.2 * rng.standard_normal((m, n))
    X1 = rng.standard_normal((m, k))
    return A, X1, rng


def _series_inverse_sqrt(F):
    """(I + F)^{-1/2} - I by the binomial series, with the number of terms chosen from
    ||F||_F as the FP32 path does (remainder ~0.3 ||F||^(m+1) below 3e-8)."""
    nf = np.linalg.norm(F)
    assert nf <= 0.06
    m, pw = 1, nf
    while m < 8 and 0.3 * pw * nf > 3e-8:
        pw *= nf
        m += 1
    c = [1.0]
    for j in range(1, m + 1):
        c.append(c[-1] * (1 - 2 * j) / (2 * j))
    k = F.shape[0]
    P = c[m] * np.eye(k)
    for j in range(m - 1, 0, -1):
        P = c[j] * np.eye(k) + F @ P
    return F @ P, m


def _basis_from_previous(X1, X1_prev, exact):
    """Q and R with X1 = Q R from the previous iterate's triangular factor and the
    symmetric second factor (I + F)^{1/2}, its inverse either exact (eigendecomposition)
    or the truncated series."""
    k = X1.shape[1]
    _, Rp = np.linalg.qr(X1_prev)
    Q1 = X1 @ np.linalg.inv(Rp)
    F = Q1.T @ Q1 - np.eye(k)
    if exact:
        w, V = np.linalg.eigh(np.eye(k) + F)
        M = (V / np.sqrt(w)) @ V.T
        terms = 0
    else:
        N, terms = _series_inverse_sqrt(F)
        M = np.eye(k) + N
    Q = Q1 @ M
    R = np.linalg.solve(M, Rp)          # X1 = Q1 Rp = Q M^{-1} Rp
    return Q, R, np.linalg.norm(F), terms


@pytest.mark.parametrize("seed,step", [(0, 1e-3), (1, 1e-2), (2, 2.5e-2)])
def test_symmetric_second_factor_gives_the_same_step(seed, step):
    A, X1, rng = _problem(seed)
    k, s = X1.shape[1], 3
    A2 = A[:, k:]
    X1_prev = X1 + step * rng.standard_normal(X1.shape) * np.abs(X1).mean()
    ref = oracle.cd_step(A2, X1, s)
    Q, R, nf, _ = _basis_from_previous(X1, X1_prev, exact=True)
    assert nf <= 0.06
    # Q orthonormal and spanning range(X1), R not triangular
    assert np.abs(Q.T @ Q - np.eye(k)).max() < 1e-12
    assert np.abs(Q @ R - X1).max() < 1e-10 * np.abs(X1).max()
    assert np.abs(np.tril(R, -1)).max() > 1e-6
    B = Q.T @ A2
    C = np.linalg.solve(R, B)
    assert np.abs(C - ref.C).max() < 1e-9 * max(1.0, np.abs(ref.C).max())
    assert np.abs(Q @ Q.T - ref.Q @ ref.Q.T).max() < 1e-12
    assert abs(np.sum(B * B) - np.sum(ref.B * ref.B)) < 1e-10 * np.sum(ref.B * ref.B)
    P = A2 - Q @ B
    assert np.abs(oracle.hard_threshold(P, s) - ref.D).max() < 1e-9 * max(1.0, np.abs(ref.D).max())
    # the truncated series is that factor to within its remainder bound (float precision)
    Qs, Rs, _, terms = _basis_from_previous(X1, X1_prev, exact=False)
    assert 1 <= terms <= 8
    assert np.abs(Qs.T @ Qs - np.eye(k)).max() < 1e-7
    Cs = np.linalg.solve(Rs, Qs.T @ A2)
    assert np.abs(Cs - ref.C).max() < 1e-6 * max(1.0, np.abs(ref.C).max())


def test_symmetric_square_root_of_the_gram_gives_the_same_C_and_D():
    # the plainest non-triangular factor: R = (X1^T X1)^{1/2} (eigendecomposition)
    A, X1, _ = _problem(3)
    k, s = X1.shape[1], 2
    A2 = A[:, k:]
    w, V = np.linalg.eigh(X1.T @ X1)
    R = (V * np.sqrt(w)) @ V.T
    Q = X1 @ np.linalg.inv(R)
    ref = oracle.cd_step(A2, X1, s)
    C = np.linalg.solve(R, Q.T @ A2)
    assert np.abs(C - ref.C).max() < 1e-9 * max(1.0, np.abs(ref.C).max())
    D = oracle.hard_threshold(A2 - Q @ (Q.T @ A2), s)
    assert np.abs(D - ref.D).max() < 1e-9 * max(1.0, np.abs(ref.D).max())


@pytest.mark.parametrize("target", [1e-5, 1e-3, 1e-2, 0.05])
def test_series_term_rule_keeps_Q_orthonormal(target):
    # F of the size the rule admits: the truncated series leaves Q^T Q within 1e-8 of I
    rng = np.random.default_rng(7)
    m, k = 400, 20
    Q0, _ = np.linalg.qr(rng.standard_normal((m, k)))
    E = rng.standard_normal((m, k))
    Q1 = Q0 + E * (target / (2 * np.linalg.norm(Q0.T @ E + E.T @ Q0)))
    F = Q1.T @ Q1 - np.eye(k)
    if np.linalg.norm(F) > 0.06:
        pytest.skip("perturbation above the series' range")
    N, terms = _series_inverse_sqrt(F)
    Q = Q1 @ (np.eye(k) + N)
    assert np.abs(Q.T @ Q - np.eye(k)).max() < 1e-8
    assert 1 <= terms <= 8
