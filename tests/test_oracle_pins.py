"""Pins for the FP64 oracle: each test checks the oracle against something the paper
or the mathematics fixes independently of the oracle's own formulas (closed forms,
constructions with a known answer, brute-force minimisation of the plain objective,
published generator outputs)."""
import math

import numpy as np
import pytest
from scipy.optimize import minimize

import oracle

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _orth(rng, m, n):
    q, _ = np.linalg.qr(rng.standard_normal((m, n)))
    return q


def _small_problem(seed=0, m=40, n=12, k=3, r=5, wlo=2.0, whi=6.0):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, 3)) @ rng.standard_normal((3, n)) + 0.3 * rng.standard_normal((m, n))
    W1 = rng.uniform(wlo, whi, size=(m, k))
    X0 = rng.standard_normal((m, k))
    return A, W1, X0, k, r


# ---------------------------------------------------------------- random init
def test_splitmix64_published_vector():
    # First outputs of SplitMix64 seeded with 0 (reference implementation by
    # Vigna, prng.di.unimi.it/splitmix64.c; Steele, Lea & Flood 2014).
    out = oracle.splitmix64(0, np.arange(3, dtype=np.uint64))
    assert [int(v) for v in out] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_random_init_is_standard_normal():
    from scipy import stats
    x = oracle.random_normal_init(20000, 3, seed=12345)
    assert x.shape == (20000, 3)
    for a in range(3):
        assert stats.kstest(x[:, a], "norm").pvalue > 1e-3
    # column-major counter layout: element (i, a) depends only on i + a*m
    y = oracle.random_normal_init(20000, 1, seed=12345)
    assert np.array_equal(x[:, 0], y[:, 0])


# ---------------------------------------------------------------- L0 closed forms
def test_hard_threshold_matches_construction():
    # A built from a known SVD: H_r(A) = U_r S_r V_r^T exactly (Eq. 2).
    rng = np.random.default_rng(1)
    U, V = _orth(rng, 30, 8), _orth(rng, 10, 8)
    sig = np.array([9.0, 7.0, 5.0, 4.0, 3.0, 2.0, 1.0, 0.5])
    A = (U * sig) @ V.T
    for r in (0, 1, 3, 8):
        ref = (U[:, :r] * sig[:r]) @ V[:, :r].T
        assert np.allclose(oracle.hard_threshold(A, r), ref, atol=1e-12)
        # Eckart-Young: the residual energy is the discarded singular values squared
        assert np.sum((A - oracle.hard_threshold(A, r)) ** 2) == pytest.approx(np.sum(sig[r:] ** 2), rel=1e-12, abs=1e-12)


def test_objective_hand_computed():
    # Eq. 8 on a 2x2 case computed by hand:
    # A = [[1,2],[3,4]], k=1, W1 = [[2],[1]], X1 = [[0],[1]], C = [[1]], D = 0
    # (1-0)^2*4 + (3-1)^2*1 + (2-0)^2 + (4-1)^2 = 4 + 4 + 4 + 9 = 21
    A = np.array([[1.0, 2.0], [3.0, 4.0]])
    F = oracle.objective(A, np.array([[2.0], [1.0]]), np.array([[0.0], [1.0]]),
                         np.array([[1.0]]), np.zeros((2, 1)))
    assert F == 21.0


def test_ghs_exact_on_constructed_input():
    # A2 = A1 c + D0 with rank(D0) = r - k: the constrained problem (Eq. 3) has zero
    # residual, so Theorem 1 must return A2 itself.
    rng = np.random.default_rng(2)
    m, k, n2, r = 20, 3, 9, 5
    A1 = rng.standard_normal((m, k))
    D0 = rng.standard_normal((m, r - k)) @ rng.standard_normal((r - k, n2))
    A2 = A1 @ rng.standard_normal((k, n2)) + D0
    assert np.allclose(oracle.ghs(A1, A2, r), A2, atol=1e-11)
    # and with r = k the answer is the plain projection onto range(A1)
    X2 = oracle.ghs(A1, A2, k)
    P = A1 @ np.linalg.lstsq(A1, A2, rcond=None)[0]
    assert np.allclose(X2, P, atol=1e-11)


def test_ghs_bruteforce_tiny():
    # Theorem 1 against a direct numerical minimisation of ||A2 - X2||^2 over all
    # X2 = A1 c + u v^T (every X2 with rank(A1 X2) <= 2 when k = 1).
    rng = np.random.default_rng(3)
    m, n2, r = 4, 3, 2
    A1 = rng.standard_normal((m, 1))
    A2 = rng.standard_normal((m, n2))

    def f(z):
        c, u, v = z[:n2], z[n2:n2 + m], z[n2 + m:]
        X2 = A1 @ c[None, :] + np.outer(u, v)
        return np.sum((A2 - X2) ** 2)

    best = min(minimize(f, rng.standard_normal(n2 + m + n2), method="BFGS", options={"gtol": 1e-12}).fun
               for _ in range(20))
    ghs_val = np.sum((A2 - oracle.ghs(A1, A2, r)) ** 2)
    assert ghs_val == pytest.approx(best, rel=1e-8, abs=1e-10)


# ---------------------------------------------------------------- L3 steps
def test_cd_step_is_the_minimiser_over_C_and_D():
    # For fixed X1, no (C, rank-s D) does better than the closed form of Section 3.
    rng = np.random.default_rng(4)
    m, n2, k, s = 5, 4, 1, 1
    A2 = rng.standard_normal((m, n2))
    X1 = rng.standard_normal((m, k))
    cd = oracle.cd_step(A2, X1, s)
    val = np.sum((A2 - X1 @ cd.C - cd.D) ** 2)

    def f(z):
        C = z[:n2].reshape(k, n2)
        u, v = z[n2:n2 + m], z[n2 + m:]
        return np.sum((A2 - X1 @ C - np.outer(u, v)) ** 2)

    best = min(minimize(f, rng.standard_normal(n2 + m + n2), method="BFGS", options={"gtol": 1e-12}).fun
               for _ in range(20))
    assert val == pytest.approx(best, rel=1e-8, abs=1e-10)
    # X1 C is the orthogonal projection of A2 onto range(X1)
    P = X1 @ np.linalg.lstsq(X1, A2, rcond=None)[0]
    assert np.allclose(X1 @ cd.C, P, atol=1e-12)
    # QR sign convention does not matter: Q Q^T and C are invariant
    assert np.allclose(cd.Q @ cd.Q.T @ A2, P, atol=1e-12)


def _F_of_X1(A, W1, X1, C, D):
    return oracle.objective(A, W1, X1, C, D)


def test_x1_update_is_stationary_and_minimal():
    # Eq. 9: the row update is the exact minimiser of F(., C_p, D_p).  Checked with a
    # central-difference gradient of the plain objective and random perturbations.
    A, W1, X0, k, r = _small_problem(seed=5, m=8, n=7, k=2, r=3)
    cd = oracle.cd_step(A[:, k:], X0, r - k)
    X1 = oracle.x1_update(A, W1, cd.C, cd.D)
    F0 = _F_of_X1(A, W1, X1, cd.C, cd.D)
    h = 1e-5
    g = np.zeros_like(X1)
    for i in range(X1.shape[0]):
        for a in range(k):
            Xp, Xm = X1.copy(), X1.copy()
            Xp[i, a] += h
            Xm[i, a] -= h
            g[i, a] = (_F_of_X1(A, W1, Xp, cd.C, cd.D) - _F_of_X1(A, W1, Xm, cd.C, cd.D)) / (2 * h)
    scale = np.abs(A).max() * (W1.max() ** 2 + np.abs(cd.C).max() ** 2)
    assert np.abs(g).max() < 1e-6 * scale
    rng = np.random.default_rng(6)
    for _ in range(20):
        assert _F_of_X1(A, W1, X1 + 1e-3 * rng.standard_normal(X1.shape), cd.C, cd.D) > F0


def test_row_constant_weights_identity():
    rng = np.random.default_rng(7)
    m, n, k, r = 50, 14, 4, 6
    A = rng.standard_normal((m, n))
    w = rng.uniform(1.0, 9.0, size=m)
    W1 = np.repeat(w[:, None], k, axis=1)
    X0 = rng.standard_normal((m, k))
    cd = oracle.cd_step(A[:, k:], X0, r - k)
    a = oracle.x1_update(A, W1, cd.C, cd.D)
    b = oracle.x1_update_row_constant(A, w, cd.C, cd.D)
    assert np.allclose(a, b, rtol=1e-12, atol=1e-12 * np.abs(a).max())


# ---------------------------------------------------------------- L3/L4 iteration
def test_objective_non_increasing():
    # Block-coordinate descent: (C, D) exact given X1 (Theorem 2) and the X1 step
    # exact given (C, D) (Eq. 9), so F_p cannot increase.
    A, W1, X0, k, r = _small_problem(seed=8, m=60, n=15, k=3, r=6)
    res = oracle.swlr(A, W1, r, X0, max_iter=40, stop="none")
    F = np.array(res.F)
    assert np.all(F[1:] <= F[:-1] * (1 + 1e-12))


def test_rank_bound_and_theorem2_structure():
    A, W1, X0, k, r = _small_problem(seed=9, m=60, n=15, k=3, r=6)
    res = oracle.swlr(A, W1, r, X0, max_iter=30, stop="none")
    X = np.hstack([res.X1, res.X2])
    sig = np.linalg.svd(X, compute_uv=False)
    assert sig[r] <= 1e-12 * sig[0]            # rank (X1 X2) <= r  (Section 3)
    # Theorem 2 form for the returned pair: X2 = GHS(X1, A2)
    assert np.allclose(res.X2, oracle.ghs(res.X1, A[:, k:], r), atol=1e-10 * np.abs(A).max())


def test_eckart_young_reduction_unit_weights():
    # W1 = 1: Eq. 5 is Eq. 1, whose optimum is H_r(A) with value sum_{j>r} sigma_j^2.
    rng = np.random.default_rng(10)
    m, n, k, r = 40, 12, 3, 5
    U, V = _orth(rng, m, n), _orth(rng, n, n)
    sig = np.geomspace(10.0, 0.1, n)
    A = (U * sig) @ V.T
    W1 = np.ones((m, k))
    Fstar = float(np.sum(sig[r:] ** 2))
    # H_r(A)'s first k columns are a fixed point of the iteration
    Xr = oracle.hard_threshold(A, r)
    st = oracle.swlr_step(A, W1, Xr[:, :k], r)
    assert st.F == pytest.approx(Fstar, rel=1e-11)
    assert np.allclose(st.X1_next, Xr[:, :k], atol=1e-10)
    # and from a random start the iteration reaches the global optimum
    res = oracle.swlr(A, W1, r, rng.standard_normal((m, k)), max_iter=400, stop="none")
    assert res.F[-1] <= Fstar * (1 + 1e-10)
    assert np.allclose(np.hstack([res.X1, res.X2]), Xr, atol=1e-6)


def test_ghs_limit_large_weights():
    # W1 = w * 1 with w -> infinity: X1 -> A1 and X2 -> the GHS closed form (Theorem 1)
    # with error O(w^-2).
    rng = np.random.default_rng(11)
    m, n, k, r = 30, 10, 2, 4
    A = rng.standard_normal((m, 3)) @ rng.standard_normal((3, n)) + 0.2 * rng.standard_normal((m, n))
    A1, A2 = A[:, :k], A[:, k:]
    ref = oracle.ghs(A1, A2, r)
    ws = np.array([1e2, 1e3, 1e4])
    e1, e2 = [], []
    for w in ws:
        W1 = np.full((m, k), w)
        res = oracle.swlr(A, W1, r, A1.copy(), max_iter=60, stop="none")
        e1.append(np.linalg.norm(res.X1 - A1))
        e2.append(np.linalg.norm(res.X2 - ref))
    s1 = np.polyfit(np.log(ws), np.log(e1), 1)[0]
    s2 = np.polyfit(np.log(ws), np.log(e2), 1)[0]
    assert -2.2 < s1 < -1.8
    assert -2.2 < s2 < -1.8


def test_bruteforce_tiny_global_minimum():
    # m = n = 4, k = 1, r = 2: minimise the plain objective of Eq. 5 over all rank-2
    # X = L R^T by multi-start BFGS, and compare with Algorithm 1 run from 50 starts.
    rng = np.random.default_rng(12)
    m, n, k, r = 4, 4, 1, 2
    A = rng.standard_normal((m, n))
    W1 = rng.uniform(1.0, 3.0, size=(m, k))

    def f(z):
        L, R = z[:m * r].reshape(m, r), z[m * r:].reshape(n, r)
        X = L @ R.T
        return np.sum(((A[:, :k] - X[:, :k]) * W1) ** 2) + np.sum((A[:, k:] - X[:, k:]) ** 2)

    brute = min(minimize(f, rng.standard_normal((m + n) * r), method="BFGS", options={"gtol": 1e-12}).fun
                for _ in range(40))
    algo = min(oracle.swlr(A, W1, r, rng.standard_normal((m, k)), max_iter=500, stop="none").F[-1]
               for _ in range(50))
    assert algo == pytest.approx(brute, rel=1e-8, abs=1e-12)


def test_r_equals_k_gives_zero_D():
    A, W1, X0, k, r = _small_problem(seed=13, m=30, n=9, k=3, r=3)
    cd = oracle.cd_step(A[:, k:], X0, 0)
    assert np.all(cd.D == 0)
    res = oracle.swlr(A, W1, 3, X0, max_iter=10, stop="none")
    assert np.linalg.matrix_rank(np.hstack([res.X1, res.X2]), tol=1e-9) <= 3


def test_stopping_rule():
    A, W1, X0, k, r = _small_problem(seed=14)
    res = oracle.swlr(A, W1, r, X0, eps=1e-3, max_iter=500, stop="relative")
    assert res.converged and res.rel_error[-1] < 1e-3
    assert all(e >= 1e-3 for e in res.rel_error[:-1])
    res2 = oracle.swlr(A, W1, r, X0, eps=1e-3, max_iter=3, stop="none")
    assert res2.iters == 3 and not res2.converged
    # the absolute test of Section 4.1 fires on its own when eps is large
    res3 = oracle.swlr(A, W1, r, X0, eps=1e9, max_iter=50, stop="paper")
    assert res3.iters == 1 and res3.converged


def test_only_weighted_columns_change_with_identical_A2_zero():
    # A2 = 0: C = 0 and D = 0, so the row solve gives X1 = A1 exactly.
    rng = np.random.default_rng(15)
    m, k = 10, 3
    A = np.hstack([rng.standard_normal((m, k)), np.zeros((m, 4))])
    W1 = rng.uniform(1, 2, size=(m, k))
    st = oracle.swlr_step(A, W1, rng.standard_normal((m, k)), 5)
    assert np.allclose(st.X1_next, A[:, :k], atol=1e-13)
