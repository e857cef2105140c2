"""Weighted frames at arbitrary columns (wlr_set_data_cols) and the result in the caller's
column order (wlr_get_x).  Eq. 5 takes the weighted frames first; the oracle here is the
plain oracle run on A with its columns permuted that way, with its X1, X2 put back."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def wlr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_1703_06303_gb300 import wlr as w
    return w


def _problem(seed, m, n, k):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, 3)) @ rng.standard_normal((3, n)) + 0.05 * rng.standard_normal((m, n))
    W1 = rng.uniform(5.0, 50.0, (m, k))
    return np.asfortranarray(A), np.asfortranarray(W1)


def _perm(cols, n):
    return list(cols) + [q for q in range(n) if q not in cols]


@pytest.mark.parametrize("mem", ["host", "device"])
def test_cols_match_the_oracle_on_the_permuted_problem(wlr, mem):
    m, n, k, r = 300, 20, 3, 6
    cols = [7, 2, 11]
    A, W1 = _problem(1, m, n, k)
    perm = _perm(cols, n)
    iters = 6
    ref = oracle.swlr(A[:, perm], W1, r, A[:, cols].copy(), max_iter=iters, stop="none")
    s = wlr.Solver(m, n, k, r, precision=wlr.WLR_PREC_FP64, stop=wlr.WLR_STOP_NONE, eig_block=14,
                   eig_iters=60, eig_iters_cold=400)
    if mem == "device":
        s.set_data_cols(torch.from_numpy(A).cuda(), torch.from_numpy(W1).cuda(), cols)
    else:
        s.set_data_cols(A, W1, cols)
    s.set_init(wlr.WLR_INIT_A1)
    s.solve(0.0, iters)
    X = np.zeros((m, n), order="F")
    s.x(X)
    want = np.empty((m, n))
    want[:, perm] = np.hstack([ref.X1, ref.X2])
    assert np.abs(X - want).max() <= 1e-10 * np.abs(want).max()
    Fh, _ = s.history()
    assert np.allclose(Fh, ref.F[:iters], rtol=1e-10, atol=0)
    s.close()


def test_cols_equal_the_prepermuted_problem_bit_for_bit(wlr):
    m, n, k, r = 4800, 90, 6, 10
    rng = np.random.default_rng(2)
    cols = sorted(rng.choice(n, size=k, replace=False).tolist(), reverse=True)
    A, W1 = _problem(3, m, n, k)
    A32, W32 = A.astype(np.float32), W1.astype(np.float32)
    perm = _perm(cols, n)
    tA, tW = torch.from_numpy(np.asfortranarray(A32)).cuda(), torch.from_numpy(W32).cuda().T.contiguous().T
    tP = torch.from_numpy(np.asfortranarray(A32[:, perm])).cuda()
    s1 = wlr.Solver(m, n, k, r, precision=wlr.WLR_PREC_FP32, stop=wlr.WLR_STOP_NONE)
    s2 = wlr.Solver(m, n, k, r, precision=wlr.WLR_PREC_FP32, stop=wlr.WLR_STOP_NONE)
    s1.set_data_cols(tA, tW, cols)
    s2.set_data(tP, tW)
    for s in (s1, s2):
        s.set_init(wlr.WLR_INIT_A1)
        s.solve(0.0, 12)
    F1, _ = s1.history()
    F2, _ = s2.history()
    assert np.array_equal(F1, F2)
    X = torch.empty((n, m), dtype=torch.float32, device="cuda").T
    s1.x(X)
    X1 = np.zeros((m, k), dtype=np.float32, order="F")
    X2 = np.zeros((m, n - k), dtype=np.float32, order="F")
    s2.result(X1, X2)
    Xh = X.cpu().numpy()
    assert np.array_equal(Xh[:, cols], X1)
    assert np.array_equal(Xh[:, perm[k:]], X2)
    # without an index set, wlr_get_x is (X1, X2)
    Y = np.zeros((m, n), dtype=np.float32, order="F")
    s2.x(Y)
    assert np.array_equal(Y[:, :k], X1) and np.array_equal(Y[:, k:], X2)
    s1.close()
    s2.close()


def test_bad_index_sets_are_rejected(wlr):
    m, n, k, r = 100, 10, 2, 4
    A, W1 = _problem(4, m, n, k)
    s = wlr.Solver(m, n, k, r, precision=wlr.WLR_PREC_FP64)
    for cols in ([3, 3], [0, 10], [-1, 2]):
        with pytest.raises(wlr.WlrError) as e:
            s.set_data_cols(A, W1, cols)
        assert e.value.status == wlr.WLR_ERR_INVALID_ARG
    with pytest.raises(ValueError):
        s.set_data_cols(A, W1, [1])
    s.close()
