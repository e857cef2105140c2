"""The allocation-free X1 update (wlr_x1_update_noalloc), checked through the C ABI
against the handle-based path (wlr_step) on two calls in a row.

It exists for callers that cannot allocate device memory (a fixed memory budget owned
by another allocator, or code where a cudaMalloc/cudaFree that can synchronise the
device is not acceptable); its scratch is one fixed device array inside the library.
This file sorts last so that a run stopping at the first failure has run every other
test first."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# Both sides run the same row-pass kernel on the same FP32 X1, C and V_s; only C C^T and
# C V_s are summed in a different order (here by prep_rowpass, in wlr_step by the D-step
# cluster kernel), so X1_{p+1} agrees to a few ulp times the row systems' condition.
TOL = 1e-4


@pytest.fixture(scope="module")
def wlr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_1703_06303_gb300 import wlr as w
    return w


def _col(a, dev):
    return torch.from_numpy(np.asfortranarray(a)).to(dev)


def test_noalloc_matches_step_twice(wlr):
    from paper_1703_06303_gb300 import synth
    dev = torch.device("cuda:0")
    spec = synth.ClipSpec(H=60, W=80, n=120, k=12, r=17, rho=4, coverage=0.05, sigma=0.02,
                          w_const=None, w_range=(5.0, 50.0), discs=True, seed=77)
    clip = synth.make_clip(spec)
    m, n, k, r = spec.m, spec.n, spec.k, spec.r
    A = clip["A"].astype(np.float32)
    W1 = clip["W1"].astype(np.float32)
    tA, tW = _col(A, dev), _col(W1, dev)
    s = wlr.Solver(m, n, k, r, precision=wlr.WLR_PREC_FP32, stop=wlr.WLR_STOP_NONE)
    s.set_data(tA, tW)
    s.set_init(wlr.WLR_INIT_A1)
    X_cur = torch.empty((k, m), dtype=torch.float32, device=dev).T
    s.result(X_cur)
    wterm = torch.zeros(1, dtype=torch.float64, device=dev)
    status = torch.full((1,), -1, dtype=torch.int32, device=dev)
    for call in range(2):
        C, Vs, _ = s.factors()                       # factors of the current X1
        tC = _col(C.astype(np.float32), dev)
        tV = _col(Vs.astype(np.float32), dev)
        out = torch.full((k, m), float("nan"), dtype=torch.float32, device=dev).T
        wlr.wlr_x1_update_noalloc(tA, tW, X_cur, k, r, tC, tV, out, wterm, status)
        s.step(want_objective=False)                 # existing entry point
        ref = torch.empty((k, m), dtype=torch.float32, device=dev).T
        s.result(ref)
        torch.cuda.synchronize()
        got, want = out.cpu().numpy(), ref.cpu().numpy()
        err = np.abs(got - want).max() / np.abs(want).max()
        assert np.isfinite(got).all()
        assert err <= TOL, (call, err)
        assert int(status.item()) == 0
        x = X_cur.cpu().numpy().astype(np.float64)
        w_ref = np.sum(((A[:, :k].astype(np.float64) - x) * W1.astype(np.float64)) ** 2)
        assert abs(wterm.item() - w_ref) <= 1e-5 * w_ref
        X_cur = ref.clone(memory_format=torch.preserve_format)
    s.close()


def test_noalloc_without_unweighted_frames(wlr):
    # n = k (so r = k): no A2, C and V_s are empty, and the row systems are diagonal,
    # diag(W1(i,:)^2) x = A1(i,:) o W1(i,:)^2, so X1_{p+1} = A1 to rounding
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(5)
    m, k = 1000, 6
    A = rng.standard_normal((m, k)).astype(np.float32)
    W1 = rng.uniform(5.0, 50.0, (m, k)).astype(np.float32)
    X = rng.standard_normal((m, k)).astype(np.float32)
    tA, tW, tX = _col(A, dev), _col(W1, dev), _col(X, dev)
    out = torch.full((k, m), float("nan"), dtype=torch.float32, device=dev).T
    wterm = torch.zeros(1, dtype=torch.float64, device=dev)
    status = torch.full((1,), -1, dtype=torch.int32, device=dev)
    for _ in range(2):
        wlr.wlr_x1_update_noalloc(tA, tW, tX, k, k, None, None, out, wterm, status)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.abs(got - A).max() <= 1e-6 * np.abs(A).max()
        assert int(status.item()) == wlr.WLR_OK
        w_ref = np.sum(((A.astype(np.float64) - X.astype(np.float64)) * W1.astype(np.float64)) ** 2)
        assert abs(wterm.item() - w_ref) <= 1e-5 * w_ref
        tX = out.clone(memory_format=torch.preserve_format)
        X = got


def test_noalloc_reports_breakdown(wlr):
    # A non-finite weight on one row makes that row's system diag(W1(i,:)^2) + C C^T
    # unusable: the status word must read WLR_ERR_NOT_SPD (the header's code), and a
    # clean call afterwards must read WLR_OK again (the error word is cleared per call).
    from paper_1703_06303_gb300 import synth
    dev = torch.device("cuda:0")
    spec = synth.ClipSpec(H=30, W=40, n=50, k=5, r=8, rho=3, coverage=0.04, sigma=0.01,
                          w_const=20.0, seed=9)
    clip = synth.make_clip(spec)
    m, n, k, r = spec.m, spec.n, spec.k, spec.r
    A = clip["A"].astype(np.float32)
    W1 = clip["W1"].astype(np.float32)
    s = wlr.Solver(m, n, k, r, precision=wlr.WLR_PREC_FP32, stop=wlr.WLR_STOP_NONE)
    tA, tW = _col(A, dev), _col(W1, dev)
    s.set_data(tA, tW)
    s.set_init(wlr.WLR_INIT_A1)
    C, Vs, _ = s.factors()
    tC = _col(C.astype(np.float32), dev)
    tV = _col(Vs.astype(np.float32), dev)
    X = _col(A[:, :k].copy(), dev)
    out = torch.empty((k, m), dtype=torch.float32, device=dev).T
    status = torch.full((1,), -1, dtype=torch.int32, device=dev)
    Wbad = W1.copy()
    Wbad[123, 2] = np.nan
    wlr.wlr_x1_update_noalloc(tA, _col(Wbad, dev), X, k, r, tC, tV, out, None, status)
    torch.cuda.synchronize()
    assert int(status.item()) == wlr.WLR_ERR_NOT_SPD
    wlr.wlr_x1_update_noalloc(tA, tW, X, k, r, tC, tV, out, None, status)
    torch.cuda.synchronize()
    assert int(status.item()) == wlr.WLR_OK
    assert np.isfinite(out.cpu().numpy()).all()
    s.close()


def test_noalloc_rejects_oversize(wlr):
    # n - k = 7980 frames need more than the fixed scratch: rejected before any GPU work
    m, n, k, r = 300000, 8000, 20, 25
    tiny = torch.zeros((1, 1), dtype=torch.float32, device="cuda:0")
    p = tiny.data_ptr()
    st = wlr._lib.wlr_x1_update_noalloc(p, m, p, m, p, m, n, k, r, p, p, p, None, None, None)
    assert st == wlr.WLR_ERR_UNSUPPORTED
    assert "scratch" in wlr.wlr_last_error(None)
