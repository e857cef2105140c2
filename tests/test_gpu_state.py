"""Checkpoint and resume through the C ABI (wlr_get_state / wlr_set_state).

A handle restored from a checkpoint must continue the same iteration bit for bit: the
loop state of Algorithm 1 (X1_p, p, the history) plus what this build carries between
iterations (the (C, D) factors the next loop body reads, the subspace basis, the previous
R^{-1}).  Checked in FP32 on the 19200 x 400 clip (past the full-CholeskyQR warm-up, so
the resumed run replays CUDA graphs) and in FP64 on a ragged problem; foreign, truncated
and mismatched buffers are rejected.
"""
import numpy as np
import pytest

from paper_1703_06303_gb300 import synth

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


DEV = "cuda:0"


def _dev(a, dtype):
    return torch.from_numpy(np.asfortranarray(a, dtype=dtype)).to(DEV)


def _x1(s, m, k):
    X = np.zeros((m, k), dtype=np.float64, order="F")
    s.result(X)
    return X


def _run_and_resume(wlr, A, W1, dims, precision, before, after, init_kind, X0=None):
    m, n, k, r = dims
    dt = np.float32 if precision == wlr.WLR_PREC_FP32 else np.float64
    Ad, Wd = _dev(A, dt), _dev(W1, dt)
    s1 = wlr.Solver(m, n, k, r, precision=precision)
    s1.set_data(Ad, Wd)
    s1.set_init(init_kind, X0)
    for _ in range(before):
        s1.step(False)
    state = s1.get_state()
    p0 = s1.iteration()
    for _ in range(after):
        s1.step(False)
    Xa = _x1(s1, m, k)
    Fa, _ = s1.history()

    s2 = wlr.Solver(m, n, k, r, precision=precision)
    s2.set_data(Ad, Wd)
    s2.set_state(state)
    assert s2.iteration() == p0
    for _ in range(after):
        s2.step(False)
    Xb = _x1(s2, m, k)
    Fb, _ = s2.history()
    s1.close()
    s2.close()
    return Xa, Xb, Fa, Fb, p0


def test_resume_fp32_config2_bit_identical(wlr):
    spec = synth.CONFIGS[2]
    clip = synth.make_clip(spec)
    dims = (spec.m, spec.n, spec.k, spec.r)
    Xa, Xb, Fa, Fb, p0 = _run_and_resume(wlr, clip["A"], clip["W1"], dims, wlr.WLR_PREC_FP32,
                                         before=30, after=20, init_kind=wlr.WLR_INIT_A1)
    assert p0 == 30
    assert len(Fa) == len(Fb) == 50
    assert np.array_equal(Xa, Xb)
    assert np.array_equal(Fa, Fb)


def test_resume_fp64_ragged_bit_identical(wlr):
    rng = np.random.default_rng(11)
    m, n, k, r = 257, 70, 20, 26
    A = rng.standard_normal((m, 3)) @ rng.standard_normal((3, n)) + 0.1 * rng.standard_normal((m, n))
    W1 = rng.uniform(5.0, 50.0, size=(m, k))
    X0 = np.asfortranarray(rng.standard_normal((m, k)))
    Xa, Xb, Fa, Fb, p0 = _run_and_resume(wlr, A, W1, (m, n, k, r), wlr.WLR_PREC_FP64,
                                         before=7, after=6, init_kind=wlr.WLR_INIT_USER, X0=X0)
    assert p0 == 7 and len(Fb) == 13
    assert np.array_equal(Xa, Xb)
    assert np.array_equal(Fa, Fb)


def test_resume_from_a_fresh_init(wlr):
    # checkpoint before any step: nothing of the (C, D) step exists yet
    rng = np.random.default_rng(12)
    m, n, k, r = 300, 40, 8, 12
    A = rng.standard_normal((m, n))
    W1 = rng.uniform(1.0, 10.0, size=(m, k))
    Xa, Xb, Fa, Fb, p0 = _run_and_resume(wlr, A, W1, (m, n, k, r), wlr.WLR_PREC_FP32,
                                         before=0, after=8, init_kind=wlr.WLR_INIT_A1)
    assert p0 == 0
    assert np.array_equal(Xa, Xb)
    assert np.array_equal(Fa, Fb)


def test_state_buffers_are_checked(wlr):
    rng = np.random.default_rng(13)
    m, n, k, r = 128, 24, 4, 6
    A = rng.standard_normal((m, n))
    W1 = rng.uniform(1.0, 10.0, size=(m, k))
    Ad, Wd = _dev(A, np.float32), _dev(W1, np.float32)
    s = wlr.Solver(m, n, k, r, precision=wlr.WLR_PREC_FP32)
    with pytest.raises(wlr.WlrError) as e:
        s.set_state(b"\0" * 64)
    assert e.value.status == wlr.WLR_ERR_NOT_READY
    s.set_data(Ad, Wd)
    s.set_init(wlr.WLR_INIT_A1)
    s.step(False)
    state = s.get_state()
    for bad in (state[:40], state[:-8], b"XXXX" + state[4:]):
        with pytest.raises(wlr.WlrError) as e:
            s.set_state(bad)
        assert e.value.status == wlr.WLR_ERR_INVALID_ARG
    other = wlr.Solver(m, n, k, r + 1, precision=wlr.WLR_PREC_FP32)
    other.set_data(Ad, Wd)
    with pytest.raises(wlr.WlrError) as e:
        other.set_state(state)
    assert e.value.status == wlr.WLR_ERR_INVALID_ARG
    f64 = wlr.Solver(m, n, k, r, precision=wlr.WLR_PREC_FP64)
    f64.set_data(_dev(A, np.float64), _dev(W1, np.float64))
    with pytest.raises(wlr.WlrError) as e:
        f64.set_state(state)
    assert e.value.status == wlr.WLR_ERR_INVALID_ARG
    s.set_state(state)   # its own checkpoint is accepted
    for h in (s, other, f64):
        h.close()


def test_bounded_wait_gives_up_and_the_context_stays_usable(wlr):
    """A bounded mbarrier wait that nothing completes (10 ms limit) returns
    WLR_ERR_DEVICE_TIMEOUT, twice in a row, and a solve on a fresh handle then runs."""
    import time
    for _ in range(2):
        t0 = time.perf_counter()
        st = wlr.wlr_selftest_bounded_wait(10_000_000)
        assert st == wlr.WLR_ERR_DEVICE_TIMEOUT
        assert time.perf_counter() - t0 < 5.0
        assert "gave up" in wlr.wlr_last_error(None)
    assert wlr.wlr_selftest_bounded_wait(0) == wlr.WLR_ERR_INVALID_ARG
    rng = np.random.default_rng(3)
    m, n, k, r = 500, 40, 4, 7
    A = np.asfortranarray(rng.standard_normal((m, n)).astype(np.float32))
    W1 = np.asfortranarray(rng.uniform(5, 50, (m, k)).astype(np.float32))
    s = wlr.Solver(m, n, k, r, precision=wlr.WLR_PREC_FP32, stop=wlr.WLR_STOP_NONE)
    s.set_data(torch.from_numpy(A).cuda(), torch.from_numpy(W1).cuda())
    s.set_init(wlr.WLR_INIT_A1)
    it, F, _ = s.solve(0.0, 10)
    assert it == 10 and np.isfinite(F)
    s.close()
