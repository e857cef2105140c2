"""FP64 refinement sweep (wlr_refine) against the FP64 oracle.

After an FP32 solve, one loop body of Algorithm 1 (Section 3) is taken in FP64 from the
FP32 iterate X1_p: X1_{p+1}, F~(X1_p) and F~(X1_{p+1}) must equal one oracle step from the
same X1_p to FP64 accuracy (1e-10 relative), at a small size and at the 320x240, n=1000,
k=50, r=60 clip; the handle's own iteration is left as it was.
"""
import numpy as np
import pytest

import oracle
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


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _x1(s, m, k):
    X = np.zeros((m, k), order="F")
    s.result(X)
    return X


def _refine_vs_oracle(wlr, A32, W32, r, iters, precision, tol):
    m, n = A32.shape
    k = W32.shape[1]
    dt = np.float32 if precision == wlr.WLR_PREC_FP32 else np.float64
    s = wlr.Solver(m, n, k, r, precision=precision, stop=wlr.WLR_STOP_NONE)
    s.set_data(torch.from_numpy(np.asfortranarray(A32.astype(dt))).to(DEV),
               torch.from_numpy(np.asfortranarray(W32.astype(dt))).to(DEV))
    s.set_init(wlr.WLR_INIT_A1)
    s.solve(0.0, iters)
    Xp = _x1(s, m, k)                       # the handle's iterate, exactly (widened)
    p0 = s.iteration()
    Xd = torch.zeros((k, m), dtype=torch.float64, device=DEV).T   # column-major on the device
    Fp, Fn = s.refine(Xd)
    Xh = np.zeros((m, k), order="F")
    Fp2, Fn2 = s.refine(Xh)                 # host output, same values
    assert s.iteration() == p0
    assert np.array_equal(Xh, Xd.cpu().numpy()) and Fp == Fp2 and Fn == Fn2
    A, W1 = A32.astype(np.float64), W32.astype(np.float64)
    st = oracle.swlr_step(A, W1, Xp, r)
    assert _rel(Xh, st.X1_next) < tol
    assert abs(Fp - st.F) <= tol * st.F
    Fo = oracle.objective_tilde(A, W1, st.X1_next, r)
    assert abs(Fn - Fo) <= tol * Fo
    assert Fn <= Fp * (1 + 1e-12)           # the objective does not increase (Theorem 2)
    s.close()
    return Xp, st


def test_refine_small_fp32(wlr):
    spec = synth.CONFIGS[1]
    clip = synth.make_clip(spec)
    _refine_vs_oracle(wlr, clip["A"].astype(np.float32), clip["W1"].astype(np.float32), spec.r,
                      12, wlr.WLR_PREC_FP32, 1e-10)


def test_refine_fp64_handle(wlr):
    rng = np.random.default_rng(31)
    m, n, k, r = 333, 57, 6, 11
    A = rng.standard_normal((m, 3)) @ rng.standard_normal((3, n)) + 0.05 * rng.standard_normal((m, n))
    W1 = rng.uniform(2.0, 30.0, size=(m, k))
    _refine_vs_oracle(wlr, A, W1, r, 5, wlr.WLR_PREC_FP64, 1e-10)


def test_refine_keeps_the_iteration(wlr):
    spec = synth.CONFIGS[1]
    clip = synth.make_clip(spec)
    A32 = torch.from_numpy(np.asfortranarray(clip["A"].astype(np.float32))).to(DEV)
    W32 = torch.from_numpy(np.asfortranarray(clip["W1"].astype(np.float32))).to(DEV)
    a, b = (wlr.Solver(spec.m, spec.n, spec.k, spec.r, stop=wlr.WLR_STOP_NONE) for _ in range(2))
    for s in (a, b):
        s.set_data(A32, W32)
        s.set_init(wlr.WLR_INIT_A1)
        s.solve(0.0, 7)
    a.refine()
    for s in (a, b):
        s.solve(0.0, 5)
    assert np.array_equal(_x1(a, spec.m, spec.k), _x1(b, spec.m, spec.k))
    assert np.array_equal(a.history()[0], b.history()[0])
    with pytest.raises(ValueError):
        a.refine(np.zeros((spec.m, spec.k)))   # C order: rejected
    fresh = wlr.Solver(spec.m, spec.n, spec.k, spec.r)
    with pytest.raises(wlr.WlrError) as e:
        fresh.refine()
    assert e.value.status == wlr.WLR_ERR_NOT_READY
    for s in (a, b, fresh):
        s.close()


def test_refine_at_320x240(wlr):
    """The mixed policy at n=1000, k=50, r=60: FP32 iterations, then one FP64 sweep.
    Per output against the oracle: the refined X1 and both objectives to 1e-10; the FP32
    path's own step from the same X1_p within its FP32 tolerances."""
    spec = synth.CONFIGS[3]
    clip = synth.make_clip(spec)
    A32, W32 = clip["A"].astype(np.float32), clip["W1"].astype(np.float32)
    Xp, st = _refine_vs_oracle(wlr, A32, W32, spec.r, 6, wlr.WLR_PREC_FP32, 1e-10)
    # the FP32 step from the same X1_p, for comparison
    s = wlr.Solver(spec.m, spec.n, spec.k, spec.r, precision=wlr.WLR_PREC_FP32, eig_iters_cold=200)
    s.set_data(torch.from_numpy(np.asfortranarray(A32)).to(DEV),
               torch.from_numpy(np.asfortranarray(W32)).to(DEV))
    s.set_init(wlr.WLR_INIT_USER, Xp.astype(np.float32))
    F = s.step()
    assert abs(F - st.F) <= 1e-4 * st.F
    assert _rel(_x1(s, spec.m, spec.k), st.X1_next) < 2e-3
    s.close()
