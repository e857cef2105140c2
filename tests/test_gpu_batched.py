"""Batched solve through the C ABI (wlr_solve_batched).

Independent problems of uneven m, n, k, r (one with s = 0, one with k > 32, one in FP64)
advance together in one CUDA graph launch per three iterations.  Each problem must come out
bit for bit as the same problem solved alone with wlr_solve (same kernels, fixed-order
reductions), and the FP64 member must follow the oracle's trajectory of Algorithm 1.
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

# (H, W, n, k, r, precision)
SHAPES = [
    (15, 20, 60, 5, 9, "fp32"),
    (30, 40, 150, 12, 15, "fp32"),
    (20, 35, 90, 3, 3, "fp32"),       # s = 0: no D-step
    (30, 40, 200, 36, 40, "fp32"),    # k > 32
    (24, 32, 130, 8, 14, "fp32"),
    (15, 20, 50, 4, 7, "fp64"),
]


def _clip(i, H, W, n, k, r):
    spec = synth.ClipSpec(H=H, W=W, n=n, k=k, r=r, rho=3, coverage=0.04, sigma=0.01,
                          w_const=20.0, seed=500 + i)
    return synth.make_clip(spec)


def _make(wlr, i, shape, use_graph=1, eig_iters=0):
    H, W, n, k, r, prec = shape
    clip = _clip(i, H, W, n, k, r)
    dt = np.float32 if prec == "fp32" else np.float64
    p = wlr.WLR_PREC_FP32 if prec == "fp32" else wlr.WLR_PREC_FP64
    kw = dict(eig_block=32, eig_iters_cold=400, eig_iters=60) if prec == "fp64" else dict(eig_iters=eig_iters)
    s = wlr.Solver(H * W, n, k, r, precision=p, stop=wlr.WLR_STOP_NONE, use_graph=use_graph, **kw)
    A = torch.from_numpy(np.asfortranarray(clip["A"].astype(dt))).to(DEV)
    Wt = torch.from_numpy(np.asfortranarray(clip["W1"].astype(dt))).to(DEV)
    s.set_data(A, Wt)
    s.set_init(wlr.WLR_INIT_A1)
    s._keep = (A, Wt)
    return s, clip


def _x1(s, m, k):
    X = np.zeros((m, k), order="F")
    s.result(X)
    return X


@pytest.mark.parametrize("iters", [14, 4])
def test_batched_equals_solved_alone(wlr, iters):
    batch = [_make(wlr, i, sh)[0] for i, sh in enumerate(SHAPES)]
    alone = [_make(wlr, i, sh)[0] for i, sh in enumerate(SHAPES)]
    # one member without graphs runs alone inside the batch call
    batch.append(_make(wlr, 1, SHAPES[1], use_graph=0)[0])
    alone.append(_make(wlr, 1, SHAPES[1], use_graph=0)[0])
    wlr.solve_batched(batch, iters)
    for s in alone:
        s.solve(0.0, iters)
    for q, (sb, sa) in enumerate(zip(batch, alone)):
        H, W, n, k, r, _ = SHAPES[q] if q < len(SHAPES) else SHAPES[1]
        assert sb.iteration() == sa.iteration() == iters
        assert np.array_equal(_x1(sb, H * W, k), _x1(sa, H * W, k)), q
        Fb, _ = sb.history()
        Fa, _ = sa.history()
        assert np.array_equal(Fb, Fa), q
    # a second call continues from where the first one left off
    wlr.solve_batched(batch, 5)
    for s in alone:
        s.solve(0.0, 5)
    for q, (sb, sa) in enumerate(zip(batch, alone)):
        H, W, n, k, r, _ = SHAPES[q] if q < len(SHAPES) else SHAPES[1]
        assert np.array_equal(_x1(sb, H * W, k), _x1(sa, H * W, k)), q
    for s in batch + alone:
        s.close()


def test_batched_fp64_member_follows_oracle(wlr):
    iters = 12
    members = [_make(wlr, i, sh) for i, sh in enumerate(SHAPES)]
    wlr.solve_batched([s for s, _ in members], iters)
    q = len(SHAPES) - 1
    H, W, n, k, r, _ = SHAPES[q]
    s, clip = members[q]
    A, W1 = clip["A"], clip["W1"]
    ref = oracle.swlr(A, W1, r, A[:, :k].copy(), max_iter=iters, stop="none")
    Fh, _ = s.history()
    assert np.allclose(Fh, ref.F[:iters], rtol=1e-9, atol=0)
    X1 = _x1(s, H * W, k)
    assert float(np.abs(X1 - ref.X1).max() / np.abs(ref.X1).max()) < 1e-8
    for s, _ in members:
        s.close()


def test_batched_errors(wlr):
    s0, _ = _make(wlr, 0, SHAPES[0])
    s1, _ = _make(wlr, 4, SHAPES[4])
    X = _x1(s1, 24 * 32, 8)
    wlr.wlr_solve_batched([], 5)                 # empty batch: nothing to do
    wlr.solve_batched([s0, s1], 0)               # no iterations: nothing changes
    assert s0.iteration() == 0 and np.array_equal(_x1(s1, 24 * 32, 8), X)
    with pytest.raises(wlr.WlrError) as e:
        wlr.solve_batched([s0, s1, s0], 3)
    assert e.value.status == wlr.WLR_ERR_INVALID_ARG
    with pytest.raises(wlr.WlrError) as e:
        wlr.solve_batched([s0, s1], -1)
    assert e.value.status == wlr.WLR_ERR_INVALID_ARG
    fresh = wlr.Solver(300, 60, 5, 9, precision=wlr.WLR_PREC_FP32)
    with pytest.raises(wlr.WlrError) as e:
        wlr.solve_batched([s0, fresh], 6)
    assert e.value.status == wlr.WLR_ERR_NOT_READY and e.value.index == 1
    for s in (s0, s1, fresh):
        s.close()


@pytest.mark.parametrize("eig_iters,tol", [(3, 1e-4), (0, 3e-4)])
def test_batched_fp32_members_follow_the_oracle(wlr, eig_iters, tol):
    """FP32 members after 30 iterations of the joined graph launches, against the FP64
    oracle's own 30 iterations of Algorithm 1 on the same clip from X1_0 = A1: the FP64
    objective of each GPU iterate within tol of the oracle's F_30, for a k > 32 member and
    an s = 0 member too.  With 3 warm subspace steps per iteration the rank-(r-k) step
    tracks the oracle's exact SVD and the reduced-precision tolerance 1e-4 holds; the
    default single warm step trails it in the early transient (1.2e-4 measured at p = 30 on
    the 15 x 20 member; within 1.5e-5 over 2500 iterations on the 160 x 120 clip)."""
    shapes = [SHAPES[0], SHAPES[1], SHAPES[2], SHAPES[3], SHAPES[4]]
    made = [_make(wlr, 20 + i, sh, eig_iters=eig_iters) for i, sh in enumerate(shapes)]
    wlr.solve_batched([s for s, _ in made], 30)
    for (s, clip), sh in zip(made, shapes):
        H, W, n, k, r, _ = sh
        A = clip["A"].astype(np.float32).astype(np.float64)
        W1 = clip["W1"].astype(np.float32).astype(np.float64)
        ref = oracle.swlr(A, W1, r, A[:, :k].copy(), max_iter=30, stop="none")
        F = s.objective()
        assert s.iteration() == 30
        assert abs(F - ref.F[30]) <= tol * ref.F[30], (sh, F, ref.F[30])
        s.close()


def test_autotuned_handles_agree_and_follow_the_oracle(wlr):
    """options.autotune: the first wlr_set_data of a shape times candidate row chunkings of
    the per-iteration Gram and caches the fastest; a second handle of the same shape takes
    the cached choice, so the two compute the same iterates bit for bit, and the objective
    stays within the reduced-precision tolerance of the oracle's trajectory."""
    H, W, n, k, r = 60, 80, 160, 10, 14
    spec = synth.ClipSpec(H=H, W=W, n=n, k=k, r=r, rho=3, coverage=0.04, sigma=0.01, w_const=20.0, seed=777)
    clip = synth.make_clip(spec)
    A32 = np.asfortranarray(clip["A"].astype(np.float32))
    W32 = np.asfortranarray(clip["W1"].astype(np.float32))
    tA, tW = torch.from_numpy(A32).to(DEV), torch.from_numpy(W32).to(DEV)
    hist = []
    for _ in range(2):
        s = wlr.Solver(spec.m, n, k, r, precision=wlr.WLR_PREC_FP32, stop=wlr.WLR_STOP_NONE, autotune=1,
                       eig_iters=3)
        s.set_data(tA, tW)
        s.set_init(wlr.WLR_INIT_A1)
        s.solve(0.0, 30)
        Fh, _ = s.history()
        hist.append((Fh, s.objective()))
        s.close()
    assert np.array_equal(hist[0][0], hist[1][0])
    ref = oracle.swlr(A32.astype(np.float64), W32.astype(np.float64), r, A32[:, :k].astype(np.float64),
                      max_iter=30, stop="none")
    assert abs(hist[0][1] - ref.F[30]) <= 1e-4 * ref.F[30]
