"""The learned warm start's kernels (include/wlr.h, wlr_ws_*) against the FP64 oracle of
oracle/warmstart.py, through the C ABI.

Tolerances: the network's float kernels sum in float what the oracle sums in double, with
the same bfloat16-rounded weights on both sides (the parameters given to the GPU are
bfloat16 numbers, so its rounding leaves them unchanged): outputs within 1e-4 relative
(max-abs error over max-abs value), gradients within 1e-4 relative in the Frobenius norm
(a relu whose input is within rounding of zero may flip one entry's mask).  Double
reductions (the basis, the weighted projection) within 1e-8 relative."""
import numpy as np
import pytest

from oracle import warmstart as ows
import oracle
from paper_1703_06303_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SHAPE = dict(h=30, w=40, c1=16, c2=32, hidden=384, r_max=64)
DEV = "cuda:0"


@pytest.fixture(scope="module")
def wlr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_1703_06303_gb300 import wlr as w
    return w


def _col(a):
    return torch.from_numpy(np.asfortranarray(a)).to(DEV)


def _rows(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(DEV)


def _rel_max(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _rel_fro(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _oracle_params(seed):
    """Oracle initialisation rounded to bfloat16, as (list of pairs, flat float32 vector)."""
    p = ows.net_init(SHAPE["h"], SHAPE["w"], SHAPE["c1"], SHAPE["c2"], SHAPE["hidden"], SHAPE["r_max"], seed)
    rng = np.random.default_rng(seed + 1)
    p = [(ows.round_bf16(W), ows.round_bf16(0.05 * rng.standard_normal(b.shape))) for W, b in p]
    flat = np.concatenate([a.ravel() for pair in p for a in pair]).astype(np.float32)
    return p, flat


def _split(flat, like):
    out, o = [], 0
    for W, b in like:
        nW, nb = W.size, b.size
        out.append((flat[o:o + nW].reshape(W.shape).astype(np.float64), flat[o + nW:o + nW + nb].astype(np.float64)))
        o += nW + nb
    return out


def _clip(H, W, n, k, r, seed):
    spec = synth.ClipSpec(H=H, W=W, n=n, k=k, r=r, rho=3, coverage=0.05, sigma=0.02, w_const=None,
                          w_range=(5.0, 50.0), discs=True, seed=seed)
    c = synth.make_clip(spec)
    return c["A"].astype(np.float32), c["W1"].astype(np.float32)


@pytest.mark.parametrize("H,W", [(30, 40), (240, 320)])
def test_prepare_matches_oracle(wlr, H, W):
    A, W1 = _clip(H, W, 9, 3, 5, 31)
    net = wlr.WarmStartNet(**SHAPE, max_frames=64)
    X = torch.empty((9, 2, 30, 40), dtype=torch.float32, device=DEV)
    net.prepare(_col(A), _col(W1), H, W, 3, X)
    want = ows.prepare_input(A.astype(np.float64), W1.astype(np.float64), H, W, H // 30)
    assert _rel_max(X.cpu().numpy(), want) < 1e-5
    net.close()


def test_forward_backward_match_oracle(wlr):
    pairs, flat = _oracle_params(3)
    net = wlr.WarmStartNet(**SHAPE, max_frames=64)
    net.set_params(flat)
    assert np.array_equal(net.params(), flat)
    rng = np.random.default_rng(4)
    sizes = (7, 5)
    Xh = rng.standard_normal((12, 2, 30, 40)).astype(np.float32)
    X = _rows(Xh)
    Om = torch.empty((12, 64), dtype=torch.float32, device=DEV)
    net.forward(X, [0, 7, 12], Om)
    want, cache = ows.net_forward(pairs, Xh.astype(np.float64), sizes)
    assert _rel_max(Om.cpu().numpy(), want) < 1e-4
    dOm = rng.standard_normal((12, 64)).astype(np.float32)
    net.backward(_rows(dOm))
    g = _split(net.grads(), pairs)
    gw = ows.net_backward(pairs, cache, dOm.astype(np.float64))
    for li in range(4):
        for which in (0, 1):
            assert _rel_fro(g[li][which], gw[li][which]) < 1e-4, (li, which)
    net.close()


def test_frames_of_other_clips_do_not_interact(wlr):
    # the context mean couples a clip's own frames only (Omega of clip 0 unchanged when
    # clip 1's frames change)
    _, flat = _oracle_params(5)
    net = wlr.WarmStartNet(**SHAPE, max_frames=64)
    net.set_params(flat)
    rng = np.random.default_rng(6)
    Xh = rng.standard_normal((10, 2, 30, 40)).astype(np.float32)
    O1 = torch.empty((10, 64), dtype=torch.float32, device=DEV)
    net.forward(_rows(Xh), [0, 4, 10], O1)
    Xh[6:] += 1.0
    O2 = torch.empty((10, 64), dtype=torch.float32, device=DEV)
    net.forward(_rows(Xh), [0, 4, 10], O2)
    assert torch.equal(O1[:4], O2[:4])
    assert not torch.equal(O1[4:], O2[4:])
    net.close()


@pytest.mark.parametrize("r,k", [(1, 1), (6, 2), (20, 0), (20, 7)])
def test_loss_and_gradient_match_oracle(wlr, r, k):
    rng = np.random.default_rng(7 + r)
    m, n = 1200, 40
    A = rng.standard_normal((m, n)).astype(np.float32)
    Om = (rng.standard_normal((n, 64)) * 0.3).astype(np.float32)
    V, _ = np.linalg.qr(rng.standard_normal((m, r)))
    net = wlr.WarmStartNet(**SHAPE, max_frames=64)
    loss = torch.zeros(1, dtype=torch.float64, device=DEV)
    dOm = torch.full((n, 64), np.nan, dtype=torch.float32, device=DEV)
    net.loss(_col(A), k, _rows(Om), r, _col(V.astype(np.float32)), loss, dOm)
    Lw, dw = ows.omega_loss(A.astype(np.float64), Om.astype(np.float64), r, V.astype(np.float32).astype(np.float64), k)
    assert abs(loss.item() - Lw) <= 1e-5 * max(Lw, 1e-3)
    got = dOm.cpu().numpy()
    assert np.all(got[:, r:] == 0.0)
    assert _rel_max(got, dw) < 1e-4
    net.close()


def test_adam_step_matches_oracle(wlr):
    pairs, flat = _oracle_params(8)
    net = wlr.WarmStartNet(**SHAPE, max_frames=64)
    net.set_params(flat)
    rng = np.random.default_rng(9)
    X = _rows(rng.standard_normal((6, 2, 30, 40)))
    Om = torch.empty((6, 64), dtype=torch.float32, device=DEV)
    net.forward(X, [0, 6], Om)
    net.backward(_rows(rng.standard_normal((6, 64))))
    G = net.grads().astype(np.float64)
    P0 = flat.astype(np.float64)
    m = np.zeros_like(P0)
    v = np.zeros_like(P0)
    net.adam(1e-3, grad_scale=0.5)
    want, m, v = ows.adam_step(P0, 0.5 * G, m, v, 1, lr=1e-3)
    assert _rel_max(net.params().astype(np.float64) - P0, want - P0) < 1e-4
    net.adam(1e-3, grad_scale=0.5)
    want, m, v = ows.adam_step(want, 0.5 * G, m, v, 2, lr=1e-3)
    assert _rel_max(net.params().astype(np.float64) - P0, want - P0) < 1e-4
    net.close()


def test_basis_of_the_solution(wlr):
    # FP64 handle with the rank-(r-k) step converged: the basis spans X1 and the kept
    # left singular vectors (oracle cd_step for the same X1)
    A, W1 = _clip(30, 40, 60, 5, 8, 12)
    A64, W64 = A.astype(np.float64), W1.astype(np.float64)
    m, n, k, r = 1200, 60, 5, 8
    s = wlr.Solver(m, n, k, r, precision=wlr.WLR_PREC_FP64, stop=wlr.WLR_STOP_NONE, eig_block=32,
                   eig_iters=60, eig_iters_cold=400)
    s.set_data(_col(A64), _col(W64))
    s.set_init(wlr.WLR_INIT_A1)
    s.solve(0.0, 5)
    V = torch.empty((r, m), dtype=torch.float32, device=DEV).T
    s.basis(V)
    Vh = V.cpu().numpy().astype(np.float64)
    X1 = np.zeros((m, k), order="F")
    s.result(X1)
    cd = oracle.cd_step(A64[:, k:], X1, r - k)
    Bref = np.hstack([cd.Q, cd.U])
    assert np.abs(Vh.T @ Vh - np.eye(r)).max() < 1e-6
    assert np.linalg.norm(Vh @ Vh.T - Bref @ Bref.T) < 1e-5
    s.close()


def test_learned_init_is_the_weighted_projection(wlr):
    H, W, n, k, r = 30, 40, 24, 4, 9
    A, W1 = _clip(H, W, n, k, r, 13)
    _, flat = _oracle_params(10)
    net = wlr.WarmStartNet(**SHAPE, max_frames=64)
    net.set_params(flat)
    tA, tW = _col(A), _col(W1)
    s = wlr.Solver(H * W, n, k, r, precision=wlr.WLR_PREC_FP32, stop=wlr.WLR_STOP_NONE)
    s.set_data(tA, tW)
    s.set_init_learned(net, H, W)
    X1 = np.zeros((H * W, k), dtype=np.float32, order="F")
    s.result(X1)
    # the same network output through the separate entry points
    X = torch.empty((n, 2, 30, 40), dtype=torch.float32, device=DEV)
    net.prepare(tA, tW, H, W, k, X)
    Om = torch.empty((n, 64), dtype=torch.float32, device=DEV)
    net.forward(X, [0, n], Om)
    U = ows.omega_basis(A.astype(np.float64), Om.cpu().numpy().astype(np.float64), r, k)
    want = ows.warm_start_x1_weighted(A[:, :k].astype(np.float64), U, W1.astype(np.float64))
    assert _rel_max(X1.astype(np.float64), want) < 1e-5
    assert s.iteration() == 0
    s.step()                                      # the iteration starts from it
    s.close()
    net.close()


def test_training_lowers_the_loss(wlr):
    # a few clips, converged targets from the FP64 path, 40 Adam steps: the loss falls
    net = wlr.WarmStartNet(**SHAPE, max_frames=512, seed=11)
    clips = []
    for q in range(4):
        H, W, n, k, r = 30, 40, 30 + 5 * q, 3 + q, 6 + q
        A, W1 = _clip(H, W, n, k, r, 100 + q)
        tA, tW = _col(A), _col(W1)
        s = wlr.Solver(H * W, n, k, r, precision=wlr.WLR_PREC_FP32, stop=wlr.WLR_STOP_NONE)
        s.set_data(tA, tW)
        s.set_init(wlr.WLR_INIT_A1)
        s.solve(0.0, 300)
        V = torch.empty((r, H * W), dtype=torch.float32, device=DEV).T
        s.basis(V)
        X = torch.empty((n, 2, 30, 40), dtype=torch.float32, device=DEV)
        net.prepare(tA, tW, H, W, k, X)
        clips.append((tA, X, V, n, r))
        s.close()
    k_of = [3 + q for q in range(4)]
    Xall = torch.cat([c[1] for c in clips])
    starts = np.cumsum([0] + [c[3] for c in clips])
    F = int(starts[-1])
    Om = torch.empty((F, 64), dtype=torch.float32, device=DEV)
    dOm = torch.empty((F, 64), dtype=torch.float32, device=DEV)
    loss = torch.zeros(1, dtype=torch.float64, device=DEV)
    hist = []
    for it in range(40):
        net.forward(Xall, starts, Om)
        loss.zero_()
        for c, (tA, _, V, n, r) in enumerate(clips):
            a, b = int(starts[c]), int(starts[c + 1])
            net.loss(tA, k_of[c], Om[a:b], r, V, loss, dOm[a:b])
        hist.append(loss.item() / len(clips))
        net.backward(dOm)
        net.adam(1e-3, grad_scale=1.0 / len(clips))
    assert all(np.isfinite(hist))
    assert hist[-1] < 0.7 * hist[0], hist
    net.close()


def test_fallback_keeps_the_start_with_the_lower_objective(wlr):
    # an untrained network's start lies far above X1_0 = A1 in F~: the fallback keeps A1
    H, W, n, k, r = 30, 40, 30, 4, 8
    A, W1 = _clip(H, W, n, k, r, 14)
    _, flat = _oracle_params(11)
    net = wlr.WarmStartNet(**SHAPE, max_frames=64)
    net.set_params(flat)
    tA, tW = _col(A), _col(W1)
    s = wlr.Solver(H * W, n, k, r, precision=wlr.WLR_PREC_FP32, stop=wlr.WLR_STOP_NONE)
    s.set_data(tA, tW)
    assert s.set_init_learned(net, H, W, fallback=False) is True
    XL = np.zeros((H * W, k), dtype=np.float32, order="F")
    s.result(XL)
    F_learned = s.step()
    s.set_init(wlr.WLR_INIT_A1)
    F_a1 = s.step()
    used = s.set_init_learned(net, H, W, fallback=True)
    assert used == (F_learned < F_a1)
    assert s.iteration() == 0
    X1 = np.zeros((H * W, k), dtype=np.float32, order="F")
    s.result(X1)
    assert np.array_equal(X1, XL if used else A[:, :k])
    s.close()
    net.close()
