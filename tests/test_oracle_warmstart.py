"""Pins of the warm-start oracle (oracle/warmstart.py) against what mathematics fixes: exact
results on constant and affine images, projection identities, the closed form of the
projector distance, and gradients against central differences."""
import numpy as np
import pytest

from oracle import warmstart as ws


def _affine_frames(H, W, n, rng):
    """Frames a + b y + c x (row-major, index y W + x), one column per frame."""
    yy, xx = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    cols = []
    for _ in range(n):
        a, b, c = rng.standard_normal(3)
        cols.append((a + b * yy + c * xx).reshape(-1))
    return np.stack(cols, axis=1)


def test_downsample_block_means():
    rng = np.random.default_rng(0)
    H, W, f = 24, 32, 8
    A = _affine_frames(H, W, 3, rng)
    D = ws.downsample_frames(A, H, W, f)
    assert D.shape == ((H // f) * (W // f), 3)
    # the mean of an affine function over a block is its value at the block centre
    yy, xx = np.meshgrid(np.arange(H // f), np.arange(W // f), indexing="ij")
    for j in range(3):
        full = A[:, j].reshape(H, W)
        a = full[0, 0]
        b = full[1, 0] - full[0, 0]
        c = full[0, 1] - full[0, 0]
        want = a + b * (f * yy + (f - 1) / 2) + c * (f * xx + (f - 1) / 2)
        assert np.allclose(D[:, j].reshape(H // f, W // f), want, atol=1e-12)
    # the frame mean is kept
    assert np.allclose(D.mean(axis=0), A.mean(axis=0), atol=1e-12)


def test_upsample_exact_on_affine_maps_away_from_the_border():
    rng = np.random.default_rng(1)
    h, w, f = 5, 7, 4
    yy, xx = np.meshgrid(np.arange(h), np.arange(w), indexing="ij")
    a, b, c = rng.standard_normal(3)
    U = (a + b * yy + c * xx).reshape(-1, 1)
    up = ws.upsample_bilinear(U, h, w, f).reshape(f * h, f * w)
    Y, X = np.meshgrid(np.arange(f * h), np.arange(f * w), indexing="ij")
    sy, sx = (Y + 0.5) / f - 0.5, (X + 0.5) / f - 0.5
    want = a + b * sy + c * sx
    inner = (sy >= 0) & (sy <= h - 1) & (sx >= 0) & (sx <= w - 1)
    assert np.allclose(up[inner], want[inner], atol=1e-12)
    # clamped at the border: the border rows/columns repeat the nearest sample
    const = ws.upsample_bilinear(np.full((h * w, 2), 3.25), h, w, f)
    assert np.allclose(const, 3.25, atol=1e-15)


def test_down_then_up_keeps_constant_frames():
    H, W, f = 16, 24, 4
    A = np.full((H * W, 2), -1.5)
    D = ws.downsample_frames(A, H, W, f)
    assert np.allclose(ws.upsample_bilinear(D, H // f, W // f, f), A, atol=1e-15)


def test_warm_start_projection_identities():
    rng = np.random.default_rng(2)
    m, k, r = 60, 4, 6
    U = rng.standard_normal((m, r))
    A1 = rng.standard_normal((m, k))
    X = ws.warm_start_x1(A1, U)
    assert np.allclose(ws.warm_start_x1(X, U), X, atol=1e-12)            # idempotent
    M = rng.standard_normal((r, r)) + 3 * np.eye(r)
    assert np.allclose(ws.warm_start_x1(A1, U @ M), X, atol=1e-10)      # basis-free
    inside = U @ rng.standard_normal((r, k))
    assert np.allclose(ws.warm_start_x1(inside, U), inside, atol=1e-11)  # A1 in span(U)
    assert np.allclose(U.T @ (A1 - X), 0.0, atol=1e-11)                  # residual orthogonal


def test_projector_distance_closed_forms():
    rng = np.random.default_rng(3)
    # one dimension: ||P_y - P_v||_F^2 = 2 sin^2(theta)
    th = 0.37
    y = np.array([[np.cos(th)], [np.sin(th)], [0.0]]) * 2.5
    v = np.array([[1.0], [0.0], [0.0]])
    assert abs(ws.projector_distance(y, v) - 2 * np.sin(th) ** 2) < 1e-14
    m, r = 40, 5
    V, _ = np.linalg.qr(rng.standard_normal((m, r)))
    Y = rng.standard_normal((m, r))
    L = ws.projector_distance(Y, V)
    Q, _ = np.linalg.qr(Y)
    assert abs(L - (2 * r - 2 * np.sum((Q.T @ V) ** 2))) < 1e-11
    M = rng.standard_normal((r, r)) + 2 * np.eye(r)
    assert abs(ws.projector_distance(Y @ M, V) - L) < 1e-10
    assert ws.projector_distance(V @ M, V) < 1e-20                      # equal spans
    assert 0.0 <= L <= 2 * r


@pytest.mark.parametrize("seed", [4, 5])
def test_projector_distance_gradient_central_differences(seed):
    rng = np.random.default_rng(seed)
    m, r = 12, 3
    V, _ = np.linalg.qr(rng.standard_normal((m, r)))
    Y = rng.standard_normal((m, r))
    G = ws.projector_distance_grad(Y, V)
    h = 1e-6
    num = np.zeros_like(Y)
    for i in range(m):
        for j in range(r):
            E = np.zeros_like(Y)
            E[i, j] = h
            num[i, j] = (ws.projector_distance(Y + E, V) - ws.projector_distance(Y - E, V)) / (2 * h)
    assert np.max(np.abs(G - num)) < 1e-7 * max(1.0, np.max(np.abs(G)))
    # Y^T (I - P_Y) = 0, so the gradient has no component along span(Y) taken row-wise
    assert np.allclose(Y.T @ G, 0.0, atol=1e-10)


def test_mlp_gradients_central_differences():
    rng = np.random.default_rng(6)
    params = ws.mlp_init([7, 9, 8, 5], seed=11)
    X = rng.standard_normal((4, 7))
    T = rng.standard_normal((4, 5))

    def loss(ps, x):
        y, _ = ws.mlp_forward(ps, x)
        return 0.5 * np.sum((y - T) ** 2)

    y, pre = ws.mlp_forward(params, X)
    grads, dX = ws.mlp_backward(params, pre, y - T)
    h = 1e-6
    for li, (Wl, bl) in enumerate(params):
        for arr, g in ((Wl, grads[li][0]), (bl, grads[li][1])):
            num = np.zeros_like(arr)
            for idx in np.ndindex(arr.shape):
                old = arr[idx]
                arr[idx] = old + h
                lp = loss(params, X)
                arr[idx] = old - h
                lm = loss(params, X)
                arr[idx] = old
                num[idx] = (lp - lm) / (2 * h)
            assert np.max(np.abs(num - g)) < 1e-6
    numx = np.zeros_like(X)
    for idx in np.ndindex(X.shape):
        E = np.zeros_like(X)
        E[idx] = h
        numx[idx] = (loss(params, X + E) - loss(params, X - E)) / (2 * h)
    assert np.max(np.abs(numx - dX)) < 1e-6


def test_mlp_last_layer_is_linear():
    params = ws.mlp_init([3, 4, 2], seed=1)
    x = np.ones((1, 3))
    y1, _ = ws.mlp_forward(params, x)
    params[-1] = (2 * params[-1][0], 2 * params[-1][1])
    y2, _ = ws.mlp_forward(params, x)
    assert np.allclose(y2, 2 * y1)


# ------------------------------------------------------------------ the warm-start network
def test_conv_is_strided_cross_correlation():
    # one input and one output channel: the 'same' cross-correlation (a library routine)
    # sampled at even positions; several channels add up
    from scipy.signal import correlate2d
    rng = np.random.default_rng(11)
    for h, w in ((7, 9), (8, 10), (30, 40)):
        X = rng.standard_normal((2, 3, h, w))
        Wc = rng.standard_normal((4, 3, 3, 3))
        b = rng.standard_normal(4)
        Z = ws.conv3x3s2_forward(X, Wc, b)
        assert Z.shape == (2, 4, (h + 1) // 2, (w + 1) // 2)
        for f in range(2):
            for o in range(4):
                want = b[o] + sum(correlate2d(X[f, c], Wc[o, c], mode="same")[::2, ::2] for c in range(3))
                assert np.allclose(Z[f, o], want, atol=1e-12)


def test_conv_of_a_delta_and_of_a_constant():
    # Z[y, x] sums W[u, v] X[2y + u - 1, 2x + v - 1]: a unit impulse at the even position
    # (2, 4) reaches only the output (1, 2), through the centre tap
    Wc = np.arange(9, dtype=float).reshape(1, 1, 3, 3) + 1.0
    X = np.zeros((1, 1, 8, 8))
    X[0, 0, 2, 4] = 1.0
    Z = ws.conv3x3s2_forward(X, Wc, np.zeros(1))
    assert Z[0, 0, 1, 2] == Wc[0, 0, 1, 1]
    assert np.count_nonzero(Z) == 1
    # an impulse at (3, 5) reaches outputs (1, 2), (1, 3), (2, 2), (2, 3) through the corner taps
    X[:] = 0.0
    X[0, 0, 3, 5] = 1.0
    Z = ws.conv3x3s2_forward(X, Wc, np.zeros(1))
    assert Z[0, 0, 1, 2] == Wc[0, 0, 2, 2] and Z[0, 0, 2, 3] == Wc[0, 0, 0, 0]
    assert Z[0, 0, 1, 3] == Wc[0, 0, 2, 0] and Z[0, 0, 2, 2] == Wc[0, 0, 0, 2]
    # a constant image: interior outputs are c * sum(W) + b
    Z = ws.conv3x3s2_forward(np.full((1, 1, 9, 9), 2.0), Wc, np.array([0.5]))
    assert np.allclose(Z[0, 0, 1:-1, 1:-1], 2.0 * Wc.sum() + 0.5)


def _num_grad(f, x, idx, h=1e-6):
    xp, xm = x.copy(), x.copy()
    xp[idx] += h
    xm[idx] -= h
    return (f(xp) - f(xm)) / (2 * h)


def test_conv_backward_central_differences():
    rng = np.random.default_rng(12)
    X = rng.standard_normal((2, 2, 7, 6))
    Wc = rng.standard_normal((3, 2, 3, 3))
    b = rng.standard_normal(3)
    G = rng.standard_normal((2, 3, 4, 3))          # dL/dZ of L = <G, Z>
    dX, dW, db = ws.conv3x3s2_backward(X, Wc, G)
    L = lambda X_, W_, b_: float(np.sum(G * ws.conv3x3s2_forward(X_, W_, b_)))
    for idx in [(0, 0, 0, 0), (1, 1, 6, 5), (0, 1, 3, 2), (1, 0, 4, 0)]:
        assert abs(_num_grad(lambda t: L(t, Wc, b), X, idx) - dX[idx]) < 1e-7
    for idx in [(0, 0, 0, 0), (2, 1, 2, 2), (1, 0, 1, 2)]:
        assert abs(_num_grad(lambda t: L(X, t, b), Wc, idx) - dW[idx]) < 1e-7
    for o in range(3):
        assert abs(_num_grad(lambda t: L(X, Wc, t), b, (o,)) - db[o]) < 1e-7


def _tiny_net(seed):
    rng = np.random.default_rng(seed)
    params = ws.net_init(6, 8, 2, 3, 5, 4, seed)
    params = [(Wl, rng.standard_normal(bl.shape) * 0.1) for Wl, bl in params]
    sizes = (3, 2)
    X = rng.standard_normal((5, 2, 6, 8))
    return params, X, sizes


def test_net_backward_central_differences():
    params, X, sizes = _tiny_net(13)
    rng = np.random.default_rng(14)
    G = rng.standard_normal((5, 4))                 # dL/dOmega of L = <G, Omega>
    Om, cache = ws.net_forward(params, X, sizes)
    assert Om.shape == (5, 4)
    grads = ws.net_backward(params, cache, G)

    def loss_with(li, which, t):
        ps = [list(p) for p in params]
        ps[li][which] = t
        return float(np.sum(G * ws.net_forward([tuple(p) for p in ps], X, sizes)[0]))

    for li in range(4):
        for which in (0, 1):
            arr = params[li][which]
            for _ in range(3):
                idx = tuple(int(rng.integers(0, d)) for d in arr.shape)
                num = _num_grad(lambda t: loss_with(li, which, t), arr, idx)
                assert abs(num - grads[li][which][idx]) <= 1e-6 * max(1.0, abs(num)), (li, which, idx)


def test_net_frames_are_exchangeable_within_a_clip():
    # permuting the frames of a clip permutes its Omega rows and changes no other clip's
    params, X, sizes = _tiny_net(15)
    Om, _ = ws.net_forward(params, X, sizes)
    perm = [2, 0, 1, 3, 4]
    Om2, _ = ws.net_forward(params, X[perm], sizes)
    assert np.allclose(Om2, Om[perm], atol=1e-12)
    # the context term couples the frames of one clip only
    X3 = X.copy()
    X3[4] += 1.0
    Om3, _ = ws.net_forward(params, X3, sizes)
    assert np.allclose(Om3[:3], Om[:3], atol=1e-12)


def test_omega_loss_gradient_prior_and_zero():
    rng = np.random.default_rng(16)
    m, n, r, k, rmax = 30, 8, 4, 2, 5
    A = rng.standard_normal((m, n))
    V, _ = np.linalg.qr(rng.standard_normal((m, r)))
    Om = rng.standard_normal((n, rmax))
    L, dOm = ws.omega_loss(A, Om, r, V, k)
    assert 0.0 <= L <= 1.0
    assert np.all(dOm[:, r:] == 0.0)
    for idx in [(0, 0), (7, 2), (3, 1), (5, 3)]:
        assert abs(_num_grad(lambda t: ws.omega_loss(A, t, r, V, k)[0], Om, idx) - dOm[idx]) < 1e-7
    # the basis is the weighted frames plus mixtures scaled by 1 / n
    Y = ws.omega_basis(A, Om, r, k)
    assert np.allclose(Y[:, :k], A[:, :k] + A @ Om[:, :k] / n, atol=1e-13)
    assert np.allclose(Y[:, k:], A @ Om[:, k:r] / n, atol=1e-13)
    # with r = k and Omega = 0 the basis is A1 itself: the loss is A1's distance to V
    Vk, _ = np.linalg.qr(rng.standard_normal((m, k)))
    Lk, _ = ws.omega_loss(A, np.zeros((n, rmax)), k, Vk, k)
    assert abs(Lk - ws.projector_distance(A[:, :k], Vk) / (2 * k)) < 1e-12
    # zero when the target is the predicted span itself
    V3, _ = np.linalg.qr(Y)
    assert ws.omega_loss(A, Om, r, V3, k)[0] < 1e-24


def test_weighted_projection():
    rng = np.random.default_rng(17)
    m, r, k = 40, 4, 3
    U = rng.standard_normal((m, r))
    A1 = rng.standard_normal((m, k))
    W1 = rng.uniform(5.0, 50.0, (m, k))
    X = ws.warm_start_x1_weighted(A1, U, W1)
    # in span(U), and the weighted residual is orthogonal to span(U) (normal equations)
    Q, _ = np.linalg.qr(U)
    assert np.allclose(Q @ (Q.T @ X), X, atol=1e-12)
    for a in range(k):
        assert np.abs(U.T @ (W1[:, a] ** 2 * (A1[:, a] - X[:, a]))).max() < 1e-8
        # no other point of span(U) is closer in the weighted norm
        f = lambda x: np.sum(W1[:, a] ** 2 * (A1[:, a] - x) ** 2)
        for _ in range(5):
            assert f(X[:, a]) <= f(X[:, a] + U @ (1e-3 * rng.standard_normal(r)))
    # weights constant along each column: the plain orthogonal projection
    Wc = np.tile(rng.uniform(5.0, 50.0, (1, k)), (m, 1))
    assert np.allclose(ws.warm_start_x1_weighted(A1, U, Wc), ws.warm_start_x1(A1, U), atol=1e-12)


def test_round_bf16():
    torch = pytest.importorskip("torch")
    one = 1.0
    assert ws.round_bf16(np.array([one]))[0] == 1.0
    assert ws.round_bf16(np.array([1.0 + 2.0 ** -8]))[0] == 1.0                 # tie -> even
    assert ws.round_bf16(np.array([1.0 + 3 * 2.0 ** -8]))[0] == 1.0 + 2.0 ** -6  # tie -> even
    assert ws.round_bf16(np.array([1.0 + 2.0 ** -8 + 2.0 ** -20]))[0] == 1.0 + 2.0 ** -7
    x = np.random.default_rng(18).standard_normal(10000).astype(np.float32) * 10
    lib = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy().astype(np.float64)
    assert np.array_equal(ws.round_bf16(x), lib)


def test_adam_first_step_and_descent():
    rng = np.random.default_rng(19)
    th = rng.standard_normal(6)
    g = rng.standard_normal(6)
    t1, m1, v1 = ws.adam_step(th, g, np.zeros(6), np.zeros(6), 1, lr=0.01)
    # bias correction makes the first step lr * g / (|g| + eps)
    assert np.allclose(t1, th - 0.01 * g / (np.abs(g) + 1e-8), atol=1e-15)
    assert np.allclose(m1, 0.1 * g) and np.allclose(v1, 0.001 * g * g)
    # minimises a convex quadratic
    c = rng.standard_normal(6)
    th, m, v = np.zeros(6), np.zeros(6), np.zeros(6)
    for t in range(1, 3001):
        th, m, v = ws.adam_step(th, 2 * (th - c), m, v, t, lr=0.01)
    assert np.abs(th - c).max() < 1e-3


def test_prepare_input_scales():
    rng = np.random.default_rng(20)
    H, W, f, n, k = 12, 16, 2, 5, 3
    A = rng.standard_normal((H * W, n)) + 2.0
    W1 = rng.uniform(5.0, 50.0, (H * W, k))
    X = ws.prepare_input(A, W1, H, W, f)
    assert X.shape == (n, 2, H // f, W // f)
    assert abs(np.sqrt(np.mean(X[:, 0] ** 2)) - 1.0) < 1e-12
    assert abs(np.mean(X[0, 1]) - 1.0) < 1e-12
    assert np.allclose(X[:, 1], X[:1, 1])
    Xc = ws.prepare_input(A, np.full((H * W, k), 7.0), H, W, f)
    assert np.allclose(Xc[:, 1], 1.0)
    # channel 0 is the block means scaled
    D = ws.downsample_frames(A, H, W, f)
    assert np.allclose(X[2, 0].reshape(-1) * np.sqrt(np.mean(D * D)), D[:, 2])
