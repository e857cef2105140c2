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
