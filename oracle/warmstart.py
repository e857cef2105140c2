"""FP64 CPU oracle for a learned warm start of the sWLR iteration (the initialisation of
Algorithm 1; Section 4.1 starts from a random matrix, which a predicted basis replaces).

TEST INFRASTRUCTURE ONLY, under the same rules as fp64.py: only the test suite may import
it, and it imports nothing from the product package.  It fixes what the warm start's GPU
kernels have to compute, one function per step, in plain float64 NumPy:

  * downsample_frames:   every H x W frame (a column of A, vectorised row-major, index
                         y W + x) to h x w by the mean of its f x f blocks (H = f h, W = f w);
  * upsample_bilinear:   an h x w map back to H x W by bilinear interpolation with
                         half-pixel centres: output pixel (Y, X) samples the input at
                         ((Y + 1/2)/f - 1/2, (X + 1/2)/f - 1/2), clamped to the border;
  * warm_start_x1:       X1_0 = P_U A1 = U (U^T U)^{-1} U^T A1, the projection of the
                         weighted frames onto the span of a full-resolution basis U (m x r);
  * projector_distance:  L(Y) = ||P_Y - P_V||_F^2 between the span of a predicted basis Y
                         (any full column rank) and an orthonormal target V; its gradient
                         dL/dY = -4 (I - P_Y) P_V Y (Y^T Y)^{-1};
  * mlp_forward / mlp_backward: a plain ReLU multilayer perceptron (features -> basis
                         entries) and its gradients by the chain rule.

Pins (tests/test_oracle_warmstart.py): block means and bilinear interpolation are exact on
constant and affine images; the projection is idempotent, equals A1 when span(U) holds A1's
columns, and does not depend on the basis of span(U); the projector distance has the closed
form 2 sin^2(theta) for one dimension, is invariant under Y -> Y M, vanishes exactly on
equal spans and equals 2r - 2 ||Q^T V||_F^2; both gradients match central differences.
The network of the warm start (per clip: n frames, k weighted, rank r <= r_max):
  * prepare_input:       per frame two h x w channels: the frame's block means divided by
                         the clip's RMS, and the mean of W1's k columns (block means)
                         divided by its own mean;
  * conv3x3s2_forward /  3 x 3 convolution (cross-correlation), stride 2, zero padding 1,
    conv3x3s2_backward:  plus bias; output ceil(h/2) x ceil(w/2);
  * net_forward /        relu(conv1) -> relu(conv2) -> flattened features f_j of frame j;
    net_backward:        z_j = [f_j | mean of f over the frames of j's clip] -> relu(fc1)
                         -> fc2 -> omega_j (r_max numbers): the row j of the frame-mixing
                         matrix Omega (n x r_max) of the clip;
  * omega_basis /        the clip's predicted basis is Y = [A1 | 0] + A Omega[:, :r] / n (full
    omega_loss:          resolution, m x r): the weighted frames plus frame mixtures (the W1
                         term of Eq. 5 keeps X1 close to A1, so the solution's span holds
                         A1's columns up to small corrections); loss = ||P_Y - P_V||_F^2 / (2 r)
                         with V the converged solution's column space; gradient
                         d/dOmega = A^T dL/dY / n;
  * warm_start_x1_weighted: X1_0(:, a) = U (U^T D_a U)^{-1} U^T D_a A1(:, a), D_a =
                         diag(W1(:, a)^2): the weighted least-squares fit of each weighted
                         frame inside span(U) (the minimiser of the first term of Eq. 5 over
                         X1 with columns in span(U));
  * round_bf16, adam_step: the weight storage (round to nearest even, 8 mantissa bits) and
                         the optimiser (Kingma & Ba, ICLR 2015, Algorithm 1).

Parity unpinned: what a trained network predicts (its worth is measured by the
iterations of Algorithm 1 it saves, not by a closed form).
"""
from __future__ import annotations

import numpy as np

__all__ = ["downsample_frames", "upsample_bilinear", "warm_start_x1", "projector_distance",
           "projector_distance_grad", "mlp_init", "mlp_forward", "mlp_backward",
           "prepare_input", "conv3x3s2_forward", "conv3x3s2_backward", "net_init", "net_forward",
           "net_backward", "omega_basis", "omega_loss", "warm_start_x1_weighted", "round_bf16", "adam_step"]


def downsample_frames(A: np.ndarray, H: int, W: int, f: int) -> np.ndarray:
    """Columns of A (m = H W pixels, row-major) averaged over f x f blocks: (H/f)(W/f) x n."""
    m, n = A.shape
    assert m == H * W and H % f == 0 and W % f == 0
    h, w = H // f, W // f
    frames = A.T.reshape(n, h, f, w, f)
    return frames.mean(axis=(2, 4)).reshape(n, h * w).T


def _bilinear_weights(out_len: int, in_len: int, f: int):
    """Source indices i0, i1 and weight t of output coordinate o: the sample position
    (o + 1/2)/f - 1/2 clamped to [0, in_len - 1]; value = (1 - t) v[i0] + t v[i1]."""
    pos = (np.arange(out_len) + 0.5) / f - 0.5
    pos = np.clip(pos, 0.0, in_len - 1.0)
    i0 = np.floor(pos).astype(int)
    i1 = np.minimum(i0 + 1, in_len - 1)
    t = pos - i0
    return i0, i1, t


def upsample_bilinear(U: np.ndarray, h: int, w: int, f: int) -> np.ndarray:
    """Columns of U (h w entries, row-major h x w maps) interpolated to (f h)(f w) rows."""
    hw, r = U.shape
    assert hw == h * w
    H, W = f * h, f * w
    y0, y1, ty = _bilinear_weights(H, h, f)
    x0, x1, tx = _bilinear_weights(W, w, f)
    maps = U.T.reshape(r, h, w)
    top = (1 - tx)[None, None, :] * maps[:, y0][:, :, x0] + tx[None, None, :] * maps[:, y0][:, :, x1]
    bot = (1 - tx)[None, None, :] * maps[:, y1][:, :, x0] + tx[None, None, :] * maps[:, y1][:, :, x1]
    out = (1 - ty)[None, :, None] * top + ty[None, :, None] * bot
    return out.reshape(r, H * W).T


def warm_start_x1(A1: np.ndarray, U: np.ndarray) -> np.ndarray:
    """X1_0 = U (U^T U)^{-1} U^T A1 (U: m x r, full column rank), through a Householder QR
    of U (library step): P_U = Q Q^T."""
    Q, _ = np.linalg.qr(U, mode="reduced")
    return Q @ (Q.T @ A1)


def projector_distance(Y: np.ndarray, V: np.ndarray) -> float:
    """||P_Y - P_V||_F^2 with P_Y = Y (Y^T Y)^{-1} Y^T and V orthonormal (m x r each)."""
    PY = Y @ np.linalg.solve(Y.T @ Y, Y.T)
    PV = V @ V.T
    return float(np.sum((PY - PV) ** 2))


def projector_distance_grad(Y: np.ndarray, V: np.ndarray) -> np.ndarray:
    """dL/dY = -4 (I - P_Y) P_V Y (Y^T Y)^{-1}: L = 2r - 2 tr(P_Y P_V) because both are
    rank-r projectors, and d tr(P_Y P_V) = 2 tr((I - P_Y) P_V Y (Y^T Y)^{-1} dY^T)."""
    G = Y.T @ Y
    PY = Y @ np.linalg.solve(G, Y.T)
    PV = V @ V.T
    return -4.0 * (np.eye(Y.shape[0]) - PY) @ PV @ Y @ np.linalg.inv(G)


def mlp_init(sizes, seed: int):
    """Weights W_l (out x in) ~ N(0, 2 / in), biases 0, for layer sizes sizes[0] -> ... ."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return [(rng.standard_normal((b, a)) * np.sqrt(2.0 / a), np.zeros(b))
            for a, b in zip(sizes[:-1], sizes[1:])]


def mlp_forward(params, X: np.ndarray):
    """Rows of X (batch x in) through h_{l+1} = relu(h_l W_l^T + b_l), the last layer
    without the relu.  Returns the output and the pre-activations of every layer."""
    h = X
    pre = []
    for li, (Wl, bl) in enumerate(params):
        z = h @ Wl.T + bl
        pre.append((h, z))
        h = z if li == len(params) - 1 else np.maximum(z, 0.0)
    return h, pre


def mlp_backward(params, pre, dY: np.ndarray):
    """Gradients (dW_l, db_l) of a loss with dL/d(output) = dY, and dL/dX."""
    grads = [None] * len(params)
    g = dY
    for li in range(len(params) - 1, -1, -1):
        h_in, z = pre[li]
        if li != len(params) - 1:
            g = g * (z > 0.0)
        Wl, _ = params[li]
        grads[li] = (g.T @ h_in, g.sum(axis=0))
        g = g @ Wl
    return grads, g


# ----------------------------------------------------------------- the warm-start network
def prepare_input(A: np.ndarray, W1: np.ndarray, H: int, W: int, f: int) -> np.ndarray:
    """Network input of one clip, shape (n, 2, h, w): channel 0 holds each frame's f x f
    block means divided by the RMS of all of them; channel 1 the block means of the
    per-pixel mean of W1 over its k columns, divided by their mean (same for every frame)."""
    n = A.shape[1]
    h, w = H // f, W // f
    a = downsample_frames(A, H, W, f)                         # (h w) x n
    a = a / np.sqrt(np.mean(a * a))
    wm = downsample_frames(np.mean(W1, axis=1, keepdims=True), H, W, f)[:, 0]
    wm = wm / np.mean(wm)
    X = np.empty((n, 2, h, w))
    X[:, 0] = a.T.reshape(n, h, w)
    X[:, 1] = wm.reshape(h, w)[None]
    return X


def conv3x3s2_forward(X: np.ndarray, Wc: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Z[f, o, y, x] = b[o] + sum_{c, u, v} Wc[o, c, u, v] X[f, c, 2y + u - 1, 2x + v - 1],
    X read as zero outside its h x w; Z is (F, O, ceil(h/2), ceil(w/2))."""
    F, C, h, w = X.shape
    ho, wo = (h + 1) // 2, (w + 1) // 2
    Xp = np.zeros((F, C, h + 2, w + 2))
    Xp[:, :, 1:h + 1, 1:w + 1] = X
    Z = np.zeros((F, Wc.shape[0], ho, wo)) + b[None, :, None, None]
    for u in range(3):
        for v in range(3):
            patch = Xp[:, :, u:u + 2 * ho:2, v:v + 2 * wo:2]   # X[2y + u - 1, 2x + v - 1]
            Z += np.einsum("oc,fcyx->foyx", Wc[:, :, u, v], patch)
    return Z


def conv3x3s2_backward(X: np.ndarray, Wc: np.ndarray, dZ: np.ndarray):
    """Gradients (dX, dWc, db) of a loss with dL/dZ = dZ for Z = conv3x3s2_forward(X, Wc, b)."""
    F, C, h, w = X.shape
    ho, wo = dZ.shape[2], dZ.shape[3]
    Xp = np.zeros((F, C, h + 2, w + 2))
    Xp[:, :, 1:h + 1, 1:w + 1] = X
    dXp = np.zeros_like(Xp)
    dW = np.zeros_like(Wc)
    for u in range(3):
        for v in range(3):
            patch = Xp[:, :, u:u + 2 * ho:2, v:v + 2 * wo:2]
            dW[:, :, u, v] = np.einsum("foyx,fcyx->oc", dZ, patch)
            dXp[:, :, u:u + 2 * ho:2, v:v + 2 * wo:2] += np.einsum("oc,foyx->fcyx", Wc[:, :, u, v], dZ)
    return dXp[:, :, 1:h + 1, 1:w + 1], dW, dZ.sum(axis=(0, 2, 3))


def net_init(h: int, w: int, c1: int, c2: int, hidden: int, r_max: int, seed: int):
    """Parameters [(Wc1, b1), (Wc2, b2), (W3, b3), (W4, b4)]: weights N(0, 2 / fan_in),
    biases 0; conv weights (out, in, 3, 3), fc weights (out, in)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    h2, w2 = ((h + 1) // 2 + 1) // 2, ((w + 1) // 2 + 1) // 2
    D = c2 * h2 * w2
    shapes = [((c1, 2, 3, 3), 18), ((c2, c1, 3, 3), 9 * c1), ((hidden, 2 * D), 2 * D), ((r_max, hidden), hidden)]
    return [(rng.standard_normal(sh) * np.sqrt(2.0 / fan), np.zeros(sh[0])) for sh, fan in shapes]


def _clip_mean(feat: np.ndarray, sizes) -> np.ndarray:
    """Each row replaced by the mean of the rows of its clip (clips = consecutive runs of
    `sizes` rows)."""
    out = np.empty_like(feat)
    o = 0
    for nc in sizes:
        out[o:o + nc] = feat[o:o + nc].mean(axis=0, keepdims=True)
        o += nc
    return out


def net_forward(params, X: np.ndarray, sizes):
    """Omega rows (F x r_max) of the frames X (F, 2, h, w) of consecutive clips of `sizes`
    frames, and the cache for net_backward."""
    (Wc1, b1), (Wc2, b2), (W3, b3), (W4, b4) = params
    z1 = conv3x3s2_forward(X, Wc1, b1)
    a1 = np.maximum(z1, 0.0)
    z2 = conv3x3s2_forward(a1, Wc2, b2)
    a2 = np.maximum(z2, 0.0)
    feat = a2.reshape(a2.shape[0], -1)
    z = np.hstack([feat, _clip_mean(feat, sizes)])
    z3 = z @ W3.T + b3
    a3 = np.maximum(z3, 0.0)
    Om = a3 @ W4.T + b4
    return Om, (X, z1, a1, z2, a2, z, z3, a3, tuple(sizes))


def net_backward(params, cache, dOm: np.ndarray):
    """Gradients [(dWc1, db1), (dWc2, db2), (dW3, db3), (dW4, db4)] for dL/dOmega = dOm."""
    (Wc1, b1), (Wc2, b2), (W3, b3), (W4, b4) = params
    X, z1, a1, z2, a2, z, z3, a3, sizes = cache
    dW4, db4 = dOm.T @ a3, dOm.sum(axis=0)
    dz3 = (dOm @ W4) * (z3 > 0.0)
    dW3, db3 = dz3.T @ z, dz3.sum(axis=0)
    dz = dz3 @ W3
    D = dz.shape[1] // 2
    dfeat = dz[:, :D] + _clip_mean(dz[:, D:], sizes)
    dz2 = dfeat.reshape(z2.shape) * (z2 > 0.0)
    da1, dWc2, db2 = conv3x3s2_backward(a1, Wc2, dz2)
    dz1 = da1 * (z1 > 0.0)
    _, dWc1, db1 = conv3x3s2_backward(X, Wc1, dz1)
    return [(dWc1, db1), (dWc2, db2), (dW3, db3), (dW4, db4)]


def omega_basis(A: np.ndarray, Om: np.ndarray, r: int, k: int) -> np.ndarray:
    """The clip's predicted basis Y = [A1 | 0] + A Omega[:, :r] / n (m x r): the k weighted
    frames plus frame mixtures, so that an output near zero starts from span(A1)."""
    n = A.shape[1]
    Y = A @ Om[:, :r] / n
    Y[:, :k] += A[:, :k]
    return Y


def omega_loss(A: np.ndarray, Om: np.ndarray, r: int, V: np.ndarray, k: int):
    """Loss ||P_Y - P_V||_F^2 / (2 r) of the clip basis Y = omega_basis(A, Omega, r, k)
    against the orthonormal target V (m x r), and its gradient with respect to Omega
    (n x r_max; the columns beyond r get zero): d/dOmega = A^T dL/dY / n."""
    n = A.shape[1]
    Y = omega_basis(A, Om, r, k)
    L = projector_distance(Y, V) / (2.0 * r)
    dY = projector_distance_grad(Y, V) / (2.0 * r)
    dOm = np.zeros_like(Om)
    dOm[:, :r] = A.T @ dY / n
    return L, dOm


def warm_start_x1_weighted(A1: np.ndarray, U: np.ndarray, W1: np.ndarray) -> np.ndarray:
    """X1_0(:, a) = U (U^T D_a U)^{-1} U^T D_a A1(:, a) with D_a = diag(W1(:, a)^2): for
    each weighted frame the point of span(U) closest to it in the W1-weighted norm of the
    first term of Eq. 5 (one dense solve per column; library step)."""
    X = np.empty_like(A1, dtype=np.float64)
    for a in range(A1.shape[1]):
        d = W1[:, a] ** 2
        X[:, a] = U @ np.linalg.solve(U.T @ (U * d[:, None]), U.T @ (d * A1[:, a]))
    return X


def round_bf16(x: np.ndarray) -> np.ndarray:
    """float32 values rounded to bfloat16 (the upper 16 bits of an IEEE binary32), round to
    nearest with ties to even, returned as float64."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (b >> np.uint64(16)) & np.uint64(1)
    b = (b + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def adam_step(theta, g, m, v, t: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-8):
    """One Adam update (Kingma & Ba 2015, Algorithm 1) at step t >= 1: returns the new
    (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
