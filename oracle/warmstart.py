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
Parity unpinned: what a trained network predicts (its worth is measured by the
iterations of Algorithm 1 it saves, not by a closed form).
"""
from __future__ import annotations

import numpy as np

__all__ = ["downsample_frames", "upsample_bilinear", "warm_start_x1", "projector_distance",
           "projector_distance_grad", "mlp_init", "mlp_forward", "mlp_backward"]


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
