"""Planted mistakes in the oracle (on the CPU only): each plausible slip in the
method's arithmetic must make at least one pin fail."""
import numpy as np
import pytest
from scipy.linalg import solve_triangular

import oracle
import oracle.fp64 as sw
from tests import test_oracle_pins as pins


def _cd_no_rinv(A2, X1, s):
    cd = sw._orig_cd_step(A2, X1, s)
    cd.C = cd.B.copy()                       # forgot R^{-1}
    return cd


def _cd_extra_rank(A2, X1, s):
    return sw._orig_cd_step(A2, X1, s + 1)   # one singular triplet too many in D


def _x1_weight_not_squared(A, W1, C, D, chunk=4096):
    k = W1.shape[1]
    A1, A2 = A[:, :k], A[:, k:]
    E = A1 * W1 + (A2 - D) @ C.T             # W1 instead of W1 o W1
    G = C @ C.T
    out = np.empty((A.shape[0], k))
    for i in range(A.shape[0]):
        out[i] = np.linalg.solve(np.diag(W1[i] ** 2) + G, E[i])
    return out


def _x1_drop_D(A, W1, C, D, chunk=4096):
    return sw._orig_x1_update(A, W1, C, np.zeros_like(D), chunk)


def _x1_transposed_G(A, W1, C, D, chunk=4096):
    k = W1.shape[1]
    A1, A2 = A[:, :k], A[:, k:]
    E = A1 * W1 * W1 + (A2 - D) @ C.T
    G = C @ C.T
    G = G + np.triu(G, 1) * 0.5              # asymmetric slip in C C^T
    out = np.empty((A.shape[0], k))
    for i in range(A.shape[0]):
        out[i] = np.linalg.solve(np.diag(W1[i] ** 2) + G, E[i])
    return out


MUTATIONS = {
    "C without R^-1": ("cd_step", _cd_no_rinv),
    "D with rank s+1": ("cd_step", _cd_extra_rank),
    "E weight not squared": ("x1_update", _x1_weight_not_squared),
    "E drops D": ("x1_update", _x1_drop_D),
    "G slip": ("x1_update", _x1_transposed_G),
}

PINS = [
    pins.test_cd_step_is_the_minimiser_over_C_and_D,
    pins.test_x1_update_is_stationary_and_minimal,
    pins.test_objective_non_increasing,
    pins.test_rank_bound_and_theorem2_structure,
    pins.test_eckart_young_reduction_unit_weights,
    pins.test_ghs_limit_large_weights,
]


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, monkeypatch):
    attr, fn = MUTATIONS[name]
    monkeypatch.setattr(sw, "_orig_cd_step", sw.cd_step, raising=False)
    monkeypatch.setattr(sw, "_orig_x1_update", sw.x1_update, raising=False)
    monkeypatch.setattr(sw, attr, fn)
    monkeypatch.setattr(oracle, attr, fn)
    failed = []
    for pin in PINS:
        try:
            with np.errstate(all="ignore"):
                pin()
        except (AssertionError, np.linalg.LinAlgError, ValueError):
            failed.append(pin.__name__)
    assert failed, f"no pin caught the planted mistake '{name}'"


# ---------------------------------------------------------------- warm-start oracle
import oracle.warmstart as ws  # noqa: E402
from tests import test_oracle_warmstart as wpins  # noqa: E402


def _grad_sign(Y, V):
    return -ws._orig["projector_distance_grad"](Y, V)


def _grad_no_gram_inverse(Y, V):
    PY = Y @ np.linalg.solve(Y.T @ Y, Y.T)
    return -4.0 * (np.eye(Y.shape[0]) - PY) @ (V @ V.T) @ Y


def _upsample_no_half_pixel(U, h, w, f):
    hw, r = U.shape
    H, W = f * h, f * w
    yi = np.minimum(np.arange(H) / f, h - 1.0)
    xi = np.minimum(np.arange(W) / f, w - 1.0)
    y0, x0 = np.floor(yi).astype(int), np.floor(xi).astype(int)
    y1, x1 = np.minimum(y0 + 1, h - 1), np.minimum(x0 + 1, w - 1)
    ty, tx = yi - y0, xi - x0
    maps = U.T.reshape(r, h, w)
    top = (1 - tx) * maps[:, y0][:, :, x0] + tx * maps[:, y0][:, :, x1]
    bot = (1 - tx) * maps[:, y1][:, :, x0] + tx * maps[:, y1][:, :, x1]
    return ((1 - ty)[None, :, None] * top + ty[None, :, None] * bot).reshape(r, H * W).T


def _downsample_first_pixel(A, H, W, f):
    m, n = A.shape
    return A.T.reshape(n, H // f, f, W // f, f)[:, :, 0, :, 0].reshape(n, -1).T


def _warm_start_unnormalised(A1, U):
    return U @ (U.T @ A1)


def _mlp_backward_no_relu_mask(params, pre, dY):
    grads = [None] * len(params)
    g = dY
    for li in range(len(params) - 1, -1, -1):
        h_in, _ = pre[li]
        Wl, _ = params[li]
        grads[li] = (g.T @ h_in, g.sum(axis=0))
        g = g @ Wl
    return grads, g


def _conv_flipped(X, Wc, b):
    return ws._orig["conv3x3s2_forward"](X, Wc[:, :, ::-1, ::-1], b)


def _net_backward_no_context(params, cache, dOm):
    (Wc1, b1), (Wc2, b2), (W3, b3), (W4, b4) = params
    X, z1, a1, z2, a2, z, z3, a3, sizes = cache
    dW4, db4 = dOm.T @ a3, dOm.sum(axis=0)
    dz3 = (dOm @ W4) * (z3 > 0.0)
    dW3, db3 = dz3.T @ z, dz3.sum(axis=0)
    dz = dz3 @ W3
    dfeat = dz[:, :dz.shape[1] // 2]
    dz2 = dfeat.reshape(z2.shape) * (z2 > 0.0)
    da1, dWc2, db2 = ws.conv3x3s2_backward(a1, Wc2, dz2)
    _, dWc1, db1 = ws.conv3x3s2_backward(X, Wc1, da1 * (z1 > 0.0))
    return [(dWc1, db1), (dWc2, db2), (dW3, db3), (dW4, db4)]


def _weighted_projection_w1(A1, U, W1):
    return ws._orig["warm_start_x1_weighted"](A1, U, np.sqrt(W1))


def _bf16_truncated(x):
    b = np.asarray(x, dtype=np.float32).view(np.uint32) & np.uint32(0xFFFF0000)
    return b.view(np.float32).astype(np.float64)


def _adam_no_bias_correction(theta, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    return theta - lr * m / (np.sqrt(v) + eps), m, v


WS_MUTATIONS = {
    "convolution with the kernel flipped": ("conv3x3s2_forward", _conv_flipped),
    "network backward without the context term": ("net_backward", _net_backward_no_context),
    "weighted projection with W1 instead of W1^2": ("warm_start_x1_weighted", _weighted_projection_w1),
    "bf16 by truncation": ("round_bf16", _bf16_truncated),
    "adam without bias correction": ("adam_step", _adam_no_bias_correction),
    "loss gradient sign": ("projector_distance_grad", _grad_sign),
    "loss gradient without (Y^T Y)^-1": ("projector_distance_grad", _grad_no_gram_inverse),
    "upsampling without half-pixel centres": ("upsample_bilinear", _upsample_no_half_pixel),
    "downsampling by the first pixel": ("downsample_frames", _downsample_first_pixel),
    "projection without orthonormal basis": ("warm_start_x1", _warm_start_unnormalised),
    "backward without the relu mask": ("mlp_backward", _mlp_backward_no_relu_mask),
}

WS_PINS = [
    wpins.test_downsample_block_means,
    wpins.test_upsample_exact_on_affine_maps_away_from_the_border,
    wpins.test_down_then_up_keeps_constant_frames,
    wpins.test_warm_start_projection_identities,
    wpins.test_projector_distance_closed_forms,
    lambda: wpins.test_projector_distance_gradient_central_differences(4),
    wpins.test_mlp_gradients_central_differences,
    wpins.test_conv_is_strided_cross_correlation,
    wpins.test_conv_of_a_delta_and_of_a_constant,
    wpins.test_conv_backward_central_differences,
    wpins.test_net_backward_central_differences,
    wpins.test_net_frames_are_exchangeable_within_a_clip,
    wpins.test_omega_loss_gradient_prior_and_zero,
    wpins.test_weighted_projection,
    wpins.test_round_bf16,
    wpins.test_adam_first_step_and_descent,
    wpins.test_prepare_input_scales,
]


@pytest.mark.parametrize("name", sorted(WS_MUTATIONS))
def test_planted_warm_start_mistake_is_caught(name, monkeypatch):
    attr, fn = WS_MUTATIONS[name]
    monkeypatch.setattr(ws, "_orig", {a: getattr(ws, a) for a, _ in WS_MUTATIONS.values()}, raising=False)
    monkeypatch.setattr(ws, attr, fn)
    caught = 0
    for pin in WS_PINS:
        try:
            with np.errstate(all="ignore"):
                pin()
        except AssertionError:
            caught += 1
    assert caught, f"no pin caught the planted mistake '{name}'"
