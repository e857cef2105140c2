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
