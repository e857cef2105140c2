"""Seeded synthetic video-shaped inputs for the sWLR problem.

This module only draws random inputs; it holds none of the method's arithmetic and
is shared by the tests, the benchmark and the oracle-based checks.  It stands in
for the Stuttgart synthetic video sequences used in the paper's experiments
(Section 4.2), which are not available here: no content of that dataset is
reproduced, only its shape (frames as columns, a low-rank background, sparse
moving foreground objects, sensor noise; the first k frames "almost pure
background", Section 1).

Recipe (all draws from numpy PCG64(seed)):
  * frames are H x W images vectorised row-major (pixel y*W + x); m = H*W and the
    n frames are the columns of A (column-major storage, Section 1);
  * background L = U V^T / sqrt(rho) scaled per frame by a gain g_j, with U (m x rho)
    and V (n x rho) i.i.d. N(0,1) (optional slow drift g_j = 1 + a sin(2 pi j / n));
  * foreground objects (axis-aligned squares, optionally discs) of side 6/40 of the
    frame width, random start and integer velocity, reflecting at the borders,
    values U[0.5, 1], replacing (occluding) the background pixels; they appear only
    in frames k..n-1 so the first k frames are background plus noise; the object
    count is the smallest whose measured coverage reaches the target fraction;
  * additive N(0, sigma^2) noise everywhere;
  * W1 (m x k) either a constant or i.i.d. U[lo, hi].
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = ["ClipSpec", "CONFIGS", "make_clip", "initial_x1", "batched_specs"]


@dataclass(frozen=True)
class ClipSpec:
    H: int
    W: int
    n: int
    k: int
    r: int
    rho: int = 3
    coverage: float = 0.04
    sigma: float = 0.01
    w_const: float | None = 20.0
    w_range: tuple = (5.0, 50.0)
    discs: bool = False
    drift: float = 0.0
    seed: int = 0

    @property
    def m(self) -> int:
        return self.H * self.W


# Workloads: 1 = small FP64 case, 2 = FP32 headline case, 3 = large mixed-precision
# case, 5 = the warm-start evaluation shape.  (4 is the batched set, batched_specs.)
CONFIGS = {
    1: ClipSpec(H=30, W=40, n=60, k=5, r=8, rho=3, coverage=0.04, sigma=0.01,
                w_const=20.0, seed=0),
    2: ClipSpec(H=120, W=160, n=400, k=20, r=25, rho=5, coverage=0.06, sigma=0.02,
                w_const=None, w_range=(5.0, 50.0), discs=True, seed=1),
    3: ClipSpec(H=240, W=320, n=1000, k=50, r=60, rho=8, coverage=0.08, sigma=0.02,
                w_const=None, w_range=(5.0, 50.0), discs=True, drift=0.2, seed=2),
    5: ClipSpec(H=240, W=320, n=600, k=30, r=40, rho=8, coverage=0.08, sigma=0.02,
                w_const=None, w_range=(5.0, 50.0), discs=True, drift=0.2, seed=200000),
}


def _object_masks(rng: np.random.Generator, spec: ClipSpec, n_obj: int) -> np.ndarray:
    """Boolean (n, H, W) occupancy and float (n, H, W) values for n_obj objects."""
    H, W, n = spec.H, spec.W, spec.n
    side = max(2, int(round(W * 6 / 40)))
    occ = np.zeros((n, H, W), dtype=bool)
    val = np.zeros((n, H, W), dtype=np.float64)
    yy, xx = np.mgrid[0:H, 0:W]
    for o in range(n_obj):
        y = int(rng.integers(0, max(1, H - side)))
        x = int(rng.integers(0, max(1, W - side)))
        vy = int(rng.integers(-2, 3))
        vx = int(rng.integers(1, 4)) * (1 if rng.random() < 0.5 else -1)
        level = rng.uniform(0.5, 1.0)
        is_disc = spec.discs and (o % 2 == 1)
        for j in range(spec.k, n):
            if is_disc:
                c = (side - 1) / 2.0
                shape = (yy - (y + c)) ** 2 + (xx - (x + c)) ** 2 <= (side / 2.0) ** 2
            else:
                shape = (yy >= y) & (yy < y + side) & (xx >= x) & (xx < x + side)
            occ[j] |= shape
            val[j][shape] = level
            # integer velocity, reflecting at the borders
            ny, nx = y + vy, x + vx
            if ny < 0 or ny > H - side:
                vy = -vy
                ny = y + vy
            if nx < 0 or nx > W - side:
                vx = -vx
                nx = x + vx
            y = min(max(ny, 0), max(0, H - side))
            x = min(max(nx, 0), max(0, W - side))
    return occ, val


def make_clip(spec: ClipSpec, seed: int | None = None, dtype=np.float64) -> dict:
    """Draw one clip.  Returns a dict with A (m x n, Fortran order), W1 (m x k,
    Fortran order), the foreground mask (m x n), the measured coverage of the
    frames k..n-1, and the spec."""
    seed = spec.seed if seed is None else seed
    rng = np.random.Generator(np.random.PCG64(seed))
    m, n, k, rho = spec.m, spec.n, spec.k, spec.rho
    U = rng.standard_normal((m, rho))
    V = rng.standard_normal((n, rho))
    j = np.arange(n)
    gain = 1.0 + spec.drift * np.sin(2.0 * np.pi * j / n)
    L = (U @ V.T) / math.sqrt(rho) * gain[None, :]

    # object count: smallest whose measured coverage reaches the target
    area = max(2, int(round(spec.W * 6 / 40))) ** 2
    n_obj = max(1, int(round(spec.coverage * m / area)))
    state = rng.bit_generator.state
    best = None
    for trial in range(n_obj, n_obj + 64):
        rng.bit_generator.state = state
        occ, val = _object_masks(rng, spec, trial)
        cov = float(occ[k:].mean()) if n > k else 0.0
        best = (occ, val, cov, trial)
        if cov >= spec.coverage - 0.01:
            break
    occ, val, cov, n_obj = best
    mask = occ.reshape(n, m).T            # m x n, pixel index y*W + x
    fg = val.reshape(n, m).T
    A = np.where(mask, fg, L)
    A = A + spec.sigma * rng.standard_normal((m, n))
    if spec.w_const is not None:
        W1 = np.full((m, k), float(spec.w_const))
    else:
        W1 = rng.uniform(spec.w_range[0], spec.w_range[1], size=(m, k))
    return {
        "A": np.asfortranarray(A.astype(dtype)),
        "W1": np.asfortranarray(W1.astype(dtype)),
        "mask": mask,
        "coverage": cov,
        "n_objects": n_obj,
        "spec": spec,
    }


def initial_x1(m: int, k: int, seed: int, dtype=np.float64) -> np.ndarray:
    """An explicit i.i.d. N(0,1) initial X1 (m x k, Fortran order) drawn from
    PCG64(seed + 7919); passed to both the oracle and the CUDA path."""
    rng = np.random.Generator(np.random.PCG64(seed + 7919))
    return np.asfortranarray(rng.standard_normal((m, k)).astype(dtype))


def batched_specs(count: int = 96, base_seed: int = 1000) -> list:
    """The uneven batched workload: m in {4800, 19200, 76800}, n ~ U[100, 800],
    k ~ U[5, 40], r = k + U[3, 10], generator as in the small case, seed
    base_seed + clip index."""
    shapes = [(60, 80), (120, 160), (240, 320)]
    rng = np.random.Generator(np.random.PCG64(base_seed))
    out = []
    for c in range(count):
        H, W = shapes[int(rng.integers(0, 3))]
        n = int(rng.integers(100, 801))
        k = int(rng.integers(5, 41))
        r = k + int(rng.integers(3, 11))
        out.append(ClipSpec(H=H, W=W, n=n, k=k, r=r, rho=3, coverage=0.04, sigma=0.01,
                            w_const=20.0, seed=base_seed + c))
    return out
