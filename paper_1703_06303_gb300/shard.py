"""Row partition and exchange layout of a row-sharded sWLR iteration (host logic only).

Every per-row step of Algorithm 1 (Section 3: the E_p rows and the m independent row
updates, the weighted objective term) touches only its own pixel row, and every cross-row
quantity is a sum over rows.  So G ranks can each own a contiguous block of rows of A, W1
and X1 and exchange only summed partials:

  once per clip      K = A2^T A2 (n2 x n2) and ||A2||_F^2
  per iteration   1: S1 = X1^T X1 (k x k) -> R1 (first CholeskyQR factor)
                  2: Q1^T [Q1 A2] (k x (k + n2)) -> R2, B = Q^T A2, C = R^{-1} B
                  3: the two objective terms of F_p (scalars; they can travel with the
                     next iteration's exchange 1)

Everything between the exchanges (the factors R1, R2, C, the rank-(r-k) eigensolve of
K - B^T B) is formed redundantly on every rank from the same sums.  This module fixes the
partition (whole 64-row blocks, the row pass's block height, so that no row block of a
kernel straddles two ranks) and the flat float64 layout of each exchange buffer; the
sharding identity (summed partials reproduce the unsharded step) is pinned on CPU ranks.
"""
from __future__ import annotations

import numpy as np

ROW_BLOCK = 64

__all__ = ["ROW_BLOCK", "row_ranges", "exchange_sizes", "exchange_bytes_per_iteration",
           "pack", "unpack"]


def row_ranges(m: int, world: int, align: int = ROW_BLOCK):
    """Contiguous [r0, r1) row blocks for ranks 0..world-1: every boundary is a multiple
    of `align` (except m itself), the blocks cover 0..m without overlap, and their sizes
    differ by at most one `align` block."""
    if m < 0 or world < 1 or align < 1:
        raise ValueError("need m >= 0, world >= 1, align >= 1")
    nblk = -(-m // align)
    base, extra = divmod(nblk, world)
    out, b = [], 0
    for rank in range(world):
        nb = base + (1 if rank < extra else 0)
        r0, r1 = min(m, b * align), min(m, (b + nb) * align)
        out.append((r0, r1))
        b += nb
    return out


def exchange_sizes(n: int, k: int):
    """Float64 element counts of the three per-iteration exchanges and the setup one."""
    n2 = n - k
    return {"setup": n2 * n2 + 1, "x1_gram": k * k + 2, "coef": k * (k + n2)}


def exchange_bytes_per_iteration(n: int, k: int) -> int:
    """Bytes each rank contributes to the per-iteration all-reduces (exchanges 1 and 2,
    the objective scalars riding with exchange 1)."""
    e = exchange_sizes(n, k)
    return 8 * (e["x1_gram"] + e["coef"])


def pack(*parts) -> np.ndarray:
    """Flat float64 buffer of the given arrays / scalars, in order (column-major)."""
    return np.concatenate([np.asarray(p, dtype=np.float64).reshape(-1, order="F") for p in parts])


def unpack(buf: np.ndarray, *shapes):
    """Inverse of pack: arrays of the given shapes (() for a scalar), in order."""
    out, off = [], 0
    for sh in shapes:
        n = int(np.prod(sh)) if len(sh) else 1
        v = np.asarray(buf[off:off + n], dtype=np.float64)
        out.append(float(v[0]) if len(sh) == 0 else v.reshape(sh, order="F"))
        off += n
    if off != len(buf):
        raise ValueError("buffer size does not match the shapes")
    return out
