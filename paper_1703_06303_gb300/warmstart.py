"""Training and evaluation of the learned warm start (host orchestration only: every step
runs in libwlr.so's kernels, through the wlr_ws_* and wlr_* entry points of include/wlr.h).

Algorithm 1 starts from an initial X1 ("Initialize (X1)_0"; Section 4.1 uses a random
matrix).  The network predicts frame-mixing weights Omega from a downsampled clip and its
weights; the basis U = [A1 | 0] + A Omega(:, 1:r) / n then gives X1_0 as the weighted
projection of A1 onto span(U).  It is trained on solutions that the method itself computes:

  * clips: the seeded synthetic video generator (synth.py), 30 x 40-pixel frames (the
    network's input size, so f = 1), n ~ U[40, 100] frames, k ~ U[3, 12], r = k + U[2, 8],
    background rank 2..4, 3..8% foreground, noise 0.005..0.02, W1 ~ U[5, 50] per entry;
  * "converged solution": the iterate after `target_iters` FP32 iterations of Algorithm 1
    from X1_0 = A1 (all clips of a group advanced together by wlr_solve_batched); its
    target is the orthonormal basis of span(X1, X1 C + D) (wlr_get_basis);
  * loss: ||P_Y - P_V||_F^2 / (2r) per clip, averaged over a minibatch, Adam.

Evaluation counts the iterations Algorithm 1 needs to reach a relative objective of
`target` (F_p - F*) / F* from X1_0 = A1 and from the learned X1_0 on held-out clips, in
FP64 (the FP32 rounding floor of these small clips lies near 1e-6), with F* the lowest
objective either run reaches.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass

import numpy as np

from . import synth, wlr

FRAME_H, FRAME_W = 30, 40


def family_spec(seed: int) -> synth.ClipSpec:
    """One clip of the training / evaluation family (all draws from the seed)."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(40, 101))
    k = int(rng.integers(3, 13))
    r = k + int(rng.integers(2, 9))
    return synth.ClipSpec(H=FRAME_H, W=FRAME_W, n=n, k=k, r=r, rho=int(rng.integers(2, 5)),
                          coverage=float(rng.uniform(0.03, 0.08)), sigma=float(rng.uniform(0.005, 0.02)),
                          w_const=None, w_range=(5.0, 50.0), discs=bool(seed % 2), seed=seed)


@dataclass
class ClipData:
    spec: synth.ClipSpec
    A: object      # m x n float32 CUDA tensor (column-major)
    W1: object     # m x k
    X: object      # (n, 2, h, w) network input
    V: object      # m x r target basis (None for evaluation clips)


def _col(a, dev):
    import torch
    return torch.from_numpy(np.asfortranarray(a)).to(dev)


def load_clips(specs, net, dev):
    """Upload the clips and prepare the network inputs (no targets)."""
    import torch
    out = []
    for sp in specs:
        c = synth.make_clip(sp)
        tA = _col(c["A"].astype(np.float32), dev)
        tW = _col(c["W1"].astype(np.float32), dev)
        X = torch.empty((sp.n, 2, net.h, net.w), dtype=torch.float32, device=dev)
        net.prepare(tA, tW, sp.H, sp.W, sp.k, X)
        out.append(ClipData(sp, tA, tW, X, None))
    return out


def solve_targets(clips, target_iters: int, group: int = 96, stream=None):
    """Target bases: each clip solved from X1_0 = A1 for target_iters FP32 iterations
    (groups of `group` clips advanced together), then V = basis of span(X1, X1 C + D)."""
    import torch
    for g0 in range(0, len(clips), group):
        part = clips[g0:g0 + group]
        hs = []
        for c in part:
            sp = c.spec
            s = wlr.Solver(sp.m, sp.n, sp.k, sp.r, precision=wlr.WLR_PREC_FP32, stop=wlr.WLR_STOP_NONE,
                           stream=stream)
            s.set_data(c.A, c.W1)
            s.set_init(wlr.WLR_INIT_A1)
            hs.append(s)
        wlr.solve_batched(hs, target_iters)
        for c, s in zip(part, hs):
            V = torch.empty((c.spec.r, c.spec.m), dtype=torch.float32, device=c.A.device).T
            s.basis(V)
            c.V = V
            s.close()
    return clips


def damp_output(net, factor: float = 0.1):
    """Scale the last layer's weights and bias (the flat layout's tail) by `factor`, so an
    untrained network starts close to X1_0 = A1 (the basis prior [A1 | 0])."""
    p = net.params()
    h, w, c1, c2, hidden, r_max = net.shape
    n_last = r_max * hidden + r_max
    p[-n_last:] *= factor
    net.set_params(p)


def _batch_frames(clips):
    import torch
    X = torch.cat([c.X for c in clips])
    starts = np.cumsum([0] + [c.spec.n for c in clips]).astype(np.int32)
    return X, starts


def batch_loss(net, clips, grad=True):
    """Mean loss of the clips (forward, per-clip loss; backward if grad).  Returns a float."""
    import torch
    X, starts = _batch_frames(clips)
    F = int(starts[-1])
    dev = X.device
    Om = torch.empty((F, net.r_max), dtype=torch.float32, device=dev)
    dOm = torch.empty((F, net.r_max), dtype=torch.float32, device=dev)
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    net.forward(X, starts, Om)
    for q, c in enumerate(clips):
        a, b = int(starts[q]), int(starts[q + 1])
        net.loss(c.A, c.spec.k, Om[a:b], c.spec.r, c.V, loss, dOm[a:b])
    if grad:
        net.backward(dOm)
    return loss.item() / len(clips)


def train(net, clips, steps: int, batch: int = 32, lr: float = 3e-4, seed: int = 0,
          val=None, log_every: int = 100, log=None):
    """Adam on random minibatches of `batch` clips, cosine learning rate from lr to lr/10.
    Returns the history [(step, train loss, validation loss or None)]."""
    rng = np.random.default_rng(seed)
    hist = []
    for t in range(steps):
        idx = rng.choice(len(clips), size=min(batch, len(clips)), replace=False)
        part = [clips[i] for i in idx]
        L = batch_loss(net, part, grad=True)
        lr_t = lr * (0.1 + 0.9 * 0.5 * (1 + math.cos(math.pi * t / max(steps - 1, 1))))
        net.adam(lr_t, grad_scale=1.0 / len(part))
        if (t + 1) % log_every == 0 or t == 0 or t == steps - 1:
            vl = None
            if val:
                vl = float(np.mean([batch_loss(net, val[i:i + batch], grad=False)
                                    for i in range(0, len(val), batch)]))
            hist.append((t + 1, L, vl))
            if log:
                log(f"step {t + 1} loss {L:.4f} val {vl}")
    return hist


def learned_x1(net, c, stream=None, fallback=False):
    """X1_0 of clip c from the network (through wlr_set_init_learned of a float handle),
    as a float64 host array, the seconds that call took and whether the network's start
    was kept (with fallback, the start with the lower FP64 objective among it and A1)."""
    import torch
    sp = c.spec
    s = wlr.Solver(sp.m, sp.n, sp.k, sp.r, precision=wlr.WLR_PREC_FP32, stop=wlr.WLR_STOP_NONE,
                   stream=stream)
    s.set_data(c.A, c.W1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    used = s.set_init_learned(net, sp.H, sp.W, fallback)
    dt = time.perf_counter() - t0
    X1 = np.zeros((sp.m, sp.k), order="F")
    s.result(X1)
    s.close()
    return X1, dt, used


def first_below(F, Fstar, target):
    rel = (np.asarray(F) - Fstar) / Fstar
    idx = np.nonzero(rel <= target)[0]
    return int(idx[0]) if idx.size else None


def evaluate(net, clips, iters: int, target: float = 1e-6, group: int = 48, stream=None,
             fallback=False):
    """Iterations of FP64 Algorithm 1 to reach (F_p - F*)/F* <= target from X1_0 = A1 and
    from the learned X1_0 (with fallback: the better of it and A1 by the FP64 objective),
    per clip.  F* = the lowest F_p of the two runs (iters each)."""
    import torch
    rows = []
    for g0 in range(0, len(clips), group):
        part = clips[g0:g0 + group]
        hs, inits = [], []
        for c in part:
            sp = c.spec
            A64 = c.A.double()
            W64 = c.W1.double()
            X1L, t_inf, used = learned_x1(net, c, stream, fallback)
            for arm in ("A1", "learned"):
                s = wlr.Solver(sp.m, sp.n, sp.k, sp.r, precision=wlr.WLR_PREC_FP64, stop=wlr.WLR_STOP_NONE,
                               eig_iters=4, stream=stream)
                s.set_data(A64, W64)
                if arm == "A1":
                    s.set_init(wlr.WLR_INIT_A1)
                else:
                    s.set_init(wlr.WLR_INIT_USER, X1L)
                s._keep = (A64, W64)
                hs.append(s)
            inits.append((t_inf, used))
        wlr.solve_batched(hs, iters)
        for q, c in enumerate(part):
            FA, _ = hs[2 * q].history()
            FL, _ = hs[2 * q + 1].history()
            Fstar = min(FA.min(), FL.min())
            rows.append({"seed": c.spec.seed, "m": c.spec.m, "n": c.spec.n, "k": c.spec.k, "r": c.spec.r,
                         "F_star": float(Fstar), "iters_A1": first_below(FA, Fstar, target),
                         "iters_learned": first_below(FL, Fstar, target),
                         "F0_rel_A1": float((FA[0] - Fstar) / Fstar), "F0_rel_learned": float((FL[0] - Fstar) / Fstar),
                         "end_gap": float(abs(FA[-1] - FL[-1]) / Fstar), "inference_s": inits[q][0],
                         "used_learned": bool(inits[q][1])})
        for s in hs:
            s.close()
    return rows


def summarize(rows, iters: int):
    """Median and mean iteration ratios (A1 / learned), counting a run that did not reach the
    target as `iters` iterations; clips whose two runs end in different minima are reported
    apart."""
    same = [r for r in rows if r["end_gap"] <= 1e-6]
    pa = np.array([r["iters_A1"] if r["iters_A1"] is not None else iters for r in same], dtype=float)
    pl = np.array([r["iters_learned"] if r["iters_learned"] is not None else iters for r in same], dtype=float)
    ratio = pa / np.maximum(pl, 1.0)
    return {"clips": len(rows), "same_limit": len(same),
            "iters_A1_mean": float(pa.mean()) if len(same) else None,
            "iters_learned_mean": float(pl.mean()) if len(same) else None,
            "total_iters_ratio": float(pa.sum() / max(pl.sum(), 1.0)) if len(same) else None,
            "median_ratio": float(np.median(ratio)) if len(same) else None,
            "learned_faster": int(np.sum(pl < pa)), "learned_slower": int(np.sum(pl > pa)),
            "F0_rel_A1_median": float(np.median([r["F0_rel_A1"] for r in rows])),
            "F0_rel_learned_median": float(np.median([r["F0_rel_learned"] for r in rows])),
            "inference_s_mean": float(np.mean([r["inference_s"] for r in rows])),
            "used_learned": int(sum(r.get("used_learned", True) for r in rows))}
