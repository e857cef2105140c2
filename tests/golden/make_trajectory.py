"""Write the FP64 oracle's objective trajectory for one synthetic workload.

Calls only the oracle and the seeded input generator.  Output: a JSON fixture with
F_p = F(X1_p, C_p, D_p) for every iteration p of Algorithm 1 started from X1_0 = A1,
used as an independent reference for the best-known objective F* of that clip.

usage: python tests/golden/make_trajectory.py CONFIG ITERS OUT.json
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_1703_06303_gb300 import synth  # noqa: E402


def main():
    cfg, iters, out = int(sys.argv[1]), int(sys.argv[2]), sys.argv[3]
    spec = synth.CONFIGS[cfg]
    clip = synth.make_clip(spec)
    # the float32-rounded data, which is what the FP32 GPU path sees
    A = clip["A"].astype(np.float32).astype(np.float64)
    W1 = clip["W1"].astype(np.float32).astype(np.float64)
    t0 = time.time()
    res = oracle.swlr(A, W1, spec.r, A[:, :spec.k].copy(), max_iter=iters, stop="none")
    doc = {
        "what": "FP64 oracle trajectory of Algorithm 1 (sWLR), X1_0 = A1, float32-rounded A and W1",
        "config": {"H": spec.H, "W": spec.W, "n": spec.n, "k": spec.k, "r": spec.r, "seed": spec.seed},
        "iterations": res.iters,
        "F": res.F,
        "rel_error": res.rel_error,
        "seconds_per_iteration": (time.time() - t0) / max(iters, 1),
    }
    with open(out, "w") as f:
        json.dump(doc, f)


if __name__ == "__main__":
    main()
