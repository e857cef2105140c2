"""Sharding identity of the row-sharded iteration (no GPU): two gloo ranks each own a
block of pixel rows, all-reduce the summed partials (K and ||A2||^2 once; X1^T X1 and
Q1^T [Q1 A2] per iteration; the objective terms), form C and V_s redundantly and update
their own rows.  The gathered result must equal the unsharded FP64 oracle step (Householder
QR and a dense SVD) to 1e-10, over several iterations.  Unmeasured on hardware: every run
of this build has one GPU."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_1703_06303_gb300 import shard  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    from paper_1703_06303_gb300 import synth
    spec = synth.ClipSpec(H=20, W=30, n=40, k=5, r=9, rho=3, coverage=0.04, sigma=0.01,
                          w_const=None, w_range=(5.0, 50.0), seed=21)
    clip = synth.make_clip(spec)
    return clip["A"], clip["W1"], spec.k, spec.r


ITERS = 3


def _allreduce(x):
    t = torch.from_numpy(np.ascontiguousarray(x))
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t.numpy()


def _rank_main(rank, world, port, out_dir):
    from oracle import sharded
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    A, W1, k, r = _problem()
    m, n = A.shape
    n2, s = n - k, r - k
    r0, r1 = shard.row_ranges(m, world)[rank]
    Ar, Wr = A[r0:r1], W1[r0:r1]
    X = Ar[:, :k].copy()                                  # X1_0 = A1 (this rank's rows)
    Kp, a2p = sharded.setup_partials(Ar, k)
    K, _a2 = shard.unpack(_allreduce(shard.pack(Kp, a2p)), (n2, n2), ())
    Fs, Xs = [], []
    for _ in range(ITERS):
        S1 = shard.unpack(_allreduce(shard.pack(sharded.gram_x1(X))), (k, k))[0]
        R1 = sharded.qr_factor(S1)
        Qa = shard.unpack(_allreduce(shard.pack(sharded.coef_partials(Ar, X, R1, k))), (k, k + n2))[0]
        C, Vs, _ = sharded.global_factors(R1, Qa, K, s)
        Xn, wt, rt = sharded.rows_update(Ar, Wr, X, C, Vs)
        F = float(_allreduce(np.array([wt + rt]))[0])
        Fs.append(F)
        X = Xn
        Xs.append(X)
    np.savez(os.path.join(out_dir, f"rank{rank}.npz"), r0=r0, r1=r1, F=np.array(Fs),
             X=np.stack(Xs), C=C)
    dist.barrier()
    dist.destroy_process_group()


def test_row_ranges_cover_aligned_and_balanced():
    for m in (0, 1, 63, 64, 65, 1200, 19200, 76801):
        for world in (1, 2, 3, 4, 8):
            rr = shard.row_ranges(m, world)
            assert len(rr) == world
            assert rr[0][0] == 0 and rr[-1][1] == m
            for (a0, a1), (b0, b1) in zip(rr, rr[1:]):
                assert a1 == b0
            for r0, r1 in rr:
                assert r0 <= r1
                assert r0 == m or r0 % shard.ROW_BLOCK == 0    # empty trailing ranks sit at m
                assert r1 == m or r1 % shard.ROW_BLOCK == 0
            blocks = [-(-(r1 - r0) // shard.ROW_BLOCK) for r0, r1 in rr]
            assert max(blocks) - min(blocks) <= 1


def test_pack_roundtrip_and_exchange_size():
    rng = np.random.default_rng(0)
    a, b = rng.standard_normal((3, 4)), rng.standard_normal((2, 5))
    a2, c, b2 = shard.unpack(shard.pack(a, 7.5, b), (3, 4), (), (2, 5))
    assert np.array_equal(a, a2) and np.array_equal(b, b2) and c == 7.5
    with pytest.raises(ValueError):
        shard.unpack(shard.pack(a), (2, 2))
    # 320x240 clip, n = 1000, k = 50: about 0.42 MB per rank per iteration
    assert shard.exchange_bytes_per_iteration(1000, 50) == 8 * (50 * 50 + 2 + 50 * 1000)


def test_two_gloo_ranks_reproduce_the_unsharded_oracle_step(tmp_path):
    import oracle
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    A, W1, k, r = _problem()
    m = A.shape[0]
    parts = [np.load(tmp_path / f"rank{q}.npz") for q in range(2)]
    assert parts[0]["r1"] == parts[1]["r0"] and parts[1]["r1"] == m
    assert 0 < int(parts[0]["r1"]) < m                   # both ranks hold rows
    X = A[:, :k].copy()
    for it in range(ITERS):
        st = oracle.swlr_step(A, W1, X, r)
        Xg = np.vstack([p["X"][it] for p in parts])
        assert np.abs(Xg - st.X1_next).max() <= 1e-10 * np.abs(st.X1_next).max(), it
        for p in parts:
            assert abs(p["F"][it] - st.F) <= 1e-10 * st.F, (it, p["F"][it], st.F)
        X = st.X1_next
    assert np.abs(parts[0]["C"] - parts[1]["C"]).max() == 0.0   # same sums, same factors
    assert np.abs(parts[0]["C"] - st.cd.C).max() <= 1e-10 * np.abs(st.cd.C).max()
