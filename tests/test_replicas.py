"""Host logic of the multi-process path (bench.py under torchrun): independent replicas,
one clip per rank, the step time taken as the maximum over ranks, and a reference arm that
only rank 0 runs.  Two gloo ranks on the CPU; no GPU."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import bench
    from paper_1703_06303_gb300 import synth
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    local = 10.0 + 3.5 * rank                      # each rank's own step time
    t = bench.max_over_ranks(local, torch.device("cpu"))
    spec = synth.CONFIGS[1]
    clip = synth.make_clip(spec, seed=bench.replica_seed(spec.seed, rank))
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"max": t, "a00": float(clip["A"][0, 0]), "asum": float(clip["A"].sum())}, f)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_distinct_clips(tmp_path):
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    r0 = json.load(open(tmp_path / "r0.json"))
    r1 = json.load(open(tmp_path / "r1.json"))
    assert r0["max"] == r1["max"] == 13.5
    assert r0["asum"] != r1["asum"]               # each rank solves its own clip


def test_replica_seed_rank0_is_the_single_gpu_clip():
    import bench
    from paper_1703_06303_gb300 import synth
    spec = synth.CONFIGS[2]
    assert bench.replica_seed(spec.seed, 0) == spec.seed
    assert len({bench.replica_seed(spec.seed, r) for r in range(8)}) == 8


def test_reference_arm_other_ranks_exit_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1", CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2"],
                       capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
