"""The bench's multi-GPU path on CPU: two `gloo` ranks (replicas only).

`bench.py --gpus N` under torchrun runs one independent replica per GPU; the
only collective is the final combination of the per-rank figures: the
slowest rank's times (MAX) and all ranks' commits (SUM).  Here two CPU
processes run exactly that combination with the gloo backend.
"""
import json
import os
import socket
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        # per-rank figures as bench_ours returns them: ms of the timed steps,
        # e2e seconds, commits of the timed steps, e2e commits
        ms = 20.0 + 5.0 * rank
        e2e_s = 0.5 + 0.25 * rank
        committed = 4_000_000 * (rank + 1) + 3
        e2e_commit = 1_000_000 * (rank + 1)
        dist.barrier()
        got = bench.combine_ranks(torch, dist, "cpu", ms, e2e_s, committed, e2e_commit)
        if rank == 0:
            with open(out, "w") as f:
                json.dump(got, f)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_combine_like_the_bench(tmp_path):
    out = str(tmp_path / "combined.json")
    mp.start_processes(_rank, args=(2, _free_port(), out), nprocs=2, join=True,
                       start_method="spawn")
    ms, e2e_s, committed, e2e_commit = json.load(open(out))
    assert ms == 25.0 and e2e_s == 0.75                 # slowest rank
    assert committed == 4_000_003 + 8_000_003          # all ranks' commits
    assert e2e_commit == 3_000_000
    # value = whole-job commits / slowest rank's time
    assert abs(committed / (ms * 1e-3) - 12_000_006 / 0.025) < 1e-6
