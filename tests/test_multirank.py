"""The multi-GPU path of bench.py on CPU ranks (gloo, world size 2): every
rank solves its own replica, and the reported figures are the whole job's,
i.e. the maximum time over ranks and the sum of the work units over ranks,
with a barrier on both sides of the timed region.  The reference arm runs on
rank 0 only.  No GPU and no data-path collective are involved."""
import argparse
import contextlib
import io
import json
import os
import socket

import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=2)
    try:
        # rank r: times (10 + 5r, 3 + 3r) ms, counts (100 + r, 7)
        bench.rank_barrier(2)
        times, counts = bench.reduce_over_ranks(2, "cpu", [10.0 + 5 * rank, 3.0 * (rank + 1)], [100 + rank, 7])
        bench.rank_barrier(2)
        with open(f"{out}.{rank}", "w") as f:
            json.dump({"t": times, "c": counts}, f)
    finally:
        dist.destroy_process_group()


def test_reduce_over_ranks_gloo_world2(tmp_path):
    mp.spawn(_worker, args=(_free_port(), str(tmp_path / "r")), nprocs=2, join=True)
    for rank in range(2):
        d = json.load(open(tmp_path / f"r.{rank}"))
        assert d["t"] == [15.0, 6.0]        # max over ranks
        assert d["c"] == [201.0, 14.0]      # sum over ranks


def test_single_rank_is_identity():
    assert bench.reduce_over_ranks(1, "cpu", [4.5, 1.0], [3, 2]) == ([4.5, 1.0], [3.0, 2.0])


def test_reference_arm_runs_on_rank0_only():
    args = argparse.Namespace(cpu_iters=2, warmup=1, steps=1, mass_div=None)
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(args, rank=1, world=2)
    assert buf.getvalue() == ""
