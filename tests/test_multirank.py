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


def test_reference_arm_json_line(tmp_path):
    """`bench.py --impl reference` (the FP64 oracle on the host cores) prints
    one JSON line with the contract's keys, on the grid workload's metric,
    unit and config, with the CPU baseline and an end-to-end figure equal to
    its own value and no host-device traffic."""
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "1"],
                         cwd=root, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["metric"] == "sinkhorn_iters_per_s" and d["unit"] == "iters/s"
    assert d["higher_is_better"] is True and d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 1
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["config"]["workload"].startswith("grid2d-256x256")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
