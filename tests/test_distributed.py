"""The N > 1 path of bench.py on CPU with two gloo ranks: every rank runs an
independent replica (no data-path collective); the timing is the maximum
over ranks, the barrier holds the ranks together, and under torchrun only
rank 0 runs and prints the reference arm."""
import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    ws, r, local = bench.dist_env()
    assert (ws, r, local) == (world, rank, rank)
    bench.init_dist(ws, "gloo")
    # the step time of the job is the slowest rank's
    got = bench.max_over_ranks(10.0 + rank * 5.0, ws)
    bench.barrier(ws)
    # the reference arm: rank 0 alone prints, the others return without work
    args = type("A", (), dict(workload="er4096", steps=1, warmup=0, gpus=world))()
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(args)
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"max": got, "out": buf.getvalue()}, f)
    dist.destroy_process_group()


def test_two_ranks_gloo(tmp_path):
    world = 2
    port = _free_port()
    mp.start_processes(_worker, args=(world, port, str(tmp_path)), nprocs=world, join=True, start_method="spawn")
    r0 = json.load(open(tmp_path / "rank0.json"))
    r1 = json.load(open(tmp_path / "rank1.json"))
    assert r0["max"] == r1["max"] == 15.0
    assert r1["out"] == ""
    line = json.loads(r0["out"].strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == world
    assert line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
