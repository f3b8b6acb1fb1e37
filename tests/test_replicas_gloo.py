"""The N > 1 path of bench.py on CPU: two gloo ranks as replicas.

Replicas solve independent problems; the only collective is the MAX of the
timed-region lengths after the timed region, and the whole-job throughput is the
solves of all ranks over the slowest rank's time.  The reference arm under
torchrun runs on rank 0 only; other ranks return without work.
"""
import contextlib
import io
import json
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local = [1.5, 2.5][rank]
        total, value = bench.replica_throughput(local, steps=4, world=world, device="cpu")
        dist.barrier()
        buf = io.StringIO()
        with contextlib.redirect_stdout(buf):
            if rank != 0:  # rank 0 would run the oracle; only the non-zero ranks' no-op is checked here
                bench.run_reference(None, rank, world)
        with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
            json.dump({"total": total, "value": value, "ref_out": buf.getvalue()}, f)
    finally:
        dist.destroy_process_group()


def test_two_replicas_max_time_and_aggregate_throughput(tmp_path):
    world = 2
    mp.spawn(_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / f"r{r}.json")) for r in range(world)]
    for r in res:
        assert r["total"] == pytest.approx(2.5)          # the slowest rank's time on every rank
        assert r["value"] == pytest.approx(4 * 2 / 2.5)  # solves of all ranks / whole-job time
    assert res[1]["ref_out"] == ""


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    total, value = bench.replica_throughput(2.0, steps=5, world=1)
    assert total == 2.0 and value == 2.5
