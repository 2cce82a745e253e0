"""Multi-rank host logic of bench.py on CPU (gloo, world size 2).

The bench runs one independent replica per rank (the mesh is not
partitioned): the job's step time is the maximum over ranks and the value
sums every rank's work.  The reference arm prints from rank 0 only.
"""
import json
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = bench.job_step_ms(1.5 + rank, world, "cpu")
    q.put((rank, ms, bench.job_value(world, 1000, 10, ms)))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_step_time_is_max_over_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [2.5, 2.5]                 # slowest replica
    assert out[0][2] == pytest.approx(2 * 1000 * 10 / 2.5e-3 / 1e9)


def test_single_rank_passthrough_and_value():
    import bench
    assert bench.job_step_ms(3.0, 1, "cpu") == 3.0
    assert bench.job_value(1, 933120, 313, 8.0) == pytest.approx(933120 * 313 / 8e-3 / 1e9)


def test_reference_arm_prints_on_rank_zero_only(capsys):
    import argparse
    import bench
    args = argparse.Namespace(gpus=2, steps=1, warmup=0)
    bench.run_reference(args, 1)
    assert capsys.readouterr().out == ""


def test_reference_arm_line_on_rank_zero(capsys):
    import argparse
    import bench
    args = argparse.Namespace(gpus=1, steps=1, warmup=0)
    bench.run_reference(args, 0)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "cpu_baseline", "e2e", "config"):
        assert key in line
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
