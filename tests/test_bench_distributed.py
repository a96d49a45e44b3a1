"""The multi-rank path of bench.py on CPU with two gloo ranks (no GPU involved).

bench.py runs one independent replica per rank (the lattice is not sharded): the job
time is the maximum over ranks, the job throughput counts every replica's nodes, and
under torchrun only rank 0 prints the reference arm's line.
"""
import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    t = bench.max_over_ranks(1.0 + rank, dist)  # rank 1 is the slower replica
    dist.barrier()

    class A:
        steps, warmup, gpus = 2, 1, world

    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(A)
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, t, buf.getvalue()))


def test_two_gloo_ranks_take_the_slowest_time_and_rank0_reports():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, t0, out0), (r1, t1, out1) = res
    assert t0 == t1 == 2.0
    assert out1.strip() == ""  # only rank 0 prints
    line = json.loads(out0.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "MLUPS" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"


def test_job_throughput_counts_every_replica():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.job_mlups(4, 256 ** 3, 1000, 2.0) == pytest.approx(4 * 256 ** 3 * 1000 / 2.0 / 1e6)
    assert bench.max_over_ranks(3.5) == 3.5
