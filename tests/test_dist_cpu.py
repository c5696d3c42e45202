"""The multi-process (torchrun) path of bench.py on CPU with gloo, world size 2.

Each rank multiplies its own matrix (weak scaling, no data-path collective);
the job's time is the maximum over ranks and the job's rate counts the units
of every rank. The products here run on the CPU oracle, so only the host
logic of the N > 1 path is exercised.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist

    import bench
    import h2gen
    import oracle

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    cfg = bench.replica_config("2d_n4096", rank)
    A = h2gen.generate(**cfg)
    x = h2gen.vectors(77 + rank, A.n, 1)
    y = oracle.matvec(A, x)
    local = 1.0 + rank  # a stand-in time that differs per rank
    job = bench.max_over_ranks(local, dist, "cpu")
    ys = [torch.zeros(A.n, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(ys, torch.from_numpy(np.ascontiguousarray(y[:, 0])))
    if rank == 0:  # small results only: the parent reads them before joining
        out.put((cfg["seed"], job, bench.job_rate(10.0, world, job), float(np.linalg.norm(ys[0] - ys[1]))))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_replicas_and_max_time():
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.SimpleQueue()
    port = _free_port()
    procs = [mp.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    seed0, job, rate, diff = q.get()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    assert job == 2.0                       # the slowest rank's time
    assert rate == pytest.approx(10.0 * 2 / 2.0)
    assert diff > 1.0                       # independent matrices per rank
