"""The N>1 path of bench.py on the CPU: world size 2 over gloo. Each rank runs its own replica
(its own seeded field; no data exchange), the job time is the max over ranks and the job
throughput the sum of points over that time."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    sys.path.insert(0, os.path.join(root, "tests"))
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import oracle
    from paper_2306_13002_gb300 import inputs
    n = 6
    U = inputs.rhs_field(n, halo=2, seed=inputs.SEED_RHS_LARGE + rank)     # the bench's per-rank seed
    R = oracle.rhs(U)
    elapsed = 1.0 + rank                                                   # stand-in per-rank times
    job_ms = bench.reduce_over_ranks(dist, elapsed, "max", "cpu")
    pts = bench.reduce_over_ranks(dist, float(n ** 3), "sum", "cpu")
    q.put((rank, job_ms, pts, float(np.sum(R))))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replicas_aggregate_without_data_exchange():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [2.0, 2.0]            # max over ranks
    assert [r[2] for r in res] == [2 * 216.0] * 2       # points of both replicas
    assert res[0][3] != res[1][3]                       # independent replicas


def test_reduce_is_identity_without_process_group():
    import bench
    assert bench.reduce_over_ranks(None, 3.5, "max", "cpu") == 3.5
