"""The N>1 path of bench.py on the CPU: world size 2 over gloo. Each rank runs its own replica
(its own seeded field, real work: the oracle's RHS), timed by the bench's own replica helpers;
the job time is the max over ranks and the job throughput the points of all ranks over that
time. No data is exchanged. Also: how bench.py decides to run, relaunch itself under
torchrun, or refuse, from --gpus and WORLD_SIZE."""
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
    n = 10 + 6 * rank                                                      # uneven replicas
    U = inputs.rhs_field(n, halo=2, seed=inputs.SEED_RHS_LARGE + rank)     # the bench's per-rank seed
    out = {}

    def step():
        out["R"] = oracle.rhs(U, threads=1)

    steps = 3
    local_ms = bench.timed_replica_region(dist, step, steps, bench.wall_timer)
    ms, value, pts = bench.replica_throughput(dist, local_ms, steps, n ** 3, "cpu")
    q.put((rank, local_ms, ms, value, pts, float(np.sum(out["R"]))))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replicas_aggregate_without_data_exchange():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    local = [r[1] for r in res]
    assert all(t > 0 for t in local)
    job_ms = max(local) / 3
    assert [r[2] for r in res] == pytest.approx([job_ms, job_ms])            # max over ranks, per step
    pts = 10 ** 3 + 16 ** 3
    assert [r[4] for r in res] == [pts, pts]                                 # points of both replicas
    assert [r[3] for r in res] == pytest.approx([pts / (job_ms * 1e-3) / 1e9] * 2)
    assert res[0][5] != res[1][5]                                            # independent replicas


def test_reduce_is_identity_without_process_group():
    import bench
    assert bench.reduce_over_ranks(None, 3.5, "max", "cpu") == 3.5
    ms, value, pts = bench.replica_throughput(None, 30.0, 3, 1e6, "cpu")
    assert (ms, pts) == (10.0, 1e6) and value == pytest.approx(0.1)


def test_launch_plan_never_measures_fewer_replicas_than_asked():
    import bench
    assert bench.launch_plan(1, {}) == "run"
    assert bench.launch_plan(4, {}) == "relaunch"
    assert bench.launch_plan(4, {"WORLD_SIZE": "4"}) == "run"
    assert bench.launch_plan(8, {"WORLD_SIZE": "1"}).startswith("error")
    assert bench.launch_plan(1, {"WORLD_SIZE": "2"}).startswith("error")
