"""The N > 1 host path of bench.py, on two gloo ranks on the CPU.

With several GPUs, bench.py runs independent replicas: each rank solves its own
problem, seeded by its rank, with no exchange on the data path.  The only
collective is the maximum of the timings over the ranks, and the job's rate is
the units of all ranks divided by that maximum.  This runs that reduction and
that arithmetic as two real processes over gloo (127.0.0.1).
"""

import json
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, outdir):
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    import bench
    # per-rank timings: each entry's maximum sits on a different rank
    mine = [10.0 + rank, 20.0 - rank, 5.0 * (rank + 1)]
    got = bench.max_over_ranks(mine, dist, "cpu")
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(outdir, f"rank{rank}.json"), "w") as f:
        json.dump({"got": got, "seed": bench.replica_seed(rank)}, f)


def test_two_rank_max_and_rate(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    for r in res:
        assert r["got"] == [11.0, 20.0, 10.0]
    # replicas are independent problems
    assert res[0]["seed"] != res[1]["seed"]

    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench
    # 2 ranks x 100 steps in 0.5 s (the slower rank) = 400 steps/s for the job
    assert bench.job_rate(100, 500.0, world) == pytest.approx(400.0)
    assert bench.job_rate(100, 500.0, 1) == pytest.approx(200.0)


def test_single_process_passthrough():
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks((1.0, 2.0), None, "cpu") == [1.0, 2.0]


def test_replica_fields_differ():
    """Each rank's seed draws a different coefficient field of the same shape."""
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench
    import workloads as W
    a0 = W.lognormal_coefficient(W.grf(np.random.default_rng(bench.replica_seed(0)), 32, 2, 0.05), 1e4)
    a1 = W.lognormal_coefficient(W.grf(np.random.default_rng(bench.replica_seed(1)), 32, 2, 0.05), 1e4)
    assert a0.shape == a1.shape and not np.allclose(a0, a1)
