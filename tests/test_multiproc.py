"""Multi-GPU is replicas only (queries are independent; a single query would
need two exchanges per round).  The rank logic of bench.py -- every rank
solves its own queries, the job's throughput is the edges of all ranks over
the slowest rank's time -- runs here as world-size-2 gloo processes on the
CPU, each rank solving with the oracle."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    import graphgen as gg
    import oracle

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # Each rank: its own sources on the same graph (a replica).
        g = gg.random_graph(2000, 6, 1, 50, 3)
        edges = 0
        for s in range(rank, 8, world):
            edges += oracle.round_r(g, s).stats["out_scanned"]
        local_ms = 10.0 * (rank + 1)            # rank 1 is the slower one
        ms, units = bench.reduce_over_ranks(dist, "cpu", local_ms, edges)
        out[rank] = (ms, units, edges)
    finally:
        dist.destroy_process_group()


def test_replica_reduction_two_ranks():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world,
                       start_method="spawn", join=True)
    ms0, units0, e0 = out[0]
    ms1, units1, e1 = out[1]
    assert ms0 == ms1 == 20.0                    # slowest rank's time
    assert units0 == units1 == e0 + e1           # all ranks' work
    assert e0 > 0 and e1 > 0


def test_single_process_reduction_is_identity():
    import bench
    assert bench.reduce_over_ranks(None, "cpu", 3.5, 17) == (3.5, 17)
