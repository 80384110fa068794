"""The benchmark's N > 1 path on CPU ranks (gloo, world size 2): replicas
only, one independent system per rank (replica index = rank), the job's time
is the slowest rank's, and the whole-job value counts every rank's
particles.  No GPU and no data-path collective are involved."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp

import bench
import oracle


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 10.0 * (rank + 1)                  # rank 1 is the slower one
    total = bench.max_over_ranks(dist, local_ms, "cpu")
    # each rank steps its own replica: the oracle's RBM-1 step with replica = rank
    n = 64
    prm = oracle.make_params(n, 2, p=2, dt=1e-2, sigma=0.1, k="gauss_agg", seed=5, replica=rank)
    X = oracle.rbm_step(prm, np.zeros((n, 2)), 0)
    out[rank] = (total, bench.weak_value(world, n, 10, total), float(X.sum()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_replicas_only():
    world = 2
    port = _free_port()
    manager = mp.Manager()
    out = manager.dict()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    (t0, v0, s0), (t1, v1, s1) = out[0], out[1]
    assert t0 == t1 == 20.0                       # the slowest rank's time on every rank
    assert v0 == v1 == world * 64 * 10 / 20e-3    # every rank's particles, the job's time
    assert s0 != s1                               # independent replicas (replica index in the counters)
