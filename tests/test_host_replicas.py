"""Replica (multi-GPU) host logic of bench.py on CPU: two gloo ranks.  Each rank works on
its own right-hand sides (distinct seeds, distinct vectors) and the job time is the
slowest rank's; no data-path collective is involved."""
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


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    from synth import random_probe
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench._max_over_ranks(dist, 1.0 + rank)  # rank r "took" 1 + r seconds
    x1, x2 = random_probe(2, 1, 2, seed=bench.replica_seed(rank), nrhs=2)
    out.put((rank, t, float(np.abs(x2).sum())))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_replicas():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0][1] == res[1][1] == 2.0     # max over ranks
    assert res[0][2] != res[1][2]            # disjoint right-hand sides
