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


def _bench_line(cmd, env):
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable] + cmd, cwd=root, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    return json.loads(lines[0])


@pytest.mark.parametrize("launcher", ["self", "torchrun"])
def test_bench_launches_two_replica_ranks(launcher):
    """bench.py --gpus 2 sees two ranks whether it starts them itself or torchrun does: both
    ranks report with distinct replica seeds, the time is the max over ranks, and only rank 0
    prints (a CPU dry run that stops before the library)."""
    env = dict(os.environ, LRCC_BENCH_BACKEND="gloo")
    env.pop("WORLD_SIZE", None)
    args = ["bench.py", "--gpus", "2", "--steps", "1", "--warmup", "0", "--dry-run"]
    if launcher == "torchrun":
        args = ["-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
                "127.0.0.1", "--master-port", str(_free_port())] + args
    line = _bench_line(args, env)
    assert line["n_gpus"] == 2
    assert sorted(r[0] for r in line["ranks"]) == [0, 1]
    assert sorted(r[1] for r in line["ranks"]) == [0, 1]      # LOCAL_RANK: one GPU per rank
    assert len({r[2] for r in line["ranks"]}) == 2             # disjoint right-hand sides
    assert line["max_over_ranks"] == 2.0
