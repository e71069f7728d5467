"""Replica (weak-scaling) path of bench.py on the CPU: two gloo ranks on
127.0.0.1.  Each rank advances its own manifest (seed = rank) with no data
exchange; the job's time is the slowest rank's and its particle-steps the sum
over ranks.  The same reductions run over NCCL-free gloo on a GPU machine."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, local = bench.dist_env()

    class A:
        runs, scale = 6, 0.01
    cfgs = bench.manifest(r, A, steps=10)
    ms, ps = bench.combine_ranks(10.0 + 5.0 * r, 1000 * (r + 1))
    dist.barrier()
    dist.destroy_process_group()
    q.put((r, w, local, [c.seed for c in cfgs], [c.n_particles for c in cfgs], ms, ps))


def test_two_ranks_weak_scaling_reductions():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, l0, s0, n0, ms0, ps0), (r1, w1, l1, s1, n1, ms1, ps1) = out
    assert (r0, r1, w0, w1, l0, l1) == (0, 1, 2, 2, 0, 1)
    assert ms0 == ms1 == 15.0          # slowest rank
    assert ps0 == ps1 == 3000.0        # all ranks' particle-steps
    assert not set(s0) & set(s1)       # each rank its own manifest
    assert n0 != n1
