"""The multi-rank host logic of bench.py on two CPU processes (gloo): each rank takes its
own ensemble (disorder streams offset by 64 x rank, same ribbon sizes), the timing scalars
are combined with max and sum, and the reference arm runs on rank 0 only."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    import workloads as wl

    w, r, local = bench.dist_setup(None)
    assert (w, r, local) == (world, rank, rank)
    ms = bench.max_over_ranks(10.0 + rank, w)
    tot = bench.sum_over_ranks(1.0 + rank, w)
    ens = wl.RibbonEnsemble(stream0=rank * 64)
    bench.barrier(w)
    out.put((rank, ms, tot, ens.sizes[:3], float(ens.ribbon(0).onsite()[0])))
    import torch.distributed as dist

    dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [x[1] for x in res] == [11.0, 11.0]   # max over ranks
    assert [x[2] for x in res] == [3.0, 3.0]     # sum over ranks
    assert res[0][3] == res[1][3]                 # same ribbon sizes on every rank
    assert res[0][4] != res[1][4]                 # different disorder streams
