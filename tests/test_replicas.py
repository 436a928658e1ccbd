"""Multi-GPU mode is replicas only (no data-path collective): the host logic of
bench.py's N > 1 path -- disjoint configurations per rank in every step and the
job time as the maximum over ranks -- run as 2 gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, local = bench.dist_env()
    seeds = [bench.seed_for(s, r, w) for s in range(5)]
    ms = bench.max_over_ranks(100.0 + 50.0 * rank)
    gathered = [None] * w
    dist.all_gather_object(gathered, seeds)
    if rank == 0:
        out.put((gathered, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_replicas():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    gathered, ms = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert ms == 150.0  # the slower rank's time
    for step in range(5):  # every step: two different configurations
        assert gathered[0][step] != gathered[1][step]


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(12.5) == 12.5
    assert [bench.seed_for(s, 0, 1) for s in range(12)] == [s % 10 for s in range(12)]
