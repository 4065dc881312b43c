"""Host logic of the replica runs (one GPU per rank), on CPU with gloo ranks."""
import os
import socket

import pytest
import torch
import torch.multiprocessing as mp

from paper_2310_09467_gb300 import replicas


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, loc = replicas.rank_env()
    ms, nbytes = replicas.aggregate(10.0 + 5.0 * rank, 1000 * (rank + 1))
    seeds = [replicas.frame_seed(r, i, k, 3) for i in range(4) for k in range(3)]
    q.put((r, w, loc, ms, nbytes, seeds))
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, l0, ms0, b0, s0), (r1, w1, l1, ms1, b1, s1) = got
    assert (r0, r1, w0, w1, l0, l1) == (0, 1, 2, 2, 0, 1)
    assert ms0 == ms1 == 15.0          # the slowest rank's time
    assert b0 == b1 == 3000            # bytes of all ranks
    assert not set(s0) & set(s1)       # each rank compresses its own frames
    assert s0 == [1 + k + 3 * i for i in range(4) for k in range(3)]  # rank 0 = the single-GPU frames
    assert replicas.throughput_mbps(ms0, b0) == pytest.approx(3000 / 1e6 / 0.015)


def test_replicas_single_process():
    assert replicas.aggregate(12.5, 777) == (12.5, 777)
    assert replicas.throughput_mbps(0.0, 5) == 0.0
