"""Replica logic of the data-parallel path on CPU: two gloo ranks, no GPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2609_32505_gb300 import replicas


@pytest.mark.parametrize("batch,ws", [(8, 2), (7, 2), (5, 4), (1, 3), (0, 2)])
def test_shard_partitions_the_batch(batch, ws):
    parts = [list(replicas.shard(batch, r, ws)) for r in range(ws)]
    flat = [i for p in parts for i in p]
    assert flat == list(range(batch))
    assert max(map(len, parts)) - min(map(len, parts)) <= 1


def _worker(rank, ws, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(ws), MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    r, w = replicas.init("gloo")
    assert (r, w) == (rank, ws)
    vals = replicas.max_over_ranks([10.0 + rank, 5.0 - rank])
    out.put((rank, vals, list(replicas.shard(9, r, w))))
    import torch.distributed as dist
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_with_two_gloo_ranks():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict((r, (v, sh)) for r, v, sh in (q.get(timeout=120) for _ in procs))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(2):
        assert res[r][0] == [11.0, 5.0]            # the slowest rank's time, everywhere
    assert res[0][1] + res[1][1] == list(range(9))
