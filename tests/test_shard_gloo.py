"""Multi-rank sharding on CPU with gloo, world size 2: each rank scans its
shard (the oracle stands in for the GPU scan), results are gathered, and the
merge equals the single-rank result -- no exchange is needed during the scan."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import workloads as W
from paper_1704_02278_gb300 import shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = W.config2(2 * W.MiB + 99)
        maxlen = int(w.patterns.lengths().max())
        lo, hi, rd = shard.text_shard(w.nbytes, rank, world, maxlen)
        part = shard.keep_owned(oracle.ac(w.text[lo:rd], w.patterns.csr()), lo, hi)
        got = [None] * world
        dist.all_gather_object(got, part)
        merged = shard.merge_ranked(got)
        # batch: whole segments per rank
        p = W.config4_patterns()
        sizes = W.config4_sizes(40)
        seg = np.zeros(41, np.uint64)
        seg[1:] = np.cumsum(sizes)
        t = W.syslog_files(W.seed(4, 0), W.seed(4, 2), seg, 0.02, p)
        s_lo, s_hi = shard.segment_shard(seg, rank, world)
        sub = seg[s_lo:s_hi + 1] - seg[s_lo]
        b = oracle.batch(t[int(seg[s_lo]):int(seg[s_hi])], sub, p.csr()) if s_hi > s_lo else np.zeros((0, 3), np.uint32)
        b = b.copy()
        b[:, 0] += s_lo
        gb = [None] * world
        dist.all_gather_object(gb, b)
        if rank == 0:
            q.put((merged, np.concatenate([x for x in gb if len(x)])))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_two_ranks_equal_one(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    merged, batch = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    w = W.config2(2 * W.MiB + 99)
    assert np.array_equal(merged, oracle.ac(w.text, w.patterns.csr()))
    p4 = W.config4_patterns()
    sizes = W.config4_sizes(40)
    seg = np.zeros(41, np.uint64)
    seg[1:] = np.cumsum(sizes)
    t = W.syslog_files(W.seed(4, 0), W.seed(4, 2), seg, 0.02, p4)
    assert np.array_equal(batch, oracle.batch(t, seg, p4.csr()))


def test_shard_bounds():
    assert shard.text_shard(10, 0, 3, 4) == (0, 4, 7)
    assert shard.text_shard(10, 2, 3, 4) == (8, 10, 10)
    seg = np.array([0, 5, 5, 100, 101, 300])
    spans = [shard.segment_shard(seg, r, 3) for r in range(3)]
    assert spans[0][0] == 0 and spans[-1][1] == 5
    assert all(spans[i][1] == spans[i + 1][0] for i in range(2))
