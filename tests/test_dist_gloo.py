"""The multi-rank host logic on CPU: two gloo ranks shard one matrix's job
queue, evaluate their shares (the oracle stands in for the GPU here), and
gather the 256-bit sums exactly; max-over-ranks timing; batch seeds."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1112_6072_gb300 import dist as D


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, queue):
    import torch.distributed as dist

    import oracle
    import workloads as W

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        a = W.random_small(9, 5, lo=-2, hi=3, density=0.6)
        a[np.arange(9), np.arange(9)] = 1
        jobs = oracle.jobs(a, 3)
        mine = D.shard_queue(np.arange(len(jobs)), rank, world)
        local = 0
        for j in mine:
            m, c = jobs[int(j)]
            local += c * oracle.per_bruteforce(m)
        total = D.gather_sum(D.words_from_int(local))
        t = D.max_over_ranks(1.0 + rank)
        queue.put((rank, D.int_from_words(total[0]), oracle.per_bruteforce(a), t))
    finally:
        dist.destroy_process_group()


def test_two_rank_shard_and_exact_sum():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, want, t in res:
        assert got == want
        assert t == 2.0


def test_shard_queue_partitions_in_order():
    q = np.array([5, 3, 9, 1, 0, 7, 2], dtype=np.uint32)
    parts = [D.shard_queue(q, r, 3) for r in range(3)]
    assert sorted(np.concatenate(parts).tolist()) == sorted(q.tolist())
    assert parts[0].tolist() == [5, 1, 2]
    with pytest.raises(ValueError):
        D.shard_queue(q, 3, 3)


def test_combine_words_carries():
    a = (1 << 64) - 1
    w = D.combine_words([D.words_from_int(a), D.words_from_int(1)])
    assert D.int_from_words(w) == 1 << 64
    w = D.combine_words([D.words_from_int(-5), D.words_from_int(3)])
    assert D.int_from_words(w) == -2
    assert D.batch_seed(100, 3) == 103
