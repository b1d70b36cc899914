"""A model check of the single-launch evaluator's work protocol, on the CPU.

The persistent kernel (persist.cuh) shares work through atomics only: a
queue counter, a board holding the queue position of the last posted leaf
job with several tasks, and per queue position a counter of tasks taken and
one of tasks finished; the warp that finishes a job's last task closes the
job (coef * per into its matrix).  No warp waits on another.  This test runs
that protocol as generators that yield at every atomic operation, under
many random interleavings of up to 40 warps, and checks that every task runs
exactly once, every job is closed exactly once and after all its tasks,
every warp finishes, and every queue position is taken exactly once.
"""
import random

import pytest


def warp(wid, jobs, S, log):
    """One warp's loop; yields after each shared-memory step."""
    while True:
        b = S["board"]  # read the board
        yield
        if b >= 0:
            yield from take_tasks(wid, b, jobs, S, log, sole=False)
            if S["board"] == b:  # atomicCAS(board, b, -1)
                S["board"] = -1
            yield
            continue
        q = S["qctr"]  # atomicAdd(qctr, 1)
        S["qctr"] += 1
        yield
        if q >= len(jobs):
            return
        log["taken"].append(q)
        kind, T = jobs[q]
        if kind == "leaf":
            if T > 1:
                S["board"] = q  # atomicExch(board, q)
                yield
            yield from take_tasks(wid, q, jobs, S, log, sole=(T == 1))
        else:  # a depth-first job: the warp evaluates it alone
            log["tasks"].append((q, 0))
            log["closed"].append(q)
            yield


def take_tasks(wid, q, jobs, S, log, sole):
    T = jobs[q][1]
    it = 0
    while True:
        if sole:
            if it > 0:
                return
            t = 0
        else:
            t = S["next"][q]  # atomicAdd(task_next + q, 1)
            S["next"][q] += 1
            yield
            if t >= T:
                return
        it += 1
        log["tasks"].append((q, t))  # the task's words into the job's sum
        yield
        if T == 1:
            log["closed"].append(q)
        else:
            d = S["done"][q]  # atomicAdd(task_done + q, 1) after a fence
            S["done"][q] += 1
            yield
            if d == T - 1:
                assert all((q, k) in set(log["tasks"]) for k in range(T)), "closed before its tasks"
                log["closed"].append(q)
        yield


@pytest.mark.parametrize("seed", range(40))
def test_every_task_once_every_job_closed_once(seed):
    rng = random.Random(seed)
    n = rng.randint(1, 30)
    jobs = [(rng.choice(["leaf", "leaf", "dfs"]), rng.choice([1, 1, 2, 3, 8, 17])) for _ in range(n)]
    jobs = [(k, T if k == "leaf" else 1) for k, T in jobs]
    S = {"qctr": 0, "board": -1, "next": [0] * n, "done": [0] * n}
    log = {"tasks": [], "closed": [], "taken": []}
    warps = [warp(w, jobs, S, log) for w in range(rng.randint(1, 40))]
    live = list(range(len(warps)))
    steps = 0
    while live:
        i = rng.choice(live)
        try:
            next(warps[i])
        except StopIteration:
            live.remove(i)
        steps += 1
        assert steps < 1_000_000, "a warp does not finish"
    want_tasks = sorted((q, t) for q, (_, T) in enumerate(jobs) for t in range(T))
    assert sorted(log["tasks"]) == want_tasks
    assert sorted(log["closed"]) == list(range(n))
    assert sorted(log["taken"]) == list(range(n))  # each queue position taken once (the counter hands them out in order)
