"""A model check of the traversal expansion's work hand-off, on the CPU.

The traversal kernel (walk.cu) shares subtrees through a queue of slots:
`head` hands out tickets, `tail` reserves slots, a ready flag per slot, and
`outstanding` = nodes put in the queue minus subtrees finished (the roots
start in the queue).  A warp takes a ticket and waits for its slot's ready
flag, leaving when `outstanding` falls to 0; while other warps wait (head >
tail) a warp walking a subtree gives the children after the first of each
node it splits to the queue instead of walking them itself.  This test runs
the protocol as generators that yield at every shared step, over random
trees and random interleavings, and checks that every node is visited
exactly once, every warp leaves and `outstanding` ends at 0.
"""
import random

import pytest


def make_tree(rng, nodes, roots=1):
    """children[i] of node i in a random forest rooted at nodes 0 .. roots-1."""
    children = {r: [] for r in range(roots)}
    for i in range(roots, nodes):
        p = rng.choice([v for v in range(i) if len(children[v]) < 3])  # Eq. 2: at most three children
        children[p].append(i)
        children[i] = []
    return children


def warp(roots_n, children, S, log):
    while True:
        t = S["head"]  # atomicAdd(head, 1)
        S["head"] += 1
        yield
        while True:  # wait for the slot, or for the end of the work
            if t < len(S["slots"]) and S["ready"].get(t):
                break
            if S["outstanding"] <= 0:
                return
            yield
        root = S["slots"][t]
        stack = [root]
        while stack:  # the subtree depth first
            v = stack.pop()
            log.append(v)
            yield
            kids = children[v]
            waiting = S["head"] > S["tail"]
            yield
            if kids and waiting:
                for c in kids[1:]:  # siblings to the waiting warps
                    S["outstanding"] += 1
                    slot = S["tail"]
                    S["tail"] += 1
                    yield
                    while len(S["slots"]) <= slot:
                        S["slots"].append(None)
                    S["slots"][slot] = c
                    S["ready"][slot] = True  # after a fence
                    yield
                stack.append(kids[0])
            else:
                stack.extend(reversed(kids))
        S["outstanding"] -= 1  # this subtree is done
        yield


@pytest.mark.parametrize("seed", range(40))
def test_every_node_once_and_every_warp_leaves(seed):
    rng = random.Random(seed)
    n = rng.randint(1, 80)
    nroots = rng.randint(1, min(n, 6))
    children = make_tree(rng, n, nroots)
    roots = list(range(nroots))
    S = {"head": 0, "tail": len(roots), "outstanding": len(roots), "slots": list(roots),
         "ready": {i: True for i in range(len(roots))}}
    log = []
    warps = [warp(len(roots), children, S, log) for _ in range(rng.randint(1, 24))]
    live = list(range(len(warps)))
    steps = 0
    while live:
        i = rng.choice(live)
        try:
            next(warps[i])
        except StopIteration:
            live.remove(i)
        steps += 1
        assert steps < 2_000_000, "a warp does not leave"
    assert sorted(log) == list(range(n))
    assert S["outstanding"] == 0
