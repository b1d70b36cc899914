"""A model check of how the traversal restores Algorithm PH's natural order.

The level-by-level expansion (Step 2) writes, at every level, each open
node's children in child order (a dropped child leaves no slot) and carries
every other node unchanged, as if it were its own first child; its jobs are
the last level, in slot order.  The traversal visits the same tree depth
first and in parallel and gives each job its path of child indices, one per
level, the root's index above them and levels below the job's own depth
filled with the lowest index.  This test builds random split trees
(several roots, up to three children per node, dropped children, nodes that
stop early) and checks that sorting the jobs' paths gives exactly the
level-by-level order.
"""
import random

import pytest


def random_forest(rng, roots, depth, k):
    """node -> list of (child index, child) for open nodes; None for a node that stops."""
    tree = {}
    nxt = [roots]

    def grow(v, level):
        if level >= depth or rng.random() < 0.2:
            tree[v] = None  # a job from here on (order <= L, s >= 5 without the split, ...)
            return
        kids = []
        for c in range(k):
            if rng.random() < 0.25:
                continue  # a child with a zero line: dropped
            u = nxt[0]
            nxt[0] += 1
            kids.append((c, u))
            grow(u, level + 1)
        tree[v] = kids

    for r in range(roots):
        grow(r, 0)
    return tree


def level_order(tree, roots, depth):
    level = list(range(roots))
    for _ in range(depth):
        nxt = []
        for v in level:
            kids = tree[v]
            if kids is None:
                nxt.append(v)  # carried in place
            else:
                nxt.extend(u for _, u in kids)
        level = nxt
    return level


def path_keys(tree, roots, depth):
    keys = {}

    def walk(v, path):
        kids = tree[v]
        if kids is None:
            keys[v] = tuple(path) + (0,) * (depth + 1 - len(path))
            return
        for c, u in kids:
            walk(u, path + [c])

    for r in range(roots):
        walk(r, [r])
    return keys


@pytest.mark.parametrize("seed", range(60))
def test_sorted_paths_give_the_level_order(seed):
    rng = random.Random(seed)
    roots, depth, k = rng.randint(1, 5), rng.randint(1, 7), rng.choice([2, 3])
    tree = random_forest(rng, roots, depth, k)
    want = level_order(tree, roots, depth)
    keys = path_keys(tree, roots, depth)
    assert sorted(keys) == sorted(want)  # the same jobs
    assert sorted(keys, key=keys.get) == want
