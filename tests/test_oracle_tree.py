"""Pins of the oracle's tree rebuild (oracle/tree.py) against a brute-force
definition of Sec. 3.1's division rule written separately here: a node at
level l with pixel prefix P exists iff it is a base box (l = 0) or its parent
exists and holds more than m particles (and l - 1 < r_max)."""
import numpy as np
import pytest

import oracle.healpix as hp
from oracle.tree import build_tree, leaf_of_key, leaf_of_sorted
from conftest import unit


def brute_nodes(keys, m, max_level=29):
    keys = [int(k) for k in keys]
    out = set()

    def rec(level, prefix):
        sh = 2 * (29 - level)
        cnt = sum(1 for k in keys if (k >> sh) == prefix)
        out.add((level, prefix, cnt))
        if cnt > m and level < max_level:
            for c in range(4):
                rec(level + 1, prefix * 4 + c)

    for f in range(12):
        rec(0, f)
    return out


@pytest.mark.parametrize("n,m", [(300, 1), (300, 4), (1000, 16)])
def test_matches_brute_force(n, m):
    rng = np.random.default_rng(n + m)
    v = unit(rng.normal(size=(n, 3)))
    keys = np.sort(hp.key29(v))
    t = build_tree(keys, m)
    got = {(int(l), int(p), int(c)) for l, p, c in zip(t["level"], t["prefix"], t["count"])}
    assert got == brute_nodes(keys, m)


def test_invariants_clustered():
    rng = np.random.default_rng(7)
    c = unit(rng.normal(size=3))
    v = np.vstack([unit(rng.normal(size=(3000, 3))), unit(c + 1e-6 * rng.normal(size=(2000, 3)))])
    keys = np.sort(hp.key29(v))
    m = 8
    t = build_tree(keys, m)
    leaf = t["is_leaf"]
    assert t["count"][leaf].sum() == len(keys)
    assert np.all((t["count"][leaf] <= m) | (t["level"][leaf] == 29))
    internal = ~leaf
    for i in np.nonzero(internal)[0]:
        ch = t["child0"][i] + np.arange(4)
        assert t["count"][ch].sum() == t["count"][i]
        assert np.all(t["parent"][ch] == i)
        assert np.all(t["prefix"][ch] >> np.uint64(2) == t["prefix"][i])
        assert t["first"][ch[0]] == t["first"][i]
    for i in range(len(t["level"])):
        sh = np.uint64(2 * (29 - t["level"][i]))
        seg = keys[t["first"][i]:t["first"][i] + t["count"][i]]
        assert np.all(seg >> sh == t["prefix"][i])
    # BFS order: by level, then prefix
    order = np.lexsort((t["prefix"], t["level"]))
    assert np.array_equal(order, np.arange(len(order)))
    lk = leaf_of_key(t, keys)
    assert np.array_equal(lk, leaf_of_sorted(t, len(keys)))


def test_coincident_points_stop_at_r_max():
    p = unit(np.array([0.3, 0.2, 0.9]))
    v = np.repeat(p[None, :], 10, axis=0)
    t = build_tree(np.sort(hp.key29(v)), 2)
    leaf = t["is_leaf"] & (t["count"] > 0)
    assert t["level"][leaf].tolist() == [29] and t["count"][leaf].tolist() == [10]
