"""Pins of the oracle's Algorithm 1 (oracle/walk.py).

* exactly once: for every target leaf L, the M2L pairs whose target is L or
  an ancestor of L together with the P2P pairs into L cover every source
  particle exactly once (brute force);
* every M2L pair satisfies MAC1 and MAC2 (Sec. 3.5); every P2P pair joins
  two leaves; no pair has an empty source box.
"""
import numpy as np
import pytest

import oracle.healpix as hp
from oracle.tree import build_tree
from oracle.walk import walk
from conftest import unit


def geometry(t):
    c = hp.pix2vec_nest(0, np.zeros(0, dtype=np.uint64))
    centre = np.zeros((len(t["level"]), 3))
    radius = np.zeros(len(t["level"]))
    for lvl in np.unique(t["level"]):
        sel = t["level"] == lvl
        centre[sel] = hp.pix2vec_nest(int(lvl), t["prefix"][sel])
        radius[sel] = hp.covering_radius(int(lvl), t["prefix"][sel], per_edge=1)
    return centre, radius


@pytest.mark.parametrize("n,m,clump", [(400, 1, False), (600, 4, True), (800, 8, True)])
def test_exactly_once(n, m, clump):
    rng = np.random.default_rng(n)
    v = unit(rng.normal(size=(n, 3)))
    if clump:
        c = unit(rng.normal(size=3))
        v[: n // 2] = unit(c + 3e-3 * rng.normal(size=(n // 2, 3)))
    keys = np.sort(hp.key29(v))
    t = build_tree(keys, m)
    centre, radius = geometry(t)
    m2l, p2p = walk(t, centre, radius)
    # MAC and structure
    for s, tt in m2l:
        d = 2 * np.arcsin(np.linalg.norm(centre[s] - centre[tt]) / 2)
        assert d - radius[tt] - 2.0 * radius[s] > 0 and radius[tt] < 0.5 * d
        assert t["count"][s] > 0
    for s, tt in p2p:
        assert t["is_leaf"][s] and t["is_leaf"][tt] and t["count"][s] > 0
    by_t_m2l = {}
    for s, tt in m2l:
        by_t_m2l.setdefault(tt, []).append(s)
    by_t_p2p = {}
    for s, tt in p2p:
        by_t_p2p.setdefault(tt, []).append(s)
    N = len(keys)
    for L in np.nonzero(t["is_leaf"])[0]:
        cover = np.zeros(N, dtype=np.int64)
        a = L
        while a >= 0:
            for s in by_t_m2l.get(a, []):
                cover[t["first"][s]:t["first"][s] + t["count"][s]] += 1
            a = t["parent"][a]
        for s in by_t_p2p.get(L, []):
            cover[t["first"][s]:t["first"][s] + t["count"][s]] += 1
        assert np.all(cover == 1), (L, np.unique(cover))
