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
    check_exactly_once(t, m2l, p2p, len(keys))


def check_exactly_once(t, m2l, p2p, N):
    by_t_m2l = {}
    for s, tt in m2l:
        by_t_m2l.setdefault(tt, []).append(s)
    by_t_p2p = {}
    for s, tt in p2p:
        by_t_p2p.setdefault(tt, []).append(s)
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


@pytest.mark.parametrize("sigma", [0.01, 0.05, 0.3])
def test_near_particle_mac_keeps_exactly_once(sigma):
    """With particles of angular radius sigma (Sec. 3.5's protected area): every
    M2L pair also keeps d - R_T - R_S > sigma, the lists still cover every
    source exactly once, every M2L pair of the sigma walk is an M2L pair of
    the point walk or lies below one, and the condition binds (some pair of
    the point walk violates it, and the two walks differ)."""
    rng = np.random.default_rng(int(sigma * 1000))
    v = unit(rng.normal(size=(700, 3)))
    c = unit(rng.normal(size=3))
    v[:300] = unit(c + 5e-3 * rng.normal(size=(300, 3)))
    keys = np.sort(hp.key29(v))
    t = build_tree(keys, 4)
    centre, radius = geometry(t)
    m0, p0 = walk(t, centre, radius)
    m2l, p2p = walk(t, centre, radius, sigma=sigma)
    for s, tt in m2l:
        d = 2 * np.arcsin(np.linalg.norm(centre[s] - centre[tt]) / 2)
        assert d - radius[tt] - 2.0 * radius[s] > 0 and radius[tt] < 0.5 * d
        assert d - radius[tt] - radius[s] > sigma
    check_exactly_once(t, m2l, p2p, len(keys))
    violate = [(s, tt) for s, tt in m0
               if 2 * np.arcsin(np.linalg.norm(centre[s] - centre[tt]) / 2) - radius[tt] - radius[s] <= sigma]
    assert violate and set(m2l) != set(m0)
    assert not (set(violate) & set(m2l))

    def ancestors(b):
        out = set()
        while b >= 0:
            out.add(b)
            b = t["parent"][b]
        return out

    # a sigma pair is a point-walk pair or descends (in source and target) from one
    m0s = set(m0)
    for s, tt in m2l:
        assert (s, tt) in m0s or any((a, b) in m0s for a in ancestors(s) for b in ancestors(tt))


def test_sigma_beyond_every_distance_leaves_no_far_pairs():
    """sigma = pi: no pair is far, every source reaches every target directly."""
    rng = np.random.default_rng(5)
    v = unit(rng.normal(size=(200, 3)))
    keys = np.sort(hp.key29(v))
    t = build_tree(keys, 8)
    centre, radius = geometry(t)
    m2l, p2p = walk(t, centre, radius, sigma=np.pi)
    assert m2l == []
    check_exactly_once(t, m2l, p2p, len(keys))
