"""Algorithm 1 (tree walk) with the MAC of Sec. 3.5 -- TEST INFRASTRUCTURE ONLY.

INTERACTION(B_S, B_T), called once on (root, root) where the root's children
are the 12 base boxes (Sec. 3.4):
  * B_S == B_T, not a leaf: INTERACTION(i, j) for every child pair (i, j);
    B_S == B_T, a leaf: the printed algorithm does nothing here; the leaf's
    particles must still act on each other, so the leaf direct-acts on
    itself (the self pair is excluded by the d^2 == 0 rule of the sum);
  * B_T far from B_S: B_S FMM-acts on B_T (an M2L pair);
  * neither is a leaf: split the box with the larger radius (the source only
    if r(B_S) > r(B_T), so equal radii -- equal to within 1e-12 relative --
    split the target);
  * only B_T is a leaf: split B_S;  only B_S is a leaf: split B_T;
  * both leaves: B_S direct-acts on B_T (a P2P pair).
"Far" is MAC1 d - R_T - c_s R_S > 0 and MAC2 R_T < c_t d, where d is the
angle between the two box centres and R the box radii (Sec. 3.5).  With the
Near Particle Model (particles of angular radius sigma > 0) a far pair must
also keep every particle's profile out of the target box, d - R_T - R_S > sigma,
so that the far field may treat each particle as a point (Sec. 3.5's protected
area, made explicit for a given sigma).

Two exact prunings, used by the solver too: a pair whose source box holds no
particle contributes nothing and is dropped; a pair whose target box holds no
target point is dropped when target counts are given.
"""
import sys

import numpy as np

# Radii within this relative difference are taken as equal (and the target is
# split): HEALPix boxes related by a symmetry have equal radii, whose computed
# values differ only by rounding.
TIE = 1e-12


def _angle(a, b):
    return 2.0 * np.arcsin(min(1.0, np.linalg.norm(a - b) / 2.0))


def walk(tree, centre, radius, c_s=2.0, c_t=0.5, tcount=None, sigma=0.0):
    """Return (m2l, p2p): lists of (source node, target node) pairs."""
    child0 = tree["child0"]
    count = tree["count"]
    m2l, p2p = [], []
    sys.setrecursionlimit(max(10000, sys.getrecursionlimit()))

    def is_leaf(b):
        return child0[b] < 0

    def children(b):
        return range(child0[b], child0[b] + 4)

    def keep(s, t):
        if count[s] == 0:
            return False
        if tcount is not None and tcount[t] == 0:
            return False
        return True

    def interaction(s, t):
        if not keep(s, t):
            return
        if s == t:
            if not is_leaf(s):
                for i in children(s):
                    for j in children(s):
                        interaction(i, j)
            else:
                p2p.append((s, t))
            return
        d = _angle(centre[s], centre[t])
        rs, rt = radius[s], radius[t]
        if d - rt - c_s * rs > 0.0 and rt < c_t * d and d - rt - rs > sigma:
            m2l.append((s, t))
        elif not is_leaf(s) and not is_leaf(t):
            if rs > rt * (1.0 + TIE):
                for i in children(s):
                    interaction(i, t)
            else:
                for j in children(t):
                    interaction(s, j)
        elif not is_leaf(s):
            for i in children(s):
                interaction(i, t)
        elif not is_leaf(t):
            for j in children(t):
                interaction(s, j)
        else:
            p2p.append((s, t))

    roots = np.nonzero(tree["level"] == 0)[0]
    for i in roots:
        for j in roots:
            interaction(int(i), int(j))
    return m2l, p2p


def mac_margin(centre, radius, s, t, c_s=2.0, c_t=0.5, sigma=0.0):
    """Smallest distance of the pair (s, t) from any MAC threshold (used to
    tell rounding-level disagreements from real ones)."""
    d = _angle(centre[s], centre[t])
    m = min(abs(d - radius[t] - c_s * radius[s]), abs(radius[t] - c_t * d))
    if sigma > 0.0:
        m = min(m, abs(d - radius[t] - radius[s] - sigma))
    return m
