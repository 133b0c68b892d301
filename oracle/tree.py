"""CPU rebuild of the sFMM tree -- TEST INFRASTRUCTURE ONLY.

Sec. 3.1 builds the tree by (1) putting every particle into one of the 12
HEALPix base boxes, (2) dividing every box holding more than m particles into
its 4 children, (3) repeating until no box holds more than m particles, and
stopping at the maximum depth r_max = 29.  A split always makes 4 children,
empty or not (Fig. quadtree); there is no merging.

Nodes are listed level by level and, inside a level, by key prefix: node i
has level[i], prefix[i] (its nested pixel index at N_side = 2^level),
first[i] / count[i] (its range in the key-sorted particle order), parent[i]
(-1 for the 12 base boxes) and child0[i] (-1 for a leaf; otherwise its 4
children are child0 .. child0+3 in child order 0..3).
"""
import numpy as np

ORDER_MAX = 29


def build_tree(sorted_keys, m, max_level=ORDER_MAX):
    keys = np.asarray(sorted_keys, dtype=np.uint64)
    if keys.size > 1 and np.any(keys[1:] < keys[:-1]):
        raise ValueError("keys must be sorted")
    level, prefix, first, count, parent, child0 = [], [], [], [], [], []

    def rng(lvl, pref):
        sh = np.uint64(2 * (ORDER_MAX - lvl))
        lo = np.searchsorted(keys, pref << sh, side="left")
        hi = np.searchsorted(keys, (pref + np.uint64(1)) << sh, side="left")
        return lo, hi - lo

    cur = np.arange(12, dtype=np.uint64)
    cur_parent = np.full(12, -1, dtype=np.int64)
    lvl = 0
    while cur.size:
        lo, cnt = rng(lvl, cur)
        base = len(level)
        level += [lvl] * cur.size
        prefix += list(cur)
        first += list(lo)
        count += list(cnt)
        parent += list(cur_parent)
        child0 += [-1] * cur.size
        split = (cnt > m) & (lvl < max_level)
        idx = np.nonzero(split)[0]
        nxt_base = base + cur.size
        for k, i in enumerate(idx):
            child0[base + i] = nxt_base + 4 * k
        cur = (cur[idx][:, None] * np.uint64(4) + np.arange(4, dtype=np.uint64)[None, :]).reshape(-1)
        cur_parent = np.repeat(base + idx, 4).astype(np.int64)
        lvl += 1
    t = dict(level=np.array(level, dtype=np.int64), prefix=np.array(prefix, dtype=np.uint64),
             first=np.array(first, dtype=np.int64), count=np.array(count, dtype=np.int64),
             parent=np.array(parent, dtype=np.int64), child0=np.array(child0, dtype=np.int64))
    t["is_leaf"] = t["child0"] < 0
    return t


def leaf_of_sorted(tree, n):
    """Leaf node index of each key-sorted particle."""
    out = np.full(n, -1, dtype=np.int64)
    for i in np.nonzero(tree["is_leaf"])[0]:
        out[tree["first"][i]:tree["first"][i] + tree["count"][i]] = i
    return out


def leaf_of_key(tree, keys):
    """Leaf containing each key (the deepest node whose prefix matches)."""
    keys = np.asarray(keys, dtype=np.uint64)
    leaves = np.nonzero(tree["is_leaf"])[0]
    sh = (2 * (ORDER_MAX - tree["level"][leaves])).astype(np.uint64)
    lo = tree["prefix"][leaves] << sh
    order = np.argsort(lo, kind="stable")
    lo_sorted = lo[order]
    pos = np.searchsorted(lo_sorted, keys, side="right") - 1
    return leaves[order[pos]]
