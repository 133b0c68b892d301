"""GPU parity of the CUDA path (through the C ABI) against the oracle.

* keys and the tree: bit-exact against the oracle's CPU rebuild;
* box geometry: centres and radii against the oracle's HEALPix geometry;
* each translation step on identical inputs: leaf multipoles against Lemma 1,
  internal multipoles against Lemma 2 applied to the GPU's child multipoles,
  locals against Lemma 3 over the GPU's M2L list plus Lemma 4 from the GPU's
  parent local;
* the interaction lists: exactly-once coverage, the MAC, and equality with
  the oracle's Algorithm 1 walk;
* end to end: psi and alpha against the FP64 direct sum, norm-wise relative
  error <= 1e-10 (the ratio of Euclidean norms over all targets).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle.healpix as hp
import oracle.lemmas as LM
from oracle.direct import direct_sum
from oracle.tree import build_tree
from oracle.walk import walk
from paper_2210_07021_gb300 import sfmm, workloads
from conftest import unit

TOL = 1e-10


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def solve(src, q, tgt, p=20, leaf=32, **kw):
    plan = sfmm.Plan(p=p, leaf_size=leaf, **kw)
    qd = torch.float32 if kw.get("q_f32") else torch.float64
    psi, alpha = plan.deflection(dev(src), dev(q, qd), dev(tgt))
    torch.cuda.synchronize()
    return plan, psi.cpu().numpy(), alpha.cpu().numpy()


def clustered_small(n=6000, m=4001, seed=3):
    rng = np.random.default_rng(seed)
    src = workloads.clustered(rng, n, 12)
    tgt = np.vstack([workloads.clustered(rng, m - 1000, 12), unit(rng.normal(size=(1000, 3)))])
    q = rng.lognormal(0, 0.5, n)
    return src, q, tgt


# ------------------------------------------------------------------- keys --
def test_keys_bit_exact():
    rng = np.random.default_rng(0)
    pts = [unit(rng.normal(size=(200000, 3))), workloads.clustered(rng, 100000, 20)]
    # special points: poles, axes, diagonals, pixel centres and corners at several orders
    special = [[0, 0, 1], [0, 0, -1], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0],
               [1, 1, 0], [-1, 1, 0], [1, -1, 0], [1, 1, 1], [-1, -1, -1], [0, 1, 1], [0, -1e-300, 1]]
    pts.append(unit(np.array(special, dtype=float)))
    for o in (0, 3, 9, 17, 29):
        pix = rng.integers(0, 12 * 4 ** o, 2000, dtype=np.int64).astype(np.uint64)
        pts.append(hp.pix2vec_nest(o, pix))
        f, ix, iy = hp.pix2face_xy(o, pix)
        pts.append(unit(hp.facexy2vec(o, f, ix.astype(float), iy.astype(float))))
    # near-pole and near-ring-boundary points
    z = np.concatenate([1 - np.geomspace(1e-16, 1e-2, 2000), np.full(2000, 2 / 3), -np.full(2000, 2 / 3)])
    ph = rng.uniform(0, 2 * np.pi, z.size)
    st = np.sqrt(np.maximum(0, 1 - z * z))
    pts.append(np.stack([st * np.cos(ph), st * np.sin(ph), z], 1))
    x = np.vstack(pts)
    got = sfmm.keys(dev(x)).cpu().numpy().view(np.uint64)
    want = hp.key29(x)
    bad = np.nonzero(got != want)[0]
    assert bad.size == 0, (bad[:10], x[bad[:3]], got[bad[:3]], want[bad[:3]])


def test_keys_bit_exact_near_decision_boundaries():
    """The key kernel's double-float fast path defers to the FP64 routine near
    every floor decision; points placed on and within rounding of the decisions
    (order-29 pixel edges and corners, the phi = 0 wrap, octant and quadrant
    lines, the polar-cap and equatorial ring boundaries) must still give the
    oracle's keys bit for bit."""
    rng = np.random.default_rng(5)
    pts = []
    # order-29 pixel corners and edge midpoints, nudged by a few ulp in each coordinate
    o = 29
    pix = rng.integers(0, 12 * 4 ** o, 20000, dtype=np.int64).astype(np.uint64)
    f, ix, iy = hp.pix2face_xy(o, pix)
    for dx, dy in ((0.0, 0.0), (0.5, 0.0), (0.0, 0.5)):
        c = unit(hp.facexy2vec(o, f, ix.astype(float) + dx, iy.astype(float) + dy))
        for k in (0, 1, 4):
            pts.append(unit(c + k * 2.2e-16 * rng.choice([-1.0, 1.0], size=c.shape)))
    # phi just below 2 pi (x > 0, y -> 0-), on the octant and quadrant lines
    t = np.geomspace(1e-17, 1e-6, 3000)
    for zz in (0.0, 0.5, 0.9, -0.95):
        st = np.sqrt(1 - zz * zz)
        pts.append(np.stack([st * np.cos(-t), st * np.sin(-t), np.full_like(t, zz)], 1))
        pts.append(np.stack([st * np.cos(np.pi / 4 + t), st * np.sin(np.pi / 4 + t), np.full_like(t, zz)], 1))
        pts.append(np.stack([st * np.cos(np.pi / 2 - t), st * np.sin(np.pi / 2 - t), np.full_like(t, zz)], 1))
        pts.append(np.stack([st * np.cos(np.pi + t), st * np.sin(np.pi + t), np.full_like(t, zz)], 1))
    # the polar-cap boundary |z| = 2/3 from both sides, near the poles
    zb = np.concatenate([2 / 3 + np.geomspace(1e-17, 1e-9, 2000), 2 / 3 - np.geomspace(1e-17, 1e-9, 2000),
                         1 - np.geomspace(1e-18, 1e-12, 2000)])
    ph = rng.uniform(0, 2 * np.pi, zb.size)
    for sgn in (1.0, -1.0):
        z = sgn * zb
        st = np.sqrt(np.maximum(0, 1 - z * z))
        pts.append(np.stack([st * np.cos(ph), st * np.sin(ph), z], 1))
    # near the axis: tiny x, y
    tiny = np.geomspace(1e-300, 1e-15, 500)
    pts.append(np.stack([tiny, -tiny * 0.5, np.sqrt(1 - 1.25 * tiny ** 2)], 1))
    x = np.vstack(pts)
    got = sfmm.keys(dev(x)).cpu().numpy().view(np.uint64)
    want = hp.key29(x)
    bad = np.nonzero(got != want)[0]
    assert bad.size == 0, (bad.size, bad[:10], x[bad[:3]], got[bad[:3]], want[bad[:3]])


# ------------------------------------------------------------------- tree --
@pytest.fixture(scope="module")
def small_solve():
    src, q, tgt = clustered_small()
    plan, psi, alpha = solve(src, q, tgt, p=20, leaf=16)
    return dict(src=src, q=q, tgt=tgt, plan=plan, psi=psi, alpha=alpha)


def gpu_tree(plan):
    return dict(
        prefix=plan.debug(sfmm.ARR_NODE_PREFIX, np.uint64),
        level=plan.debug(sfmm.ARR_NODE_LEVEL, np.int32).astype(np.int64),
        rng=plan.debug(sfmm.ARR_NODE_RANGE, np.int32, 2).astype(np.int64),
        trng=plan.debug(sfmm.ARR_NODE_TRANGE, np.int32, 2).astype(np.int64),
        child0=plan.debug(sfmm.ARR_NODE_CHILD0, np.int32).astype(np.int64),
        parent=plan.debug(sfmm.ARR_NODE_PARENT, np.int32).astype(np.int64),
        geom=plan.debug(sfmm.ARR_NODE_GEOM, np.float64, 11),
    )


def test_tree_bit_exact(small_solve):
    S = small_solve
    plan = S["plan"]
    keys = plan.debug(sfmm.ARR_SRC_KEYS, np.uint64)
    perm = plan.debug(sfmm.ARR_SRC_PERM, np.uint32)
    want_keys = hp.key29(S["src"])
    assert np.array_equal(keys, np.sort(want_keys))
    assert np.array_equal(want_keys[perm], keys)
    # stable: equal keys keep the input order
    eq = keys[1:] == keys[:-1]
    assert np.all(perm[1:][eq] > perm[:-1][eq])
    g = gpu_tree(plan)
    t = build_tree(np.sort(want_keys), 16)
    assert np.array_equal(g["prefix"], t["prefix"])
    assert np.array_equal(g["level"], t["level"])
    assert np.array_equal(g["rng"][:, 0], t["first"]) and np.array_equal(g["rng"][:, 1], t["count"])
    assert np.array_equal(g["child0"], t["child0"])
    assert np.array_equal(g["parent"], t["parent"])
    tk = np.sort(hp.key29(S["tgt"]))
    assert np.array_equal(plan.debug(sfmm.ARR_TGT_KEYS, np.uint64), tk)
    sh = (2 * (29 - t["level"])).astype(np.uint64)
    lo = np.searchsorted(tk, t["prefix"] << sh)
    hi = np.searchsorted(tk, (t["prefix"] + np.uint64(1)) << sh)
    assert np.array_equal(g["trng"][:, 0], lo) and np.array_equal(g["trng"][:, 1], hi - lo)


def test_geometry(small_solve):
    g = gpu_tree(small_solve["plan"])
    for lvl in np.unique(g["level"]):
        sel = g["level"] == lvl
        c = hp.pix2vec_nest(int(lvl), g["prefix"][sel])
        np.testing.assert_allclose(g["geom"][sel, 0:3], c, atol=4e-16)
        R = hp.covering_radius(int(lvl), g["prefix"][sel], per_edge=1)
        np.testing.assert_allclose(g["geom"][sel, 9], R + 2e-15, rtol=1e-12, atol=2e-15)
        _, et, ep = LM.basis(c)
        np.testing.assert_allclose(g["geom"][sel, 3:6], et, atol=1e-15)
        np.testing.assert_allclose(g["geom"][sel, 6:9], ep, atol=1e-15)


# ------------------------------------------------------------ expansions --
def _scaled(A, r, local):
    l = np.arange(1, A.shape[-1] + 1)
    return A * (r ** l if local else r ** (-l.astype(float)))


def test_p2m_m2m_l2l_m2l_steps(small_solve):
    S = small_solve
    plan = S["plan"]
    p = plan.order
    g = gpu_tree(plan)
    mp = plan.debug(sfmm.ARR_MULTIPOLE, np.float64, 2 * p + 2)
    lc = plan.debug(sfmm.ARR_LOCAL, np.float64, 2 * p + 2)
    perm = plan.debug(sfmm.ARR_SRC_PERM, np.uint32)
    ys, qs = S["src"][perm], S["q"][perm]
    cen, r = g["geom"][:, 0:3], g["geom"][:, 10]

    def exp_of(row):
        return row[0], row[1], row[2::2] + 1j * row[3::2]

    rng = np.random.default_rng(1)
    leaves = np.nonzero((g["child0"] < 0) & (g["rng"][:, 1] > 0))[0]
    for i in rng.choice(leaves, 40, replace=False):
        f, n = g["rng"][i]
        C, Q, A = LM.p2m(cen[i], ys[f:f + n], qs[f:f + n], p)
        gc, gq, ga = exp_of(mp[i])
        np.testing.assert_allclose([gc, gq], [C, Q], rtol=1e-13, atol=1e-15)
        np.testing.assert_allclose(_scaled(ga, r[i], False), _scaled(A, r[i], False), rtol=0, atol=1e-13 * abs(Q) + 1e-300)
    internal = np.nonzero((g["child0"] >= 0) & (g["rng"][:, 1] > 0))[0]
    for i in rng.choice(internal, min(30, internal.size), replace=False):
        acc = None
        for c in range(g["child0"][i], g["child0"][i] + 4):
            if g["rng"][c, 1] == 0:
                continue
            e = LM.m2m(cen[c], cen[i], exp_of(mp[c]))
            acc = e if acc is None else (acc[0] + e[0], acc[1] + e[1], acc[2] + e[2])
        gc, gq, ga = exp_of(mp[i])
        np.testing.assert_allclose(gc, acc[0], rtol=1e-12)
        np.testing.assert_allclose(_scaled(ga, r[i], False), _scaled(acc[2], r[i], False), atol=1e-12 * abs(gq))
    # locals: sum of Lemma 3 over the M2L list plus Lemma 4 of the parent's local
    m2l = plan.debug(sfmm.ARR_M2L, np.int32, 2)
    by_t = {}
    for s_, t_ in m2l:
        by_t.setdefault(int(t_), []).append(int(s_))
    withloc = np.nonzero(g["trng"][:, 1] > 0)[0]
    checked = 0
    for i in rng.permutation(withloc):
        if g["level"][i] == 0 or checked >= 40:
            continue
        par = g["parent"][i]
        acc = LM.l2l(cen[par], cen[i], exp_of(lc[par]))
        for s_ in by_t.get(int(i), []):
            e = LM.m2l(cen[s_], cen[i], exp_of(mp[s_]))
            acc = (acc[0] + e[0], acc[1] + e[1], acc[2] + e[2])
        gc, gq, ga = exp_of(lc[i])
        np.testing.assert_allclose([gc, gq], [acc[0], acc[1]], rtol=1e-11, atol=1e-14)
        scale = max(abs(gq), np.abs(_scaled(ga, r[i], True)).max(), 1e-30)
        np.testing.assert_allclose(_scaled(ga, r[i], True), _scaled(acc[2], r[i], True), atol=1e-11 * scale)
        checked += 1
    assert checked > 10


# ------------------------------------------------------------------ lists --
def test_lists_match_algorithm_1(small_solve):
    S = small_solve
    plan = S["plan"]
    g = gpu_tree(plan)
    t = dict(level=g["level"], prefix=g["prefix"], first=g["rng"][:, 0], count=g["rng"][:, 1],
             parent=g["parent"], child0=g["child0"], is_leaf=g["child0"] < 0)
    cen = np.zeros((len(t["level"]), 3))
    rad = np.zeros(len(t["level"]))
    for lvl in np.unique(t["level"]):
        sel = t["level"] == lvl
        cen[sel] = hp.pix2vec_nest(int(lvl), t["prefix"][sel])
        rad[sel] = hp.covering_radius(int(lvl), t["prefix"][sel], per_edge=1) + 2e-15
    m2l_o, p2p_o = walk(t, cen, rad, tcount=g["trng"][:, 1])
    m2l = plan.debug(sfmm.ARR_M2L, np.int32, 2)
    p2p = plan.debug(sfmm.ARR_P2P, np.int32, 2)
    assert set(map(tuple, m2l.tolist())) == set(m2l_o)
    assert set(map(tuple, p2p.tolist())) == set(p2p_o)
    assert len(m2l) == len(m2l_o) and len(p2p) == len(p2p_o)
    # grouped by target
    assert np.all(np.diff(m2l[:, 1]) >= 0) and np.all(np.diff(p2p[:, 1]) >= 0)


# ------------------------------------------------------------- end to end --
def check_against_oracle(src, q, tgt, psi, alpha, tol=TOL, idx=None):
    if idx is None:
        idx = np.arange(tgt.shape[0])
    ref = direct_sum(src, q, tgt[idx])
    ep, ea = rel(psi[idx], ref["psi"]), rel(alpha[idx], ref["alpha"])
    assert ep <= tol and ea <= tol, (ep, ea)
    return ep, ea


def test_end_to_end_small_clustered(small_solve):
    S = small_solve
    plan, psi, alpha = solve(S["src"], S["q"], S["tgt"], p=32, leaf=16)
    check_against_oracle(S["src"], S["q"], S["tgt"], psi, alpha)


def test_random_sky_targets_are_sources():
    d = workloads.random_sky(4096)
    plan, psi, alpha = solve(d["src"], d["q"], d["tgt"], p=32, leaf=32)
    check_against_oracle(d["src"], d["q"], d["tgt"], psi, alpha)


@pytest.mark.parametrize("n,m,leaf", [(1, 1, 32), (5, 3, 32), (33, 17, 32), (100, 2, 1), (2049, 4099, 8)])
def test_ragged_and_tiny(n, m, leaf):
    rng = np.random.default_rng(n * 7 + m)
    src = unit(rng.normal(size=(n, 3)))
    tgt = unit(rng.normal(size=(m, 3)))
    q = rng.random(n) + 0.1
    plan, psi, alpha = solve(src, q, tgt, p=32, leaf=leaf)
    check_against_oracle(src, q, tgt, psi, alpha)


def test_empty_inputs():
    plan = sfmm.Plan(p=10)
    tgt = dev(unit(np.random.default_rng(0).normal(size=(7, 3))))
    psi, alpha = plan.deflection(dev(np.zeros((0, 3))), dev(np.zeros(0)), tgt)
    assert torch.all(psi == 0) and torch.all(alpha == 0)
    psi, alpha = plan.deflection(dev(np.zeros((3, 3)) + [0, 0, 1.0]), dev(np.ones(3)), dev(np.zeros((0, 3))))
    assert psi.numel() == 0


def test_coincident_points_and_poles():
    rng = np.random.default_rng(9)
    base = unit(np.array([0.1, 0.2, 0.97]))
    src = np.vstack([np.repeat(base[None], 50, 0), unit(base + 1e-9 * rng.normal(size=(50, 3))),
                     [[0, 0, 1.0], [0, 0, -1.0]], unit(rng.normal(size=(400, 3)))])
    q = rng.random(len(src)) + 0.5
    tgt = np.vstack([src[:60], [[0, 0, 1.0], [0, 0, -1.0]], unit(rng.normal(size=(100, 3)))])
    plan, psi, alpha = solve(src, q, tgt, p=32, leaf=8)
    check_against_oracle(src, q, tgt, psi, alpha)


def test_host_entry_point_and_options():
    src, q, tgt = clustered_small(3000, 2000, seed=5)
    plan, psi, alpha = solve(src, q, tgt, p=24)
    hpsi, halpha = plan.deflection_host(src, q, tgt)
    np.testing.assert_array_equal(hpsi, psi)
    np.testing.assert_array_equal(halpha, alpha)
    # potential-only agrees with the deflection call's psi
    pot = plan.potential(dev(src), dev(q), dev(tgt)).cpu().numpy()
    np.testing.assert_array_equal(pot, psi)
    # no-psi deflection gives the same alpha
    _, a2 = plan.deflection(dev(src), dev(q), dev(tgt), with_psi=False)
    np.testing.assert_array_equal(a2.cpu().numpy(), alpha)
    # zero mean adds sum(q)/(4 pi)
    zplan, zpsi, zalpha = solve(src, q, tgt, p=24, zero_mean=True)
    np.testing.assert_allclose(zpsi - psi, q.sum() / (4 * np.pi), rtol=1e-12)
    # float32 masses
    q32 = q.astype(np.float32)
    fplan, fpsi, falpha = solve(src, q32, tgt, p=24, q_f32=True)
    ref = direct_sum(src, q32.astype(np.float64), tgt[:300])
    assert rel(fpsi[:300], ref["psi"]) < TOL and rel(falpha[:300], ref["alpha"]) < TOL


def test_rotation_invariance_of_the_solver():
    """The tree is not rotation invariant, so this checks the FMM's error too."""
    src, q, tgt = clustered_small(4000, 1500, seed=8)
    Rm, _ = np.linalg.qr(np.random.default_rng(2).normal(size=(3, 3)))
    _, psi, _ = solve(src, q, tgt, p=28)
    _, psi_r, _ = solve(src @ Rm.T, q, tgt @ Rm.T, p=28)
    assert rel(psi_r, psi) < TOL


@pytest.mark.slow
def test_clustered_sky_million_sampled():
    """1e6 clustered sources -> 3,145,728 grid targets; oracle on a seeded
    subsample of targets (the launch configuration of the benchmark)."""
    d = workloads.clustered_sky()
    plan, psi, alpha = solve(d["src"], d["q"], d["tgt"], p=32, leaf=32)
    idx = workloads.subsample(d["tgt"].shape[0], 512, 2)
    check_against_oracle(d["src"], d["q"], d["tgt"], psi, alpha, idx=idx)
