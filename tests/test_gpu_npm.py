"""GPU parity of the Near Particle Model (sfmm_options.sigma > 0; Secs. 3.2,
4.2) against the oracle's NPM direct sum and its walk with the sigma MAC
condition (both pinned in test_oracle_npm.py).  Stated error 1e-10."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle.healpix as hp
from oracle.direct import direct_sum
from oracle.walk import walk
from paper_2210_07021_gb300 import sfmm, workloads
from conftest import unit
from test_gpu_parity import gpu_tree

TOL = 1e-10


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def solve(src, q, tgt, sigma, p=32, leaf=32, **kw):
    plan = sfmm.Plan(p=p, leaf_size=leaf, sigma=sigma, **kw)
    psi, alpha = plan.deflection(dev(src), dev(q), dev(tgt))
    torch.cuda.synchronize()
    return plan, psi.cpu().numpy(), alpha.cpu().numpy()


def test_npm_random_sky_paper_sigma():
    """sigma = sqrt(4 pi / N), the paper's choice; targets = sources."""
    d = workloads.random_sky(4096)
    sigma = np.sqrt(4 * np.pi / 4096)
    _, psi, alpha = solve(d["src"], d["q"], d["tgt"], sigma)
    ref = direct_sum(d["src"], d["q"], d["tgt"], sigma=sigma)
    assert rel(psi, ref["psi"]) < TOL and rel(alpha, ref["alpha"]) < TOL, (rel(psi, ref["psi"]), rel(alpha, ref["alpha"]))
    # and it differs from the point-mass answer (pairs inside sigma exist)
    pt = direct_sum(d["src"], d["q"], d["tgt"])
    assert rel(alpha, pt["alpha"]) > 1e-6


def test_npm_clustered_and_lists_follow_the_sigma_mac():
    rng = np.random.default_rng(31)
    src = workloads.clustered(rng, 20000, 15)
    tgt = np.vstack([workloads.clustered(rng, 5000, 15), unit(rng.normal(size=(1000, 3)))])
    q = rng.lognormal(0, 0.5, 20000)
    sigma = 2e-3
    plan, psi, alpha = solve(src, q, tgt, sigma, leaf=16)
    idx = workloads.subsample(tgt.shape[0], 800, 31)
    ref = direct_sum(src, q, tgt[idx], sigma=sigma)
    assert rel(psi[idx], ref["psi"]) < TOL and rel(alpha[idx], ref["alpha"]) < TOL
    g = gpu_tree(plan)
    t = dict(level=g["level"], prefix=g["prefix"], first=g["rng"][:, 0], count=g["rng"][:, 1],
             parent=g["parent"], child0=g["child0"], is_leaf=g["child0"] < 0)
    cen = np.zeros((len(t["level"]), 3))
    rad = np.zeros(len(t["level"]))
    for lvl in np.unique(t["level"]):
        sel = t["level"] == lvl
        cen[sel] = hp.pix2vec_nest(int(lvl), t["prefix"][sel])
        rad[sel] = hp.covering_radius(int(lvl), t["prefix"][sel], per_edge=1) + 2e-15
    m2l_o, p2p_o = walk(t, cen, rad, tcount=g["trng"][:, 1], sigma=sigma)
    m2l = plan.debug(sfmm.ARR_M2L, np.int32, 2)
    p2p = plan.debug(sfmm.ARR_P2P, np.int32, 2)
    assert set(map(tuple, m2l.tolist())) == set(m2l_o)
    assert set(map(tuple, p2p.tolist())) == set(p2p_o)
    # every M2L pair keeps the particles' profiles out of the target box
    d = 2 * np.arcsin(np.minimum(1, np.linalg.norm(cen[m2l[:, 0]] - cen[m2l[:, 1]], axis=1) / 2))
    assert np.all(d - rad[m2l[:, 1]] - rad[m2l[:, 0]] > sigma)


def test_sigma_zero_is_the_point_mass_path_and_checks():
    rng = np.random.default_rng(32)
    src = unit(rng.normal(size=(3000, 3)))
    q = rng.lognormal(0, 0.5, 3000)
    tgt = unit(rng.normal(size=(2000, 3)))
    _, p0, a0 = solve(src, q, tgt, 0.0)
    plan = sfmm.Plan(p=32, leaf_size=32)
    p1, a1 = plan.deflection(dev(src), dev(q), dev(tgt))
    assert np.array_equal(p0, p1.cpu().numpy()) and np.array_equal(a0, a1.cpu().numpy())
    with pytest.raises(sfmm.SfmmError):
        sfmm.Plan(p=16, sigma=0.01, precision=sfmm.SFMM_MIXED)
    with pytest.raises(sfmm.SfmmError):
        sfmm.Plan(p=16, sigma=-1.0)
    plan = sfmm.Plan(p=16, sigma=0.01)
    with pytest.raises(sfmm.SfmmError):
        plan.shear(dev(src), dev(q), dev(tgt))
