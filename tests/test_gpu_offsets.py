"""The (hi, lo) FP32 offsets of the reduced-precision paths, formed on the GPU
without FP64 instructions (an exact integer difference of the FP64 mantissas,
split into two floats), against the FP64 data: every sorted source's offset
from its leaf centre and its mass, every sorted target's offset from its leaf
centre, to 2^-47 relative (the 48 bits a float pair carries)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2210_07021_gb300 import sfmm, workloads
from conftest import unit

REL = 2.0 ** -46          # 2^-47 of the split, with room for the reference's own rounding


def points(rng):
    """Clustered points plus coordinates of every scale: exact zeros (great
    circles), the poles, coordinates of 1e-20 to 1e-3, near-duplicates."""
    base = workloads.clustered(rng, 40000, 20)
    eq = unit(np.c_[rng.normal(size=(300, 2)), np.zeros(300)])                    # z = 0 exactly
    tiny = unit(np.c_[10.0 ** rng.uniform(-20, -3, 300), rng.normal(size=(300, 2))])
    poles = np.array([[0.0, 0.0, 1.0], [0.0, 0.0, -1.0], [1.0, 0.0, 0.0], [0.0, -1.0, 0.0]])
    dup = unit(base[:200] + 1e-12 * rng.normal(size=(200, 3)))
    return np.vstack([base, eq, tiny, poles, dup])


def check_split(hi, lo, exact, what):
    got = hi.astype(np.longdouble) + lo.astype(np.longdouble)
    err = np.abs(got - exact)
    bound = REL * np.abs(exact) + 2.0 ** -126
    bad = np.nonzero(err > bound)[0]
    assert bad.size == 0, (what, bad[:5], err[bad[:5]], exact[bad[:5]])
    # lo is the rounding remainder of hi
    assert np.all(np.abs(lo) <= np.abs(hi) * 2.0 ** -24 * (1 + 1e-6)), what


@pytest.mark.parametrize("precision", [sfmm.SFMM_MIXED, sfmm.SFMM_MIXED_DF])
def test_source_and_target_offsets_exact_to_48_bits(precision):
    rng = np.random.default_rng(41)
    src = points(rng)
    tgt = points(np.random.default_rng(42))
    q = rng.lognormal(0, 0.5, src.shape[0])
    plan = sfmm.Plan(p=12, leaf_size=32, precision=precision)
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")
    plan.deflection(dev(src), dev(q), dev(tgt))
    torch.cuda.synchronize()
    geom = plan.debug(sfmm.ARR_NODE_GEOM, np.float64, 11)
    child0 = plan.debug(sfmm.ARR_NODE_CHILD0, np.int32)
    rng_s = plan.debug(sfmm.ARR_NODE_RANGE, np.int32, 2)
    rng_t = plan.debug(sfmm.ARR_NODE_TRANGE, np.int32, 2)
    perm = plan.debug(sfmm.ARR_SRC_PERM, np.int32)
    soff = plan.debug(sfmm.ARR_SRC_OFFSETS, np.float32, 8)
    toff = plan.debug(sfmm.ARR_TGT_OFFSETS, np.float32, 8)
    assert soff.shape == (src.shape[0], 8) and toff.shape == (tgt.shape[0], 8)
    leaf = child0 < 0
    # the sorted sources' leaf centres
    cs = np.full((src.shape[0], 3), np.nan)
    for n in np.nonzero(leaf & (rng_s[:, 1] > 0))[0]:
        f, c = rng_s[n]
        cs[f:f + c] = geom[n, :3]
    assert not np.isnan(cs).any()
    xs = src[perm].astype(np.longdouble)
    for k in range(3):
        check_split(soff[:, k], soff[:, 4 + k], xs[:, k] - cs[:, k].astype(np.longdouble), f"source {k}")
    check_split(soff[:, 3], soff[:, 7], q[perm].astype(np.longdouble), "mass")
    # the sorted targets: the original targets ordered by their keys (a stable sort)
    tkeys = plan.debug(sfmm.ARR_TGT_KEYS, np.uint64)
    own_keys = sfmm.keys(dev(tgt)).cpu().numpy().view(np.uint64)
    order = np.argsort(own_keys, kind="stable")
    assert np.array_equal(own_keys[order], tkeys)
    ct = np.full((tgt.shape[0], 3), np.nan)
    for n in np.nonzero(leaf & (rng_t[:, 1] > 0))[0]:
        f, c = rng_t[n]
        ct[f:f + c] = geom[n, :3]
    assert not np.isnan(ct).any()
    xt = tgt[order].astype(np.longdouble)
    for k in range(3):
        check_split(toff[:, k], toff[:, 4 + k], xt[:, k] - ct[:, k].astype(np.longdouble), f"target {k}")
    assert np.all(toff[:, 3] == 0) and np.all(toff[:, 7] == 0)


def test_offsets_absent_on_the_fp64_path():
    plan = sfmm.Plan(p=8, precision=sfmm.SFMM_FP64)
    x = torch.as_tensor(unit(np.random.default_rng(1).normal(size=(500, 3))), device="cuda")
    plan.deflection(x, torch.ones(500, dtype=torch.float64, device="cuda"), x)
    torch.cuda.synchronize()
    assert plan.debug(sfmm.ARR_SRC_OFFSETS, np.float32).size == 0
