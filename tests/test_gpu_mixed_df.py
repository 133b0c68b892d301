"""GPU parity of the double-float path (SFMM_MIXED_DF) against the oracle.

This path keeps the expansions and every translation in FP64 and runs the
near-field pair loop in double-float arithmetic (unevaluated sums of two
float32 numbers) on the FP32 pipe; its stated error is 1e-10, the norm-wise
relative error of psi and alpha used throughout the tests.  The masses enter
the pair loop as (hi, lo) pairs, so float64 masses that float32 cannot hold
keep their precision (the lognormal masses below would show a dropped low part
at the 1e-8 level)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.direct import direct_sum
from paper_2210_07021_gb300 import sfmm, workloads
from conftest import unit

TOL_DF = 1e-10


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def solve(src, q, tgt, precision=sfmm.SFMM_MIXED_DF, p=32, leaf=32, **kw):
    plan = sfmm.Plan(p=p, leaf_size=leaf, precision=precision, **kw)
    qd = torch.float32 if kw.get("q_f32") else torch.float64
    psi, alpha = plan.deflection(dev(src), dev(q, qd), dev(tgt))
    torch.cuda.synchronize()
    return plan, psi.cpu().numpy(), alpha.cpu().numpy()


def check(psi, alpha, ref):
    e_psi, e_al = rel(psi, ref["psi"]), rel(alpha, ref["alpha"])
    assert e_psi < TOL_DF and e_al < TOL_DF, (e_psi, e_al)


def test_random_sky_df():
    d = workloads.random_sky(4096)
    _, psi, alpha = solve(d["src"], d["q"], d["tgt"])
    check(psi, alpha, direct_sum(d["src"], d["q"], d["tgt"]))


def test_clustered_df_float64_masses_and_same_lists_as_fp64():
    rng = np.random.default_rng(14)
    clumps = workloads.clump_set(rng, 30)
    src = workloads.clustered(rng, 60000, 30, clumps=clumps)
    tgt = workloads.clustered(rng, 20001, 30, clumps=clumps)
    q = rng.lognormal(0, 0.5, 60000)
    pm, psi_m, al_m = solve(src, q, tgt)
    pd, psi_d, al_d = solve(src, q, tgt, precision=sfmm.SFMM_FP64)
    assert np.array_equal(pm.debug(sfmm.ARR_M2L, np.int32, 2), pd.debug(sfmm.ARR_M2L, np.int32, 2))
    assert np.array_equal(pm.debug(sfmm.ARR_P2P, np.int32, 2), pd.debug(sfmm.ARR_P2P, np.int32, 2))
    idx = workloads.subsample(tgt.shape[0], 800, 14)
    check(psi_m[idx], al_m[idx], direct_sum(src, q, tgt[idx]))
    # the far field is the FP64 path's own: the two differ only in the near field
    assert rel(psi_m, psi_d) < TOL_DF and rel(al_m, al_d) < TOL_DF


def test_df_coincident_points_and_poles():
    rng = np.random.default_rng(19)
    base = unit(np.array([0.1, 0.2, 0.97]))
    src = np.vstack([np.repeat(base[None], 50, 0), unit(base + 1e-9 * rng.normal(size=(50, 3))),
                     [[0, 0, 1.0], [0, 0, -1.0]], unit(rng.normal(size=(4000, 3)))])
    q = rng.random(len(src)) + 0.5
    tgt = np.vstack([src[:60], src[50:100], [[0, 0, 1.0], [0, 0, -1.0]], unit(rng.normal(size=(1000, 3)))])
    _, psi, alpha = solve(src, q, tgt, leaf=8)
    check(psi, alpha, direct_sum(src, q, tgt))


def test_df_equal_masses_product_logarithm():
    """Equal masses take the product form of sum q log d^2 (one logarithm per
    block of sources): targets on the sources themselves (coincident pairs
    skipped), duplicates, a clump 1e-9 rad wide (d^2 near 1e-18, products of
    many small mantissas and exponents) and the poles, against the oracle."""
    rng = np.random.default_rng(29)
    base = unit(np.array([-0.4, 0.7, 0.2]))
    src = np.vstack([np.repeat(base[None], 20, 0), unit(base + 1e-9 * rng.normal(size=(60, 3))),
                     [[0, 0, 1.0], [0, 0, -1.0]], workloads.clustered(rng, 20000, 40)])
    q = np.full(len(src), 4 * np.pi / len(src))
    _, psi, alpha = solve(src, q, src, leaf=16)
    ref = direct_sum(src, q, src)
    check(psi, alpha, ref)
    idx = np.arange(100)           # the duplicates and the tight clump, pointwise
    na = np.linalg.norm(ref["alpha"][idx], axis=1)
    assert (np.linalg.norm(alpha[idx] - ref["alpha"][idx], axis=1) <= 1e-10 * na.max()).all()


def test_df_without_psi_odd_stages_and_both_mass_forms():
    """The near field without psi (no logarithm, the PSI = false kernels) gives
    the alpha of the solve with psi.  The sources sit in clumps of odd sizes, so
    stages of odd counts (a massless partner in the packed loop's last pair) meet
    both mass forms: equal masses (the product logarithm) and lognormal ones."""
    rng = np.random.default_rng(19)
    centres = unit(rng.normal(size=(37, 3)))
    sizes = rng.integers(1, 40, size=37) * 2 + 1
    src = unit(np.concatenate([c + 2e-3 * rng.normal(size=(k, 3)) for c, k in zip(centres, sizes)]))
    tgt = unit(np.concatenate([src[::7] + 1e-4 * rng.normal(size=(len(src[::7]), 3)), rng.normal(size=(3001, 3))]))
    for q in (np.full(len(src), 4 * np.pi / len(src)), rng.lognormal(0.0, 0.5, len(src))):
        plan = sfmm.Plan(p=32, leaf_size=32, precision=sfmm.SFMM_MIXED_DF)
        psi, alpha = plan.deflection(dev(src), dev(q), dev(tgt))
        none, alpha2 = plan.deflection(dev(src), dev(q), dev(tgt), with_psi=False)
        torch.cuda.synchronize()
        assert none is None
        a1, a2 = alpha.cpu().numpy(), alpha2.cpu().numpy()
        # the far field reaches each box through FP64 atomic additions: equal to their rounding
        assert rel(a2, a1) < 1e-13
        ref = direct_sum(src, q, tgt)
        check(psi.cpu().numpy(), a1, ref)
        assert rel(a2, ref["alpha"]) < TOL_DF


def test_df_log_and_reciprocal_over_the_exponent_range():
    """One source, targets from 1e-4 to pi away: every pair in the near field of
    the source's leaf runs the table-driven double-float logarithm and the
    Newton-corrected reciprocal over d^2 from 1e-8 to 4; each target is checked
    on its own."""
    rng = np.random.default_rng(23)
    y = unit(np.array([0.3, -0.5, 0.8]))
    e1 = unit(np.cross(y, [0.0, 0.0, 1.0]))
    e2 = np.cross(y, e1)
    th = np.concatenate([10.0 ** rng.uniform(-4, 0, 400), rng.uniform(1, np.pi, 200), [np.pi]])
    ph = rng.uniform(0, 2 * np.pi, th.size)
    tgt = unit(np.cos(th)[:, None] * y + np.sin(th)[:, None] * (np.cos(ph)[:, None] * e1 + np.sin(ph)[:, None] * e2))
    q = np.array([1.3])
    _, psi, alpha = solve(y[None], q, tgt)
    ref = direct_sum(y[None], q, tgt)
    check(psi, alpha, ref)
    near = th < 1.0          # inside the MAC radius of the source's base box: P2P only
    assert np.abs(psi - ref["psi"])[near].max() < 1e-12 * q[0]
    na = np.linalg.norm(ref["alpha"], axis=1)
    assert (np.linalg.norm(alpha - ref["alpha"], axis=1) <= 1e-10 * na + 1e-14)[near].all()


def test_df_float32_masses_zero_mean_and_ragged_sizes():
    rng = np.random.default_rng(20)
    for n, m in ((1, 1), (33, 7), (30000, 5000)):
        src = workloads.clustered(rng, n, 20) if n > 100 else unit(rng.normal(size=(n, 3)))
        tgt = unit(rng.normal(size=(m, 3)))
        q = np.full(n, 4 * np.pi / n, dtype=np.float32)
        _, psi, alpha = solve(src, q, tgt, q_f32=True, zero_mean=True)
        ref = direct_sum(src, q.astype(np.float64), tgt)
        assert rel(psi, ref["psi"] + q.astype(np.float64).sum() / (4 * np.pi)) < TOL_DF
        assert rel(alpha, ref["alpha"]) < TOL_DF


def test_df_empty():
    plan = sfmm.Plan(p=16, precision=sfmm.SFMM_MIXED_DF)
    psi, alpha = plan.deflection(dev(np.zeros((0, 3))), dev(np.zeros(0)), dev(unit(np.ones((3, 3)))))
    torch.cuda.synchronize()
    assert np.all(psi.cpu().numpy() == 0) and np.all(alpha.cpu().numpy() == 0)


@pytest.mark.parametrize("p", [8, 26, 32])
def test_df_multipoles_match_fp64(p):
    """The double-float P2M (from (hi, lo) offsets, table logarithm) and M2M give
    the FP64 path's multipoles to double-float accuracy, node by node."""
    rng = np.random.default_rng(30 + p)
    src = workloads.clustered(rng, 50000, 25)
    tgt = unit(rng.normal(size=(2000, 3)))
    q = rng.lognormal(0, 0.5, 50000)
    pm, _, _ = solve(src, q, tgt, p=p, leaf=64)
    pd, _, _ = solve(src, q, tgt, precision=sfmm.SFMM_FP64, p=p, leaf=64)
    m_df = pm.debug(sfmm.ARR_MULTIPOLE, np.float64, 2 * p + 2)
    m_64 = pd.debug(sfmm.ARR_MULTIPOLE, np.float64, 2 * p + 2)
    r = pd.debug(sfmm.ARR_NODE_GEOM, np.float64, 11)[:, 10]
    ell = np.arange(1, p + 1)
    # compare the scaled coefficients A_l / r^l, which are O(|Q|) at every level
    s_df = (m_df[:, 2::2] + 1j * m_df[:, 3::2]) / r[:, None] ** ell
    s_64 = (m_64[:, 2::2] + 1j * m_64[:, 3::2]) / r[:, None] ** ell
    scale = np.abs(m_64[:, 1]).max()
    assert np.abs(s_df - s_64).max() < 1e-12 * scale
    assert np.abs(m_df[:, :2] - m_64[:, :2]).max() < 1e-12 * np.abs(m_64[:, :2]).max()
