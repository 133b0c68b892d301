"""GPU parity of the all-FP32 path (SFMM_FP32) against the oracle.

This path runs the expansions, the translations (M2L on the tensor cores as
split-BF16 products) and the near-field pair loop in FP32, keeping FP64 only
for the recentring and the final psi sum.  Its error has a floor near
eps_f32 Q / |alpha| where the near and far fields nearly cancel (targets in
smooth or empty sky; up to ~1.2e-5 on a uniform sky), so its stated error is
3e-5; on the skies below, where the targets follow the mass, it stays under
1e-6, which is what these tests check (norm-wise relative error of psi and
alpha, the reading of the paper's relative error used throughout the tests)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.direct import direct_sum
from paper_2210_07021_gb300 import sfmm, workloads
from conftest import unit

TOL_FP32 = 1e-6


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def solve(src, q, tgt, precision, p=20, leaf=32, **kw):
    plan = sfmm.Plan(p=p, leaf_size=leaf, precision=precision, **kw)
    qd = torch.float32 if kw.get("q_f32") else torch.float64
    psi, alpha = plan.deflection(dev(src), dev(q, qd), dev(tgt))
    torch.cuda.synchronize()
    return plan, psi.cpu().numpy(), alpha.cpu().numpy()


def test_random_sky_fp32():
    d = workloads.random_sky(4096)
    _, psi, alpha = solve(d["src"], d["q"], d["tgt"], sfmm.SFMM_FP32)
    ref = direct_sum(d["src"], d["q"], d["tgt"])
    assert rel(psi, ref["psi"]) < TOL_FP32 and rel(alpha, ref["alpha"]) < TOL_FP32, \
        (rel(psi, ref["psi"]), rel(alpha, ref["alpha"]))


def test_clustered_fp32_and_same_lists_as_fp64():
    rng = np.random.default_rng(4)
    clumps = workloads.clump_set(rng, 30)
    src = workloads.clustered(rng, 60000, 30, clumps=clumps)
    tgt = workloads.clustered(rng, 20001, 30, clumps=clumps)
    q = rng.lognormal(0, 0.5, 60000)
    pm, psi_m, al_m = solve(src, q, tgt, sfmm.SFMM_FP32, leaf=32)
    pd, psi_d, al_d = solve(src, q, tgt, sfmm.SFMM_FP64, p=32, leaf=32)
    assert np.array_equal(pm.debug(sfmm.ARR_M2L, np.int32, 2), pd.debug(sfmm.ARR_M2L, np.int32, 2))
    assert np.array_equal(pm.debug(sfmm.ARR_P2P, np.int32, 2), pd.debug(sfmm.ARR_P2P, np.int32, 2))
    idx = workloads.subsample(tgt.shape[0], 800, 4)
    ref = direct_sum(src, q, tgt[idx])
    assert rel(psi_m[idx], ref["psi"]) < TOL_FP32 and rel(al_m[idx], ref["alpha"]) < TOL_FP32, \
        (rel(psi_m[idx], ref["psi"]), rel(al_m[idx], ref["alpha"]))
    # and against the FP64 path on every target
    assert rel(psi_m, psi_d) < TOL_FP32 and rel(al_m, al_d) < TOL_FP32


def test_fp32_coincident_points_and_poles():
    rng = np.random.default_rng(9)
    base = unit(np.array([0.1, 0.2, 0.97]))
    src = np.vstack([np.repeat(base[None], 50, 0), unit(base + 1e-9 * rng.normal(size=(50, 3))),
                     [[0, 0, 1.0], [0, 0, -1.0]], unit(rng.normal(size=(4000, 3)))])
    q = rng.random(len(src)) + 0.5
    tgt = np.vstack([src[:60], [[0, 0, 1.0], [0, 0, -1.0]], unit(rng.normal(size=(1000, 3)))])
    _, psi, alpha = solve(src, q, tgt, sfmm.SFMM_FP32, leaf=8)
    ref = direct_sum(src, q, tgt)
    assert rel(psi, ref["psi"]) < TOL_FP32 and rel(alpha, ref["alpha"]) < TOL_FP32


def test_fp32_targets_are_the_sources_same_or_copied_array():
    """Targets that are the sources: passed as the very same array the pair loop
    tests every pair for d = 0; passed as a copy it finds each target's own
    source by the non-finite block sum and sums that block again.  Both agree
    with each other and with the oracle (which leaves out d = 0)."""
    d = workloads.random_sky(4096, config_index=11)
    plan = sfmm.Plan(p=20, leaf_size=32, precision=sfmm.SFMM_FP32, c_s=1.3)
    x, q = dev(d["src"]), dev(d["q"])
    psi_s, al_s = plan.deflection(x, q, x)
    psi_c, al_c = plan.deflection(x, q, x.clone())
    torch.cuda.synchronize()
    psi_s, al_s, psi_c, al_c = (t.cpu().numpy() for t in (psi_s, al_s, psi_c, al_c))
    assert np.all(np.isfinite(psi_c)) and np.all(np.isfinite(al_c))
    assert rel(psi_s, psi_c) < 1e-12 and rel(al_s, al_c) < 1e-12
    ref = direct_sum(d["src"], d["q"], d["src"])
    for psi, al in ((psi_s, al_s), (psi_c, al_c)):
        assert rel(psi, ref["psi"]) < TOL_FP32 and rel(al, ref["alpha"]) < TOL_FP32


def test_fp32_float32_masses_zero_mean():
    rng = np.random.default_rng(10)
    src = workloads.clustered(rng, 30000, 20)
    tgt = unit(rng.normal(size=(5000, 3)))
    q = np.full(30000, 4 * np.pi / 30000, dtype=np.float32)
    _, psi, alpha = solve(src, q, tgt, sfmm.SFMM_FP32, q_f32=True, zero_mean=True)
    ref = direct_sum(src, q.astype(np.float64), tgt)
    assert rel(psi, ref["psi"] + q.astype(np.float64).sum() / (4 * np.pi)) < TOL_FP32
    assert rel(alpha, ref["alpha"]) < TOL_FP32


@pytest.mark.parametrize("p", [6, 12, 16, 20, 24, 27, 32])
def test_tensor_core_m2l_matches_warp_kernel(p):
    """The tcgen05 M2L (split-BF16 GEMMs, FP32 accumulation) and the FP32 warp
    kernel produce the same local expansions and results to FP32 accuracy."""
    rng = np.random.default_rng(p)
    src = workloads.clustered(rng, 40000, 25)
    tgt = unit(rng.normal(size=(20000, 3)))
    q = rng.lognormal(0, 0.5, 40000)
    pt, psi_t, al_t = solve(src, q, tgt, sfmm.SFMM_FP32, p=p, m2l_tensor_cores=True)
    pw, psi_w, al_w = solve(src, q, tgt, sfmm.SFMM_FP32, p=p, m2l_tensor_cores=False)
    lt = pt.debug(sfmm.ARR_LOCAL, np.float64, 2 * p + 2)
    lw = pw.debug(sfmm.ARR_LOCAL, np.float64, 2 * p + 2)
    r = pt.debug(sfmm.ARR_NODE_GEOM, np.float64, 11)[:, 10]
    ell = np.arange(1, p + 1)
    st = (lt[:, 2::2] + 1j * lt[:, 3::2]) * r[:, None] ** ell      # scaled coefficients, O(1)
    sw = (lw[:, 2::2] + 1j * lw[:, 3::2]) * r[:, None] ** ell
    scale = np.abs(sw).max()
    assert np.abs(st - sw).max() < 2e-5 * scale
    assert np.abs(lt[:, :2] - lw[:, :2]).max() < 2e-5 * np.abs(lw[:, :2]).max()
    assert rel(psi_t, psi_w) < 1e-6 and rel(al_t, al_w) < 1e-6
    if p >= 16:   # at p = 12 the truncation error of this sky is above 1e-6 for both paths
        ref = direct_sum(src, q, tgt[:2000])
        assert rel(psi_t[:2000], ref["psi"]) < TOL_FP32 and rel(al_t[:2000], ref["alpha"]) < TOL_FP32


def test_fp32_host_entry_point_matches_device_and_survives_empty_calls():
    """The host-array entry point (targets copied on the auxiliary stream while
    the sources are copied and sorted) gives the device path's results bit for
    bit, also after calls that return early (no sources; no targets)."""
    rng = np.random.default_rng(31)
    clumps = workloads.clump_set(rng, 20)
    src = workloads.clustered(rng, 50000, 20, clumps=clumps)
    tgt = workloads.clustered(rng, 30001, 20, clumps=clumps)
    q = np.full(50000, 4 * np.pi / 50000, dtype=np.float32)
    plan = sfmm.Plan(p=20, leaf_size=64, c_s=1.3, precision=sfmm.SFMM_FP32, q_f32=True)
    psi, alpha = plan.deflection(dev(src), dev(q, torch.float32), dev(tgt))
    torch.cuda.synchronize()
    psi, alpha = psi.cpu().numpy(), alpha.cpu().numpy()
    e_psi, e_al = plan.deflection_host(np.zeros((0, 3)), np.zeros(0, dtype=np.float32), tgt)
    assert np.all(e_psi == 0) and np.all(e_al == 0)
    plan.deflection_host(src, q, np.zeros((0, 3)))
    for _ in range(2):
        hpsi, halpha = plan.deflection_host(src, q, tgt)
        np.testing.assert_array_equal(hpsi, psi)
        np.testing.assert_array_equal(halpha, alpha)


def test_tensor_core_wait_time_out_is_reported_and_the_plan_recovers():
    """The tensor-core M2L's mbarrier waits are bounded.  With a limit of one
    non-blocking poll they run out: the solve returns SFMM_ETIMEOUT (the kernel
    drains its MMAs with the full bound and frees its tensor memory, so the
    context stays usable), and the same plan with the default bound then solves
    correctly."""
    rng = np.random.default_rng(77)
    src = workloads.clustered(rng, 40000, 25)
    tgt = unit(rng.normal(size=(5000, 3)))
    q = rng.lognormal(0, 0.5, 40000)
    plan = sfmm.Plan(p=20, leaf_size=32, precision=sfmm.SFMM_FP32)
    plan.set_wait_limit(1)
    for _ in range(2):
        with pytest.raises(sfmm.SfmmError, match=f"status {sfmm.SFMM_ETIMEOUT}:"):
            plan.deflection(dev(src), dev(q), dev(tgt))
    plan.set_wait_limit(0)
    psi, alpha = plan.deflection(dev(src), dev(q), dev(tgt))
    torch.cuda.synchronize()
    ref = direct_sum(src, q, tgt[:1000])
    assert rel(psi.cpu().numpy()[:1000], ref["psi"]) < TOL_FP32
    assert rel(alpha.cpu().numpy()[:1000], ref["alpha"]) < TOL_FP32
