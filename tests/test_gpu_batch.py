"""Batched shells (sfmm_deflection_batch) and the autotuner.

Each shell of a batch must give exactly what a single solve with the same
settings gives (the FP64 kernels are deterministic), whichever lane solves it;
empty shells are allowed; the autotuner's choice meets its stated error."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.direct import direct_sum
from paper_2210_07021_gb300 import sfmm, tune, workloads
from conftest import unit


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def shells(seed, sizes):
    rng = np.random.default_rng(seed)
    out = []
    for n, m in sizes:
        src = workloads.clustered(rng, n, max(1, n // 500)) if n > 1000 else unit(rng.normal(size=(n, 3)))
        tgt = unit(rng.normal(size=(m, 3)))
        q = rng.lognormal(0, 0.5, n)
        out.append((src, q, tgt))
    return out


@pytest.mark.parametrize("lanes", [1, 3])
def test_batch_equals_single_solves_fp64(lanes):
    sh = shells(41, [(20000, 3000), (500, 100), (0, 50), (60000, 4000), (7000, 0), (3000, 2000)])
    plan = sfmm.Plan(p=24, leaf_size=32)
    outs = plan.deflection_batch([(dev(s), dev(q), dev(t)) for s, q, t in sh], lanes=lanes)
    torch.cuda.synchronize()
    single = sfmm.Plan(p=24, leaf_size=32)
    for (s, q, t), (psi, alpha) in zip(sh, outs):
        p1, a1 = single.deflection(dev(s), dev(q), dev(t))
        assert np.array_equal(psi.cpu().numpy(), p1.cpu().numpy())
        assert np.array_equal(alpha.cpu().numpy(), a1.cpu().numpy())
    s, q, t = sh[3]
    ref = direct_sum(s, q, t[:500])
    assert rel(outs[3][1].cpu().numpy()[:500], ref["alpha"]) < 1e-9


def test_batch_mixed_without_psi():
    sh = shells(42, [(30000, 5000), (8000, 3000), (15000, 1000)])
    plan = sfmm.Plan(p=16, leaf_size=64, precision=sfmm.SFMM_MIXED)
    outs = plan.deflection_batch([(dev(s), dev(q), dev(t)) for s, q, t in sh], with_psi=False, lanes=2)
    torch.cuda.synchronize()
    for (s, q, t), (psi, alpha) in zip(sh, outs):
        assert psi is None
        ref = direct_sum(s, q, t[:400])
        assert rel(alpha.cpu().numpy()[:400], ref["alpha"]) < 1e-6


def test_autotune_meets_its_stated_error():
    rng = np.random.default_rng(43)
    clumps = workloads.clump_set(rng, 40)
    src = workloads.clustered(rng, 200000, 40, clumps=clumps)
    tgt = workloads.clustered(rng, 100000, 40, clumps=clumps)
    q = np.full(200000, 4 * np.pi / 200000)
    r = tune.autotune(dev(src), dev(q), dev(tgt), sfmm.SFMM_MIXED, 1e-6, sample=500)
    assert all(row["ms"] > 0 for row in r["table"])
    plan = sfmm.Plan(precision=sfmm.SFMM_MIXED, **r["best"])
    psi, alpha = plan.deflection(dev(src), dev(q), dev(tgt))
    idx = workloads.subsample(tgt.shape[0], 300, 43)
    ref = direct_sum(src, q, tgt[idx])
    assert rel(alpha.cpu().numpy()[idx], ref["alpha"]) < 1e-6 and rel(psi.cpu().numpy()[idx], ref["psi"]) < 1e-6


def test_autotune_falls_back_to_a_format_that_reaches_the_target():
    """A target below the FP32 path's reach (1e-9): its candidates all fail, the
    double-float fallback is tuned instead and its choice meets the target."""
    rng = np.random.default_rng(44)
    clumps = workloads.clump_set(rng, 20)
    src = workloads.clustered(rng, 60000, 20, clumps=clumps)
    tgt = workloads.clustered(rng, 30000, 20, clumps=clumps)
    q = np.full(60000, 4 * np.pi / 60000)
    r = tune.autotune(dev(src), dev(q), dev(tgt), sfmm.SFMM_MIXED, 1e-9, sample=300,
                      candidates=[dict(p=20, leaf_size=64, c_s=1.3, c_t=0.5)], fallback=sfmm.SFMM_MIXED_DF,
                      fallback_candidates=[dict(p=28, leaf_size=64, c_s=2.0, c_t=0.45)])
    assert r["precision"] == sfmm.SFMM_MIXED_DF
    assert [row["precision"] for row in r["table"]] == [sfmm.SFMM_MIXED, sfmm.SFMM_MIXED_DF]
    assert not r["table"][0]["ok"] and r["table"][1]["ok"]
    plan = sfmm.Plan(precision=r["precision"], **r["best"])
    psi, alpha = plan.deflection(dev(src), dev(q), dev(tgt))
    idx = workloads.subsample(tgt.shape[0], 200, 44)
    ref = direct_sum(src, q, tgt[idx])
    assert rel(alpha.cpu().numpy()[idx], ref["alpha"]) < 1e-9 and rel(psi.cpu().numpy()[idx], ref["psi"]) < 1e-9
