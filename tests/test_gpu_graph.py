"""Graph-launched shells (sfmm_graph_capture / sfmm_graph_launch): the solves
of a batch of shells recorded into one CUDA graph with no host
synchronisation inside, replayed, and checked against per-shell synchronised
solves of the same plan settings and against the oracle.

Two solves of the same shell need not be bit-identical: the M2L sums reach
each target box through FP64 atomic additions, whose order varies from run to
run.  So the graph's results are held to the agreement of two synchronised
solves with each other (measured here, a few ulps of FP64 on the far field)
with a bound of 1e-12 of the largest deflection, and to the stated error
against the oracle.  The overflow path (a shell whose new data outgrows the
capacities planned at capture) is driven by replacing a uniform shell's data
with a much more clustered one."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.direct import direct_sum
from paper_2210_07021_gb300 import sfmm, workloads
from conftest import unit

SET = dict(p=20, leaf_size=64, c_s=1.5, c_t=0.5)
AGREE = 1e-12          # graph vs per-shell solve, relative to the largest |alpha| of the shell


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def shell_data(seed, n, m, clumps):
    rng = np.random.default_rng(seed)
    src = workloads.clustered(rng, n, clumps) if clumps else unit(rng.normal(size=(n, 3)))
    tgt = unit(rng.normal(size=(m, 3)))
    q = rng.lognormal(0.0, 0.5, n)
    return src, q, tgt


def per_shell(shells, precision=sfmm.SFMM_MIXED, **kw):
    plan = sfmm.Plan(precision=precision, **(kw or SET))
    out = []
    for src, q, tgt in shells:
        psi, alpha = plan.deflection(src, q, tgt)
        out.append((psi.clone(), alpha.clone()))
    torch.cuda.synchronize()
    plan.close()
    return out


def max_rel(a, b):
    return float((a - b).abs().max() / b.abs().max().clamp_min(1e-300))


def assert_agree(got, ref, tol=AGREE):
    worst = 0.0
    for (gp, ga), (rp, ra) in zip(got, ref):
        if ra.numel() == 0:
            continue
        worst = max(worst, max_rel(ga, ra))
        if gp is not None:
            worst = max(worst, max_rel(gp, rp))
    assert worst < tol, worst
    return worst


def make_shells(specs):
    host = [shell_data(*s) for s in specs]
    return host, [(dev(s), dev(q), dev(t)) for s, q, t in host]


SPECS = [(1, 200_000, 50_000, 400), (2, 3_000, 4_000, 6), (3, 60_000, 30_000, 120), (4, 20_000, 20_000, 0),
         (5, 120_000, 10_000, 240)]


def test_graph_matches_per_shell_solves_and_oracle():
    host, sh = make_shells(SPECS)
    plan = sfmm.Plan(precision=sfmm.SFMM_MIXED, **SET)
    outs = plan.graph_capture(sh, with_psi=True)
    ref = per_shell(sh)
    # two synchronised solves agree to FP64 atomic-order rounding; the graph as closely
    base = assert_agree(per_shell(sh), ref)
    assert_agree(outs, ref)
    for rep in range(3):
        for _, a in outs:
            a.fill_(np.nan)
        plan.graph_launch()
        torch.cuda.synchronize()
        worst = assert_agree(outs, ref)
    info = plan.graph_info()
    assert info["n_shells"] == len(SPECS) and info["launches"] == 3
    assert info["overflows"] == 0 and info["recaptures"] == 0
    assert info["kernel_nodes"] > 20 * len(SPECS)
    stats_nodes = info["n_nodes"]
    assert stats_nodes > 0 and info["n_m2l"] > 0 and info["n_p2p"] > 0
    # the stated 1e-6 against the oracle on every shell (a target sample of each)
    for k, ((src, q, tgt), (psi, alpha)) in enumerate(zip(host, outs)):
        idx = workloads.subsample(tgt.shape[0], 300, 5, stream=k)
        r = direct_sum(src, q, tgt[idx])
        a = alpha.cpu().numpy()[idx]
        p = psi.cpu().numpy()[idx]
        ea = np.linalg.norm(a - r["alpha"]) / np.linalg.norm(r["alpha"])
        ep = np.linalg.norm(p - r["psi"]) / np.linalg.norm(r["psi"])
        assert ea < 1e-6 and ep < 1e-6, (k, ea, ep)
    print(f"graph vs per-shell {worst:.2e} (two per-shell solves {base:.2e}), {info}")
    plan.close()


def test_new_data_in_place_and_overflow_recapture():
    """New data of the same sizes written into the bound tensors: the replay
    solves it.  Then a shell's uniform sky replaced by one tight clump (a far
    deeper tree than the capacities allow): the replay detects the overflow on
    the device, the launch re-solves that shell synchronously and records the
    graph again, and the next replay needs no fallback."""
    specs = [(11, 50_000, 20_000, 100), (12, 40_000, 20_000, 0), (13, 8_000, 5_000, 16)]
    host, sh = make_shells(specs)
    plan = sfmm.Plan(precision=sfmm.SFMM_MIXED, **SET)
    outs = plan.graph_capture(sh, with_psi=False, slack=0.1)
    # same distributions, new draws
    for (s, q, t), k in zip(sh, (21, 22, 23)):
        ns, nq, nt = shell_data(k, s.shape[0], t.shape[0], 100 if k != 22 else 0)
        s.copy_(dev(ns)); q.copy_(dev(nq)); t.copy_(dev(nt))
    plan.graph_launch()
    assert_agree(outs, per_shell(sh))
    # shell 1: uniform -> one clump of radius 1e-4 rad
    rng = np.random.default_rng(99)
    c = unit(rng.normal(size=3))
    tight = unit(c + 1e-4 * rng.normal(size=(sh[1][0].shape[0], 3)))
    sh[1][0].copy_(dev(tight))
    plan.graph_launch()
    info = plan.graph_info()
    assert info["overflows"] >= 1 and info["recaptures"] >= 1, info
    ref = per_shell(sh)
    assert_agree(outs, ref)
    plan.graph_launch()
    info2 = plan.graph_info()
    assert info2["overflows"] == info["overflows"] and info2["recaptures"] == info["recaptures"], (info, info2)
    assert_agree(outs, ref)
    plan.close()


def test_empty_shells_and_double_float_path():
    """Shells with no sources (psi = alpha = 0) and no targets inside a
    graph; the 1e-10 path (SFMM_MIXED_DF) through the graph."""
    host, sh = make_shells([(31, 30_000, 10_000, 60), (32, 5_000, 3_000, 10)])
    empty_src = (torch.zeros((0, 3), dtype=torch.float64, device="cuda"),
                 torch.zeros(0, dtype=torch.float64, device="cuda"), dev(unit(np.ones((7, 3)))))
    empty_tgt = (sh[0][0], sh[0][1], torch.zeros((0, 3), dtype=torch.float64, device="cuda"))
    batch = [sh[0], empty_src, sh[1], empty_tgt]
    kw = dict(p=32, leaf_size=64, c_s=1.5, c_t=0.45)
    plan = sfmm.Plan(precision=sfmm.SFMM_MIXED_DF, **kw)
    outs = plan.graph_capture(batch, with_psi=True)
    plan.graph_launch()
    ref = per_shell(batch, sfmm.SFMM_MIXED_DF, **kw)
    assert_agree([outs[0], outs[2]], [ref[0], ref[2]])
    assert torch.all(outs[1][1] == 0) and torch.all(outs[1][0] == 0)
    assert outs[3][1].shape == (0, 2)
    src, q, tgt = host[1]
    r = direct_sum(src, q, tgt)
    a = outs[2][1].cpu().numpy()
    assert np.linalg.norm(a - r["alpha"]) / np.linalg.norm(r["alpha"]) < 1e-10
    plan.close()


def test_fp64_graph_matches_per_shell_solves():
    """The FP64 path through the graph: the same results as per-shell FP64 solves
    (deterministic kernels, the same lists) and the oracle to 1e-10."""
    host, sh = make_shells([(51, 40_000, 8_000, 80), (52, 6_000, 3_000, 0), (53, 15_000, 5_000, 30)])
    kw = dict(p=32, leaf_size=32, c_s=1.5, c_t=0.45)       # the FP64 path's settings for 1e-10
    plan = sfmm.Plan(precision=sfmm.SFMM_FP64, **kw)
    outs = plan.graph_capture(sh, with_psi=True)
    plan.graph_launch()
    torch.cuda.synchronize()
    assert_agree(outs, per_shell(sh, sfmm.SFMM_FP64, **kw))
    for k, ((src, q, tgt), (psi, alpha)) in enumerate(zip(host, outs)):
        idx = workloads.subsample(tgt.shape[0], 300, 6, stream=k)
        r = direct_sum(src, q, tgt[idx])
        a = alpha.cpu().numpy()[idx]
        assert np.linalg.norm(a - r["alpha"]) / np.linalg.norm(r["alpha"]) < 1e-10, k
    plan.close()


def test_graph_refuses_fp32_and_release():
    sh = make_shells([(41, 2_000, 1_000, 4)])[1]
    plan = sfmm.Plan(precision=sfmm.SFMM_FP32, p=16)
    with pytest.raises(sfmm.SfmmError):
        plan.graph_capture(sh)
    assert plan.graph_info()["n_shells"] == 0
    plan.close()
    plan = sfmm.Plan(precision=sfmm.SFMM_MIXED, **SET)
    plan.graph_capture(sh)
    plan.graph_release()
    with pytest.raises(sfmm.SfmmError):
        plan.graph_launch()
    # the plan still solves on its own after the graph is gone
    psi, alpha = plan.deflection(*sh[0])
    torch.cuda.synchronize()
    assert torch.isfinite(alpha).all()
    plan.close()
