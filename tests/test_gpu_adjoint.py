"""GPU parity of the adjoint sFMM (sfmm_adjoint) and its autograd wrapper
against the oracle's adjoint (pinned by finite differences of the forward
oracle in test_oracle_adjoint.py).  Stated error 1e-10, norm-wise."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.direct import adjoint as oracle_adjoint, direct_sum
from paper_2210_07021_gb300 import autograd as sfa
from paper_2210_07021_gb300 import sfmm, workloads
from conftest import unit

TOL = 1e-10


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def run(src, q, tgt, g_psi, g_alpha, p=32, leaf=32, **kw):
    plan = sfmm.Plan(p=p, leaf_size=leaf, **kw)
    qd = torch.float32 if kw.get("q_f32") else torch.float64
    gq, gs = plan.adjoint(dev(src), dev(q, qd), dev(tgt), g_psi=None if g_psi is None else dev(g_psi),
                          g_alpha=None if g_alpha is None else dev(g_alpha))
    torch.cuda.synchronize()
    return gq.cpu().numpy(), gs.cpu().numpy()


@pytest.mark.parametrize("which", ["both", "alpha", "psi"])
def test_adjoint_random_sky(which):
    rng = np.random.default_rng(11)
    src = unit(rng.normal(size=(3000, 3)))
    tgt = unit(rng.normal(size=(2500, 3)))
    q = rng.lognormal(0, 0.5, 3000)
    g_psi = rng.normal(size=2500) if which in ("both", "psi") else None
    g_alpha = rng.normal(size=(2500, 2)) if which in ("both", "alpha") else None
    gq, gs = run(src, q, tgt, g_psi, g_alpha)
    rq, rs = oracle_adjoint(src, q, tgt, g_alpha, g_psi)
    assert rel(gq, rq) < TOL and rel(gs, rs) < TOL, (rel(gq, rq), rel(gs, rs))
    assert np.abs(np.sum(gs * src, 1)).max() < 1e-12 * np.abs(gs).max()       # tangent


def test_adjoint_clustered_near_field_heavy_and_mixed_plan():
    """Clustered sources and targets, small leaves; the FP64 adjoint and the
    double-float one (the adjoint of a plan made for the mixed path)."""
    rng = np.random.default_rng(12)
    clumps = workloads.clump_set(rng, 20)
    src = workloads.clustered(rng, 40000, 20, clumps=clumps)
    tgt = workloads.clustered(rng, 30001, 20, clumps=clumps)
    q = rng.lognormal(0, 0.5, 40000)
    g_psi = rng.normal(size=30001)
    g_alpha = rng.normal(size=(30001, 2))
    for prec in (sfmm.SFMM_FP64, sfmm.SFMM_MIXED):
        gq, gs = run(src, q, tgt, g_psi, g_alpha, leaf=16, precision=prec)
        idx = workloads.subsample(40000, 600, 12)
        rq, rs = oracle_adjoint(src[idx], q[idx], tgt, g_alpha, g_psi)
        assert rel(gq[idx], rq) < TOL and rel(gs[idx], rs) < TOL, (prec, rel(gq[idx], rq), rel(gs[idx], rs))


def test_adjoint_self_targets_zero_mean_f32_masses():
    """Targets equal to the sources (coincident pairs skipped, as in the
    forward sum), the zero-mean constant, float32 masses."""
    rng = np.random.default_rng(13)
    src = unit(rng.normal(size=(2048, 3)))
    q = rng.lognormal(0, 0.5, 2048).astype(np.float32)
    g_psi = rng.normal(size=2048)
    g_alpha = rng.normal(size=(2048, 2))
    gq, gs = run(src, q, src, g_psi, g_alpha, q_f32=True, zero_mean=True)
    rq, rs = oracle_adjoint(src, q.astype(np.float64), src, g_alpha, g_psi, zero_mean=True)
    assert rel(gq, rq) < TOL and rel(gs, rs) < TOL, (rel(gq, rq), rel(gs, rs))


def test_adjoint_edges():
    rng = np.random.default_rng(14)
    src = unit(rng.normal(size=(100, 3)))
    q = np.ones(100)
    # no targets, or no loss terms: zero gradients
    gq, gs = run(src, q, np.zeros((0, 3)), None, None)
    assert np.all(gq == 0) and np.all(gs == 0)
    tgt = unit(rng.normal(size=(10, 3)))
    gq, gs = run(src, q, tgt, None, None)
    assert np.all(gq == 0) and np.all(gs == 0)
    # a target at a pole: its dipole uses the phi = 0 basis
    tgt = np.array([[0, 0, 1.0], [0, 0, -1.0], [1.0, 0, 0]])
    g_alpha = rng.normal(size=(3, 2))
    gq, gs = run(src, q, tgt, None, g_alpha)
    rq, rs = oracle_adjoint(src, q, tgt, g_alpha, None)
    assert rel(gq, rq) < TOL and rel(gs, rs) < TOL


def test_autograd_loss_matches_oracle_gradient():
    """L = sum w |alpha - a_ref|^2 + sum v (psi - p_ref)^2 through torch autograd."""
    rng = np.random.default_rng(15)
    src = unit(rng.normal(size=(4096, 3)))
    tgt = unit(rng.normal(size=(3000, 3)))
    q = rng.lognormal(0, 0.5, 4096)
    w = rng.uniform(0.5, 1.5, 3000)
    v = rng.uniform(0.5, 1.5, 3000)
    a_ref = rng.normal(size=(3000, 2))
    p_ref = rng.normal(size=3000)
    plan = sfmm.Plan(p=32, leaf_size=32)
    ts = dev(src).requires_grad_(True)
    tq = dev(q).requires_grad_(True)
    psi, alpha = sfa.deflection(ts, tq, dev(tgt), plan)
    L = (dev(w)[:, None] * (alpha - dev(a_ref)) ** 2).sum() + (dev(v) * (psi - dev(p_ref)) ** 2).sum()
    L.backward()
    r = direct_sum(src, q, tgt)
    rq, rs = oracle_adjoint(src, q, tgt, 2 * w[:, None] * (r["alpha"] - a_ref), 2 * v * (r["psi"] - p_ref))
    assert rel(tq.grad.cpu().numpy(), rq) < TOL and rel(ts.grad.cpu().numpy(), rs) < TOL
    with pytest.raises(NotImplementedError):
        tt = dev(tgt).requires_grad_(True)
        psi, alpha = sfa.deflection(dev(src), dev(q), tt, plan)
        alpha.sum().backward()


def test_gradient_workload_matches_central_differences():
    """The gradient workload (N = 1e6 clustered sources, the 786,432 N_side = 256
    pixel centres, L = sum_i w_i |alpha_i - alpha_ref,i|^2), gradient through
    autograd.deflection (forward on the 1e-10 path, backward the adjoint sFMM),
    on 64 seeded particles:

    * dL/dq_j against central differences with h = 1e-6 of the same forward: L
      is quadratic in q, so the difference is exact but for rounding (1e-9);
    * dL/dy_j (the covariant gradient) against the oracle's analytic adjoint
      evaluated at these particles (1e-10);
    * dL/dy_j against central differences of the forward along e_theta and
      e_phi (steps of h = 1e-6 and 2h, renormalised; Richardson combination).
      Moving one source changes the rounding of every sum above it (its leaf's
      multipole, their parents', the locals): the forward's L moves by about
      eps L whatever the step, so a difference resolves a derivative only to
      about eps L / h.  The particles are taken where the step keeps their
      cell at the tree's deepest level (same tree and lists on both sides) and
      at least 1.2e-3 rad from every target (the O((h/d)^4) error of the
      Richardson combination below 1e-12); the check is that each difference
      agrees with the analytic gradient within 16 eps L / h."""
    from oracle.healpix import key29
    d = workloads.loss_sky()
    N, M = d["src"].shape[0], d["tgt"].shape[0]
    plan = sfmm.Plan(p=32, leaf_size=64, c_s=2.0, c_t=0.45, precision=sfmm.SFMM_MIXED_DF)
    src = dev(d["src"]).requires_grad_(True)
    q = dev(d["q"]).requires_grad_(True)
    tgt, w = dev(d["tgt"]), dev(d["w"])
    with torch.no_grad():
        _, a0 = plan.deflection(src, q, tgt)
        a_ref = float(torch.sqrt((a0 ** 2).mean())) * dev(d["xi"])

    def alpha_of(s_, q_):
        return plan.deflection(s_, q_, tgt, with_psi=False)[1]

    def central(ap, am, step):
        # (L(+) - L(-)) / (2 step), summed as w (a+ - a-) . (a+ + a- - 2 a_ref): the same difference
        # without cancelling two losses of ~3 M |alpha|^2
        return float((w[:, None] * (ap - am) * (ap + am - 2.0 * a_ref)).sum()) / (2 * step)

    _, alpha = sfa.deflection(src, q, tgt, plan)
    loss = (w[:, None] * (alpha - a_ref) ** 2).sum()
    loss.backward()
    L = float(loss)
    gq, gs = q.grad.cpu().numpy(), src.grad.cpu().numpy()
    g_alpha = (2.0 * w[:, None] * (alpha.detach() - a_ref)).cpu().numpy()
    depth = plan.stats()["depth"]
    h = 1e-6
    y = d["src"]
    rng = np.random.default_rng(55)
    cand = rng.permutation(N)[:400]
    rho = np.sqrt(y[cand, 0] ** 2 + y[cand, 1] ** 2)
    et = np.stack([y[cand, 2] * y[cand, 0] / rho, y[cand, 2] * y[cand, 1] / rho, -rho], 1)
    ep = np.stack([-y[cand, 1] / rho, y[cand, 0] / rho, np.zeros_like(rho)], 1)
    shift = np.uint64(2 * (29 - depth))
    k0 = key29(y[cand]) >> shift
    same = np.ones(cand.size, dtype=bool)
    for t in (et, ep):
        for sg in (2.0, 1.0, -1.0, -2.0):
            same &= (key29(unit(y[cand] + sg * h * t)) >> shift) == k0
    far = np.array([(d["tgt"] @ y[c]).max() for c in cand]) < np.cos(1.2e-3)
    sel = np.nonzero(same & far)[0][:64]
    assert sel.size == 64
    js = cand[sel]
    # the position gradient against the oracle's analytic adjoint at these particles
    _, rs = oracle_adjoint(y[js], d["q"][js], d["tgt"], g_alpha, None)
    assert rel(gs[js], rs) < 1e-10, rel(gs[js], rs)
    fd_q, fd_y, ad_y = [], [], []
    with torch.no_grad():
        for i in sel:
            j = int(cand[i])
            qp, qm = q.detach().clone(), q.detach().clone()
            qp[j] += h
            qm[j] -= h
            fd_q.append(central(alpha_of(src, qp), alpha_of(src, qm), h))
            for t in (et[i], ep[i]):
                dd = []
                for hh in (h, 2 * h):
                    sp, sm = src.detach().clone(), src.detach().clone()
                    sp[j] = dev(unit(y[j] + hh * t))
                    sm[j] = dev(unit(y[j] - hh * t))
                    dd.append(central(alpha_of(sp, q), alpha_of(sm, q), hh))
                fd_y.append((4 * dd[0] - dd[1]) / 3)
                ad_y.append(float(gs[j] @ t))
    assert rel(gq[js], np.array(fd_q)) < 1e-9, rel(gq[js], np.array(fd_q))
    bound = 16 * np.finfo(float).eps * L / h
    dev_y = np.abs(np.array(fd_y) - np.array(ad_y))
    assert dev_y.max() < bound, (dev_y.max(), bound, L)
