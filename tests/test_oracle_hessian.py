"""Pins of the oracle's covariant Hessian, shear and magnification (Sec. 2.2):
the paper's definitions by finite differences of the (pinned) potential and
deflection in (theta, phi), the Laplacian identity tr H = -sum q / 4pi off the
masses (Delta G = delta - 1/4pi), and the single-mass closed form."""
import numpy as np

from oracle.direct import direct_sum, hessian, lensing
from conftest import unit


def sph(theta, phi):
    return np.stack([np.sin(theta) * np.cos(phi), np.sin(theta) * np.sin(phi), np.cos(theta)], -1)


def test_hessian_matches_the_papers_definitions_by_differences():
    rng = np.random.default_rng(1)
    src = unit(rng.normal(size=(30, 3)))
    q = rng.lognormal(0, 0.5, 30)
    th = rng.uniform(0.3, 2.8, 20)
    ph = rng.uniform(0, 2 * np.pi, 20)
    H = hessian(src, q, sph(th, ph))
    h = 1e-5
    for i in range(20):
        t, p = th[i], ph[i]
        a = lambda tt, pp: direct_sum(src, q, sph(np.array([tt]), np.array([pp])))["alpha"][0]
        # alpha = (dpsi/dtheta, (1/sin theta) dpsi/dphi)
        d_t = (a(t + h, p) - a(t - h, p)) / (2 * h)
        d_p = (a(t, p + h) - a(t, p - h)) / (2 * h)
        a0 = a(t, p)
        h11 = d_t[0]
        h12 = d_t[1]
        h22 = d_p[1] / np.sin(t) + a0[0] / np.tan(t)
        scale = np.abs(H[i]).max()
        assert abs(H[i, 0] - h11) < 1e-7 * scale and abs(H[i, 2] - h12) < 1e-7 * scale
        assert abs(H[i, 1] - h22) < 1e-7 * scale
        # and the symmetric partner d/dphi(alpha_theta)/sin theta - cot theta alpha_phi (torsion-free)
        h21 = d_p[0] / np.sin(t) - a0[1] / np.tan(t)
        assert abs(H[i, 2] - h21) < 1e-7 * scale


def test_second_differences_of_psi():
    rng = np.random.default_rng(2)
    src = unit(rng.normal(size=(25, 3)))
    q = rng.lognormal(0, 0.5, 25)
    t, p = 1.1, 0.7
    psi = lambda tt, pp: direct_sum(src, q, sph(np.array([tt]), np.array([pp])))["psi"][0]
    h = 1e-4
    H = hessian(src, q, sph(np.array([t]), np.array([p])))[0]
    h11 = (psi(t + h, p) - 2 * psi(t, p) + psi(t - h, p)) / h ** 2
    assert abs(H[0] - h11) < 1e-5 * np.abs(H).max()


def test_trace_is_minus_total_mass_over_4pi():
    rng = np.random.default_rng(3)
    src = unit(rng.normal(size=(200, 3)))
    q = rng.lognormal(0, 0.5, 200)
    tgt = unit(rng.normal(size=(300, 3)))
    L = lensing(src, q, tgt)
    assert np.allclose(L["kappa"], -q.sum() / (4 * np.pi), rtol=1e-10, atol=1e-12 * np.abs(hessian(src, q, tgt)).max())


def test_single_mass_closed_form():
    """psi = (q/4pi) 2 log sin(theta/2) for a mass at the north pole:
    H11 = -(q/4pi) / (2 sin^2(theta/2)), H22 = (q/4pi) cot theta cot(theta/2), H12 = 0."""
    q = np.array([1.7])
    th = np.linspace(0.05, 3.0, 40)
    tgt = sph(th, np.full_like(th, 0.4))
    H = hessian(np.array([[0, 0, 1.0]]), q, tgt)
    c = q[0] / (4 * np.pi)
    assert np.allclose(H[:, 0], -c / (2 * np.sin(th / 2) ** 2), rtol=1e-12)
    assert np.allclose(H[:, 1], c / np.tan(th) / np.tan(th / 2), rtol=1e-11, atol=1e-14)
    assert np.abs(H[:, 2]).max() < 1e-13
    L = lensing(np.array([[0, 0, 1.0]]), q, tgt)
    g1 = 0.5 * (H[:, 0] - H[:, 1])
    assert np.allclose(L["mu"], 1 / ((1 + c / 2) ** 2 - g1 ** 2), rtol=1e-12)
