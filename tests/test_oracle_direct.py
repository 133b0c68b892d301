"""Pins of the oracle's direct sum (oracle/direct.c) against what the paper
and the mathematics fix -- none of them re-types the oracle's formula.

* a single point mass: psi = (q/2pi) log sin(Theta/2) and alpha =
  q cot(Theta/2)/(4pi) along +e_theta when the mass sits on the north pole
  (Sec. 2.1, Eq. GRE_FUN; App. A's point-mass deflection shape);
* symmetric configurations (octahedron, icosahedron): alpha = 0 by symmetry
  and psi in closed form from the vertex inner products;
* a Y_lm density gives psi = -Y_lm / (l (l+1)) (Eq. POI_EQU with the
  normalisation of Eq. LAP_GRE), and a uniform density gives psi = -1;
* Delta psi = -sum(q)/(4 pi) away from the masses (Eq. LAP_GRE);
* alpha equals the finite-difference covariant gradient of psi (Eq. ALP_PSI);
* invariance under a random rotation, linearity, order independence;
* a 30-digit mpmath evaluation of the same sum.
"""
import numpy as np
import pytest

from oracle.direct import direct_sum
from conftest import unit


def sph(theta, phi):
    return np.stack([np.sin(theta) * np.cos(phi), np.sin(theta) * np.sin(phi), np.cos(theta)], axis=-1)


def test_single_point_mass_on_the_pole():
    q = 1.7
    th = np.array([1e-6, 1e-3, 0.1, 0.7, 1.5, 2.5, 3.1])
    ph = np.array([0.0, 0.3, 1.0, 2.0, 3.0, 4.0, 5.5])
    tgt = sph(th, ph)
    r = direct_sum(np.array([[0.0, 0.0, 1.0]]), [q], tgt, want=("psi", "alpha", "alpha3"))
    np.testing.assert_allclose(r["psi"], q / (2 * np.pi) * np.log(np.sin(th / 2)), rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(r["alpha"][:, 0], q / (4 * np.pi) / np.tan(th / 2), rtol=1e-12)
    np.testing.assert_allclose(r["alpha"][:, 1], 0.0, atol=1e-12 * np.abs(r["alpha"][:, 0]).max())
    # tangent to the sphere
    tang = np.sum(r["alpha3"] * tgt, axis=1) / np.linalg.norm(r["alpha3"], axis=1)
    # the radial residual is set by |x|^2 - 1 ~ 1e-16 of the inputs, relative to Theta
    assert np.all(np.abs(tang) <= 1e-15 / th + 1e-14)


def test_single_mass_points_away_everywhere():
    rng = np.random.default_rng(11)
    y = unit(rng.normal(size=3))
    x = unit(rng.normal(size=(50, 3)))
    r = direct_sum(y[None, :], [1.0], x, want=("alpha3",))
    away = x - y
    away -= np.sum(away * x, axis=1)[:, None] * x          # tangent direction away from y
    cos_t = x @ y
    theta = np.arccos(np.clip(cos_t, -1, 1))
    mag = 1 / (4 * np.pi) / np.tan(theta / 2)
    np.testing.assert_allclose(r["alpha3"], unit(away) * mag[:, None], rtol=1e-11, atol=1e-13)


def octahedron():
    return np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], float)


def icosahedron():
    g = (1 + 5 ** 0.5) / 2
    v = []
    for a in (-1, 1):
        for b in (-g, g):
            v += [[0, a, b], [a, b, 0], [b, 0, a]]
    return unit(np.array(v, float))


@pytest.mark.parametrize("poly,psi_vertex", [
    (octahedron, lambda q: -q * np.log(2) / np.pi),                 # 4 at 90 deg, 1 antipodal
    (icosahedron, lambda q: -5 * q * np.log(5) / (4 * np.pi)),      # 5 at cos 1/sqrt5, 5 at -1/sqrt5, 1 antipodal
])
def test_symmetric_polyhedra(poly, psi_vertex):
    v = poly()
    q = 0.9
    r = direct_sum(v, np.full(len(v), q), v)
    assert r["skipped"] == len(v)                         # self pairs excluded
    np.testing.assert_allclose(r["psi"], psi_vertex(q), rtol=1e-14)
    np.testing.assert_allclose(r["alpha"], 0.0, atol=1e-14)
    # face centres of the octahedron / any point mapped by the symmetry group: alpha = 0
    if len(v) == 6:
        f = unit(np.array([[s1, s2, s3] for s1 in (-1, 1) for s2 in (-1, 1) for s3 in (-1, 1)], float))
        rf = direct_sum(v, np.full(6, q), f)
        np.testing.assert_allclose(rf["alpha"], 0.0, atol=1e-14)
        np.testing.assert_allclose(rf["psi"], rf["psi"][0], rtol=1e-14)


def _sphere_quadrature(n_t, n_p):
    t, w = np.polynomial.legendre.leggauss(n_t)             # t = cos(theta)
    ph = (np.arange(n_p) + 0.5) * 2 * np.pi / n_p
    T, P = np.meshgrid(t, ph, indexing="ij")
    W = np.repeat(w[:, None], n_p, axis=1) * (2 * np.pi / n_p)
    st = np.sqrt(1 - T ** 2)
    pts = np.stack([st * np.cos(P), st * np.sin(P), T], axis=-1).reshape(-1, 3)
    return pts, W.reshape(-1)


# real spherical harmonics (unnormalised), their degree l and gradients
def _Y(kind, x):
    th = np.arccos(np.clip(x[:, 2], -1, 1))
    ph = np.arctan2(x[:, 1], x[:, 0])
    c, s = np.cos(th), np.sin(th)
    if kind == "Y00":
        return np.ones_like(c), 0, np.zeros_like(c), np.zeros_like(c)
    if kind == "Y10":
        return c, 1, -s, np.zeros_like(c)
    if kind == "Y20":
        return (3 * c * c - 1) / 2, 2, -3 * c * s, np.zeros_like(c)
    if kind == "Y22":
        return s * s * np.cos(2 * ph), 2, 2 * s * c * np.cos(2 * ph), -2 * s * np.sin(2 * ph)
    if kind == "Y31":
        f = (5 * c * c - 1) * s
        df = -10 * c * s * s + (5 * c * c - 1) * c
        return f * np.cos(ph), 3, df * np.cos(ph), -f * np.sin(ph) / s
    raise KeyError(kind)


@pytest.mark.parametrize("kind", ["Y00", "Y10", "Y20", "Y22", "Y31"])
def test_Ylm_density(kind):
    """kappa = Y_lm (sampled on a Gauss-Legendre x uniform grid) gives
    psi = -Y_lm / (l(l+1)) for l >= 1 and psi = -1 for l = 0 (int G = -1).

    Raw form: masses Y(y_j) w_j; psi converges under refinement.  Subtracted
    form (per target x): masses (Y(y_j) - Y(x)) w_j, which removes the
    singular part of the quadrature; since int G = -1 and int grad G = 0,
    psi = sum - Y(x) and alpha = sum exactly, so both must match closely."""
    rng = np.random.default_rng(5)
    tgt = unit(rng.normal(size=(8, 3)))
    Yt, l, dth, dph = _Y(kind, tgt)
    lam = -1.0 if l == 0 else -1.0 / (l * (l + 1))
    errs = []
    for n_t in (96, 192):
        pts, w = _sphere_quadrature(n_t, 2 * n_t)
        Yv = _Y(kind, pts)[0]
        r = direct_sum(pts, Yv * w, tgt)
        errs.append(np.abs(r["psi"] - lam * Yt).max())
    assert errs[1] < 1e-4 and errs[1] < errs[0], errs
    pts, w = _sphere_quadrature(192, 384)
    Yv = _Y(kind, pts)[0]
    for i in range(len(tgt)):
        r = direct_sum(pts, (Yv - Yt[i]) * w, tgt[i:i + 1])
        np.testing.assert_allclose(r["psi"][0] - Yt[i], lam * Yt[i], atol=2e-5)
        np.testing.assert_allclose(r["alpha"][0], lam * np.array([dth[i], dph[i]]), atol=2e-4)


def _exp_map(x, e1, e2, u, v):
    r = np.hypot(u, v)
    if r == 0:
        return x
    return np.cos(r) * x + np.sin(r) * (u * e1 + v * e2) / r


def _tangent_frame(x):
    a = np.array([0.0, 0.0, 1.0]) if abs(x[2]) < 0.9 else np.array([1.0, 0.0, 0.0])
    e1 = unit(np.cross(x, a))
    return e1, np.cross(x, e1)


def test_laplacian_is_minus_mean_density():
    """Delta psi = delta - sum(q)/(4 pi): away from the masses, the spherical
    Laplacian of psi is -sum(q)/(4 pi) (Eq. LAP_GRE)."""
    rng = np.random.default_rng(8)
    x = unit(np.array([0.2, -0.4, 0.9]))
    src = unit(rng.normal(size=(40, 3)))
    src = src[np.arccos(np.clip(src @ x, -1, 1)) > 0.6]
    q = rng.random(len(src)) + 0.5
    e1, e2 = _tangent_frame(x)
    h = 2e-3
    pts = np.array([_exp_map(x, e1, e2, u, v) for u, v in
                    [(0, 0), (h, 0), (-h, 0), (0, h), (0, -h), (2 * h, 0), (-2 * h, 0), (0, 2 * h), (0, -2 * h)]])
    p = direct_sum(src, q, pts)["psi"]
    lap_h = (p[1] + p[2] + p[3] + p[4] - 4 * p[0]) / h ** 2
    lap_2h = (p[5] + p[6] + p[7] + p[8] - 4 * p[0]) / (2 * h) ** 2
    lap = (4 * lap_h - lap_2h) / 3                       # Richardson
    np.testing.assert_allclose(lap, -q.sum() / (4 * np.pi), rtol=1e-6)


def test_alpha_is_covariant_gradient_of_psi():
    rng = np.random.default_rng(9)
    src = unit(rng.normal(size=(30, 3)))
    q = rng.lognormal(0, 0.5, 30)
    x = unit(rng.normal(size=(6, 3)))
    r = direct_sum(src, q, x, want=("psi", "alpha"))
    h = 1e-5
    for i in range(len(x)):
        th = np.arccos(x[i, 2])
        ph = np.arctan2(x[i, 1], x[i, 0])
        pp = direct_sum(src, q, sph(np.array([th + h, th - h, th, th]),
                                    np.array([ph, ph, ph + h, ph - h])))["psi"]
        d_th = (pp[0] - pp[1]) / (2 * h)
        d_ph = (pp[2] - pp[3]) / (2 * h) / np.sin(th)
        np.testing.assert_allclose(r["alpha"][i], [d_th, d_ph], rtol=2e-6, atol=1e-8)


def test_rotation_invariance():
    rng = np.random.default_rng(12)
    src = unit(rng.normal(size=(200, 3)))
    q = rng.lognormal(0, 0.5, 200)
    x = unit(rng.normal(size=(50, 3)))
    Rm, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    if np.linalg.det(Rm) < 0:
        Rm[:, 0] *= -1
    a = direct_sum(src, q, x, want=("psi", "alpha3"))
    b = direct_sum(src @ Rm.T, q, x @ Rm.T, want=("psi", "alpha3"))
    np.testing.assert_allclose(b["psi"], a["psi"], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(b["alpha3"], a["alpha3"] @ Rm.T, rtol=1e-10, atol=1e-11)


def test_linearity_and_order():
    rng = np.random.default_rng(13)
    src = unit(rng.normal(size=(300, 3)))
    q1, q2 = rng.random(300), rng.random(300)
    x = unit(rng.normal(size=(40, 3)))
    a = direct_sum(src, q1, x)
    b = direct_sum(src, q2, x)
    c = direct_sum(src, 2 * q1 - 3 * q2, x)
    np.testing.assert_allclose(c["psi"], 2 * a["psi"] - 3 * b["psi"], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(c["alpha"], 2 * a["alpha"] - 3 * b["alpha"], rtol=1e-11, atol=1e-11)
    perm = rng.permutation(300)
    d = direct_sum(src[perm], q1[perm], x)
    np.testing.assert_allclose(d["psi"], a["psi"], rtol=1e-14, atol=1e-14)
    np.testing.assert_allclose(d["alpha"], a["alpha"], rtol=1e-13, atol=1e-13)


def test_mpmath_thirty_digits():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    rng = np.random.default_rng(14)
    src = unit(rng.normal(size=(128, 3)))
    src[:3] = unit(src[0] + np.array([[0, 0, 0], [1e-7, 0, 0], [0, 2e-6, 1e-6]]))   # near-coincident pairs
    q = rng.lognormal(0, 0.5, 128)
    x = np.vstack([src[0] + [3e-7, -1e-7, 0], unit(rng.normal(size=(3, 3)))])
    x = unit(x)
    r = direct_sum(src, q, x, want=("psi", "alpha3"))
    for i in range(len(x)):
        X = [mp.mpf(float(c)) for c in x[i]]
        sp = mp.mpf(0)
        g = [mp.mpf(0)] * 3
        for j in range(len(src)):
            Y = [mp.mpf(float(c)) for c in src[j]]
            e = [X[k] - Y[k] for k in range(3)]
            d2 = sum(t * t for t in e)
            qq = mp.mpf(float(q[j]))
            sp += qq * mp.log(d2 / 4) / (4 * mp.pi)
            g = [g[k] + qq * (e[k] - d2 / 2 * X[k]) / (2 * mp.pi * d2) for k in range(3)]
        assert abs(float(sp) - r["psi"][i]) <= 1e-14 * abs(float(sp)) + 1e-15
        for k in range(3):
            assert abs(float(g[k]) - r["alpha3"][i, k]) <= 1e-13 * max(abs(float(gg)) for gg in g)
