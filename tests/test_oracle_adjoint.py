"""Pins of the oracle's adjoint (dL/dq and dL/dy of a loss of psi and alpha).

The adjoint formulas are checked against finite differences of the loss
computed by the forward oracle (itself pinned by closed forms): the loss is
quadratic in the masses, so central differences in q are exact up to
rounding; positions move along great circles y(t) = cos t y + sin t u with u
a unit tangent, and dL/dt(0) must equal dL/dy . u."""
import numpy as np
import pytest

from oracle.direct import adjoint, direct_sum, tangent_basis
from conftest import unit

pytestmark = pytest.mark.filterwarnings("ignore")


def problem(seed, n=40, m=30):
    rng = np.random.default_rng(seed)
    src = unit(rng.normal(size=(n, 3)))
    tgt = unit(rng.normal(size=(m, 3)))
    q = rng.lognormal(0, 0.5, n)
    w = rng.uniform(0.5, 1.5, m)
    v = rng.uniform(0.5, 1.5, m)
    a_ref = rng.normal(size=(m, 2))
    p_ref = rng.normal(size=m)
    return src, tgt, q, w, v, a_ref, p_ref


def loss(src, q, tgt, w, v, a_ref, p_ref, zero_mean=False):
    r = direct_sum(src, q, tgt)
    psi = r["psi"] + (q.sum() / (4 * np.pi) if zero_mean else 0.0)
    return float(np.sum(w[:, None] * (r["alpha"] - a_ref) ** 2) + np.sum(v * (psi - p_ref) ** 2))


def grads(src, q, tgt, w, v, a_ref, p_ref, zero_mean=False):
    r = direct_sum(src, q, tgt)
    psi = r["psi"] + (q.sum() / (4 * np.pi) if zero_mean else 0.0)
    g_alpha = 2 * w[:, None] * (r["alpha"] - a_ref)
    g_psi = 2 * v * (psi - p_ref)
    return adjoint(src, q, tgt, g_alpha, g_psi, zero_mean=zero_mean)


@pytest.mark.parametrize("zero_mean", [False, True])
def test_dq_equals_central_differences(zero_mean):
    src, tgt, q, w, v, a_ref, p_ref = problem(1)
    dq, _ = grads(src, q, tgt, w, v, a_ref, p_ref, zero_mean)
    h = 1e-3
    fd = np.empty_like(q)
    for j in range(q.size):
        qp, qm = q.copy(), q.copy()
        qp[j] += h
        qm[j] -= h
        fd[j] = (loss(src, qp, tgt, w, v, a_ref, p_ref, zero_mean) - loss(src, qm, tgt, w, v, a_ref, p_ref, zero_mean)) / (2 * h)
    assert np.allclose(dq, fd, rtol=1e-7, atol=1e-7 * np.abs(fd).max())


def test_dy_equals_great_circle_differences():
    src, tgt, q, w, v, a_ref, p_ref = problem(2)
    _, dy = grads(src, q, tgt, w, v, a_ref, p_ref)
    # the gradient is tangent at each source
    assert np.abs(np.sum(dy * src, 1)).max() < 1e-12 * np.abs(dy).max()
    rng = np.random.default_rng(3)
    t = 1e-6
    for j in range(src.shape[0]):
        e_th, e_ph = tangent_basis(src[j:j + 1])
        ang = rng.uniform(0, 2 * np.pi)
        u = np.cos(ang) * e_th[0] + np.sin(ang) * e_ph[0]
        sp, sm = src.copy(), src.copy()
        sp[j] = np.cos(t) * src[j] + np.sin(t) * u
        sm[j] = np.cos(t) * src[j] - np.sin(t) * u
        fd = (loss(sp, q, tgt, w, v, a_ref, p_ref) - loss(sm, q, tgt, w, v, a_ref, p_ref)) / (2 * t)
        assert abs(fd - dy[j] @ u) < 1e-6 * max(1.0, abs(fd)), (j, fd, dy[j] @ u)


def test_dipole_term_is_the_derivative_of_a_point_mass():
    """One dipole g at x equals the limit of masses +1/h at x + h g/|g| ... : the
    potential of g is d/ds G(x(s), y) along the great circle through x in the
    direction g, at s = 0 (central difference, h = 1e-5)."""
    from oracle.direct import dipole_field
    rng = np.random.default_rng(4)
    x = unit(rng.normal(size=(1, 3)))
    e_th, e_ph = tangent_basis(x)
    g = 0.7 * e_th + -1.3 * e_ph
    gn = np.linalg.norm(g)
    y = unit(rng.normal(size=(50, 3)))
    phi, grad = dipole_field(x, None, g, y)
    h = 1e-5
    xp = np.cos(h) * x + np.sin(h) * g / gn
    xm = np.cos(h) * x - np.sin(h) * g / gn
    fd = gn * (direct_sum(xp, np.ones(1), y)["psi"] - direct_sum(xm, np.ones(1), y)["psi"]) / (2 * h)
    assert np.allclose(phi, fd, rtol=1e-7, atol=1e-9)
    # and its gradient is the gradient of that difference quotient
    fdg = gn * (direct_sum(xp, np.ones(1), y, want=("alpha3",))["alpha3"]
                - direct_sum(xm, np.ones(1), y, want=("alpha3",))["alpha3"]) / (2 * h)
    assert np.allclose(grad, fdg, rtol=1e-6, atol=1e-8)
