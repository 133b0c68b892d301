"""Pins of the oracle's Near Particle Model (Sec. 3.2, Sec. 4.2 Eq. KERNEL):
beyond sigma the sum is the point-mass sum bit for bit; inside, alpha is the
derivative of psi, both are continuous at the cap's edge, and the spherical
Laplacian of psi equals the profile q W minus the background q/4pi (Delta G =
delta - 1/4pi), which fixes the normalisation N_sigma = 2 pi sin^2(sigma/2)."""
import numpy as np

from oracle.direct import direct_sum
from conftest import unit


def sph(theta, phi=0.3):
    theta = np.atleast_1d(theta)
    return np.stack([np.sin(theta) * np.cos(phi), np.sin(theta) * np.sin(phi), np.cos(theta)], -1)


NORTH = np.array([[0.0, 0.0, 1.0]])


def test_beyond_sigma_equals_point_masses():
    rng = np.random.default_rng(1)
    src = unit(rng.normal(size=(300, 3)))
    q = rng.lognormal(0, 0.5, 300)
    tgt = unit(rng.normal(size=(400, 3)))
    sigma = 1e-3                     # no pair of these random points is that close
    a = direct_sum(src, q, tgt, sigma=sigma)
    b = direct_sum(src, q, tgt)
    assert np.array_equal(a["psi"], b["psi"]) and np.array_equal(a["alpha"], b["alpha"])


def test_alpha_is_the_derivative_of_psi_inside_the_cap():
    sigma, q = 0.05, np.array([1.3])
    th = np.linspace(0.002, 0.049, 25)
    h = 1e-7
    a = direct_sum(NORTH, q, sph(th), sigma=sigma)["alpha"][:, 0]
    dpsi = (direct_sum(NORTH, q, sph(th + h), sigma=sigma)["psi"] - direct_sum(NORTH, q, sph(th - h), sigma=sigma)["psi"]) / (2 * h)
    assert np.allclose(a, dpsi, rtol=1e-6, atol=1e-9)


def test_continuous_at_the_cap_edge():
    sigma, q = 0.05, np.array([0.7])
    eps = 1e-9
    inside = direct_sum(NORTH, q, sph(sigma - eps), sigma=sigma)
    outside = direct_sum(NORTH, q, sph(sigma + eps), sigma=sigma)
    assert abs(inside["psi"][0] - outside["psi"][0]) < 1e-7
    assert abs(inside["alpha"][0, 0] - outside["alpha"][0, 0]) < 1e-5


def test_laplacian_is_the_profile_minus_the_background():
    sigma, q = 0.08, np.array([2.0])
    s = np.sin(sigma / 2) ** 2
    th = np.linspace(0.01, 0.075, 15)
    h = 1e-5
    # axisymmetric: Delta psi = (1/sin t) d/dt (sin t dpsi/dt), dpsi/dt = alpha_theta
    f = lambda t: np.sin(t) * direct_sum(NORTH, q, sph(t), sigma=sigma)["alpha"][:, 0]
    lap = (f(th + h) - f(th - h)) / (2 * h) / np.sin(th)
    u = np.sin(th / 2) ** 2
    W = (1 - u / s) / (2 * np.pi * s)
    assert np.allclose(lap, q[0] * W - q[0] / (4 * np.pi), rtol=1e-6, atol=1e-6 * q[0] * W.max())
    # outside the cap only the background remains
    th2 = np.array([0.1, 0.5, 1.5])
    lap2 = (f(th2 + h) - f(th2 - h)) / (2 * h) / np.sin(th2)
    assert np.allclose(lap2, -q[0] / (4 * np.pi), rtol=1e-6)
