"""Pins of the oracle's HEALPix keys and geometry (oracle/healpix.py).

* the nest numbering of Gorski et al. (2005) at N_side = 1, 2: base-pixel
  centres on the rings z = 2/3, 0, -2/3 and the sub-pixel layout of face 0;
* ang2pix(pix2vec(p)) == p at every pixel of orders 0-6 and at random pixels
  of order 29 (the two directions are written independently);
* the equal-area ring grid of the input generator (separate code, ring
  order) lands one-to-one on nest pixel centres;
* the key hierarchy: key29 >> 2(29 - k) equals the order-k pixel;
* equal areas: uniform points fill the 192 pixels of N_side = 4 evenly;
* the azimuth routine agrees with numpy's arctan2 to a few ulp and is exact
  on the axes;
* the 4 corners realise the covering radius (128 samples per edge never
  exceed them) and every point lies within its pixel's radius.
"""
import numpy as np
import pytest

import oracle.healpix as hp
from paper_2210_07021_gb300 import workloads
from conftest import unit


def test_base_pixels():
    c = hp.pix2vec_nest(0, np.arange(12, dtype=np.uint64))
    z = c[:, 2]
    phi = np.mod(np.arctan2(c[:, 1], c[:, 0]), 2 * np.pi)
    np.testing.assert_allclose(z[:4], 2 / 3, atol=1e-15)
    np.testing.assert_allclose(z[4:8], 0.0, atol=1e-15)
    np.testing.assert_allclose(z[8:], -2 / 3, atol=1e-15)
    np.testing.assert_allclose(phi[:4], np.pi / 4 + np.arange(4) * np.pi / 2, atol=1e-14)
    np.testing.assert_allclose(phi[4:8], np.arange(4) * np.pi / 2, atol=1e-14)
    np.testing.assert_allclose(phi[8:], np.pi / 4 + np.arange(4) * np.pi / 2, atol=1e-14)


def test_face0_subpixels_nside2():
    c = hp.pix2vec_nest(1, np.arange(4, dtype=np.uint64))
    z = c[:, 2]
    phi = np.arctan2(c[:, 1], c[:, 0])
    # pixel 0 is the southern corner of face 0, pixel 3 touches the pole,
    # pixel 1 lies east (larger phi) of pixel 2
    np.testing.assert_allclose(z, [1 / 3, 2 / 3, 2 / 3, 11 / 12], atol=1e-15)
    np.testing.assert_allclose(phi, [np.pi / 4, 3 * np.pi / 8, np.pi / 8, np.pi / 4], atol=1e-14)


@pytest.mark.parametrize("order", [0, 1, 2, 3, 4, 6])
def test_roundtrip_all_pixels(order):
    p = np.arange(12 * 4 ** order, dtype=np.uint64)
    assert np.array_equal(hp.ang2pix_nest(order, hp.pix2vec_nest(order, p)), p)


def test_roundtrip_order29():
    rng = np.random.default_rng(1)
    p = rng.integers(0, 12 * 4 ** 29, 200000, dtype=np.int64).astype(np.uint64)
    assert np.array_equal(hp.key29(hp.pix2vec_nest(29, p)), p)


def test_generator_grid_is_nest_centres():
    g = workloads.healpix_ring_centres(64)
    p = hp.ang2pix_nest(6, g)
    assert len(np.unique(p)) == 12 * 64 * 64
    np.testing.assert_allclose(hp.pix2vec_nest(6, p), g, atol=2e-15)


def test_key_hierarchy():
    rng = np.random.default_rng(2)
    v = unit(rng.normal(size=(100000, 3)))
    k = hp.key29(v)
    for o in range(0, 30, 3):
        assert np.array_equal(hp.ang2pix_nest(o, v), k >> np.uint64(2 * (29 - o)))


def test_equal_area():
    rng = np.random.default_rng(3)
    n = 960000
    v = unit(rng.normal(size=(n, 3)))
    cnt = np.bincount(hp.ang2pix_nest(2, v).astype(np.int64), minlength=192)
    e = n / 192
    chi2 = np.sum((cnt - e) ** 2 / e)
    assert chi2 < 191 + 6 * np.sqrt(2 * 191)          # ~ 6 sigma


def test_phi_quarter():
    rng = np.random.default_rng(4)
    xy = rng.normal(size=(500000, 2)) * np.exp(rng.uniform(-30, 30, size=(500000, 1)))
    tt = hp.phi_quarter(xy[:, 0], xy[:, 1])
    ref = np.mod(np.arctan2(xy[:, 1], xy[:, 0]), 2 * np.pi) / (np.pi / 2)
    d = np.abs(tt - ref)
    d = np.minimum(d, 4 - d)
    assert d.max() < 4e-15
    assert np.all((tt >= 0) & (tt < 4))
    ax = hp.phi_quarter(np.array([1.0, 0.0, -1.0, 0.0, 1.0, -1.0, -1.0, 1.0, 0.0]),
                        np.array([0.0, 1.0, 0.0, -1.0, 1.0, 1.0, -1.0, -1.0, 0.0]))
    np.testing.assert_allclose(ax, [0, 1, 2, 3, 0.5, 1.5, 2.5, 3.5, 0], atol=1e-15)


@pytest.mark.parametrize("order", [0, 1, 2, 3, 5, 9, 17, 29])
def test_covering_radius(order):
    rng = np.random.default_rng(5)
    v = unit(rng.normal(size=(20000, 3)))
    p = hp.ang2pix_nest(order, v)
    up = np.unique(p)[:2000]
    r4 = hp.covering_radius(order, up, per_edge=1)
    r128 = hp.covering_radius(order, up, per_edge=128)
    assert np.all(r128 <= r4 * (1 + 1e-12) + 1e-15)
    # points lie within their pixel's covering radius
    c = hp.pix2vec_nest(order, p)
    ang = 2 * np.arcsin(np.linalg.norm(v - c, axis=1) / 2)
    r = hp.covering_radius(order, p, per_edge=1)
    assert np.all(ang <= r * (1 + 1e-9) + 2e-15)
