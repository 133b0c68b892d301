"""The seeded input generators: determinism, unit norm, and that clump
profiles follow the projected NFW enclosed-mass CDF (Sec. 4.3, Eq. NFW)."""
import numpy as np

from paper_2210_07021_gb300 import workloads as w


def test_random_sky_deterministic():
    a = w.random_sky(1000)
    b = w.random_sky(1000)
    assert np.array_equal(a["src"], b["src"]) and np.array_equal(a["q"], b["q"])
    np.testing.assert_allclose(np.linalg.norm(a["src"], axis=1), 1.0, atol=2e-16)
    assert np.all(a["q"] > 0)


def test_nfw_profile_cdf():
    rng = np.random.default_rng(0)
    x = np.sort(w.sample_nfw_x(rng, 20000))
    # KS distance against the enclosed projected mass, by numerical
    # integration of Eq. NFW's kappa(x) x (not of the closed form used to draw)
    def kappa(t):
        t = np.asarray(t, float)
        out = np.empty_like(t)
        lo, hi = t < 1, t > 1
        out[lo] = 4 / (t[lo] ** 2 - 1) * (1 - 2 / np.sqrt(1 - t[lo] ** 2) * np.arctanh(np.sqrt((1 - t[lo]) / (1 + t[lo]))))
        out[hi] = 4 / (t[hi] ** 2 - 1) * (1 - 2 / np.sqrt(t[hi] ** 2 - 1) * np.arctan(np.sqrt((t[hi] - 1) / (t[hi] + 1))))
        out[~(lo | hi)] = 4 / 3
        return out
    grid = np.concatenate([np.geomspace(1e-8, 1, 20000, endpoint=False), np.linspace(1, 20, 20000)])
    f = kappa(grid) * grid
    cdf = np.concatenate([[0], np.cumsum(0.5 * (f[1:] + f[:-1]) * np.diff(grid))])
    cdf /= cdf[-1]
    emp = np.arange(1, len(x) + 1) / len(x)
    ks = np.abs(np.interp(x, grid, cdf) - emp).max()
    assert ks < 1.63 / np.sqrt(len(x))                 # 1% level


def test_clustered_sky_shapes():
    d = w.clustered_sky(n=20000, n_clumps=50, nside=16)
    assert d["src"].shape == (20000, 3) and d["tgt"].shape == (12 * 256, 3)
    np.testing.assert_allclose(d["q"].sum(), 4 * np.pi)
    p = w.clustered_pair(n=5000, n_clumps=10)
    assert p["q"].dtype == np.float32 and p["tgt"].shape == (5000, 3)
    assert not np.array_equal(p["src"], p["tgt"])
