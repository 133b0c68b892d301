"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no sFMM arithmetic: it only draws points and masses.  Both
the CUDA path and the oracle are fed from here (the oracle never imports the
solver and the solver never imports the oracle).

Workloads
---------
random      N directions = normalised standard-normal 3-vectors, masses
            lognormal(0, 0.5) (the paper's random sources with random masses,
            Sec. 4.1); the targets are the sources themselves.
clustered   a clustered sky: a fraction of the particles in clumps whose
            centres are uniform on S^2 and whose angular profile is the
            projected NFW profile (Sec. 4.3, Eq. NFW), scale radius
            log-uniform in [0.1, 2] arcmin, truncated at 20 scale radii; the
            rest uniform on S^2.  Equal masses q = 4 pi / N (mean kappa = 1).
grid        the centres of the 12 N_side^2 equal-area HEALPix pixels (ring
            order), used as target points.

The projected NFW profile is sampled by inverting its enclosed-mass CDF
g(x) / g(20), g(x) = ln(x/2) + F(x) with F = arccosh(1/x)/sqrt(1-x^2) (x<1),
arccos(1/x)/sqrt(x^2-1) (x>1), 1 (x=1) -- the standard closed form of the
projected NFW mass (Wright & Brainerd 2000, cited in Sec. 4.3) -- tabulated on
a fine log grid and interpolated.
"""
import numpy as np

ARCMIN = np.pi / (180.0 * 60.0)
SEED_BASE = 7021


def rng_for(config_index, stream=0):
    return np.random.Generator(np.random.PCG64([SEED_BASE + config_index, stream]))


def uniform_sphere(rng, n):
    v = rng.standard_normal((n, 3))
    return v / np.linalg.norm(v, axis=1)[:, None]


def _nfw_g(x):
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    lo = x < 1.0
    hi = x > 1.0
    eq = ~(lo | hi)
    xl = x[lo]
    out[lo] = np.log(xl / 2.0) + np.arccosh(1.0 / xl) / np.sqrt(1.0 - xl * xl)
    xh = x[hi]
    out[hi] = np.log(xh / 2.0) + np.arccos(1.0 / xh) / np.sqrt(xh * xh - 1.0)
    out[eq] = 1.0 + np.log(0.5)
    return out


def sample_nfw_x(rng, n, xmax=20.0, grid=200001):
    """Projected radius x = r / r_s drawn from the truncated projected NFW:
    the inverse of CDF(x) = g(x) / g(xmax), tabulated on a log-spaced grid of
    x in [1e-9, xmax] (the CDF is below 1e-15 at 1e-9) and interpolated."""
    u = rng.random(n)
    xs = np.geomspace(1e-9, xmax, grid)
    xs[-1] = xmax
    cdf = _nfw_g(xs) / _nfw_g(np.array([xmax]))[0]
    cdf[0] = 0.0
    cdf = np.maximum.accumulate(cdf)
    return np.interp(u, cdf, xs)


def place_around(centres, theta, phi):
    """Points at angular distance theta and azimuth phi about each centre."""
    c = centres
    a = np.where(np.abs(c[:, 2:3]) < 0.9, np.array([[0.0, 0.0, 1.0]]), np.array([[1.0, 0.0, 0.0]]))
    e1 = np.cross(c, a)
    e1 /= np.linalg.norm(e1, axis=1)[:, None]
    e2 = np.cross(c, e1)
    y = (np.cos(theta)[:, None] * c
         + np.sin(theta)[:, None] * (np.cos(phi)[:, None] * e1 + np.sin(phi)[:, None] * e2))
    return y / np.linalg.norm(y, axis=1)[:, None]


def clump_set(rng, n_clumps, rs_arcmin=(0.1, 2.0)):
    """Clump centres (uniform on S^2) and scale radii (log-uniform, radians)."""
    centres = uniform_sphere(rng, n_clumps)
    rs = np.exp(rng.uniform(np.log(rs_arcmin[0]), np.log(rs_arcmin[1]), n_clumps)) * ARCMIN
    return centres, rs


def clustered(rng, n, n_clumps, frac_clustered=0.7, rs_arcmin=(0.1, 2.0), clumps=None):
    """Clustered-sky positions [n, 3] (float64); `clumps` = (centres, rs) to
    reuse a clump set, else one is drawn from rng."""
    n_cl = int(round(frac_clustered * n))
    n_un = n - n_cl
    centres, rs = clumps if clumps is not None else clump_set(rng, n_clumps, rs_arcmin)
    which = rng.integers(0, centres.shape[0], n_cl)
    x = sample_nfw_x(rng, n_cl)
    theta = x * rs[which]
    phi = rng.uniform(0.0, 2.0 * np.pi, n_cl)
    pts = np.concatenate([place_around(centres[which], theta, phi), uniform_sphere(rng, n_un)])
    return pts[rng.permutation(n)]


def healpix_ring_centres(nside):
    """Centres of the 12 nside^2 HEALPix pixels in ring order (Gorski et al.
    2005): equal-area target points."""
    npix = 12 * nside * nside
    p = np.arange(npix, dtype=np.int64)
    ncap = 2 * nside * (nside - 1)
    z = np.empty(npix)
    phi = np.empty(npix)
    north = p < ncap
    south = p >= npix - ncap
    eq = ~(north | south)
    pn = p[north]
    ir = ((1 + np.sqrt(1.0 + 2.0 * pn)) // 2).astype(np.int64)
    ir = np.where(2 * ir * (ir - 1) > pn, ir - 1, ir)
    ir = np.where(2 * (ir + 1) * ir <= pn, ir + 1, ir)
    iphi = pn + 1 - 2 * ir * (ir - 1)
    z[north] = 1.0 - ir * ir / (3.0 * nside * nside)
    phi[north] = (iphi - 0.5) * np.pi / (2.0 * ir)
    pe = p[eq] - ncap
    ir = pe // (4 * nside) + nside
    iphi = pe % (4 * nside) + 1
    fodd = np.where(((ir + nside) & 1) == 1, 1.0, 0.5)
    z[eq] = (2 * nside - ir) * 2.0 / (3.0 * nside)
    phi[eq] = (iphi - fodd) * np.pi / (2.0 * nside)
    ps = npix - p[south]
    ir = ((1 + np.sqrt(2.0 * ps - 1.0)) // 2).astype(np.int64)
    ir = np.where(2 * ir * (ir - 1) >= ps, ir - 1, ir)
    ir = np.where(2 * (ir + 1) * ir < ps, ir + 1, ir)
    iphi = 4 * ir + 1 - (ps - 2 * ir * (ir - 1))
    z[south] = -1.0 + ir * ir / (3.0 * nside * nside)
    phi[south] = (iphi - 0.5) * np.pi / (2.0 * ir)
    st = np.sqrt((1.0 - z) * (1.0 + z))
    return np.stack([st * np.cos(phi), st * np.sin(phi), z], axis=1)


# ----------------------------------------------------------- named configs --
def random_sky(n=4096, config_index=1):
    """N random directions with lognormal(0, 0.5) masses; targets = sources."""
    rng = rng_for(config_index)
    src = uniform_sphere(rng, n)
    q = rng.lognormal(0.0, 0.5, n)
    return dict(src=src, q=q, tgt=src, workload=f"random N={n}, targets=sources")


def clustered_sky(n=1_000_000, n_clumps=2000, nside=512, config_index=2):
    """Clustered sky of N equal masses, targets on the N_side grid."""
    rng = rng_for(config_index)
    src = clustered(rng, n, n_clumps)
    q = np.full(n, 4.0 * np.pi / n)
    tgt = healpix_ring_centres(nside)
    return dict(src=src, q=q, tgt=tgt,
                workload=f"clustered N={n} ({n_clumps} clumps) -> M={tgt.shape[0]} grid (Nside={nside})")


def loss_sky(n=1_000_000, n_clumps=2000, nside=256, config_index=5):
    """The gradient workload: N equal masses on a clustered sky, targets on the
    N_side grid, per-target loss weights w ~ U[0.5, 1.5] and a reference
    direction xi ~ N(0, I_2) for the reference deflection alpha_ref = s xi
    (the caller picks the scale s, e.g. the RMS of alpha)."""
    rng = rng_for(config_index)
    src = clustered(rng, n, n_clumps)
    q = np.full(n, 4.0 * np.pi / n)
    tgt = healpix_ring_centres(nside)
    r2 = rng_for(config_index, 1)
    w = r2.uniform(0.5, 1.5, tgt.shape[0])
    xi = r2.standard_normal((tgt.shape[0], 2))
    return dict(src=src, q=q, tgt=tgt, w=w, xi=xi,
                workload=f"clustered sky N={n} ({n_clumps} clumps), M={tgt.shape[0]} N_side={nside} pixel centres, "
                         "loss sum w |alpha - s xi|^2")


def shell_sizes(n_shells=64, n_min=10_000, n_max=10_000_000, config_index=4):
    """Source counts N_k of the shells, log-uniform in [n_min, n_max]."""
    rng = rng_for(config_index)
    return np.exp(rng.uniform(np.log(n_min), np.log(n_max), n_shells)).astype(np.int64)


def shell(k, n, config_index=4):
    """Shell k of the shell set: n clustered sources (n/500 clumps), equal masses 4 pi / n."""
    src = clustered(rng_for(config_index, 1 + k), int(n), max(1, int(n) // 500))
    return src, np.full(int(n), 4.0 * np.pi / int(n))


def shell_set(n_shells=64, n_min=10_000, n_max=10_000_000, nside=256, config_index=4):
    """Independent lensing shells (the multi-layer setting): shell k has N_k
    clustered sources, N_k log-uniform in [n_min, n_max], N_k/500 clumps,
    equal masses 4 pi / N_k (float64); every shell uses the same targets, the
    12 nside^2 HEALPix pixel centres."""
    sizes = shell_sizes(n_shells, n_min, n_max, config_index)
    shells = [shell(k, n, config_index) for k, n in enumerate(sizes)]
    tgt = healpix_ring_centres(nside)
    return dict(shells=shells, tgt=tgt, sizes=sizes,
                workload=f"{n_shells} shells, N_k log-uniform in [{n_min:g}, {n_max:g}] (sum {int(sizes.sum())}), "
                         f"clustered (N_k/500 clumps), M = {tgt.shape[0]} N_side={nside} pixel centres each")


def clustered_pair(n=16_000_000, m=None, n_clumps=20_000, config_index=3, q_dtype=np.float32):
    """N sources and M targets drawn independently from the same clustered
    mix (the same clumps); masses equal, stored as float32 by default."""
    m = n if m is None else m
    clumps = clump_set(rng_for(config_index, 2), n_clumps)
    src = clustered(rng_for(config_index, 0), n, n_clumps, clumps=clumps)
    tgt = clustered(rng_for(config_index, 1), m, n_clumps, clumps=clumps)
    q = np.full(n, 4.0 * np.pi / n, dtype=q_dtype)
    return dict(src=src, q=q, tgt=tgt, clumps=clumps,
                workload=f"clustered sources and targets N=M={n} ({n_clumps} shared clumps), q {np.dtype(q_dtype).name}")


def clump_strata(tgt, clumps, k_each, config_index, trunc=20.0, pool=40_000):
    """Seeded target samples of two strata: k_each targets inside some clump's
    truncation radius (trunc scale radii: near-clump) and k_each outside every
    clump's (empty sky, where only the uniform background lies), drawn from a
    seeded pool of candidate targets.  Returns (near, empty) index arrays."""
    centres, rs = clumps
    cand = subsample(tgt.shape[0], min(pool, tgt.shape[0]), config_index, stream=21)
    inside = np.zeros(cand.size, dtype=bool)
    cos_lim = np.cos(np.minimum(trunc * rs, np.pi))
    for i in range(0, cand.size, 2048):
        dots = tgt[cand[i:i + 2048]] @ centres.T             # [chunk, clumps]
        inside[i:i + 2048] = (dots > cos_lim[None, :]).any(axis=1)
    near, empty = cand[inside], cand[~inside]
    rng = rng_for(config_index, 22)
    near = np.sort(rng.choice(near, size=min(k_each, near.size), replace=False))
    empty = np.sort(rng.choice(empty, size=min(k_each, empty.size), replace=False))
    return near, empty


def subsample(n, k, config_index, stream=7):
    """Seeded subsample of k indices out of n (for oracle checks)."""
    rng = rng_for(config_index, stream)
    k = min(k, n)
    return np.sort(rng.choice(n, size=k, replace=False))
