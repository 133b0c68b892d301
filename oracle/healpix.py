"""HEALPix nested pixelisation for the oracle -- TEST INFRASTRUCTURE ONLY.

The sFMM tree (Sec. 3.1, steps 1-3) divides the sphere into the 12 HEALPix
base boxes and then quad-splits boxes; a box at level l is a HEALPix pixel of
N_side = 2^l in the NESTED numbering (Gorski et al. 2005, cited in Sec. 3.1).
The deepest level is r_max = 29 (Sec. 3.1), so every point gets a 64-bit key
    key = face * 4^29 + interleave(ix, iy)        (ix on even bits)
and the box containing it at level l is key >> 2 (29 - l).

Keys must be bit-identical to the ones the CUDA path computes, with no shared
code.  Both sides therefore evaluate the same published formulas with the
same sequence of correctly rounded IEEE double operations (+, -, *, /, sqrt;
no fused multiply-add, no library transcendental):

* the azimuth, as a fraction of a quarter turn, comes from the Gregory series
  atan(t) = sum_k (-1)^k t^(2k+1) / (2k+1) after two textbook reductions:
  t -> (t - 1)/(t + 1) when t > tan(pi/8) (adds pi/4), then the half-angle
  identity atan(t) = 2 atan(t / (1 + sqrt(1 + t^2))), which leaves
  |t| <= tan(pi/16) ~ 0.199, where 12 terms reach double precision;
* the HEALPix ang2pix_nest mapping of Gorski et al. (2005), with
  1 - |z| evaluated as (x^2 + y^2) / (1 + |z|) in the polar caps.

Pixel centres and corners (pix2vec) use ordinary numpy trigonometry: they
feed geometry (box centres and covering radii), not keys.
"""
import numpy as np

ORDER_MAX = 29
NSIDE_MAX = 1 << ORDER_MAX

# face -> ring / azimuth offsets of the base pixels (Gorski et al. 2005)
JRLL = np.array([2, 2, 2, 2, 3, 3, 3, 3, 4, 4, 4, 4], dtype=np.int64)
JPLL = np.array([1, 3, 5, 7, 0, 2, 4, 6, 1, 3, 5, 7], dtype=np.int64)

TAN_PI_8 = 0.41421356237309503        # tan(pi/8) = sqrt(2) - 1, as a double literal
TWO_OVER_PI = 0.6366197723675814      # 2/pi, as a double literal
# Gregory-series coefficients (-1)^k / (2k+1), k = 0..11, each one correctly
# rounded double (what 1.0/(2k+1) gives).
GREGORY = [(-1.0) ** k / (2 * k + 1) for k in range(12)]


def _atan_quarter_01(t):
    """atan(t) * 2/pi for t in [0, 1] (numpy array), deterministic IEEE ops."""
    t = np.asarray(t, dtype=np.float64)
    big = t > TAN_PI_8
    # first reduction: atan(t) = pi/4 + atan((t - 1)/(t + 1))
    t1 = np.where(big, (t - 1.0) / (t + 1.0), t)
    # half-angle reduction: atan(t1) = 2 atan(t1 / (1 + sqrt(1 + t1^2)))
    t2 = t1 / (1.0 + np.sqrt(1.0 + t1 * t1))
    s = t2 * t2
    p = np.full_like(t2, GREGORY[11])
    for k in range(10, -1, -1):
        p = p * s + GREGORY[k]
    a = (2.0 * t2) * p                      # atan(t1) in radians
    v = a * TWO_OVER_PI                     # in quarter turns
    return np.where(big, 0.5 + v, v)


def phi_quarter(x, y):
    """phi = atan2(y, x) expressed in quarter turns, in [0, 4)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    ax = np.abs(x)
    ay = np.abs(y)
    swap = ay > ax
    num = np.where(swap, ax, ay)
    den = np.where(swap, ay, ax)
    zero = den == 0.0
    t = np.where(zero, 0.0, num / np.where(zero, 1.0, den))
    u = _atan_quarter_01(t)
    v = np.where(swap, 1.0 - u, u)          # atan2(|y|, |x|) in quarter turns, [0, 1]
    xpos = x >= 0.0
    ypos = y >= 0.0
    tt = np.where(xpos & ypos, v,
         np.where(~xpos & ypos, 2.0 - v,
         np.where(~xpos & ~ypos, 2.0 + v, 4.0 - v)))
    tt = np.where(tt >= 4.0, tt - 4.0, tt)
    return np.where(zero, 0.0, tt)


def _spread_bits(v):
    """Move bit k of v (k < 32) to bit 2k."""
    v = np.asarray(v, dtype=np.uint64)
    v = (v | (v << np.uint64(16))) & np.uint64(0x0000FFFF0000FFFF)
    v = (v | (v << np.uint64(8))) & np.uint64(0x00FF00FF00FF00FF)
    v = (v | (v << np.uint64(4))) & np.uint64(0x0F0F0F0F0F0F0F0F)
    v = (v | (v << np.uint64(2))) & np.uint64(0x3333333333333333)
    v = (v | (v << np.uint64(1))) & np.uint64(0x5555555555555555)
    return v


def _compact_bits(v):
    """Inverse of _spread_bits: bit 2k of v -> bit k."""
    v = np.asarray(v, dtype=np.uint64) & np.uint64(0x5555555555555555)
    v = (v | (v >> np.uint64(1))) & np.uint64(0x3333333333333333)
    v = (v | (v >> np.uint64(2))) & np.uint64(0x0F0F0F0F0F0F0F0F)
    v = (v | (v >> np.uint64(4))) & np.uint64(0x00FF00FF00FF00FF)
    v = (v | (v >> np.uint64(8))) & np.uint64(0x0000FFFF0000FFFF)
    v = (v | (v >> np.uint64(16))) & np.uint64(0x00000000FFFFFFFF)
    return v


def ang2pix_nest(order, xyz):
    """Nested pixel index at N_side = 2^order of unit vectors xyz [n,3] (uint64)."""
    xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
    x, y, z = xyz[:, 0], xyz[:, 1], xyz[:, 2]
    nside = float(1 << order)
    ns = np.int64(1 << order)
    mask = ns - 1
    za = np.abs(z)
    tt = phi_quarter(x, y)

    # equatorial belt, |z| <= 2/3
    temp1 = nside * (0.5 + tt)
    temp2 = nside * z * 0.75
    jp_e = (temp1 - temp2).astype(np.int64)
    jm_e = (temp1 + temp2).astype(np.int64)
    ifp = jp_e >> order
    ifm = jm_e >> order
    face_e = np.where(ifp == ifm, ifp | 4, np.where(ifp < ifm, ifp, ifm + 8))
    ix_e = jm_e & mask
    iy_e = ns - (jp_e & mask) - 1

    # polar caps, |z| > 2/3
    ntt = np.minimum(3, tt.astype(np.int64))
    tp = tt - ntt
    one_m_za = (x * x + y * y) / (1.0 + za)
    tmp = nside * np.sqrt(3.0 * one_m_za)
    jp_p = np.minimum((tp * tmp).astype(np.int64), ns - 1)
    jm_p = np.minimum(((1.0 - tp) * tmp).astype(np.int64), ns - 1)
    north = z > 0.0
    face_p = np.where(north, ntt, ntt + 8)
    ix_p = np.where(north, ns - jm_p - 1, jp_p)
    iy_p = np.where(north, ns - jp_p - 1, jm_p)

    eq = za <= 2.0 / 3.0
    face = np.where(eq, face_e, face_p).astype(np.uint64)
    ix = np.where(eq, ix_e, ix_p)
    iy = np.where(eq, iy_e, iy_p)
    return (face << np.uint64(2 * order)) | _spread_bits(ix) | (_spread_bits(iy) << np.uint64(1))


def key29(xyz):
    """The order-29 nested key of each unit vector (uint64)."""
    return ang2pix_nest(ORDER_MAX, xyz)


def pix2face_xy(order, pix):
    pix = np.asarray(pix, dtype=np.uint64)
    face = (pix >> np.uint64(2 * order)).astype(np.int64)
    ipf = pix & np.uint64((1 << (2 * order)) - 1)
    ix = _compact_bits(ipf).astype(np.int64)
    iy = _compact_bits(ipf >> np.uint64(1)).astype(np.int64)
    return face, ix, iy


def facexy2vec(order, face, X, Y):
    """Point at continuous face coordinates (X, Y) in [0, N_side]^2 of base
    pixel `face` -> unit vector (the inverse of the ang2pix mapping)."""
    nside = float(1 << order)
    face = np.asarray(face, dtype=np.int64)
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    jr = JRLL[face] * nside - X - Y
    north = jr < nside
    south = jr > 3.0 * nside
    nr = np.where(north, jr, np.where(south, 4.0 * nside - jr, nside))
    z = np.where(north, 1.0 - nr * nr / (3.0 * nside * nside),
        np.where(south, -1.0 + nr * nr / (3.0 * nside * nside),
                 (2.0 * nside - jr) * 2.0 / (3.0 * nside)))
    safe_nr = np.where(nr > 0.0, nr, 1.0)
    phi = np.where(nr > 0.0, (np.pi / 4.0) * (JPLL[face] + (X - Y) / safe_nr), 0.0)
    st = np.sqrt(np.maximum(0.0, (1.0 - z) * (1.0 + z)))
    return np.stack([st * np.cos(phi), st * np.sin(phi), z], axis=-1)


def pix2vec_nest(order, pix):
    """Centre of nested pixel `pix` at N_side = 2^order."""
    face, ix, iy = pix2face_xy(order, pix)
    return facexy2vec(order, face, ix + 0.5, iy + 0.5)


def pixel_boundary(order, pix, per_edge=16):
    """Points on the boundary of the pixel: the 4 corners and `per_edge`
    equispaced points along each edge -> [n, 4*per_edge, 3]."""
    face, ix, iy = pix2face_xy(order, pix)
    s = np.arange(per_edge) / per_edge
    # walk the square [ix, ix+1] x [iy, iy+1] counter-clockwise
    ex = np.concatenate([s, np.ones_like(s), 1.0 - s, np.zeros_like(s)])
    ey = np.concatenate([np.zeros_like(s), s, np.ones_like(s), 1.0 - s])
    X = ix[:, None] + ex[None, :]
    Y = iy[:, None] + ey[None, :]
    return facexy2vec(order, face[:, None], X, Y)


def covering_radius(order, pix, per_edge=16):
    """Angular radius of the circle about the pixel centre through the
    farthest sampled boundary point (the box radius of Sec. 3.5)."""
    c = pix2vec_nest(order, pix)
    b = pixel_boundary(order, pix, per_edge)
    chord = np.linalg.norm(b - c[:, None, :], axis=-1).max(axis=1)
    return 2.0 * np.arcsin(np.minimum(1.0, chord / 2.0))
