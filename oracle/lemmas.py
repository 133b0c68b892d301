"""Lemmas 1-4 and the lensing quantities of Sec. 3.6, written as printed --
TEST INFRASTRUCTURE ONLY.

Everything follows the paper's notation and conventions:

* Local frame K_P (Sec. 3.1): zenith e_r(P), azimuth reference e_theta(P);
  a point X has local coordinates (theta^(P), phi^(P)) with
  cos theta^(P) = X . e_r(P) and phi^(P) = atan2(X . e_phi(P), X . e_theta(P)).
* Basis function z^l(theta, phi) = tan^l(theta/2) e^{i l phi}.
* An expansion is the triple (C, Q, A) with A = [A_1 .. A_p] (complex).
  Multipole expansion (Lemma 1):
      psi = C + Q log(1 - cos theta) + 2 Re sum_l A_l / z^l
  Local expansion (Lemmas 3, 4):
      psi = C + Q log(1 + cos theta) + 2 Re sum_l A_l z^l
* T_{ll'}(x) = sum_{n=1}^{min(l,l')} C(l-1, n-1) C(l', n) x^{l+l'-2n} (1 + x^2)^n,
  with x = tan(theta_T^(S)/2) in Lemmas 2 and 4 and x = cot(theta_T^(S)/2) in
  Lemma 3, evaluated term by term (O(p^3)) exactly as printed.

The geometry of a translation from centre S to centre T uses
(theta_T^(S), phi_T^(S)) = coordinates of T in K_S and phi_S^(T) = azimuth of
S in K_T (Lemma 2).
"""
from math import comb

import numpy as np

INV4PI = 1.0 / (4.0 * np.pi)


# ---------------------------------------------------------------- geometry --
def spherical(P):
    """(theta, phi) of a unit vector, phi = atan2(y, x) (0 at the poles)."""
    P = np.asarray(P, dtype=np.float64)
    return np.arctan2(np.hypot(P[..., 0], P[..., 1]), P[..., 2]), np.arctan2(P[..., 1], P[..., 0])


def basis(P):
    """(e_r, e_theta, e_phi) at P (Sec. 2.2's normalised basis)."""
    th, ph = spherical(P)
    e_r = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], axis=-1)
    e_t = np.stack([np.cos(th) * np.cos(ph), np.cos(th) * np.sin(ph), -np.sin(th)], axis=-1)
    e_p = np.stack([-np.sin(ph), np.cos(ph), np.zeros_like(ph)], axis=-1)
    return e_r, e_t, e_p


def local_coords(P, X):
    """(theta^(P), phi^(P)) of the points X [..., 3] in K_P (Sec. 3.1).

    The tangent components X.e_theta(P), X.e_phi(P) are evaluated as
    (X - P).e and, when X is closer to -P than to P, as (X + P).e: the same
    numbers, since P is normal to e_theta(P) and e_phi(P), but without the
    cancellation of a full dot product for points close to P or to -P."""
    e_r, e_t, e_p = basis(P)
    X = np.asarray(X, dtype=np.float64)
    P = np.asarray(P, dtype=np.float64)
    D = X - P
    E = X + P
    use_e = np.sum(E * E, axis=-1) < np.sum(D * D, axis=-1)
    V = np.where(use_e[..., None], E, D)
    c = X @ e_r
    a = V @ e_t
    b = V @ e_p
    return np.arctan2(np.hypot(a, b), c), np.arctan2(b, a)


def zpow(theta, phi, l):
    return np.tan(theta / 2.0) ** l * np.exp(1j * l * phi)


def Tmat(x, p):
    """T_{ll'}(x), l, l' = 1..p, as printed (index [l-1, l'-1])."""
    T = np.zeros((p, p))
    for l in range(1, p + 1):
        for lp in range(1, p + 1):
            s = 0.0
            for n in range(1, min(l, lp) + 1):
                s += comb(l - 1, n - 1) * comb(lp, n) * x ** (l + lp - 2 * n) * (1.0 + x * x) ** n
            T[l - 1, lp - 1] = s
    return T


def translation_geometry(S, T):
    """theta_T^(S), phi_T^(S) and phi_S^(T) of Lemma 2."""
    th, ph_T = local_coords(S, T)
    _, ph_S = local_coords(T, S)
    return float(th), float(ph_T), float(ph_S)


# ---------------------------------------------------------------- Lemma 1 ---
def p2m(S, y, q, p):
    """Multipole expansion about S of masses q at points y (Lemma 1)."""
    y = np.asarray(y, dtype=np.float64).reshape(-1, 3)
    q = np.asarray(q, dtype=np.float64).reshape(-1)
    th, ph = local_coords(S, y)
    Q = INV4PI * q.sum()
    C = INV4PI * np.sum(2.0 * q * np.log(np.cos(th / 2.0))) - Q * np.log(2.0)
    A = np.array([-INV4PI / l * np.sum(q * zpow(th, ph, l)) for l in range(1, p + 1)])
    return C, Q, A


def eval_multipole(S, exp, X):
    """psi at points X from a multipole expansion about S (Lemma 1, Eq. LEMMA1:EXP)."""
    C, Q, A = exp
    th, ph = local_coords(S, X)
    s = np.zeros(np.shape(th), dtype=np.complex128)
    for l in range(1, len(A) + 1):
        s += A[l - 1] / zpow(th, ph, l)
    return C + Q * np.log(1.0 - np.cos(th)) + 2.0 * s.real


# ---------------------------------------------------------------- Lemma 2 ---
def m2m(S, T, exp):
    """Multipole about S -> multipole about T (Lemma 2)."""
    C, Q, A = exp
    p = len(A)
    th, phT, phS = translation_geometry(S, T)
    t = np.tan(th / 2.0)
    Tm = Tmat(t, p)
    l = np.arange(1, p + 1)
    Cn = C + 2.0 * Q * np.log(np.cos(th / 2.0)) + 2.0 * np.sum((-1.0) ** l * np.exp(-1j * l * phT) * A * t ** l).real
    inner = (-1.0) ** l * np.exp(-1j * l * phT) * A                 # indexed by l'
    An = (-Q / l * t ** l + Tm @ inner) * np.exp(1j * l * phS)
    return Cn, Q, An


# ---------------------------------------------------------------- Lemma 3 ---
def m2l(S, T, exp):
    """Multipole about S -> local expansion about T (Lemma 3)."""
    C, Q, A = exp
    p = len(A)
    th, phT, phS = translation_geometry(S, T)
    c = 1.0 / np.tan(th / 2.0)
    Tm = Tmat(c, p)
    l = np.arange(1, p + 1)
    Cn = C + 2.0 * Q * np.log(np.sin(th / 2.0)) + 2.0 * np.sum(np.exp(-1j * l * phT) * A * c ** l).real
    inner = np.exp(-1j * l * phT) * A
    An = (-Q / l * c ** l + Tm @ inner) * np.exp(-1j * l * phS)
    return Cn, Q, An


def eval_local(T, exp, X):
    """psi at points X from a local expansion about T (Eq. LEMMA_EXP3)."""
    C, Q, A = exp
    th, ph = local_coords(T, X)
    s = np.zeros(np.shape(th), dtype=np.complex128)
    for l in range(1, len(A) + 1):
        s += A[l - 1] * zpow(th, ph, l)
    return C + Q * np.log(1.0 + np.cos(th)) + 2.0 * s.real


# ---------------------------------------------------------------- Lemma 4 ---
def l2l(S, T, exp):
    """Local expansion about S -> local expansion about T (Lemma 4)."""
    C, Q, A = exp
    p = len(A)
    th, phT, phS = translation_geometry(S, T)
    t = np.tan(th / 2.0)
    Tm = Tmat(t, p)
    l = np.arange(1, p + 1)
    Cn = C + 2.0 * Q * np.log(np.cos(th / 2.0)) + 2.0 * np.sum(np.exp(1j * l * phT) * A * t ** l).real
    inner = np.exp(1j * l * phT) * A
    An = (-1.0) ** l * (-Q / l * t ** l + Tm @ inner) * np.exp(-1j * l * phS)
    return Cn, Q, An


# ------------------------------------------------------------ Sec. 3.6 L2P --
def l2p(L, exp, X):
    """psi_e and alpha_e at points X from a local expansion about L.

    psi_e   = C + Q log(1 + cos theta) + 2 Re sum A_l z^l            (Sec. 3.6)
    alpha_theta^(L) = -Q tan(theta/2) + 2 Re sum (l / sin theta) A_l z^l  (Sec. 3.6)
    alpha_phi^(L)   = (1/sin theta) d psi_e / d phi
                    = -(2 / sin theta) sum l Im(A_l z^l)   (not printed; the
                      same derivative taken along phi)
    The local components are rotated to the global (e_theta, e_phi) at X.
    Returns psi [n], alpha [n, 2], alpha3 [n, 3].
    """
    C, Q, A = exp
    X = np.asarray(X, dtype=np.float64).reshape(-1, 3)
    th, ph = local_coords(L, X)
    psi = C + Q * np.log(1.0 + np.cos(th))
    a_t = -Q * np.tan(th / 2.0)
    a_p = np.zeros_like(th)
    st = np.sin(th)
    for l in range(1, len(A) + 1):
        zl = A[l - 1] * zpow(th, ph, l)
        psi = psi + 2.0 * zl.real
        a_t = a_t + 2.0 * l / st * zl.real
        a_p = a_p - 2.0 * l / st * zl.imag
    e_r, e_t, e_p = basis(L)
    # unit vectors of the local spherical system of K_L at X
    et_loc = (np.cos(th)[:, None] * (np.cos(ph)[:, None] * e_t + np.sin(ph)[:, None] * e_p)
              - np.sin(th)[:, None] * e_r)
    ep_loc = -np.sin(ph)[:, None] * e_t + np.cos(ph)[:, None] * e_p
    a3 = a_t[:, None] * et_loc + a_p[:, None] * ep_loc
    _, gt, gp = basis(X)
    alpha = np.stack([np.sum(a3 * gt, axis=1), np.sum(a3 * gp, axis=1)], axis=1)
    return psi, alpha, a3


def mul_err_bound(Qabs, x, p):
    """Truncation bound of Eq. MUL_ERR: Qabs/(2 pi) x^(p+1) / ((p+1)(1-x))."""
    return Qabs / (2.0 * np.pi) * x ** (p + 1) / ((p + 1) * (1.0 - x))
