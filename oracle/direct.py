"""FP64 direct sum (the PPM of Sec. 4.1) -- TEST INFRASTRUCTURE ONLY.

psi(x_i)   = sum_j q_j G(x_i, y_j),  G = (1/4pi) log(d^2/4)        (Eq. SUM, GRE_FUN)
alpha(x_i) = sum_j q_j P_x(x_i - y_j) / (2 pi d^2)                  (Eq. ALP_PSI)

A pair with d^2 == 0 is skipped (self-interaction when targets == sources).
The arithmetic lives in direct.c; this module only marshals arrays.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        lib.oracle_direct.argtypes = [dp, dp, ctypes.c_int64, dp, ctypes.c_int64, dp, dp, dp]
        lib.oracle_direct.restype = ctypes.c_int64
        lib.oracle_dipole.argtypes = [dp, dp, dp, ctypes.c_int64, dp, ctypes.c_int64, dp, dp]
        lib.oracle_dipole.restype = ctypes.c_int64
        lib.oracle_hessian.argtypes = [dp, dp, ctypes.c_int64, dp, ctypes.c_int64, dp]
        lib.oracle_hessian.restype = ctypes.c_int64
        lib.oracle_direct_npm.argtypes = [dp, dp, ctypes.c_int64, dp, ctypes.c_int64, ctypes.c_double, dp, dp, dp]
        lib.oracle_direct_npm.restype = ctypes.c_int64
        lib.oracle_threads.argtypes = []
        lib.oracle_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def direct_sum(src, q, tgt, want=("psi", "alpha"), sigma=0.0):
    """Return a dict with 'psi' [M], 'alpha' [M,2] (e_theta, e_phi),
    'alpha3' [M,3] (tangent 3-vector) as requested, plus 'skipped'.
    sigma > 0: each mass smoothed by the Near Particle Model profile of
    angular radius sigma (oracle_direct_npm in direct.c)."""
    lib = _load()
    src = np.ascontiguousarray(src, dtype=np.float64).reshape(-1, 3)
    tgt = np.ascontiguousarray(tgt, dtype=np.float64).reshape(-1, 3)
    q = np.ascontiguousarray(q, dtype=np.float64).reshape(-1)
    if q.shape[0] != src.shape[0]:
        raise ValueError("q and src differ in length")
    M = tgt.shape[0]
    out = {}
    psi = np.empty(M) if "psi" in want else None
    a2 = np.empty((M, 2)) if "alpha" in want else None
    a3 = np.empty((M, 3)) if "alpha3" in want else None
    if sigma > 0.0:
        out["skipped"] = int(lib.oracle_direct_npm(_ptr(src), _ptr(q), src.shape[0], _ptr(tgt), M, float(sigma),
                                                   _ptr(psi), _ptr(a2), _ptr(a3)))
    else:
        out["skipped"] = int(lib.oracle_direct(_ptr(src), _ptr(q), src.shape[0], _ptr(tgt), M,
                                               _ptr(psi), _ptr(a2), _ptr(a3)))
    if psi is not None:
        out["psi"] = psi
    if a2 is not None:
        out["alpha"] = a2
    if a3 is not None:
        out["alpha3"] = a3
    return out


def tangent_basis(x):
    """(e_theta, e_phi) at the unit vectors x [M,3], with phi = atan2(0, 0) = 0 at
    the poles: e_theta = (cos t cos p, cos t sin p, -sin t), e_phi = (-sin p, cos p, 0)."""
    x = np.asarray(x, dtype=np.float64).reshape(-1, 3)
    rho = np.hypot(x[:, 0], x[:, 1])
    safe = np.where(rho > 0, rho, 1.0)
    cp = np.where(rho > 0, x[:, 0] / safe, 1.0)
    sp = np.where(rho > 0, x[:, 1] / safe, 0.0)
    e_th = np.stack([x[:, 2] * cp, x[:, 2] * sp, -rho], 1)
    e_ph = np.stack([-sp, cp, np.zeros_like(cp)], 1)
    return e_th, e_ph


def dipole_field(x, h, g, y):
    """Phi [N] and its covariant gradient [N,3] at y of charges h [M] and tangent
    dipoles g [M,3] at x (either may be None); see oracle_dipole in direct.c."""
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    y = np.ascontiguousarray(y, dtype=np.float64).reshape(-1, 3)
    hh = None if h is None else np.ascontiguousarray(h, dtype=np.float64).reshape(-1)
    gg = None if g is None else np.ascontiguousarray(g, dtype=np.float64).reshape(-1, 3)
    phi = np.empty(y.shape[0])
    grad = np.empty((y.shape[0], 3))
    lib.oracle_dipole(_ptr(x), _ptr(hh), _ptr(gg), x.shape[0], _ptr(y), y.shape[0], _ptr(phi), _ptr(grad))
    return phi, grad


def adjoint(src, q, tgt, g_alpha=None, g_psi=None, zero_mean=False):
    """Gradients of a loss L(psi, alpha) of the direct-sum outputs at the targets,
    given dL/dalpha [M,2] (components on (e_theta, e_phi) at each target) and
    dL/dpsi [M]:

      dL/dq_j = sum_i dL/dpsi_i G(x_i, y_j) + g_i . grad_x G(x_i, y_j)   (+ sum dL/dpsi / 4pi with zero_mean)
      dL/dy_j = q_j grad_S [ the same sum as a function of y ] (y = y_j), a tangent 3-vector,

    g_i = dL/dalpha_i[0] e_theta(x_i) + dL/dalpha_i[1] e_phi(x_i), because
    alpha_i = sum_j q_j grad_x G(x_i, y_j) is linear in q and G is symmetric.
    Returns (dL/dq [N], dL/dy [N,3])."""
    tgt = np.asarray(tgt, dtype=np.float64).reshape(-1, 3)
    q = np.asarray(q, dtype=np.float64).reshape(-1)
    g = None
    if g_alpha is not None:
        ga = np.asarray(g_alpha, dtype=np.float64).reshape(-1, 2)
        e_th, e_ph = tangent_basis(tgt)
        g = ga[:, :1] * e_th + ga[:, 1:] * e_ph
    phi, grad = dipole_field(tgt, g_psi, g, src)
    if zero_mean and g_psi is not None:
        phi = phi + np.sum(g_psi) / (4 * np.pi)
    return phi, q[:, None] * grad


def hessian(src, q, tgt):
    """Covariant Hessian of psi at the targets in (e_theta, e_phi), [M,3] =
    (H_theta_theta, H_phi_phi, H_theta_phi) (Sec. 2.2; see direct.c)."""
    lib = _load()
    src = np.ascontiguousarray(src, dtype=np.float64).reshape(-1, 3)
    tgt = np.ascontiguousarray(tgt, dtype=np.float64).reshape(-1, 3)
    q = np.ascontiguousarray(q, dtype=np.float64).reshape(-1)
    h = np.empty((tgt.shape[0], 3))
    lib.oracle_hessian(_ptr(src), _ptr(q), src.shape[0], _ptr(tgt), tgt.shape[0], _ptr(h))
    return h


def lensing(src, q, tgt):
    """Trace part, shear and magnification from the Hessian (Sec. 2.2, Eq. GAM_DEF):
    kappa - kappa_bar = tr H, gamma_1 = (H11 - H22)/2, gamma_2 = H12,
    mu = 1 / ((1 - tr H / 2)^2 - gamma_1^2 - gamma_2^2)."""
    h = hessian(src, q, tgt)
    tr = h[:, 0] + h[:, 1]
    g1 = 0.5 * (h[:, 0] - h[:, 1])
    g2 = h[:, 2]
    mu = 1.0 / ((1.0 - 0.5 * tr) ** 2 - g1 ** 2 - g2 ** 2)
    return dict(kappa=tr, gamma=np.stack([g1, g2], 1), mu=mu)


def threads() -> int:
    return int(_load().oracle_threads())
