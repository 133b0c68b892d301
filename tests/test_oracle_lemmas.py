"""Pins of the oracle's Lemmas 1-4 and L2P (oracle/lemmas.py) against the
direct sum of G (itself pinned in test_oracle_direct) at points inside each
expansion's region of convergence, against App. B's single-source series and
against the truncation bound of Eq. MUL_ERR; alpha from L2P is also checked
against the finite-difference gradient of psi from L2P."""
import numpy as np
import pytest

import oracle.lemmas as L
from oracle.direct import direct_sum
from conftest import unit, rand_cap

RNG = np.random.default_rng(21)
S = unit(np.array([0.3, 0.5, 0.8]))
Y = rand_cap(RNG, S, 0.05, 25)
Q = RNG.lognormal(0, 0.5, 25)
P = 30
FAR = unit(np.array([-0.2, 0.6, 0.7]))
XF = rand_cap(RNG, FAR, 0.05, 16)
REF = direct_sum(Y, Q, XF, want=("psi", "alpha"))


def test_single_source_series():
    """App. B: one source at (theta_S, 0) gives
    psi = 2 log cos(theta_S/2) + log(1 - cos theta) - log 2 - 2 Re sum (1/l) (z_S/z)^l
    (in units of q/4pi)."""
    thS = 0.3
    y = np.array([[np.sin(thS), 0.0, np.cos(thS)]])
    C, Qv, A = L.p2m(np.array([0.0, 0.0, 1.0]), y, [4 * np.pi], 20)
    np.testing.assert_allclose(Qv, 1.0, rtol=1e-15)
    np.testing.assert_allclose(C, 2 * np.log(np.cos(thS / 2)) - np.log(2), rtol=1e-14)
    ell = np.arange(1, 21)
    np.testing.assert_allclose(A, -np.tan(thS / 2) ** ell / ell, rtol=1e-13)


def test_p2m_matches_direct_sum():
    got = L.eval_multipole(S, L.p2m(S, Y, Q, P), XF)
    np.testing.assert_allclose(got, REF["psi"], rtol=0, atol=1e-13)


@pytest.mark.parametrize("p", [2, 4, 8, 12])
def test_p2m_truncation_bound(p):
    e = L.p2m(S, Y, Q, p)
    err = np.abs(L.eval_multipole(S, e, XF) - REF["psi"])
    thr = np.max(L.local_coords(S, Y)[0])
    th = L.local_coords(S, XF)[0]
    x = np.tan(thr / 2) / np.tan(th / 2)
    bound = L.mul_err_bound(np.abs(Q).sum(), x, p)
    assert np.all(err <= bound * (1 + 1e-9) + 1e-14)


def test_m2m_matches_direct_sum():
    T = unit(S + np.array([0.03, -0.02, 0.01]))
    e = L.m2m(S, T, L.p2m(S, Y, Q, P))
    np.testing.assert_allclose(L.eval_multipole(T, e, XF), REF["psi"], atol=1e-13)
    # the same as building the multipole about T directly
    d = L.p2m(T, Y, Q, P)
    np.testing.assert_allclose(e[0], d[0], rtol=1e-13)
    np.testing.assert_allclose(e[2][:10], d[2][:10], rtol=1e-9, atol=1e-15)


def test_m2l_matches_direct_sum():
    e = L.m2l(S, FAR, L.p2m(S, Y, Q, P))
    np.testing.assert_allclose(L.eval_local(FAR, e, XF), REF["psi"], atol=1e-13)


def test_l2l_matches_direct_sum():
    e = L.m2l(S, FAR, L.p2m(S, Y, Q, P))
    T2 = unit(FAR + np.array([0.01, 0.01, -0.005]))
    e2 = L.l2l(FAR, T2, e)
    X2 = rand_cap(RNG, T2, 0.02, 10)
    ref = direct_sum(Y, Q, X2)
    np.testing.assert_allclose(L.eval_local(T2, e2, X2), ref["psi"], atol=1e-13)


def test_l2p_psi_and_alpha():
    e = L.m2l(S, FAR, L.p2m(S, Y, Q, P))
    psi, alpha, a3 = L.l2p(FAR, e, XF)
    np.testing.assert_allclose(psi, REF["psi"], atol=1e-13)
    np.testing.assert_allclose(alpha, REF["alpha"], atol=1e-11 * np.abs(REF["alpha"]).max())
    # alpha is the gradient of psi_e (finite differences along e_theta, e_phi)
    h = 1e-6
    x = XF[0]
    th = np.arccos(x[2])
    ph = np.arctan2(x[1], x[0])

    def at(t, p):
        return np.array([[np.sin(t) * np.cos(p), np.sin(t) * np.sin(p), np.cos(t)]])

    d_th = (L.l2p(FAR, e, at(th + h, ph))[0] - L.l2p(FAR, e, at(th - h, ph))[0]) / (2 * h)
    d_ph = (L.l2p(FAR, e, at(th, ph + h))[0] - L.l2p(FAR, e, at(th, ph - h))[0]) / (2 * h) / np.sin(th)
    np.testing.assert_allclose(alpha[0], [d_th[0], d_ph[0]], rtol=1e-6)
