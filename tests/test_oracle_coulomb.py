"""Pins of the oracle's Coulomb outer region (ionic targets, residual charge z > 0).

The oracle takes F_l, G_l and the Whittaker function W from mpmath and derives
their derivatives from recurrence relations; these tests tie both to facts that
do not come from mpmath's Coulomb or Whittaker routines: the eta = 0 limit
(Riccati-Bessel functions from scipy), the small-rho normalisation
C_l(eta) rho^(l+1) (from scipy's complex log-gamma), the Wronskian, the
large-rho asymptotic phase, the terminating (hydrogenic) Whittaker functions,
the z = 0 closed-channel limit, numerical differentiation, and whole-sweep
invariants (hard sphere, symmetry, unitarity) with z > 0.
"""
import math

import numpy as np
import pytest
from scipy.special import loggamma, spherical_jn, spherical_yn

from oracle import rmatrix as o
from paper_1403_5524_gb300 import synth

mp = pytest.importorskip("mpmath")

ETAS = [-0.1, -1.0, -5.0, -30.0]


def riccati(l, x):
    j, jp = spherical_jn(l, x), spherical_jn(l, x, derivative=True)
    y, yp = spherical_yn(l, x), spherical_yn(l, x, derivative=True)
    return x * j, j + x * jp, x * y, y + x * yp


@pytest.mark.parametrize("l", [0, 1, 3, 7])
@pytest.mark.parametrize("rho", [0.5, 3.0, 20.0])
def test_eta_zero_is_riccati_bessel(l, rho):
    F, Fp, G, Gp = o.coulomb_open(l, 0.0, rho)
    jh, jhp, nh, nhp = riccati(l, rho)
    for got, want in [(F, jh), (Fp, jhp), (G, -nh), (Gp, -nhp)]:
        assert abs(got - want) <= 1e-12 * max(1.0, abs(want))


@pytest.mark.parametrize("l", [0, 2, 7])
@pytest.mark.parametrize("eta", ETAS)
def test_wronskian(l, eta):
    for rho in [0.2, 1.5, 9.0, 47.0]:
        F, Fp, G, Gp = o.coulomb_open(l, eta, rho)
        assert abs(Fp * G - F * Gp - 1.0) <= 1e-12 * max(1.0, abs(F * Gp), abs(Fp * G))


@pytest.mark.parametrize("l", [0, 1, 4])
@pytest.mark.parametrize("eta", ETAS)
def test_small_rho_normalisation(l, eta):
    # F_l -> C_l(eta) rho^(l+1) (1 + eta rho / (l+1) + ...), C_l = 2^l e^(-pi eta/2) |Gamma(l+1+i eta)| / (2l+1)!
    lnC = l * math.log(2.0) - math.pi * eta / 2.0 + loggamma(complex(l + 1, eta)).real - math.lgamma(2 * l + 2)
    rho = 1e-6
    F, Fp, _, _ = o.coulomb_open(l, eta, rho)
    C = math.exp(lnC)
    want = C * rho ** (l + 1) * (1.0 + eta * rho / (l + 1))
    dwant = C * ((l + 1) * rho ** l + eta * (l + 2) / (l + 1) * rho ** (l + 1))
    assert abs(F - want) <= 1e-9 * abs(want)
    assert abs(Fp - dwant) <= 1e-9 * abs(dwant)


@pytest.mark.parametrize("l", [0, 3])
@pytest.mark.parametrize("eta", [-0.5, -4.0])
def test_large_rho_phase(l, eta):
    rho = 4000.0
    sig = loggamma(complex(l + 1, eta)).imag
    th = rho - eta * math.log(2.0 * rho) - l * math.pi / 2.0 + sig
    F, Fp, G, Gp = o.coulomb_open(l, eta, rho)
    tol = 2.0 * (eta * eta + l * (l + 1) + 1.0) / rho
    assert abs(F - math.sin(th)) <= tol and abs(G - math.cos(th)) <= tol
    assert abs(Fp - math.cos(th)) <= tol and abs(Gp + math.sin(th)) <= tol


def test_open_derivatives_numerically():
    with mp.workdps(30):
        for l, eta, rho in [(0, -2.0, 3.0), (3, -0.7, 11.0), (5, -12.0, 0.8)]:
            F, Fp, G, Gp = o.coulomb_open(l, eta, rho)
            dF = float(mp.diff(lambda t: mp.coulombf(l, eta, t), rho))
            dG = float(mp.diff(lambda t: mp.coulombg(l, eta, t), rho))
            assert abs(Fp - dF) <= 1e-12 * max(1.0, abs(dF))
            assert abs(Gp - dG) <= 1e-12 * max(1.0, abs(dG))


@pytest.mark.parametrize("l", [0, 2, 6])
def test_whittaker_terminating(l):
    # mu - kappa + 1/2 = 0 or -1: W = x^(l+1) e^(-x/2) times 1 or (x - 2l - 2)
    for x in [0.3, 4.0, 25.0]:
        assert abs(o.whittaker_logderiv(l, l + 1.0, x) - ((l + 1) / x - 0.5)) <= 1e-13 * (1 + (l + 1) / x)
        want = -0.5 + (l + 1) / x + 1.0 / (x - 2 * l - 2)
        assert abs(o.whittaker_logderiv(l, l + 2.0, x) - want) <= 1e-12 * (1 + abs(want))


@pytest.mark.parametrize("l", [0, 1, 5])
def test_whittaker_zero_charge_is_khat(l):
    for kap, a in [(0.3, 20.0), (1.1, 30.0)]:
        assert abs(2 * kap * o.whittaker_logderiv(l, 0.0, 2 * kap * a) - kap * o.khat_logderiv(l, kap * a)) \
            <= 1e-12 * abs(kap * o.khat_logderiv(l, kap * a))


def test_whittaker_derivative_numerically():
    with mp.workdps(30):
        for l, kp, x in [(0, 0.4, 7.0), (3, 2.5, 1.2), (7, 40.0, 0.9)]:
            m = l + 0.5
            want = float(mp.diff(lambda t: mp.whitw(kp, m, t), x) / mp.whitw(kp, m, x))
            assert abs(o.whittaker_logderiv(l, kp, x) - want) <= 1e-12 * max(1.0, abs(want))


def test_channel_functions_zero_charge_unchanged():
    wl = synth.small(5, 6, 100, 1)
    w = wl.waves[0]
    for E in [0.05, 0.9, 2.5]:
        f0 = o.channel_functions(w.l, w.thresh, E, w.a)
        f1 = o.channel_functions(w.l, w.thresh, E, w.a, z=0.0)
        for k in ("s", "sp", "c", "cp", "lam"):
            assert np.array_equal(f0[k], f1[k])


def test_coulomb_hard_sphere():
    # R = 0: the solution vanishes at r = a, so K_ii = -F_l(eta, ka) / G_l(eta, ka)
    a, E, z = 12.0, 1.3, 2.0
    wave = synth.Wave(l=np.array([0, 1, 3, 1], np.int32), thresh=np.array([0.0, 0.2, 0.5, 1.5]),
                      poles=np.array([-1.0, 4.0]), W=np.zeros((4, 2)), a=a, z=z)
    out = o.sweep(wave, np.array([E]))
    assert out["n_open"][0] == 3
    K = out["K"][0]
    for i in range(3):
        k = math.sqrt(E - wave.thresh[i])
        with mp.workdps(30):
            F = float(mp.coulombf(int(wave.l[i]), -z / k, k * a))
            G = float(mp.coulombg(int(wave.l[i]), -z / k, k * a))
        assert abs(K[i, i] + F / G) <= 1e-10 * max(1.0, abs(F / G))
    assert np.abs(K[:3, :3] - np.diag(np.diag(K[:3, :3]))).max() == 0.0


def test_coulomb_sweep_invariants():
    wl = synth.small(21, 5, 120, 1, pole_lo=-2.0, pole_hi=8.0, a=15.0, z=1.0)
    w = wl.waves[0]
    E = np.array([0.07, 0.6, 1.4, 2.7])
    out = o.sweep(w, E, sel=(0, 1))
    for t in range(E.size):
        no = out["n_open"][t]
        K = out["K"][t, :no, :no]
        assert np.abs(K - K.T).max() <= 1e-10 * max(1.0, np.abs(K).max())
        S, _ = o.smatrix(K)
        assert np.abs(S @ S.conj().T - np.eye(no)).max() <= 1e-10
    # the charge matters: a neutral target gives different K
    w0 = synth.Wave(l=w.l, thresh=w.thresh, poles=w.poles, W=w.W, a=w.a, z=0.0)
    out0 = o.sweep(w0, E)
    assert np.abs(out0["K"] - out["K"]).max() > 1e-3
