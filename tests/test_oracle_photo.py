"""Pins of the oracle's photoionisation amplitudes and cross section.

The R-matrix expansion of the final state is checked against a brute-force
solve of the inner-region problem: with the Bloch operator in H, the inner
solution whose boundary derivatives are F'(a) has basis coefficients
c = (H - E O)^-1 B F', and the dipole amplitude is c . v for the dipole
source vector v; the oracle instead works from the eigen-expansion (poles
E_k, w_ik, d_k = C_k . v).  Closed channels are handled in the brute force by
eliminating them from F = a R F' with F_c = F'_c / Lambda_c, independently of
the oracle's matching solve.  Further pins: the scalar incoming-wave
normalisation |M^-|^2 = (M^K)^2 / (1 + K^2), invariance of sigma_PI under
channel and dipole sign flips, and its linear dependence on omega = E - E_0.
"""
import math

import numpy as np
import pytest
import scipy.linalg as sl

from oracle import rmatrix as o
from paper_1403_5524_gb300 import synth
from tests.test_oracle_pins import bloch_inner_region


def inner_problem(n_ch, thr, seed, a=10.0, n_basis=14):
    l = list(range(n_ch))
    H, O, Bv = bloch_inner_region(n_ch, n_basis, a, l, thr, seed=seed)
    Ek, C = sl.eigh(H, O)
    W = math.sqrt(2.0) * (Bv.T @ C)
    v = np.random.default_rng(seed + 100).normal(0.0, 1.0, H.shape[0])
    dip = C.T @ v
    return np.array(l, np.int32), H, O, Bv, Ek, W, v, dip, a


def brute_force_amplitudes(l, thr, H, O, Bv, v, R, E, a):
    # boundary derivatives of each K-normalised solution: open parts from K, closed parts from
    # (1/Lambda_c - a R_cc) F'_c = a R_co F'_o; then c = (H - E O)^-1 B F', M = c . v
    n = l.shape[0]
    f = o.channel_functions(l, thr, E, a)
    no = f["n_o"]
    K, no2, _, _ = o.kmatrix(R, l, thr, E, a)
    assert no2 == no
    M = np.zeros(no)
    op, cl = np.arange(no), np.arange(no, n)
    for m in range(no):
        Fp = np.zeros(n)
        Fp[:no] = f["cp"][:no] * K[:, m]
        Fp[m] += f["sp"][m]
        if cl.size:
            A = np.diag(1.0 / f["lam"][cl]) - a * R[np.ix_(cl, cl)]
            Fp[cl] = np.linalg.solve(A, a * R[np.ix_(cl, op)] @ Fp[:no])
        c = np.linalg.solve(H - E * O, Bv @ Fp)
        M[m] = c @ v
    return M, K


@pytest.mark.parametrize("thr,E", [([0.0, 0.1, 0.25], 0.9), ([0.0, 0.3, 2.5], 0.8), ([0.0, 1.6, 1.9], 0.55)])
def test_amplitudes_against_inner_region_solve(thr, E):
    thr = np.array(thr)
    l, H, O, Bv, Ek, W, v, dip, a = inner_problem(3, thr, seed=int(10 * E))
    R = o.rmatrix(W, Ek, E, a)
    y = o.dipole_vector(W, dip, Ek, E, a)
    MK, Mm, K = o.photo_amplitudes(R, y, l, thr, E, a)
    Mb, Kb = brute_force_amplitudes(l, thr, H, O, Bv, v, R, E, a)
    assert np.abs(MK - Mb).max() <= 1e-9 * max(1.0, np.abs(Mb).max()), (MK, Mb)
    # incoming-wave amplitudes solve (I + iK) M^- = M^K
    assert np.abs((np.eye(K.shape[0]) + 1j * K) @ Mm - MK).max() <= 1e-12 * max(1.0, np.abs(MK).max())


def test_single_channel_normalisation():
    rng = np.random.default_rng(4)
    N, a = 30, 12.0
    poles = np.sort(rng.uniform(-1, 9, N))
    W = rng.normal(0, 1 / math.sqrt(N), (1, N))
    dip = rng.normal(0, 1 / math.sqrt(N), N)
    l, thr = np.array([1], np.int32), np.array([0.0])
    for E in [0.3, 1.7, 4.4]:
        R = o.rmatrix(W, poles, E, a)
        MK, Mm, K = o.photo_amplitudes(R, o.dipole_vector(W, dip, poles, E, a), l, thr, E, a)
        assert abs(abs(Mm[0]) ** 2 - MK[0] ** 2 / (1.0 + K[0, 0] ** 2)) <= 1e-12 * MK[0] ** 2


def test_sigma_pi_invariances():
    wl = synth.small(7, 5, 160, 1, pole_lo=-2.0, pole_hi=9.0, a=14.0, dipole=True)
    w = wl.waves[0]
    E = np.array([0.08, 0.7, 1.9, 2.6])
    base = o.sweep(w, E, keep_R=False, keep_K=False)
    assert np.all(base["sig_pi"] >= 0.0) and base["sig_pi"].max() > 0.0
    # a channel's sign (row of W) and the dipole's sign are conventions
    W2 = w.W.copy()
    W2[2] *= -1.0
    for ww in (synth.Wave(l=w.l, thresh=w.thresh, poles=w.poles, W=W2, a=w.a, dip=w.dip, e0=w.e0),
               synth.Wave(l=w.l, thresh=w.thresh, poles=w.poles, W=w.W, a=w.a, dip=-w.dip, e0=w.e0)):
        other = o.sweep(ww, E, keep_R=False, keep_K=False)
        assert np.allclose(other["sig_pi"], base["sig_pi"], rtol=1e-11, atol=0)
        assert np.allclose(other["sig_pi_ch"], base["sig_pi_ch"], rtol=1e-10, atol=1e-300)
    # sigma_PI is linear in omega = E - E_0 at fixed amplitudes
    w3 = synth.Wave(l=w.l, thresh=w.thresh, poles=w.poles, W=w.W, a=w.a, dip=w.dip, e0=w.e0 - 1.0)
    other = o.sweep(w3, E, keep_R=False, keep_K=False)
    ratio = (E - w3.e0) / (E - w.e0)
    assert np.allclose(other["sig_pi"], base["sig_pi"] * ratio, rtol=1e-13)
    # channel partials sum to the total, closed channels contribute nothing
    assert np.allclose(base["sig_pi_ch"].sum(axis=1), base["sig_pi"], rtol=1e-13)
    for t in range(E.size):
        assert np.all(base["sig_pi_ch"][t, base["n_open"][t]:] == 0.0)


def test_no_dipole_no_output():
    wl = synth.small(7, 4, 60, 1)
    out = o.sweep(wl.waves[0], np.array([0.5]))
    assert "sig_pi" not in out
