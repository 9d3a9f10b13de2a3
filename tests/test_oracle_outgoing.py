"""The outgoing-wave identities the GPU cross-section path is built on, checked on the CPU.

The GPU path (rm_run / rm_xsec) never forms K.  With M = R - diag(c / (a c')) on
open and R - diag(1 / (a Lambda)) on closed channels, S_oo the Schur complement of
M's closed block, G = S_oo + diag(c / (a c')), h = c + i s (Wronskian
s c' - s' c = -1), it uses

  Z = G - diag(h / (a h')),
  T_ji = -(2i/a) (Z^-1)_ji / (h'_j h'_i) - 2i delta_ji s'_i / h'_i,
  det(I - iK) = prod_j (c'_j h'_j) det Z / (det C'^2 det S_oo), and sign det S_oo from
  the inertia of S'' = V S_oo V, V = diag(c'/|h'|),
  M^-_m = -sqrt(2) (conj(Zhat)^-1 y)_m / conj(h'_m)  (photoionisation),

all algebraically equal to the oracle's K-based quantities.  These tests restate
them in NumPy (eigenvalue inertia, dense solves: no factorisation the kernel
uses) and compare with the oracle's S, eta and M^- on neutral and Coulomb
waves, energies below, between and above the thresholds.
"""
import math

import numpy as np

from oracle import rmatrix as orc
from paper_1403_5524_gb300 import synth


def outgoing(R, l, thr, E, a, z, sel, y=None):
    n = l.shape[0]
    f = orc.channel_functions(l, thr, E, a, z)
    no = f["n_o"]
    c, cp, s, sp, lam = f["c"][:no], f["cp"][:no], f["s"][:no], f["sp"][:no], f["lam"]
    M = R.copy()
    for j in range(n):
        M[j, j] -= (c[j] / (a * cp[j])) if j < no else 1.0 / (a * lam[j])
    Moo, Moc, Mcc = M[:no, :no], M[:no, no:], M[no:, no:]
    S_oo = Moo - Moc @ np.linalg.solve(Mcc, Moc.T) if no < n else Moo
    G = S_oo + np.diag(c / (a * cp))
    h, hp = c + 1j * s, cp + 1j * sp
    Z = G - np.diag(h / (a * hp))
    Zi = np.linalg.inv(Z)
    T = -(2j / a) * Zi / (hp[:, None] * hp[None, :]) - 2j * np.diag(sp / hp)
    V = cp / np.abs(hp)
    S2 = V[:, None] * S_oo * V[None, :]
    neg = int(np.sum(np.linalg.eigvalsh(0.5 * (S2 + S2.T)) < 0))
    ph = np.sum(np.angle(hp)) + np.angle(np.linalg.det(Z)) + math.pi * (np.sum(cp < 0) - neg)
    eta = -ph
    Mm = None
    if y is not None:
        Zh = R.astype(complex).copy()
        for j in range(n):
            Zh[j, j] -= (np.conj(h[j]) / (a * np.conj(hp[j]))) if j < no else 1.0 / (a * lam[j])
        x = np.linalg.solve(Zh, y.astype(complex))
        Mm = -math.sqrt(2.0) * x[:no] / np.conj(hp)
    return no, T, eta, Mm


def check_wave(w, energies, z):
    E_all, _ = orc.nudge_energies(energies, w.poles, w.thresh)
    seen = set()
    for E in E_all:
        R = orc.rmatrix(w.W, w.poles, E, w.a)
        K, no, fl, _ = orc.kmatrix(R, w.l, w.thresh, E, w.a, z)
        if no == 0 or fl:
            continue
        seen.add(min(no, 2) if no < w.n else 3)
        _, To = orc.smatrix(K)
        y = orc.dipole_vector(w.W, w.dip, w.poles, E, w.a) if w.dip is not None else None
        no2, T, eta, Mm = outgoing(R, w.l, w.thresh, E, w.a, z, (0,), y)
        assert no2 == no
        scale = max(1.0, np.abs(To).max())
        assert np.abs(T - To).max() <= 1e-10 * scale, E
        d = eta - orc.eigenphase_sum(K)
        assert abs(orc.wrap_angle(d)) <= 1e-9, (E, d)
        if y is not None:
            _, Mo, _ = orc.photo_amplitudes(R, y, w.l, w.thresh, E, w.a, z)
            assert np.abs(Mm - Mo).max() <= 1e-10 * np.abs(Mo).max(), E
    return seen


def test_outgoing_identities_neutral():
    wl = synth.small(61, 9, 150, 40, e_lo=0.05, e_hi=2.8, thr_hi=2.0, pole_lo=-2.0, pole_hi=6.0, a=12.0,
                     dipole=True)
    seen = check_wave(wl.waves[0], wl.energies, 0.0)
    assert seen == {1, 2, 3}  # one open channel, several (some closed), all open


def test_outgoing_identities_coulomb():
    wl = synth.small(62, 7, 120, 30, e_lo=0.05, e_hi=2.6, thr_hi=2.0, pole_lo=-2.0, pole_hi=6.0, a=12.0,
                     z=1.0, dipole=True)
    seen = check_wave(wl.waves[0], wl.energies, 1.0)
    assert 3 in seen and (1 in seen or 2 in seen)


def test_eta_across_a_k_pole():
    # where an eigenvalue of S_oo crosses zero, K has a pole and eta (mod 2 pi) jumps by pi: the
    # inertia term of the outgoing-wave formula must follow the oracle on both sides
    wl = synth.small(63, 5, 80, 1, pole_lo=-1.0, pole_hi=5.0, thr_hi=1.0, a=10.0)
    w = wl.waves[0]

    def detsign(E):
        R = orc.rmatrix(w.W, w.poles, E, w.a)
        f = orc.channel_functions(w.l, w.thresh, E, w.a)
        no, n = f["n_o"], w.n
        lam = f["lam"]
        M = R.copy()
        for j in range(n):
            M[j, j] -= (f["c"][j] / (w.a * f["cp"][j])) if j < no else 1.0 / (w.a * lam[j])
        S = M[:no, :no] - (M[:no, no:] @ np.linalg.solve(M[no:, no:], M[no:, :no]) if no < n else 0.0)
        V = f["cp"][:no] / np.hypot(f["cp"][:no], f["sp"][:no])
        return np.prod(np.sign(np.linalg.eigvalsh(V[:, None] * S * V[None, :]))), no

    grid = np.linspace(1.2, 2.4, 241)  # above every threshold (all five channels open)
    signs = [detsign(E)[0] for E in grid]
    # det S_oo also changes sign where R has a pole (an eigenvalue passes through infinity): keep
    # the intervals that hold no pole
    flips = [k for k in range(len(grid) - 1) if signs[k] != signs[k + 1]
             and not np.any((w.poles > grid[k] - 1e-3) & (w.poles < grid[k + 1] + 1e-3))]
    assert flips, "no K pole on the grid"
    lo, hi = grid[flips[0]], grid[flips[0] + 1]
    s_lo = detsign(lo)[0]
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        if detsign(mid)[0] == s_lo:
            lo = mid
        else:
            hi = mid
    for E in (lo - 1e-7, hi + 1e-7):
        R = orc.rmatrix(w.W, w.poles, E, w.a)
        K, no, fl, _ = orc.kmatrix(R, w.l, w.thresh, E, w.a)
        _, T, eta, _ = outgoing(R, w.l, w.thresh, E, w.a, 0.0, (0,))
        assert abs(orc.wrap_angle(eta - orc.eigenphase_sum(K))) <= 1e-6, E
