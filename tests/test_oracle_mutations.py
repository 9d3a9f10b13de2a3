"""Plant plausible mistakes in the FP64 oracle (on the CPU) and check that the
independent pins catch every one.

Each mutation rewrites one line of an oracle function (a flipped sign, a
dropped factor, a transposed scaling, a wrong index, an inverted Cayley map,
...), compiles the result into the oracle module for the duration of the test,
and runs a compact set of pins: single-pole Breit-Wigner, Lane-Thomas l = 1,
hard sphere, the Bloch-operator resolvent, closed-channel elimination, K
symmetry / S unitarity, detailed balance, and the nudge.  A mutation that no
pin rejects would mean the oracle is not pinned where that mistake lives.
"""
import inspect
import math
import textwrap

import numpy as np
import pytest
from scipy.special import spherical_kn

from oracle import rmatrix as o
from paper_1403_5524_gb300 import synth
from tests.test_oracle_pins import (bloch_inner_region, jhat_explicit, nhat_explicit,
                                    one_channel_wave)


def mutate(func, old, new):
    src = textwrap.dedent(inspect.getsource(func))
    assert old in src, (func.__name__, old)
    ns = dict(vars(o))
    exec(compile(src.replace(old, new, 1), "<mutant>", "exec"), ns)
    return ns[func.__name__]


# ---------------------------------------------------------------- pins
def pin_breit_wigner():
    a, w, E1, E = 20.0, 0.7, 2.5, 1.1
    out = o.sweep(one_channel_wave(0, w, E1, a), np.array([E]))
    k = math.sqrt(E)
    d = -k * a + math.atan(k * w * w / (2.0 * (E1 - E)))
    sig = 4.0 * math.pi / k ** 2 * math.sin(d) ** 2
    S, _ = o.smatrix(out["K"][0, :1, :1])
    return (abs(math.sin(math.atan(out["K"][0, 0, 0]) - d)) < 1e-10
            and abs(out["sig_sel"][0, 0, 0] - sig) < 1e-10 * sig
            and abs(math.sin(out["eta"][0] - d)) < 1e-10
            and abs(S[0, 0] - np.exp(2j * d)) < 1e-10)


def pin_lane_thomas():
    a, w, E1, E, l = 20.0, 0.5, 2.5, 0.6, 1
    out = o.sweep(one_channel_wave(l, w, E1, a), np.array([E]))
    k = math.sqrt(E)
    x = k * a
    j, jp = jhat_explicit(l, x)
    n, np_ = nhat_explicit(l, x)
    O, Op = complex(-n, j), complex(-np_, jp)
    L = x * Op / O
    R = w * w / (2.0 * a * (E1 - E))
    d = -np.angle(O) + math.atan2(L.imag * R, 1.0 - L.real * R)
    return abs(math.sin(math.atan(out["K"][0, 0, 0]) - d)) < 1e-10


def pin_hard_sphere():
    a, E = 12.0, 1.3
    wave = synth.Wave(l=np.array([0, 1, 2, 1], np.int32), thresh=np.array([0.0, 0.2, 0.5, 1.5]),
                      poles=np.array([-1.0, 4.0]), W=np.zeros((4, 2)), a=a)
    out = o.sweep(wave, np.array([E]))
    K = out["K"][0]
    ok = out["n_open"][0] == 3 and np.all(np.isfinite(K))
    for i in range(3):
        x = math.sqrt(E - wave.thresh[i]) * a
        j, _ = jhat_explicit(int(wave.l[i]), x)
        n, _ = nhat_explicit(int(wave.l[i]), x)
        ok &= abs(K[i, i] - j / n) <= 1e-10 * max(1.0, abs(j / n))
    return ok


def pin_bloch():
    import scipy.linalg as sl
    a = 10.0
    H, O, Bv = bloch_inner_region(2, 10, a, [0, 1], [0.0, 0.35], seed=11)
    Ek, C = sl.eigh(H, O)
    W = math.sqrt(2.0) * (Bv.T @ C)
    E = 0.57
    Rp = o.rmatrix(W, Ek, E, a)
    Rd = (Bv.T @ np.linalg.solve(H - E * O, Bv)) / a
    return np.abs(Rp - Rd).max() <= 1e-9 * np.abs(Rd).max()


def pin_closed_channel():
    rng = np.random.default_rng(9)
    N = 25
    poles = np.sort(rng.uniform(-2, 12, N))
    W = rng.normal(0, 1 / math.sqrt(N), (2, N))
    a, lc, E = 8.0, 2, 0.9
    wave = synth.Wave(l=np.array([0, lc], np.int32), thresh=np.array([0.0, 2.0]), poles=poles, W=W, a=a)
    out = o.sweep(wave, np.array([E]))
    d0 = 1.0 / (poles - E)
    R = (W * d0[None, :]) @ W.T / (2.0 * a)   # independent of the oracle's pole sum
    kap = math.sqrt(2.0 - E)
    x = kap * a
    L1 = kap * (spherical_kn(lc, x) + x * spherical_kn(lc, x, derivative=True)) / (x * spherical_kn(lc, x))
    Reff = R[0, 0] + a * R[0, 1] * L1 * R[1, 0] / (1.0 - a * R[1, 1] * L1)
    k = math.sqrt(E)
    d = -k * a + math.atan(k * a * Reff)
    return out["n_open"][0] == 1 and abs(math.sin(math.atan(out["K"][0, 0, 0]) - d)) < 1e-10


def pin_symmetry_unitarity_balance():
    wl = synth.config(1)
    w = wl.waves[0]
    out = o.sweep(w, wl.energies[600:1000:80], sel=(0, 1, 2, 3))
    ok = True
    for t in range(out["E"].shape[0]):
        no = out["n_open"][t]
        K = out["K"][t, :no, :no]
        ok &= np.abs(K - K.T).max() <= 1e-10 * max(np.abs(K).max(), 1.0)
        S, _ = o.smatrix(K)
        ok &= np.abs(S @ S.conj().T - np.eye(no)).max() <= 1e-10
        k2 = out["E"][t] - w.thresh
        sig = out["sig_sel"][t]
        for i in range(no):
            for j in range(no):
                ok &= abs(k2[i] * sig[i, j] - k2[j] * sig[j, i]) <= 1e-9 * max(k2[i] * sig[i, j], 1e-300)
    return bool(ok)


def pin_nudge():
    En, fl = o.nudge_energies(np.array([0.5 + 5e-10, 0.9]), np.array([0.5, 1.0]), np.array([0.0, 0.7]))
    return En[0] == 0.5 + 5e-10 + 1e-6 and En[1] == 0.9 and fl[0] == o.FLAG_NUDGED and fl[1] == 0


def pin_coulomb_hard_sphere():
    # R = 0 with z > 0: K_ii = -F_l(eta, ka) / G_l(eta, ka), eta = -z/k
    import mpmath as mp
    a, E, z = 12.0, 1.3, 2.0
    wave = synth.Wave(l=np.array([0, 1, 3, 1], np.int32), thresh=np.array([0.0, 0.2, 0.5, 1.5]),
                      poles=np.array([-1.0, 4.0]), W=np.zeros((4, 2)), a=a, z=z)
    out = o.sweep(wave, np.array([E]))
    ok = out["n_open"][0] == 3
    for i in range(3):
        k = math.sqrt(E - wave.thresh[i])
        with mp.workdps(30):
            r = float(mp.coulombf(int(wave.l[i]), -z / k, k * a) / mp.coulombg(int(wave.l[i]), -z / k, k * a))
        ok &= abs(out["K"][0, i, i] + r) <= 1e-10 * max(1.0, abs(r))
    return bool(ok)


def pin_coulomb_closed_hydrogenic():
    # closed channel at kappa = z/(l+1): the decaying solution is r^(l+1) e^(-kappa r), so
    # Lambda = (l+1)/a - kappa
    a, z, lc = 9.0, 1.5, 2
    kap = z / (lc + 1)
    thr = np.array([0.0, 1.0])
    E = thr[1] - kap * kap
    f = o.channel_functions(np.array([0, lc], np.int32), thr, E, a, z=z)
    return abs(f["lam"][1] - ((lc + 1) / a - kap)) <= 1e-12


def pin_coulomb_eta_zero():
    # eta = 0 gives the Riccati-Bessel functions (scipy), and the Wronskian is 1 at eta != 0
    from scipy.special import spherical_jn, spherical_yn
    ok = True
    for l, x in [(0, 2.0), (3, 7.5)]:
        F, Fp, G, Gp = o.coulomb_open(l, 0.0, x)
        ok &= abs(F - x * spherical_jn(l, x)) <= 1e-12
        ok &= abs(G + x * spherical_yn(l, x)) <= 1e-12 * max(1.0, abs(x * spherical_yn(l, x)))
        ok &= abs(Fp - (spherical_jn(l, x) + x * spherical_jn(l, x, derivative=True))) <= 1e-12
        F, Fp, G, Gp = o.coulomb_open(l, -3.0, x)
        ok &= abs(Fp * G - F * Gp - 1.0) <= 1e-11
    # large rho: F ~ sin(theta), F' ~ cos(theta), theta = rho - eta ln 2 rho - l pi/2 + arg Gamma(l+1+i eta)
    from scipy.special import loggamma
    l, eta, rho = 1, -3.0, 4000.0
    th = rho - eta * math.log(2 * rho) - l * math.pi / 2 + loggamma(complex(l + 1, eta)).imag
    F, Fp, G, Gp = o.coulomb_open(l, eta, rho)
    tol = 2.0 * (eta * eta + l * (l + 1) + 1.0) / rho
    ok &= abs(F - math.sin(th)) <= tol and abs(Fp - math.cos(th)) <= tol and abs(Gp + math.sin(th)) <= tol
    return bool(ok)


def pin_photo():
    # amplitudes against the brute-force inner-region solve (one closed channel), scalar
    # incoming-wave normalisation, and a positive sigma_PI from the sweep
    from tests.test_oracle_photo import brute_force_amplitudes, inner_problem
    thr, E = np.array([0.0, 0.3, 2.5]), 0.8
    l, H, O, Bv, Ek, W, v, dip, a = inner_problem(3, thr, seed=8)
    R = o.rmatrix(W, Ek, E, a)
    MK, Mm, K = o.photo_amplitudes(R, o.dipole_vector(W, dip, Ek, E, a), l, thr, E, a)
    Mb, _ = brute_force_amplitudes(l, thr, H, O, Bv, v, R, E, a)
    ok = np.abs(MK - Mb).max() <= 1e-9 * max(1.0, np.abs(Mb).max())
    wave = synth.Wave(l=l, thresh=thr, poles=Ek, W=W, a=a, dip=dip, e0=-0.4)
    out = o.sweep(wave, np.array([E]))
    ok &= out["sig_pi"][0] > 0.0
    # single channel: |M^-|^2 = (M^K)^2 / (1 + K^2)
    W1, y1 = W[:1], o.dipole_vector(W[:1], dip, Ek, 1.7, a)
    MK1, Mm1, K1 = o.photo_amplitudes(o.rmatrix(W1, Ek, 1.7, a), y1, l[:1], thr[:1], 1.7, a)
    ok &= abs(abs(Mm1[0]) ** 2 - MK1[0] ** 2 / (1.0 + K1[0, 0] ** 2)) <= 1e-12 * MK1[0] ** 2
    return bool(ok)


def pin_convolution():
    # Gaussian * Gaussian on a non-uniform mesh: widths add in quadrature; weights are linear
    u = np.linspace(0.0, 1.0, 3001)
    E = 2.0 * u ** 2
    g = lambda x, mu, sd: np.exp(-0.5 * ((x - mu) / sd) ** 2) / (sd * math.sqrt(2 * math.pi))
    s1, fwhm = 0.03, 0.05
    s2 = fwhm / (2 * math.sqrt(2 * math.log(2)))
    both = o.convolve_average(E, np.vstack([g(E, 1.0, s1), g(E, 1.0, s1)]), [0.25, 0.75], fwhm)
    inner = (E > 0.6) & (E < 1.4)
    want = g(E, 1.0, math.hypot(s1, s2))
    return bool(np.abs(both[inner] - want[inner]).max() <= 1e-4 * want.max())


PINS = [pin_breit_wigner, pin_lane_thomas, pin_hard_sphere, pin_bloch, pin_closed_channel,
        pin_symmetry_unitarity_balance, pin_nudge, pin_coulomb_hard_sphere, pin_coulomb_closed_hydrogenic,
        pin_coulomb_eta_zero, pin_photo, pin_convolution]


def run_pins():
    res = {}
    for p in PINS:
        try:
            with np.errstate(all="ignore"):
                res[p.__name__] = bool(p())
        except Exception:
            res[p.__name__] = False
    return res


def test_unmutated_oracle_passes_every_pin():
    res = run_pins()
    assert all(res.values()), res


MUTATIONS = [
    ("pole sum sign", o.rmatrix, "d = 1.0 / (poles - E)", "d = 1.0 / (E - poles)"),
    ("pole sum missing 1/2", o.rmatrix, "/ (2.0 * a)", "/ a"),
    ("Lambda scales rows not columns", o.kmatrix, "a * R * f[\"lam\"][None, :]", "a * R * f[\"lam\"][:, None]"),
    ("K divided by the column's c", o.kmatrix, "K = Y[:no, :] / f[\"c\"][:no, None]", "K = Y[:no, :] / f[\"c\"][None, :no]"),
    ("B term sign", o.kmatrix, "B = -a * R[:, :no]", "B = a * R[:, :no]"),
    ("s' missing chain-rule k", o.channel_functions, "sp[i] = jhp * math.sqrt(k)", "sp[i] = jhp / math.sqrt(k)"),
    ("c sign", o.channel_functions, "c[i] = -nh / math.sqrt(k)", "c[i] = nh / math.sqrt(k)"),
    ("c' sign", o.channel_functions, "cp[i] = -nhp * math.sqrt(k)", "cp[i] = nhp * math.sqrt(k)"),
    ("closed log-derivative sign", o.channel_functions, "lam[i] = kap * khat_logderiv", "lam[i] = -kap * khat_logderiv"),
    ("khat derivative term dropped", o.khat_logderiv, "return dp / p - 1.0", "return dp / p"),
    ("inverted Cayley map", o.smatrix, "S = np.linalg.solve(I - 1j * K, I + 1j * K)",
     "S = np.linalg.solve(I + 1j * K, I - 1j * K)"),
    ("sigma uses k of the final channel", o.xsec, "(math.pi / k2[:no])[:, None]", "(math.pi / k2[:no])[None, :]"),
    ("sigma 4 pi instead of pi", o.xsec, "(math.pi / k2[:no])", "(4 * math.pi / k2[:no])"),
    ("eigenphase sign", o.eigenphase_sum, "np.sum(np.arctan(", "-np.sum(np.arctan("),
    ("nudge downwards", o.nudge_energies, "E[e] = E[e] + NUDGE_SHIFT", "E[e] = E[e] - NUDGE_SHIFT"),
    ("open count too large", o.n_open, "thresh < E", "thresh <= E + 0.5"),
    ("Coulomb eta sign", o.channel_functions, "-z / k, k * a", "z / k, k * a"),
    ("Coulomb c from F", o.channel_functions, "c[i] = G / math.sqrt(k)", "c[i] = F / math.sqrt(k)"),
    ("Whittaker argument kappa a", o.channel_functions, "2.0 * kap * a)", "kap * a)"),
    ("Whittaker order", o.channel_functions, "z / kap, 2.0 * kap * a", "-z / kap, 2.0 * kap * a"),
    ("Whittaker derivative sign", o.whittaker_logderiv, "(xx / 2 - k) * W0 - W1", "(xx / 2 - k) * W0 + W1"),
    ("Coulomb derivative coefficient", o.coulomb_open, "c2 = mp.sqrt(L * L + e * e) / L",
     "c2 = mp.sqrt(L * L + e * e) / (L + 1)"),
    ("Coulomb derivative eta term", o.coulomb_open, "c1 = (L * L / r + e) / L", "c1 = (L * L / r - e) / L"),
    ("dipole vector 1/a", o.dipole_vector, "/ (2.0 * a)", "/ a"),
    ("dipole amplitude without sqrt 2", o.photo_amplitudes, "math.sqrt(2.0) * a * (Fp.T @ y)", "a * (Fp.T @ y)"),
    ("boundary derivative without s'", o.photo_amplitudes, "+= f[\"sp\"][:no]", "+= 0.0 * f[\"sp\"][:no]"),
    ("boundary derivative Lambda by column", o.photo_amplitudes, "f[\"lam\"][:, None] * Y",
     "f[\"lam\"][None, :no] * Y"),
    ("photon energy sign", o.sweep, "(E - float(wave.e0))", "(float(wave.e0) - E)"),
    ("FWHM taken as the standard deviation", o.convolve_average,
     "sd = fwhm / (2.0 * math.sqrt(2.0 * math.log(2.0)))", "sd = fwhm"),
    ("convolution without mesh weights", o.convolve_average, ") ** 2) * tw", ") ** 2) * 1.0"),
    ("statistical weights ignored", o.convolve_average, "mixed = f @ sigma", "mixed = sigma.sum(axis=0)"),
]


@pytest.mark.parametrize("name,func,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_mutation_is_caught(monkeypatch, name, func, old, new):
    monkeypatch.setattr(o, func.__name__, mutate(func, old, new))
    res = run_pins()
    assert not all(res.values()), f"mutation '{name}' passed every pin: {res}"
