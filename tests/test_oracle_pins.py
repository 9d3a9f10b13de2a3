"""Pins of the FP64 oracle against closed forms, invariants and brute force.

None of these tests re-types the oracle's formulas: each compares the oracle
with an independent route (textbook closed forms for the Riccati functions,
the single-pole Breit-Wigner phase shift, the Lane-Thomas shift/penetration
form for l > 0, the Bloch-operator resolvent in a finite basis, SciPy's
modified spherical Bessel function, a closed-channel elimination formula) or
with an invariant the physics fixes (K symmetric, S unitary and symmetric,
detailed balance, the optical theorem, Wigner's dR/dE >= 0, the +pi rise of the
eigenphase sum across an isolated resonance).
"""
import math

import numpy as np
import pytest
from scipy.special import spherical_kn

from oracle import rmatrix as o
from paper_1403_5524_gb300 import synth

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


# ----------------------------------------------------------------------------
# textbook Riccati-Bessel functions for l <= 2 (explicit trigonometric forms)
# ----------------------------------------------------------------------------
def jhat_explicit(l, x):
    s, c = math.sin(x), math.cos(x)
    if l == 0:
        return s, c
    if l == 1:
        return s / x - c, c / x - s / x ** 2 + s
    if l == 2:
        v = (3.0 / x ** 2 - 1.0) * s - 3.0 * c / x
        dv = (-6.0 / x ** 3) * s + (3.0 / x ** 2 - 1.0) * c + 3.0 * s / x + 3.0 * c / x ** 2
        return v, dv
    raise ValueError


def nhat_explicit(l, x):
    s, c = math.sin(x), math.cos(x)
    if l == 0:
        return -c, s
    if l == 1:
        return -c / x - s, s / x + c / x ** 2 - c
    if l == 2:
        v = -(3.0 / x ** 2 - 1.0) * c - 3.0 * s / x
        dv = (6.0 / x ** 3) * c + (3.0 / x ** 2 - 1.0) * s - 3.0 * c / x + 3.0 * s / x ** 2
        return v, dv
    raise ValueError


@pytest.mark.parametrize("l", [0, 1, 2])
@pytest.mark.parametrize("x", [0.07, 0.9, 3.3, 17.0, 86.0])
def test_riccati_explicit(l, x):
    j, jp = o.riccati_jn(l, x)
    n, np_ = o.riccati_yn(l, x)
    je, jpe = jhat_explicit(l, x)
    ne, npe = nhat_explicit(l, x)
    scale = max(1.0, abs(ne))
    assert abs(j - je) <= 1e-13 * max(1.0, abs(je)) + 1e-15 * scale
    assert abs(jp - jpe) <= 1e-12 * max(1.0, abs(jpe), abs(npe))
    assert abs(n - ne) <= 1e-13 * scale
    assert abs(np_ - npe) <= 1e-12 * max(1.0, abs(npe))


@pytest.mark.parametrize("l", list(range(16)))
def test_riccati_wronskian(l):
    # jhat nhat' - jhat' nhat = 1 for every l (open-channel normalisation)
    for x in [0.5, 2.0, 7.0, 30.0, 90.0]:
        j, jp = o.riccati_jn(l, x)
        n, np_ = o.riccati_yn(l, x)
        w = j * np_ - jp * n
        assert abs(w - 1.0) < 1e-9, (l, x, w)


@pytest.mark.parametrize("l", [0, 1, 3, 7, 15])
@pytest.mark.parametrize("x", [0.03, 0.5, 4.0, 40.0])
def test_khat_logderiv_vs_scipy(l, x):
    # x k_l(x) from SciPy; log-derivative (k + x k')/(x k)
    k = spherical_kn(l, x)
    kp = spherical_kn(l, x, derivative=True)
    ref = (k + x * kp) / (x * k)
    got = o.khat_logderiv(l, x)
    assert abs(got - ref) <= 1e-12 * abs(ref)


# ----------------------------------------------------------------------------
# p1: single channel, single pole (Breit-Wigner closed form)
# ----------------------------------------------------------------------------
def one_channel_wave(l, w, E1, a):
    return synth.Wave(l=np.array([l], np.int32), thresh=np.array([0.0]),
                      poles=np.array([E1]), W=np.array([[w]]), a=a)


@pytest.mark.parametrize("E", [0.05, 0.3, 1.1, 2.4, 2.6, 3.9])
def test_breit_wigner_s_wave(E):
    a, w, E1 = 20.0, 0.7, 2.5
    wave = one_channel_wave(0, w, E1, a)
    out = o.sweep(wave, np.array([E]), sel=(0,))
    k = math.sqrt(E)
    delta = -k * a + math.atan(k * w * w / (2.0 * (E1 - E)))
    K = out["K"][0, 0, 0]
    # K = tan(delta)
    assert abs(math.atan(K) - o.wrap_angle(2 * delta) / 2) < 1e-12 or \
        abs(abs(math.atan(K) - o.wrap_angle(2 * delta) / 2) - math.pi / 2) < 1e-12
    assert abs(math.sin(math.atan(K) - delta)) < 1e-12
    # eta = delta mod pi
    assert abs(math.sin(out["eta"][0] - delta)) < 1e-12
    # sigma = (4 pi / k^2) sin^2 delta
    sig = 4.0 * math.pi / k ** 2 * math.sin(delta) ** 2
    assert abs(out["sig_sel"][0, 0, 0] - sig) <= 1e-12 * max(sig, 1e-300) + 1e-14
    assert abs(out["sig_tot"][0, 0] - sig) <= 1e-12 * max(sig, 1e-300) + 1e-14
    # S = exp(2 i delta)
    S, T = o.smatrix(np.array([[K]]))
    assert abs(S[0, 0] - np.exp(2j * delta)) < 1e-12
    # R itself: w^2 / (2 a (E1 - E))
    R = out["R"][0, 0]
    assert abs(R - w * w / (2 * a * (E1 - E))) <= 1e-15 * abs(R)


@pytest.mark.parametrize("l", [1, 2])
@pytest.mark.parametrize("E", [0.08, 0.6, 1.7, 2.45, 2.55])
def test_lane_thomas_single_channel(l, E):
    # delta_l = -phi_l + arctan(P_l R / (1 - S_l R)) with x O'/O = S_l + i P_l,
    # O_l = -nhat_l + i jhat_l ~ exp(i(x - l pi/2)), phi_l = arg O_l(ka), b = 0.
    a, w, E1 = 20.0, 0.5, 2.5
    wave = one_channel_wave(l, w, E1, a)
    out = o.sweep(wave, np.array([E]))
    k = math.sqrt(E)
    x = k * a
    j, jp = jhat_explicit(l, x)
    n, np_ = nhat_explicit(l, x)
    O = complex(-n, j)
    Op = complex(-np_, jp)
    L = x * Op / O
    Sl, Pl = L.real, L.imag
    R = w * w / (2.0 * a * (E1 - E))
    delta = -np.angle(O) + math.atan2(Pl * R, 1.0 - Sl * R)
    K = out["K"][0, 0, 0]
    assert abs(math.sin(math.atan(K) - delta)) < 1e-11
    assert abs(math.sin(out["eta"][0] - delta)) < 1e-11


# ----------------------------------------------------------------------------
# p2: hard sphere (no poles couple): K_ii = jhat_l(ka) / nhat_l(ka)
# ----------------------------------------------------------------------------
def test_hard_sphere():
    a = 12.0
    wave = synth.Wave(l=np.array([0, 1, 2, 1], np.int32), thresh=np.array([0.0, 0.2, 0.5, 3.0]),
                      poles=np.array([-1.0, 4.0]), W=np.zeros((4, 2)), a=a)
    E = 1.3
    out = o.sweep(wave, np.array([E]))
    assert out["n_open"][0] == 3
    K = out["K"][0]
    for i in range(3):
        x = math.sqrt(E - wave.thresh[i]) * a
        j, _ = jhat_explicit(int(wave.l[i]), x)
        n, _ = nhat_explicit(int(wave.l[i]), x)
        assert abs(K[i, i] - j / n) <= 1e-12 * max(1.0, abs(j / n))
    off = K[:3, :3] - np.diag(np.diag(K[:3, :3]))
    assert np.abs(off).max() == 0.0
    # s wave: K = -tan(ka)
    x0 = math.sqrt(E) * a
    assert abs(K[0, 0] + math.tan(x0)) <= 1e-12 * max(1.0, abs(math.tan(x0)))
    # the closed channel carries no cross section
    assert np.all(out["sig_sel"][0, 0, 3:] == 0.0)


# ----------------------------------------------------------------------------
# p3: uncoupled reduction (each pole couples to one channel)
# ----------------------------------------------------------------------------
def test_uncoupled_reduction():
    rng = np.random.default_rng(5)
    n, per = 4, 30
    N = n * per
    poles = np.sort(rng.uniform(-3.0, 15.0, N))
    owner = rng.permutation(np.repeat(np.arange(n), per))
    W = np.zeros((n, N))
    W[owner, np.arange(N)] = rng.normal(0, 1 / math.sqrt(N), N)
    wave = synth.Wave(l=np.array([0, 2, 1, 3], np.int32), thresh=np.array([0.0, 0.3, 0.6, 0.9]),
                      poles=poles, W=W, a=15.0)
    E = np.array([0.45, 1.2, 2.0])
    out = o.sweep(wave, E)
    for t, e in enumerate(E):
        no = out["n_open"][t]
        K = out["K"][t, :no, :no]
        assert np.abs(K - np.diag(np.diag(K))).max() <= 1e-14 * np.abs(K).max()
        for i in range(no):
            sub = synth.Wave(l=wave.l[i:i + 1], thresh=wave.thresh[i:i + 1].copy(), poles=poles,
                             W=W[i:i + 1].copy(), a=wave.a)
            ref = o.sweep(sub, np.array([e]))
            assert abs(K[i, i] - ref["K"][0, 0, 0]) <= 1e-11 * max(1.0, abs(K[i, i]))


# ----------------------------------------------------------------------------
# p4: pole sum against the Bloch-operator resolvent of a small inner region
# ----------------------------------------------------------------------------
def bloch_inner_region(n_ch, n_basis, a, l, e_thr, seed):
    """H + L_Bloch (b = 0) in a sine basis u_m(r) = sin((m - 1/2) pi r / a).

    Rydberg form: -d2/dr2 + l(l+1)/r^2 + V_ij(r) + e_i delta_ij on [0, a]; with
    u(0) = 0 the Bloch term turns the kinetic part into int u_m' u_n' dr.
    Returns (H, O, B) with B[:, i] = boundary values of channel i's basis.
    """
    rng = np.random.default_rng(seed)
    xg, wg = np.polynomial.legendre.leggauss(600)
    r = 0.5 * a * (xg + 1.0)
    wr = 0.5 * a * wg
    km = (np.arange(1, n_basis + 1) - 0.5) * math.pi / a
    u = np.sin(np.outer(km, r))
    du = km[:, None] * np.cos(np.outer(km, r))
    ua = np.sin(km * a)
    amp = rng.normal(0, 1.0, (n_ch, n_ch))
    amp = 0.5 * (amp + amp.T)
    rng_c = rng.uniform(1.0, 4.0, (n_ch, n_ch))
    rng_c = 0.5 * (rng_c + rng_c.T)
    dim = n_ch * n_basis
    H = np.zeros((dim, dim))
    O = np.zeros((dim, dim))
    Bv = np.zeros((dim, n_ch))
    ovl = (u * wr) @ u.T
    kin = (du * wr) @ du.T
    for i in range(n_ch):
        si = slice(i * n_basis, (i + 1) * n_basis)
        Bv[si, i] = ua
        O[si, si] = ovl
        for j in range(n_ch):
            sj = slice(j * n_basis, (j + 1) * n_basis)
            V = -amp[i, j] * np.exp(-r / rng_c[i, j])
            if i == j:
                V = V + l[i] * (l[i] + 1) / r ** 2 + e_thr[i]
            H[si, sj] = (u * (wr * V)) @ u.T
            if i == j:
                H[si, sj] += kin
    return H, O, Bv


def test_bloch_resolvent_brute_force():
    import scipy.linalg as sl
    a = 10.0
    n_ch, nb = 3, 14
    l = [0, 1, 2]
    e_thr = [0.0, 0.35, 0.8]
    H, O, Bv = bloch_inner_region(n_ch, nb, a, l, e_thr, seed=11)
    Ek, C = sl.eigh(H, O)                 # C^T O C = 1
    phi_a = Bv.T @ C                      # (n_ch, dim) boundary amplitudes
    W = math.sqrt(2.0) * phi_a            # w_ik = sqrt(2) psi_ik(a)
    for E in [0.13, 0.57, 1.4, 2.9]:
        R_pole = o.rmatrix(W, Ek, E, a)
        G = np.linalg.solve(H - E * O, Bv)
        R_direct = (Bv.T @ G) / a
        assert np.abs(R_pole - R_direct).max() <= 1e-10 * np.abs(R_direct).max()
        assert np.abs(R_pole - R_pole.T).max() <= 1e-14 * np.abs(R_pole).max()


# ----------------------------------------------------------------------------
# invariants on a seeded coupled workload
# ----------------------------------------------------------------------------
@pytest.fixture(scope="module")
def c1_out():
    w = synth.config(1)
    return w, o.sweep(w.waves[0], w.energies, sel=(0, 1, 2, 3))


def test_k_symmetric_s_unitary(c1_out):
    w, out = c1_out
    for t in range(out["E"].shape[0]):
        no = out["n_open"][t]
        if out["flags"][t] & o.FLAG_ILLCOND:
            continue
        K = out["K"][t, :no, :no]
        assert np.abs(K - K.T).max() <= 1e-12 * max(np.abs(K).max(), 1.0)
        S, T = o.smatrix(K)
        assert np.abs(S @ S.conj().T - np.eye(no)).max() <= 1e-12
        assert np.abs(S - S.T).max() <= 1e-12


def test_detailed_balance_and_optical_theorem(c1_out):
    w, out = c1_out
    thr = w.waves[0].thresh
    for t in range(0, out["E"].shape[0], 7):
        no = out["n_open"][t]
        E = out["E"][t]
        k2 = E - thr
        sig = out["sig_sel"][t]
        for i in range(no):
            for j in range(no):
                lhs, rhs = k2[i] * sig[i, j], k2[j] * sig[j, i]
                assert abs(lhs - rhs) <= 1e-11 * max(abs(lhs), 1e-300) + 1e-300
        S, T = o.smatrix(out["K"][t, :no, :no])
        for i in range(no):
            opt = 2 * math.pi / k2[i] * (1.0 - S[i, i].real)
            assert abs(out["sig_tot"][t, i] - opt) <= 1e-10 * max(opt, 1e-300)


def test_wigner_monotone():
    w = synth.config(1).waves[0]
    poles = w.poles
    # pick a gap between consecutive poles and two energies inside it
    gaps = np.diff(poles)
    g = int(np.argmax(gaps * ((poles[:-1] > 0.2) & (poles[1:] < 3.0))))
    E1 = poles[g] + 0.25 * gaps[g]
    E2 = poles[g] + 0.75 * gaps[g]
    dR = o.rmatrix(w.W, poles, E2, w.a) - o.rmatrix(w.W, poles, E1, w.a)
    ev = np.linalg.eigvalsh(dR)
    assert ev.min() >= -1e-14 * np.abs(ev).max()
    assert ev.max() > 0.0


def test_resonance_raises_eigenphase_by_pi():
    # smooth background from far poles plus one narrow isolated pole at Er:
    # across Er the eigenphase sum rises by pi more than the background alone
    rng = np.random.default_rng(3)
    n = 3
    far = np.concatenate([rng.uniform(-8, -2, 40), rng.uniform(12, 30, 40)])
    Er = 1.5
    poles = np.sort(np.concatenate([far, [Er]]))
    W = rng.normal(0, 0.3, (n, poles.size))
    ir = int(np.searchsorted(poles, Er))
    W[:, ir] = np.array([0.01, 0.008, 0.005])
    Wbg = W.copy()
    Wbg[:, ir] = 0.0
    E = np.linspace(Er - 0.01, Er + 0.01, 4001)
    rises = []
    for WW in (W, Wbg):
        wave = synth.Wave(l=np.array([0, 1, 0], np.int32), thresh=np.array([0.0, 0.1, 0.2]),
                          poles=poles, W=WW, a=10.0)
        out = o.sweep(wave, E, keep_R=False, keep_K=False)
        eta = np.unwrap(2.0 * out["eta"]) / 2.0      # eta is defined mod pi
        rises.append(eta[-1] - eta[0])
    assert abs(rises[0] - rises[1] - math.pi) < 0.03, rises


def test_closed_channel_elimination():
    # one open s-wave channel, one closed channel; the open-channel phase shift
    # from R_eff = R_00 + a R_01 L1 (1 - a R_11 L1)^-1 R_10, L1 from SciPy's k_l
    rng = np.random.default_rng(9)
    N = 25
    poles = np.sort(rng.uniform(-2, 12, N))
    W = rng.normal(0, 1 / math.sqrt(N), (2, N))
    a = 8.0
    lc = 2
    wave = synth.Wave(l=np.array([0, lc], np.int32), thresh=np.array([0.0, 2.0]),
                      poles=poles, W=W, a=a)
    for E in [0.3, 0.9, 1.6, 1.95]:
        out = o.sweep(wave, np.array([E]))
        assert out["n_open"][0] == 1
        R = o.rmatrix(W, poles, E, a)
        kap = math.sqrt(2.0 - E)
        x = kap * a
        kk = spherical_kn(lc, x)
        kkp = spherical_kn(lc, x, derivative=True)
        L1 = kap * (kk + x * kkp) / (x * kk)
        Reff = R[0, 0] + a * R[0, 1] * L1 * R[1, 0] / (1.0 - a * R[1, 1] * L1)
        k = math.sqrt(E)
        delta = -k * a + math.atan(k * a * Reff)
        assert abs(math.sin(math.atan(out["K"][0, 0, 0]) - delta)) < 1e-11


def test_eigenphase_from_determinant(c1_out):
    # sum arctan(lambda) == -arg det(I - iK) (mod 2 pi): the form the GPU uses
    w, out = c1_out
    for t in range(0, out["E"].shape[0], 11):
        no = out["n_open"][t]
        K = out["K"][t, :no, :no]
        d = np.linalg.det(np.eye(no) - 1j * K)
        assert abs(o.wrap_angle(out["eta"][t] + np.angle(d))) < 1e-11


def test_nudge():
    poles = np.array([0.5, 1.0])
    thr = np.array([0.0, 0.7])
    E = np.array([0.5 + 5e-10, 0.7 - 2e-10, 0.9, 1.0])
    En, fl = o.nudge_energies(E, poles, thr)
    assert En[0] == E[0] + 1e-6 and fl[0] == o.FLAG_NUDGED
    assert En[1] == E[1] + 1e-6 and fl[1] == o.FLAG_NUDGED | o.FLAG_NEAR_THRESHOLD
    assert En[2] == E[2] and fl[2] == 0
    assert En[3] == 1.0 + 1e-6


def test_near_threshold_classification():
    # flagged when the given energy is strictly within 1e-6 Ry of a threshold, from either side;
    # poles do not count; the flag comes from the energy before the nudge
    poles = np.array([0.3])
    thr = np.array([0.0, 0.7, 1.2])
    E = np.array([0.7 - 9e-7, 0.7 + 9e-7, 0.7 - 1.1e-6, 0.7 + 1.1e-6, 0.3 + 5e-7, 1.2, 1.2 + 2e-6, 5e-7])
    En, fl = o.nudge_energies(E, poles, thr)
    near = (fl & o.FLAG_NEAR_THRESHOLD) != 0
    assert near.tolist() == [True, True, False, False, False, True, False, True]
    assert fl[5] & o.FLAG_NUDGED and En[5] == 1.2 + 1e-6   # on a threshold: moved and flagged
    assert not fl[4] & o.FLAG_NUDGED                        # 5e-7 from a pole: neither


def test_pole_sum_loops_and_packing():
    w = synth.small(1, 5, 17, 3).waves[0]
    for E in [0.2, 1.7]:
        R = o.rmatrix(w.W, w.poles, E, w.a)
        R2 = o.rmatrix_loops(w.W, w.poles, E, w.a)
        assert np.abs(R - R2).max() <= 1e-14 * np.abs(R).max()
        Rp = o.pack_upper(R)
        for i in range(5):
            for j in range(i, 5):
                assert Rp[o.pair_index(5, i, j)] == R[i, j]
        assert np.abs(o.unpack_upper(Rp, 5) - R).max() <= 1e-15 * np.abs(R).max()


def test_window_split_adds_up():
    w = synth.small(2, 6, 300, 1, pole_lo=-1, pole_hi=4).waves[0]
    E = 1.234
    full = o.rmatrix(w.W, w.poles, E, w.a)
    far = o.rmatrix(w.W, w.poles, E, w.a, delta=0.05, part="far")
    near = o.rmatrix(w.W, w.poles, E, w.a, delta=0.05, part="near")
    assert np.abs(far + near - full).max() <= 1e-14 * np.abs(full).max()
    assert np.any(np.abs(w.poles - E) < 0.05)


def test_mpmath_precision_bound():
    # the oracle's own FP64 rounding on a tiny case, against 40-digit arithmetic
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    w = synth.small(4, 3, 12, 1, pole_lo=-1, pole_hi=6, a=6.0, thr_hi=0.8).waves[0]
    E = 1.37
    out = o.sweep(w, np.array([E]))
    n = 3
    a = mp.mpf(w.a)
    R = mp.matrix(n, n)
    for i in range(n):
        for j in range(n):
            R[i, j] = mp.fsum(mp.mpf(w.W[i, k]) * mp.mpf(w.W[j, k]) / (mp.mpf(w.poles[k]) - mp.mpf(E))
                              for k in range(w.N)) / (2 * a)
    Ro = o.unpack_upper(out["R"][0], n)
    assert max(abs(float(R[i, j]) - Ro[i, j]) for i in range(n) for j in range(n)) <= 1e-15 * 10

    def rj(l, x):
        return x * mp.sqrt(mp.pi / (2 * x)) * mp.besselj(l + mp.mpf(1) / 2, x)

    def ry(l, x):
        return x * mp.sqrt(mp.pi / (2 * x)) * mp.bessely(l + mp.mpf(1) / 2, x)

    no = out["n_open"][0]
    assert no == n
    s = []; sp = []; c = []; cp = []
    for i in range(n):
        k = mp.sqrt(mp.mpf(E) - mp.mpf(w.thresh[i]))
        x = k * a
        l = int(w.l[i])
        s.append(rj(l, x) / mp.sqrt(k)); sp.append(mp.diff(lambda r: rj(l, k * r), a) / mp.sqrt(k))
        c.append(-ry(l, x) / mp.sqrt(k)); cp.append(-mp.diff(lambda r: ry(l, k * r), a) / mp.sqrt(k))
    M = mp.matrix(n, n)
    B = mp.matrix(n, n)
    for i in range(n):
        for j in range(n):
            M[i, j] = (c[j] if i == j else 0) - a * R[i, j] * cp[j]
            B[i, j] = (s[j] if i == j else 0) - a * R[i, j] * sp[j]
    X = mp.matrix(n, n)
    for m in range(n):
        col = mp.lu_solve(M, mp.matrix([-B[i, m] for i in range(n)]))
        for i in range(n):
            X[i, m] = col[i]
    K = out["K"][0]
    kmax = max(abs(float(X[i, j])) for i in range(n) for j in range(n))
    err = max(abs(float(X[i, j]) - K[i, j]) for i in range(n) for j in range(n))
    assert err <= 1e-13 * kmax
