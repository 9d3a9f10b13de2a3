"""Plain FP64 CPU oracle for the R-matrix outer-region energy sweep.

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
baseline leg of the benchmark may import this module.  The product path (the
CUDA library and its binding) never imports, links or executes it, and this
module imports nothing from the product path.

What it computes, for one partial wave and one energy E (Rydberg units, radius
in bohr, k^2 = E - e_i):

1. R-matrix pole sum (Eq. 1, written as a matrix product in Eq. 2):
   R_ij(E) = (1/2a) sum_k w_ik w_jk / (E_k - E).
   Eq. 1 prints sum_k W_ik W_kj / (E - E_k) with no 1/(2a); this oracle takes
   the Rydberg-units form with surface amplitudes w_ik = sqrt(2) psi_ik(a), whose
   sign makes dR/dE positive semidefinite (Wigner causality).
2. Open/closed split: channel i is open when E > e_i; thresholds are sorted, so
   the open channels are a prefix of length n_o.
3. Zero-potential asymptotic functions at r = a (the paper does not give them;
   standard reading): open channels s_i = k^-1/2 jhat_l(kr),
   c_i = -k^-1/2 nhat_l(kr) (Riccati-Bessel, nhat_l = x y_l(x) ~ -cos(x - l pi/2)),
   so that every open channel has Wronskian s c' - s' c = -1; closed channels
   decay as khat_l(kappa r), kappa = sqrt(e_i - E).
3'. Ionic targets (residual charge z > 0, potential -2z/r in Rydberg units;
   the paper's targets are ions but it gives no outer-region formulas, so this
   is the standard Coulomb reading): open channels use the Coulomb functions
   F_l(eta, kr), G_l(eta, kr) with eta = -z/k in place of jhat_l and -nhat_l
   (s = k^-1/2 F, c = k^-1/2 G; z = 0 gives back item 3), closed channels decay
   as the Whittaker function W_{z/kappa, l+1/2}(2 kappa r).  Both come from
   mpmath (30 digits); derivatives from the standard recurrence relations.
4. Matching with Bloch constant b = 0, F(a) = a R F'(a), F_ij ~ s_i d_ij + c_i K_ij
   (open i), F_ij ~ e_i(r) x_ij (closed i).  Column j of the matching matrix is
   divided by c_j (open) or e_j (closed); the system becomes
   (I - a R Lambda) Y = -B, Lambda_j = c'_j/c_j or e'_j/e_j,
   B[:, m] = s_m delta_m - a R[:, m] s'_m, and K_jm = Y_jm / c_j.
   Solved by LU with partial pivoting (LAPACK getrf/getrs).
5. S = (I + iK)(I - iK)^-1, T = S - I, sigma_{i->j} = (pi / k_i^2) |T_ji|^2
   (statistical weight (2J+1)/g_i taken as 1), eigenphase sum
   eta = sum_m arctan(lambda_m(K)).

6. Photoionisation (a wave with a bound-free dipole vector d_k = <psi_k|D|Psi_0>
   over the inner-region eigenstates and an initial bound-state energy E_0; the
   paper names the module but prints no formulas, so this is the standard
   R-matrix reading, length form): the inner-region part of the final state is
   sum_k A_k psi_k with A_k = sum_i psi_ik(a) F_i'(a) / (E_k - E), so with
   w_ik = sqrt(2) psi_ik(a) and the dipole vector y_i = (1/2a) sum_k w_ik d_k / (E_k - E)
   the K-normalised amplitude of open solution m is
   M^K_m = sqrt(2) a sum_i F'_im y_i, F'_im = s'_m d_im + Lambda_i Y_im,
   the incoming-wave amplitudes are M^- = (I + iK)^-1 M^K, and
   sigma_PI = (4 pi alpha / 3) omega sum_m |M^-_m|^2 (a0^2; omega = E - E_0 in Ry;
   s, c normalised as k^-1/2 sin, cos, i.e. sqrt(pi) times per-Rydberg energy
   normalisation; initial statistical weight 1).

7. Post-processing to compare with experiment (the paper convolves its cross
   sections with a Gaussian of the experiment's FWHM and averages them over
   initial levels with statistical weights, e.g. 2/3 ground + 1/3 metastable):
   sigma_avg(E) = sum_s f_s int sigma_s(E') G(E - E') dE' / int G(E - E') dE',
   G a normalised Gaussian of full width at half maximum F (standard deviation
   F / (2 sqrt(2 ln 2))); on the mesh the integrals are trapezoid sums over the
   mesh, and dividing by the kernel's own sum keeps a constant a constant at
   the mesh ends.

Energies closer than 1e-9 Ry to a pole or a threshold are moved up by 1e-6 Ry,
once, and flagged.

The paper prints no worked example for this path; the tests pin every step to
closed forms and invariants instead (Breit-Wigner single pole, hard sphere,
uncoupled channels, Bloch-operator resolvent, symmetry, unitarity, detailed
balance, Wigner monotonicity, resonance causality).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg
from scipy.special import spherical_jn, spherical_yn

FLAG_NUDGED = 1
FLAG_ILLCOND = 2
FLAG_NO_OPEN = 4
FLAG_SINGULAR = 8
FLAG_NEAR_THRESHOLD = 128

NUDGE_TOL = 1e-9
NUDGE_SHIFT = 1e-6
NEAR_THRESHOLD = 1e-6
ILLCOND_RATIO = 1e-12


# ----------------------------------------------------------------------------
# energy mesh preparation
# ----------------------------------------------------------------------------
def nudge_energies(energies, poles, thresh):
    """Move every energy within 1e-9 Ry of a pole or a threshold up by 1e-6 Ry.

    Applied once per energy (no re-check after the move).  Returns the new mesh
    and a uint8 flag array with FLAG_NUDGED set where a move happened, and
    FLAG_NEAR_THRESHOLD where the given energy lies within 1e-6 Ry of a channel
    threshold: a channel opens there (k -> 0), so such energies are judged
    apart from the rest of the mesh.
    """
    E = np.array(energies, dtype=np.float64, copy=True)
    flags = np.zeros(E.shape, dtype=np.uint8)
    for e in range(E.shape[0]):
        near = False
        if poles.size:
            near |= bool(np.min(np.abs(poles - E[e])) < NUDGE_TOL)
        if thresh.size:
            dthr = float(np.min(np.abs(thresh - E[e])))
            near |= dthr < NUDGE_TOL
            if dthr < NEAR_THRESHOLD:
                flags[e] |= FLAG_NEAR_THRESHOLD
        if near:
            E[e] = E[e] + NUDGE_SHIFT
            flags[e] |= FLAG_NUDGED
    return E, flags


def n_open(thresh, E):
    """Number of open channels at energy E: #{i : e_i < E}."""
    return int(np.count_nonzero(thresh < E))


# ----------------------------------------------------------------------------
# pole sum (Eq. 1 / Eq. 2)
# ----------------------------------------------------------------------------
def rmatrix(W, poles, E, a, delta=None, part="all"):
    """R_ij(E) = (1/2a) sum_k w_ik w_jk / (E_k - E), Eq. 1 as the product of Eq. 2.

    X_ik = w_ik / (E_k - E) and Y = W^T, so R = X Y / (2a), one GEMM per energy.
    ``part`` restricts the sum to the near-pole window |E_k - E| < delta
    ("near") or to its complement ("far"); "all" is the full sum.
    """
    d = 1.0 / (poles - E)
    if part != "all":
        inside = np.abs(poles - E) < delta
        if part == "far":
            d = np.where(inside, 0.0, d)
        elif part == "near":
            d = np.where(inside, d, 0.0)
        else:
            raise ValueError(part)
    return (W * d[None, :]) @ W.T / (2.0 * a)


def rmatrix_loops(W, poles, E, a):
    """The same pole sum as three plain loops (tiny sizes only)."""
    n, N = W.shape
    R = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            s = 0.0
            for k in range(N):
                s += W[i, k] * W[j, k] / (poles[k] - E)
            R[i, j] = s / (2.0 * a)
    return R


def pair_index(n, i, j):
    """Packed upper-triangle index p(i, j) = i n - i(i-1)/2 + (j - i), i <= j."""
    return i * n - (i * (i - 1)) // 2 + (j - i)


def pack_upper(R):
    """Pack the upper triangle of a symmetric n x n matrix, row by row."""
    n = R.shape[0]
    iu = np.triu_indices(n)
    return R[iu]


def unpack_upper(Rp, n):
    R = np.zeros((n, n))
    iu = np.triu_indices(n)
    R[iu] = Rp
    R.T[iu] = Rp
    return R


# ----------------------------------------------------------------------------
# asymptotic functions at r = a
# ----------------------------------------------------------------------------
def riccati_jn(l, x):
    """jhat_l(x) = x j_l(x) and its x-derivative (SciPy spherical Bessel)."""
    j = spherical_jn(l, x)
    jp = spherical_jn(l, x, derivative=True)
    return x * j, j + x * jp


def riccati_yn(l, x):
    """nhat_l(x) = x y_l(x) (~ -cos(x - l pi/2)) and its x-derivative."""
    y = spherical_yn(l, x)
    yp = spherical_yn(l, x, derivative=True)
    return x * y, y + x * yp


def khat_logderiv(l, x):
    """x-log-derivative of the decaying Riccati function khat_l(x).

    khat_l(x) = exp(-x) p_l(x), p_l(x) = sum_{m=0}^{l} (l+m)!/(m!(l-m)!) (2x)^-m,
    so khat_l'/khat_l = p_l'/p_l - 1.
    """
    p = 0.0
    dp = 0.0
    for m in range(l + 1):
        c = math.factorial(l + m) / (math.factorial(m) * math.factorial(l - m)) / (2.0 ** m)
        p += c * x ** (-m)
        dp += -m * c * x ** (-m - 1)
    return dp / p - 1.0


def coulomb_open(l, eta, rho):
    """Coulomb functions F_l(eta, rho), G_l(eta, rho) and their rho-derivatives.

    Values from mpmath (coulombf / coulombg, 30 significant digits).  The
    derivatives follow from the relation between orders l and l + 1,
    (l+1) u_l' = ((l+1)^2 / rho + eta) u_l - sqrt((l+1)^2 + eta^2) u_{l+1}
    for u = F or G (Abramowitz & Stegun 14.2.1).
    """
    import mpmath as mp
    with mp.workdps(30):
        r = mp.mpf(rho)
        e = mp.mpf(eta)
        L = l + 1
        c1 = (L * L / r + e) / L
        c2 = mp.sqrt(L * L + e * e) / L
        F, F1 = mp.coulombf(l, e, r), mp.coulombf(l + 1, e, r)
        G, G1 = mp.coulombg(l, e, r), mp.coulombg(l + 1, e, r)
        return float(F), float(c1 * F - c2 * F1), float(G), float(c1 * G - c2 * G1)


def whittaker_logderiv(l, kp, x):
    """W'(x) / W(x) for the decaying Whittaker function W_{kp, l+1/2}(x).

    Values from mpmath (whitw, 30 digits); the derivative from
    x W'_{k,m}(x) = (x/2 - k) W_{k,m}(x) - W_{k+1,m}(x).
    """
    import mpmath as mp
    with mp.workdps(30):
        xx = mp.mpf(x)
        k = mp.mpf(kp)
        m = mp.mpf(l) + mp.mpf(1) / 2
        W0 = mp.whitw(k, m, xx)
        W1 = mp.whitw(k + 1, m, xx)
        return float(((xx / 2 - k) * W0 - W1) / (xx * W0))


def channel_functions(l, thresh, E, a, z=0.0):
    """Per-channel matching data at energy E (residual target charge z >= 0).

    Returns dict with n_o, k2 (E - e_i), and for open channels s, s', c, c'
    (r-derivatives); for every channel the scaled log-derivative Lambda used as
    column scale of the matching matrix.
    """
    n = l.shape[0]
    k2 = E - thresh
    no = n_open(thresh, E)
    s = np.zeros(n); sp = np.zeros(n); c = np.zeros(n); cp = np.zeros(n)
    lam = np.zeros(n)
    for i in range(n):
        if z != 0.0:
            if k2[i] > 0.0:
                k = math.sqrt(k2[i])
                F, Fp, G, Gp = coulomb_open(int(l[i]), -z / k, k * a)
                s[i] = F / math.sqrt(k)
                sp[i] = Fp * math.sqrt(k)
                c[i] = G / math.sqrt(k)
                cp[i] = Gp * math.sqrt(k)
                lam[i] = cp[i] / c[i]
            else:
                kap = math.sqrt(-k2[i])
                lam[i] = 2.0 * kap * whittaker_logderiv(int(l[i]), z / kap, 2.0 * kap * a)
            continue
        if k2[i] > 0.0:
            k = math.sqrt(k2[i])
            x = k * a
            jh, jhp = riccati_jn(int(l[i]), x)
            nh, nhp = riccati_yn(int(l[i]), x)
            s[i] = jh / math.sqrt(k)
            sp[i] = jhp * math.sqrt(k)
            c[i] = -nh / math.sqrt(k)
            cp[i] = -nhp * math.sqrt(k)
            lam[i] = cp[i] / c[i]
        else:
            kap = math.sqrt(-k2[i])
            lam[i] = kap * khat_logderiv(int(l[i]), kap * a)
    return {"n_o": no, "k2": k2, "s": s, "sp": sp, "c": c, "cp": cp, "lam": lam}


# ----------------------------------------------------------------------------
# matching -> K, then S, eigenphase sum, cross sections
# ----------------------------------------------------------------------------
def kmatrix(R, l, thresh, E, a, z=0.0):
    """Open-open K-matrix from the R-matrix at energy E (b = 0 matching).
    z is the residual charge of the target (0: neutral, item 3; > 0: item 3').

    Solves (I - a R Lambda) Y = -B by LU with partial pivoting; K = Y[:n_o]/c.
    Returns (K (n_o x n_o), n_o, flags, pivot ratio min|u_jj| / max|u_jj|).
    """
    n = l.shape[0]
    f = channel_functions(l, thresh, E, a, z)
    no = f["n_o"]
    flags = 0
    if no == 0:
        return np.zeros((0, 0)), 0, FLAG_NO_OPEN, 1.0
    Mt = np.eye(n) - a * R * f["lam"][None, :]
    B = -a * R[:, :no] * f["sp"][None, :no]
    B[np.arange(no), np.arange(no)] += f["s"][:no]
    lu, piv = scipy.linalg.lu_factor(Mt, check_finite=False)
    d = np.abs(np.diag(lu))
    if d.min() == 0.0:
        return np.full((no, no), np.nan), no, FLAG_SINGULAR, 0.0
    ratio = d.min() / d.max()
    if ratio < ILLCOND_RATIO:
        flags |= FLAG_ILLCOND
    Y = scipy.linalg.lu_solve((lu, piv), -B, check_finite=False)
    K = Y[:no, :] / f["c"][:no, None]
    return K, no, flags, ratio


ALPHA = 7.2973525693e-3                    # fine-structure constant (CODATA 2018)
PI_PREFACTOR = 4.0 * math.pi * ALPHA / 3.0   # sigma_PI = PI_PREFACTOR omega sum |M^-|^2


def dipole_vector(W, dip, poles, E, a):
    """y_i(E) = (1/2a) sum_k w_ik d_k / (E_k - E): the pole sum of item 6."""
    return (W @ (dip / (poles - E))) / (2.0 * a)


def photo_amplitudes(R, y, l, thresh, E, a, z=0.0):
    """Dipole amplitudes of the open final channels at energy E (item 6).

    Solves the matching system of item 4 for Y, forms the boundary derivatives
    F'_im = s'_m delta_im + Lambda_i Y_im of each K-normalised solution m, then
    M^K = sqrt(2) a F'^T y and M^- = (I + iK)^-1 M^K.  Returns (M^K, M^-, K).
    """
    n = l.shape[0]
    f = channel_functions(l, thresh, E, a, z)
    no = f["n_o"]
    if no == 0:
        return np.zeros(0), np.zeros(0, complex), np.zeros((0, 0))
    Mt = np.eye(n) - a * R * f["lam"][None, :]
    B = -a * R[:, :no] * f["sp"][None, :no]
    B[np.arange(no), np.arange(no)] += f["s"][:no]
    Y = np.linalg.solve(Mt, -B)
    K = Y[:no, :] / f["c"][:no, None]
    Fp = f["lam"][:, None] * Y
    Fp[np.arange(no), np.arange(no)] += f["sp"][:no]
    MK = math.sqrt(2.0) * a * (Fp.T @ y)
    Mm = np.linalg.solve(np.eye(no) + 1j * K, MK.astype(complex))
    return MK, Mm, K


def smatrix(K):
    """S = (I + iK)(I - iK)^-1 (= (I - iK)^-1 (I + iK) for symmetric K) and T = S - I."""
    no = K.shape[0]
    I = np.eye(no)
    S = np.linalg.solve(I - 1j * K, I + 1j * K)
    return S, S - I


def xsec(T, k2):
    """sigma[i, j] = sigma_{i->j} = (pi / k_i^2) |T_ji|^2 for open i, j (bohr^2)."""
    no = T.shape[0]
    return (math.pi / k2[:no])[:, None] * np.abs(T.T) ** 2


def eigenphase_sum(K):
    """eta = sum_m arctan(lambda_m(K)), in (-n_o pi/2, n_o pi/2)."""
    if K.shape[0] == 0:
        return 0.0
    return float(np.sum(np.arctan(np.linalg.eigvalsh(0.5 * (K + K.T)))))


# ----------------------------------------------------------------------------
# whole sweep
# ----------------------------------------------------------------------------
def sweep(wave, energies, sel=(0,), delta=0.05, part="all", keep_R=True, keep_K=True,
          energy_idx=None):
    """Run the full per-energy path for one wave.

    ``energy_idx`` restricts the work to a subset of mesh indices (the mesh is
    still nudged as a whole).  Returned arrays follow the library's layouts:
    R (m, n_p) packed upper, K (m, n, n) with the open block valid and zeros
    elsewhere, eta (m,), sig_tot (m, n_sel), sig_sel (m, n_sel, n), n_open (m,),
    flags (m,) uint8, piv_ratio (m,).
    """
    l, thr, poles, W, a = wave.l, wave.thresh, wave.poles, wave.W, wave.a
    z = float(getattr(wave, "z", 0.0))
    n = l.shape[0]
    E_all, nflags = nudge_energies(energies, poles, thr)
    idx = np.arange(E_all.shape[0]) if energy_idx is None else np.asarray(energy_idx)
    m = idx.shape[0]
    n_sel = len(sel)
    out = {
        "E": E_all[idx].copy(),
        "eta": np.zeros(m),
        "sig_tot": np.zeros((m, n_sel)),
        "sig_sel": np.zeros((m, n_sel, n)),
        "n_open": np.zeros(m, dtype=np.int32),
        "flags": np.zeros(m, dtype=np.uint8),
        "piv_ratio": np.zeros(m),
    }
    if keep_R:
        out["R"] = np.zeros((m, n * (n + 1) // 2))
    if keep_K:
        out["K"] = np.zeros((m, n, n))
    dip = getattr(wave, "dip", None)
    if dip is not None:
        out["sig_pi"] = np.zeros(m)
        out["sig_pi_ch"] = np.zeros((m, n))
    for t, e in enumerate(idx):
        E = E_all[e]
        R = rmatrix(W, poles, E, a, delta=delta, part=part)
        K, no, fl, ratio = kmatrix(R, l, thr, E, a, z)
        fl |= int(nflags[e])
        out["flags"][t] = fl
        out["n_open"][t] = no
        out["piv_ratio"][t] = ratio
        if keep_R:
            out["R"][t] = pack_upper(R)
        if no == 0 or (fl & FLAG_SINGULAR):
            continue
        if keep_K:
            out["K"][t, :no, :no] = K
        if dip is not None:
            y = dipole_vector(W, np.asarray(dip, dtype=np.float64), poles, E, a)
            _, Mm, _ = photo_amplitudes(R, y, l, thr, E, a, z)
            ch = PI_PREFACTOR * (E - float(wave.e0)) * np.abs(Mm) ** 2
            out["sig_pi_ch"][t, :no] = ch
            out["sig_pi"][t] = float(np.sum(ch))
        S, T = smatrix(K)
        sig = xsec(T, E - thr)
        out["eta"][t] = eigenphase_sum(K)
        for q, i in enumerate(sel):
            if i < no:
                out["sig_sel"][t, q, :no] = sig[i, :]
                out["sig_tot"][t, q] = float(np.sum(sig[i, :]))
    return out


def wrap_angle(x):
    """Wrap to (-pi, pi]."""
    y = np.mod(np.asarray(x) + np.pi, 2.0 * np.pi) - np.pi
    return np.where(y == -np.pi, np.pi, y)


def trapezoid_weights(E):
    """Trapezoid-rule weights of a sorted mesh: (E_{e+1} - E_{e-1}) / 2, half intervals at the ends."""
    E = np.asarray(E, dtype=np.float64)
    w = np.zeros(E.size)
    if E.size > 1:
        d = np.diff(E)
        w[:-1] += 0.5 * d
        w[1:] += 0.5 * d
    else:
        w[:] = 1.0
    return w


def convolve_average(E, sigma, weights, fwhm):
    """Item 7: sum_s f_s (G * sigma_s)(E_e) on the mesh, with sigma [n_series, n_e].

    fwhm = 0 returns the weighted sum of the series unconvolved.
    """
    E = np.asarray(E, dtype=np.float64)
    sigma = np.atleast_2d(np.asarray(sigma, dtype=np.float64))
    f = np.asarray(weights, dtype=np.float64)
    mixed = f @ sigma
    if fwhm == 0.0:
        return mixed
    sd = fwhm / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    tw = trapezoid_weights(E)
    out = np.zeros(E.size)
    for e in range(E.size):
        g = np.exp(-0.5 * ((E[e] - E) / sd) ** 2) * tw
        out[e] = np.dot(g, mixed) / np.sum(g)
    return out

