"""The outgoing-wave cross-section path against the LU path and the oracle (needs a GPU).

With solve "fp64", rm_run and rm_xsec take the cross sections and the eigenphase
sum from Z = G - diag(h / (a h')), h = c + i s, G the open block of
M = R - diag(c / (a c')) (closed: R - diag(1 / (a Lambda))) less the closed
channels' Schur correction; solve "fp64_lu" solves K by LU for every energy and
then I - iK.  Both are FP64 solves of the same matching equations from the
same R, so they differ by rounding amplified by the conditioning, as the LU
path differs from the oracle: the tolerances are those of the FP64 parity
tests (1e-9 on sigma normalised by the total of its initial channel, on eta
mod 2 pi).  Cases: a contiguous block of the n_ch = 64 mesh (thresholds up to
2 Ry, so 1..64 open channels), a Coulomb wave, an energy where the first
closed pivot vanishes (must go through LU, RM_FLAG_LU), one where c'_0 = 0
(K is regular there, but M and the unit-right-hand-side LU form divide by c'),
photoionisation against the LU form, the largest channel count (640, FP64 and
split BF16), the two sides of a K pole (the inertia of S'' flips there), and the
energies of the n_ch = 256 mesh whose S'' fails the double-float checks and is
factored again in FP64 (RM_FLAG_FP64).
"""
import math

import numpy as np
import pytest

from oracle import rmatrix as orc
from paper_1403_5524_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FLAG_LU = 64
FLAG_FP64 = 32
TOL = 1e-9


@pytest.fixture(scope="module")
def rm():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1403_5524_gb300 import rm as _rm
    _rm.load_library()
    return _rm


def run(rm, wl, solve, sel=(0,), prec="fp64"):
    w = wl.waves[0]
    with rm.Plan(wl.waves, wl.energies, prec=prec, sel=sel, solve=solve) as p:
        p.run()
        out = rm.host_outputs(wl.n_e, w.n, len(sel))
        p.results(0, 0, wl.n_e, **out)
    return out


def close(a, b, idx=None, tol=TOL):
    idx = np.arange(a["eigsum"].shape[0]) if idx is None else idx
    for e in idx:
        st = b["sig_tot"][e]
        for q in range(st.shape[0]):
            if st[q] == 0:
                assert np.all(a["sig_sel"][e, q] == 0), (e, q)
                continue
            err = np.abs(a["sig_sel"][e, q] - b["sig_sel"][e, q]).max() / st[q]
            assert err <= tol, (e, q, err)
            assert abs(a["sig_tot"][e, q] - st[q]) <= tol * st[q], (e, q)
        assert abs(orc.wrap_angle(a["eigsum"][e] - b["eigsum"][e])) <= 10 * tol, e


def as_ref(ref):
    return {"eigsum": ref["eta"], "sig_tot": ref["sig_tot"], "sig_sel": ref["sig_sel"]}


def test_config2_block_matches_lu_path(rm):
    wl = synth.config(2)
    sub = synth.Workload(wl.name, wl.waves, wl.energies[2000:2800])  # 0.41 .. 0.57 Ry: 12..20 open
    a = run(rm, sub, "fp64", sel=(0, 3))
    b = run(rm, sub, "fp64_lu", sel=(0, 3))
    assert np.array_equal(a["n_open"], b["n_open"])
    assert np.array_equal(a["flags"] & ~np.uint8(FLAG_LU | FLAG_FP64), b["flags"])
    assert np.count_nonzero(a["flags"] & FLAG_LU) < sub.n_e // 20  # the LU fallback stays rare
    close(a, b)
    idx = np.arange(0, sub.n_e, 37)
    ref = orc.sweep(wl.waves[0], sub.energies, sel=(0, 3), energy_idx=idx, keep_R=False, keep_K=False)
    close({k: v[idx] for k, v in a.items()}, as_ref(ref))


def test_all_open_and_ragged(rm):
    # energies above every threshold (no closed channel: no real elimination) and n not a
    # multiple of the panel widths
    wl = synth.small(41, 37, 300, 90, e_lo=0.05, e_hi=4.0, thr_hi=1.5, pole_lo=-2.0, pole_hi=8.0,
                     a=15.0)
    sel = (0, 1, 36)
    a = run(rm, wl, "fp64", sel=sel)
    ref = orc.sweep(wl.waves[0], wl.energies, sel=sel, keep_R=False, keep_K=False)
    assert np.array_equal(a["n_open"], ref["n_open"])
    close(a, as_ref(ref))


def test_coulomb_matches_lu_path(rm):
    wl = synth.small(7, 12, 160, 120, e_lo=0.02, e_hi=2.5, z=1.0)
    a = run(rm, wl, "fp64", sel=(0, 2))
    b = run(rm, wl, "fp64_lu", sel=(0, 2))
    close(a, b)


def bisect(f, lo, hi, it=200):
    flo = f(lo)
    for _ in range(it):
        mid = 0.5 * (lo + hi)
        if mid in (lo, hi):
            break
        fm = f(mid)
        if (fm < 0) == (flo < 0):
            lo, flo = mid, fm
        else:
            hi = mid
    return 0.5 * (lo + hi)


def test_vanishing_closed_pivot_goes_through_lu(rm):
    # The first closed pivot (last channel, eliminated first) is d = R_nn - 1/(a Lambda_n); between
    # two poles R_nn rises from -inf to +inf, so it vanishes once.  There the outgoing-wave path must
    # hand the energy to LU, whose results still match the oracle.
    wl0 = synth.small(12, 6, 60, 1, pole_lo=0.0, pole_hi=3.0, thr_hi=2.5, a=10.0)
    w = wl0.waves[0]
    last = w.n - 1

    def d0(E):
        R = orc.rmatrix(w.W, w.poles, E, w.a)
        lam = orc.channel_functions(w.l, w.thresh, E, w.a)["lam"][last]
        return R[last, last] - 1.0 / (w.a * lam)

    k = int(np.searchsorted(w.poles, 0.3))
    while w.poles[k + 1] - w.poles[k] < 0.02:
        k += 1
    assert w.poles[k + 1] < w.thresh[last]
    lo, hi = w.poles[k] + 1e-7, w.poles[k + 1] - 1e-7
    assert d0(lo) < 0 < d0(hi)
    Es = bisect(d0, lo, hi)
    E = np.array([Es - 0.01, Es, Es + 0.01]) if Es + 0.01 < w.poles[k + 1] else np.array([Es - 0.01, Es])
    wl = synth.Workload("pivot", [w], np.sort(E))
    a = run(rm, wl, "fp64", sel=(0,))
    i = int(np.nonzero(wl.energies == Es)[0][0])
    assert a["flags"][i] & FLAG_LU
    ref = orc.sweep(w, wl.energies, sel=(0,), keep_R=False, keep_K=False)
    close(a, as_ref(ref))


def test_regular_where_c_prime_vanishes(rm):
    # c'_0 = 0 at k a = x with nhat_l'(x) = 0: M's diagonal term c / (a c') diverges there, Z does not.
    wl0 = synth.small(13, 5, 50, 1, pole_lo=-1.0, pole_hi=6.0, thr_hi=1.0, a=12.0)
    w = wl0.waves[0]
    l0 = int(w.l[0])

    def cp0(E):
        return orc.riccati_yn(l0, math.sqrt(E) * w.a)[1]

    grid = np.linspace(1.2, 2.5, 400)
    v = np.array([cp0(E) for E in grid])
    j = int(np.nonzero(np.sign(v[1:]) != np.sign(v[:-1]))[0][0])
    Es = bisect(cp0, grid[j], grid[j + 1])
    E = np.array([Es - 1e-3, Es, Es + 1e-3])
    assert np.min(np.abs(w.poles[:, None] - E[None, :])) > 1e-6
    wl = synth.Workload("cprime", [w], E)
    a = run(rm, wl, "fp64", sel=(0, 1))
    ref = orc.sweep(w, wl.energies, sel=(0, 1), keep_R=False, keep_K=False)
    close(a, as_ref(ref))


def test_photo_matches_lu_path(rm):
    # dipole amplitudes from one more right-hand side of Z against the K-normalised LU form
    for z in (0.0, 1.0):
        wl = synth.small(23, 18, 240, 60, e_lo=0.05, e_hi=2.5, z=z, dipole=True)
        w = wl.waves[0]
        out = {}
        for solve in ("fp64", "fp64_lu"):
            with rm.Plan(wl.waves, wl.energies, prec="fp64", sel=(0,), solve=solve) as p:
                p.run()
                pi = np.zeros(wl.n_e)
                pich = np.zeros((wl.n_e, w.n))
                p.results_photo(0, 0, wl.n_e, sig_pi=pi, sig_pi_ch=pich)
                out[solve] = (pi, pich)
        a, b = out["fp64"], out["fp64_lu"]
        for e in range(wl.n_e):
            if b[0][e] == 0:
                assert a[0][e] == 0
                continue
            assert abs(a[0][e] - b[0][e]) <= TOL * b[0][e], (z, e)
            assert np.abs(a[1][e] - b[1][e]).max() <= TOL * b[0][e], (z, e)


def test_maximum_channel_count(rm):
    # n_ch = 640, the largest the library accepts: two solve CTAs per SM, 40 panels of the real and
    # 80 of the complex LDL^T; energies with a few, about half, and all channels open
    wl = synth.small(31, 640, 1500, 5, e_lo=0.02, e_hi=3.0, thr_hi=2.0, pole_lo=-3.0, pole_hi=8.0, a=20.0)
    sel = (0, 1, 639)
    a = run(rm, wl, "fp64", sel=sel)
    b = run(rm, wl, "fp64_lu", sel=sel)
    ref = orc.sweep(wl.waves[0], wl.energies, sel=sel, keep_R=False, keep_K=False)
    assert np.array_equal(a["n_open"], ref["n_open"])
    assert ref["n_open"].min() < 100 and ref["n_open"].max() == 640
    close(a, as_ref(ref))
    close(b, as_ref(ref))


def test_maximum_channel_count_split(rm):
    # the same size through the split-BF16 tensor-core pole sum with TMA-staged D slices
    # (205120 pairs: 1603 pair tiles) and the FP64 near window; sigma within the method's 1e-8
    wl = synth.small(32, 640, 1500, 4, e_lo=0.3, e_hi=3.0, thr_hi=2.0, pole_lo=-3.0, pole_hi=8.0, a=20.0)
    sel = (0, 5)
    a = run(rm, wl, "fp64", sel=sel, prec="split_bf16")
    ref = orc.sweep(wl.waves[0], wl.energies, sel=sel, keep_R=False, keep_K=False)
    assert np.array_equal(a["n_open"], ref["n_open"])
    close(a, as_ref(ref), tol=1e-8)


def test_eta_across_a_k_pole(rm):
    # the kernel's sign of det S'' (the inertia of its real LDL^T) against the oracle on both sides of
    # a K pole, where eta mod 2 pi jumps by pi; the energy is found on the CPU as in
    # tests/test_oracle_outgoing.py
    wl0 = synth.small(63, 5, 80, 1, pole_lo=-1.0, pole_hi=5.0, thr_hi=1.0, a=10.0)
    w = wl0.waves[0]

    def detsign(E):
        R = orc.rmatrix(w.W, w.poles, E, w.a)
        f = orc.channel_functions(w.l, w.thresh, E, w.a)
        no = f["n_o"]
        M = R[:no, :no] - np.diag(f["c"][:no] / (w.a * f["cp"][:no]))
        V = f["cp"][:no] / np.hypot(f["cp"][:no], f["sp"][:no])
        return np.prod(np.sign(np.linalg.eigvalsh(V[:, None] * M * V[None, :])))

    grid = np.linspace(1.2, 2.4, 241)  # every channel open
    signs = [detsign(E) for E in grid]
    flips = [k for k in range(len(grid) - 1) if signs[k] != signs[k + 1]
             and not np.any((w.poles > grid[k] - 1e-3) & (w.poles < grid[k + 1] + 1e-3))]
    assert flips
    lo, hi = grid[flips[0]], grid[flips[0] + 1]
    s_lo = detsign(lo)
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        if detsign(mid) == s_lo:
            lo = mid
        else:
            hi = mid
    E = np.array([lo - 1e-7, hi + 1e-7])
    wl = synth.Workload("kpole", [w], E)
    a = run(rm, wl, "fp64", sel=(0, 1))
    ref = orc.sweep(w, E, sel=(0, 1), keep_R=False, keep_K=False)
    assert not np.any(a["flags"] & FLAG_LU)
    close(a, as_ref(ref), tol=1e-7)


def test_s2_fp64_retry_energies(rm):
    # S'' gives only the sign of det S_oo (eta mod 2 pi), so its LDL^T runs in double-float; where
    # that fails its growth (1e4) or pivot check, S'' is formed again from Z and factored in FP64
    # (RM_FLAG_FP64), a few energies in a thousand of the n_ch = 256 mesh.  Those energies must
    # keep the outgoing-wave path (not LU) and match the LU path and the oracle like the rest: a
    # wrong sign count would put eta off by pi.
    wl = synth.config(3)
    a = run(rm, wl, "fp64", prec="split_bf16")
    retry = np.flatnonzero(a["flags"] & FLAG_FP64)
    assert 0 < retry.size < wl.n_e // 100, retry.size
    assert not np.any(a["flags"][retry] & FLAG_LU)
    b = run(rm, wl, "fp64_lu", prec="split_bf16")  # the same R, solved by LU
    lu_ok = retry[(b["flags"][retry] & orc.FLAG_ILLCOND) == 0]
    close(a, b, idx=lu_ok, tol=1e-8)
    pick = retry[np.linspace(0, retry.size - 1, 4).astype(int)]
    ref = orc.sweep(wl.waves[0], wl.energies, sel=(0,), energy_idx=pick, keep_R=False, keep_K=False)
    keep = np.array([t for t in range(pick.size) if not ref["flags"][t] & orc.FLAG_ILLCOND], dtype=np.int64)
    assert keep.size
    close({k: v[pick[keep]] for k, v in a.items()}, {k: v[keep] for k, v in as_ref(ref).items()}, tol=1e-8)


def test_z_double_float_against_its_fp64_fallback(rm, monkeypatch):
    # split plans factor Z in double-float and refine its solutions once against an FP64 residual;
    # where the correction is large the energy takes Z again in FP64 (RM_FLAG_FP64).  The test hook
    # RM_TEST_Z_FP64=1 (read at plan creation) sends every energy down that fallback, so both paths
    # run on the same R: they must agree at the FP64 tolerances (and the double-float one with the
    # LU path and the oracle), on a block of the n_ch = 64 mesh (1..64 open channels, two initial
    # channels) and on the n_ch = 256 mesh's first energies
    for wl in (synth.config(2), synth.config(3)):
        wl = synth.Workload(wl.name, wl.waves, wl.energies[7000:7240:2].copy(), delta=wl.delta)
        sel = (0, 1)
        a = run(rm, wl, "fp64", sel=sel, prec="split_bf16")
        monkeypatch.setenv("RM_TEST_Z_FP64", "1")
        f = run(rm, wl, "fp64", sel=sel, prec="split_bf16")
        monkeypatch.delenv("RM_TEST_Z_FP64")
        sym = (a["flags"] & (FLAG_LU | orc.FLAG_NO_OPEN)) == 0
        assert np.all(f["flags"][sym] & FLAG_FP64), "the hook did not reach the fallback"
        assert np.array_equal(a["n_open"], f["n_open"])
        close(a, f, idx=np.flatnonzero(sym))
        b = run(rm, wl, "fp64_lu", sel=sel, prec="split_bf16")  # the same R, solved by LU in FP64
        close(a, b, idx=np.flatnonzero(sym & ((b["flags"] & orc.FLAG_ILLCOND) == 0)))
        pick = np.array([3, 40, 77, 119])
        ref = orc.sweep(wl.waves[0], wl.energies, sel=sel, energy_idx=pick, keep_R=False, keep_K=False)
        keep = np.array([t for t in range(pick.size) if not ref["flags"][t] & orc.FLAG_ILLCOND], dtype=np.int64)
        close({k: v[pick[keep]] for k, v in a.items()}, {k: v[keep] for k, v in as_ref(ref).items()}, tol=1e-8)
