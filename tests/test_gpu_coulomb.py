"""Coulomb outer region (ionic targets, residual charge z > 0) on the GPU
against the oracle (needs a GPU).

Tolerances: the kernel's continued fractions stop at two ulps per partial
step and the order recurrences (F down, G up) are the stable directions, so
F, G, F', G' and the Whittaker log-derivative carry relative errors of about
1e-12 at the workloads' parameters (rho = ka >= 0.3, |eta| <= 100) and below
5e-9 at the extreme of a point nudged onto a threshold (k = 1e-3, |eta| up to
1e3; prototype against mpmath over l <= 15, |eta| <= 1000, rho >= 0.03).  An
LU solve multiplies that by cond <~ 1e3 at the tested energies, so K is held
to 1e-8 normwise and sigma to 1e-8 of sigma_tot (the Cayley map does not
amplify), eta to 1e-7 mod 2 pi; R = 0 isolates the functions themselves
(K_ii = -F/G) and is held to 1e-10.
"""
import math

import numpy as np
import pytest

from oracle import rmatrix as orc
from paper_1403_5524_gb300 import synth

torch = pytest.importorskip("torch")
mp = pytest.importorskip("mpmath")
pytestmark = pytest.mark.gpu

TOL_K = 1e-8
TOL_SIG = 1e-8


@pytest.fixture(scope="module")
def rm():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1403_5524_gb300 import rm as _rm
    _rm.load_library()
    return _rm


def run(rm, waves, E, prec="fp64", sel=(0,), delta=0.05):
    outs = []
    with rm.Plan(waves, E, prec=prec, sel=sel, delta=delta) as p:
        for g, w in enumerate(waves):
            n = w.n
            K = np.zeros((E.size, n, n))
            no = np.zeros(E.size, np.int32)
            fl = np.zeros(E.size, np.uint8)
            p.kmatrix(g, 0, E.size, K=K, n_open=no, flags=fl)
            o = rm.host_outputs(E.size, n, len(sel))
            p.xsec(g, 0, E.size, eigsum=o["eigsum"], sig_tot=o["sig_tot"], sig_sel=o["sig_sel"])
            o.update(K=K, n_open=no, flags=fl)
            outs.append(o)
    return outs


def compare(out, ref, tol_k=TOL_K, tol_sig=TOL_SIG):
    worst = {"K": 0.0, "sig": 0.0}
    for t in range(ref["E"].shape[0]):
        assert out["n_open"][t] == ref["n_open"][t]
        assert not (out["flags"][t] & orc.FLAG_SINGULAR) and not (out["flags"][t] & 16), (t, out["flags"][t])
        if ref["flags"][t] & (orc.FLAG_ILLCOND | orc.FLAG_NO_OPEN | orc.FLAG_SINGULAR):
            continue
        no = ref["n_open"][t]
        Ko = ref["K"][t, :no, :no]
        eK = np.abs(out["K"][t, :no, :no] - Ko).max() / max(np.abs(Ko).max(), 1e-300)
        assert eK <= tol_k, (t, ref["E"][t], eK)
        worst["K"] = max(worst["K"], eK)
        for q in range(ref["sig_tot"].shape[1]):
            st = ref["sig_tot"][t, q]
            if st > 0:
                eS = np.abs(out["sig_sel"][t, q] - ref["sig_sel"][t, q]).max() / st
                assert eS <= tol_sig, (t, q, eS)
                worst["sig"] = max(worst["sig"], eS)
        d = out["eigsum"][t] - ref["eta"][t]
        assert abs(np.mod(d + np.pi, 2 * np.pi) - np.pi) <= 1e-7, (t, d)
    return worst


def test_coulomb_functions_through_zero_r(rm):
    # W = 0 -> R = 0 -> K_ii = -F_l(eta, ka)/G_l(eta, ka): the kernel's F/G directly
    a, z = 20.0, 1.5
    l = np.array([0, 1, 2, 3, 5, 7, 11, 15], np.int32)
    thr = np.array([0.0, 0.0, 0.1, 0.1, 0.3, 0.3, 0.6, 0.6])
    wave = synth.Wave(l=l, thresh=thr, poles=np.array([-3.0, 50.0]), W=np.zeros((8, 2)), a=a, z=z)
    E = np.array([0.6 + 2e-4, 0.6 + 0.01, 0.7, 1.3, 2.9, 6.0])  # k from 0.014 to 2.4 in the last channels
    out = run(rm, [wave], E)[0]
    with mp.workdps(30):
        for t, En in enumerate(E):
            for i in range(8):
                if En <= thr[i]:
                    continue
                k = math.sqrt(En - thr[i])
                r = float(mp.coulombf(int(l[i]), -z / k, k * a) / mp.coulombg(int(l[i]), -z / k, k * a))
                assert abs(out["K"][t, i, i] + r) <= 1e-10 * max(1.0, abs(r)), (En, i, out["K"][t, i, i], -r)


@pytest.mark.parametrize("z", [1.0, 3.0])
@pytest.mark.parametrize("seed,n,N", [(31, 6, 150), (32, 13, 400)])
def test_coulomb_fp64_sweep(rm, z, seed, n, N):
    wl = synth.small(seed, n, N, 1, pole_lo=-2.0, pole_hi=10.0, a=18.0, z=z)
    w = wl.waves[0]
    # energies across the thresholds, two of them just above / below one (small rho, large |eta| and
    # large z/kappa), one exactly on a threshold (nudged by 1e-6 Ry: k = 1e-3)
    E = np.sort(np.concatenate([np.linspace(0.02, 3.0, 9), [w.thresh[2] + 3e-4, w.thresh[3] - 3e-4,
                                                             w.thresh[4]]]))
    out = run(rm, [w], E, sel=(0, 1))[0]
    ref = orc.sweep(w, E, sel=(0, 1), keep_R=False)
    worst = compare(out, ref)
    print("coulomb fp64 worst", worst)


def test_coulomb_split_sweep(rm):
    wl = synth.small(33, 24, 1200, 1, pole_lo=-3.0, pole_hi=12.0, a=20.0, z=2.0)
    w = wl.waves[0]
    E = np.linspace(0.03, 3.2, 14)
    out = run(rm, [w], E, prec="split_bf16", sel=(0,))[0]
    ref = orc.sweep(w, E, sel=(0,), keep_R=False)
    compare(out, ref, tol_k=1e-6, tol_sig=1e-8)


def test_grouped_mixed_charges(rm):
    # neutral and ionic waves in one plan and one rm_run
    waves = [synth.small(40 + g, n, 40 * n, 1, pole_lo=-3.0, pole_hi=10.0, a=18.0, z=z).waves[0]
             for g, (n, z) in enumerate([(7, 0.0), (11, 1.0), (5, 4.0)])]
    E = np.linspace(0.05, 2.8, 90)
    sel = (0,)
    with rm.Plan(waves, E, prec="split_bf16", delta=0.05, sel=sel) as p:
        p.run()
        outs = []
        for g, w in enumerate(waves):
            o = rm.host_outputs(E.size, w.n, 1)
            p.results(g, 0, E.size, **o)
            outs.append(o)
    idx = np.array([2, 29, 55, 88])
    for g, w in enumerate(waves):
        ref = orc.sweep(w, E, sel=sel, energy_idx=idx, keep_R=False, keep_K=False)
        for t, e in enumerate(idx):
            assert outs[g]["n_open"][e] == ref["n_open"][t]
            if ref["flags"][t] & orc.FLAG_ILLCOND:
                continue
            st = ref["sig_tot"][t, 0]
            err = np.abs(outs[g]["sig_sel"][e, 0] - ref["sig_sel"][t, 0]).max() / st
            assert err <= TOL_SIG, (g, e, err)
