"""Energies the method's accuracy targets set apart, judged on their own (needs a GPU).

The targets (R, K within 1e-6 normwise, cross sections within 1e-8 of sigma_tot for
the split form; 1e-9 for the FP64 form) apply to every energy except those whose
matching LU is ill-conditioned (RM_FLAG_ILLCOND, pivot ratio below 1e-12) and those
within 1e-6 Ry of a pole or a channel threshold.  Those are not skipped here: each
class gets its own maximum errors, printed and checked against its own bound.

* near a threshold (RM_FLAG_NEAR_THRESHOLD): a channel opens (k -> 0).  The library's
  flag must equal the oracle's classification.  sigma and eta stay well defined
  (sigma is normalised by sigma_tot), and K (outside ILLCOND) is as accurate as
  elsewhere, so the regular tolerances apply.
* near a pole: one term of the pole sum dominates R; the near window sums it in FP64
  on both sides, so the regular tolerances apply to R, K, sigma and eta.
* ILLCOND: placed where an open channel's c_j(a) vanishes (n-hat_0(k a) = 0), so
  the column scaling of the matching LU divides by a tiny number.  K from the LU
  path (rm_kmatrix) then loses up to about u / (pivot ratio) relative accuracy and is
  only reported; sigma and eta come from S, which stays bounded, and through the
  outgoing-wave form (which never divides by c_j) they keep the regular tolerances.
"""
import math

import numpy as np
import pytest

from oracle import rmatrix as orc
from paper_1403_5524_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": {"K": 1e-9, "sig": 1e-9, "eta": 1e-8},
       "split_bf16": {"K": 1e-6, "sig": 1e-8, "eta": 1e-7}}


@pytest.fixture(scope="module")
def rm():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1403_5524_gb300 import rm as _rm
    _rm.load_library()
    return _rm


def flagged_workload():
    rng = np.random.default_rng(4242)
    l = [0, 1, 0, 2, 0, 3, 1, 0, 2, 1, 0, 1]
    w = synth.make_wave(rng, len(l), 600, thr_hi=1.5, pole_lo=-3.0, pole_hi=10.0, a=18.0, l_fixed=l)
    E = list(np.linspace(0.05, 3.0, 30))
    for t in w.thresh[1:6]:
        E += [t - 4e-7, t + 3e-7, t, t + 8e-7, t - 3e-6]
    for k in (150, 200, 260):
        p = w.poles[k]
        if 0.02 < p < 3.2:
            E += [p - 5e-7, p + 5e-7, p]
    # zeros of c_j(a): n-hat_0(k a) = -cos(k a) = 0 for the l = 0 channels
    for j in np.nonzero(w.l == 0)[0][:4]:
        for m in range(3):
            E.append(w.thresh[j] + ((math.pi / 2 + m * math.pi) / w.a) ** 2)
    E = np.unique(np.array([e for e in E if 0.01 < e < 3.3]))
    return w, E


def classify(w, E, ref):
    near_pole = np.array([np.min(np.abs(w.poles - e)) < 1e-6 for e in E])
    cls = {
        "illcond": (ref["flags"] & orc.FLAG_ILLCOND) != 0,
        "near_threshold": (ref["flags"] & orc.FLAG_NEAR_THRESHOLD) != 0,
        "near_pole": near_pole,
    }
    flagged = np.zeros(E.size, bool)
    for v in cls.values():
        flagged |= v
    cls["regular"] = ~flagged & ((ref["flags"] & (orc.FLAG_NO_OPEN | orc.FLAG_SINGULAR)) == 0)
    return cls


def gpu_outputs(rm, w, E, prec, sel):
    n = w.n
    out = {}
    with rm.Plan([w], E, prec=prec, delta=0.05, sel=sel) as p:
        K = np.zeros((E.size, n, n))
        no = np.zeros(E.size, np.int32)
        fl = np.zeros(E.size, np.uint8)
        p.kmatrix(0, 0, E.size, K=K, n_open=no, flags=fl)
        x = rm.host_outputs(E.size, n, len(sel))
        p.xsec(0, 0, E.size, eigsum=x["eigsum"], sig_tot=x["sig_tot"], sig_sel=x["sig_sel"])
        p.run()
        r = rm.host_outputs(E.size, n, len(sel))
        p.results(0, 0, E.size, **r)
    out.update(K=K, n_open=no, kflags=fl, eta=x["eigsum"], sig=x["sig_sel"], run=r)
    return out


def errors(ref, g, t, sel):
    no = ref["n_open"][t]
    Ko = ref["K"][t, :no, :no]
    eK = float(np.abs(g["K"][t, :no, :no] - Ko).max() / max(np.abs(Ko).max(), 1e-300))
    eS = eSr = 0.0
    for q in range(len(sel)):
        st = ref["sig_tot"][t, q]
        if st > 0:
            eS = max(eS, float(np.abs(g["sig"][t, q] - ref["sig_sel"][t, q]).max() / st))
            eSr = max(eSr, float(np.abs(g["run"]["sig_sel"][t, q] - ref["sig_sel"][t, q]).max() / st))
    eE = float(abs(orc.wrap_angle(g["eta"][t] - ref["eta"][t])))
    eEr = float(abs(orc.wrap_angle(g["run"]["eigsum"][t] - ref["eta"][t])))
    return {"K": eK, "sig": max(eS, eSr), "eta": max(eE, eEr)}


@pytest.mark.parametrize("prec", ["fp64", "split_bf16"])
def test_flagged_energies_reported_separately(rm, prec):
    w, E = flagged_workload()
    sel = (0, 2)
    ref = orc.sweep(w, E, sel=sel)
    g = gpu_outputs(rm, w, E, prec, sel)
    # classification: n_open everywhere, the near-threshold bit from both the per-range and run paths
    assert np.array_equal(g["n_open"], ref["n_open"])
    nt = (ref["flags"] & orc.FLAG_NEAR_THRESHOLD) != 0
    assert nt.sum() >= 15
    assert np.array_equal((g["kflags"] & orc.FLAG_NEAR_THRESHOLD) != 0, nt)
    assert np.array_equal((g["run"]["flags"] & orc.FLAG_NEAR_THRESHOLD) != 0, nt)
    cls = classify(w, E, ref)
    assert cls["illcond"].sum() >= 2 and cls["near_pole"].sum() >= 3 and cls["regular"].sum() >= 20
    tol = TOL[prec]
    report = {}
    for name, mask in cls.items():
        worst = {"K": 0.0, "sig": 0.0, "eta": 0.0, "energies": int(mask.sum())}
        for t in np.nonzero(mask)[0]:
            if ref["flags"][t] & (orc.FLAG_NO_OPEN | orc.FLAG_SINGULAR):
                continue
            e = errors(ref, g, t, sel)
            for k in ("K", "sig", "eta"):
                worst[k] = max(worst[k], e[k])
            assert e["sig"] <= tol["sig"], (name, t, e)
            assert e["eta"] <= tol["eta"], (name, t, e)
            if not ref["flags"][t] & orc.FLAG_ILLCOND:
                assert e["K"] <= tol["K"], (name, t, e)
            else:
                # K of an ill-conditioned matching LU: reported; bounded by the pivot ratio
                assert e["K"] <= 1e-3 * 1e-12 / max(ref["piv_ratio"][t], 1e-300) + tol["K"], (name, t, e)
        report[name] = worst
    print(prec, "flagged-energy errors by class:", report)
