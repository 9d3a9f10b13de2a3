"""Mixed-precision matching solve (FP32 LU + double-float iterative refinement,
FP64 fallback) against the oracle (needs a GPU).

Tolerances: refinement stops when the last correction is below 1e-11 of Y, so
Y carries about that relative error plus the FP64-level rounding of the rest
of the path; K is held to the FP64 path's 1e-9 normwise, sigma to 1e-9 of
sigma_tot and the eigenphase sum (the S-step stays FP64) to 1e-8.  Energies
whose refinement stops contracting are solved in FP64 (flag 32) and must
agree just as well.
"""
import numpy as np
import pytest

from oracle import rmatrix as orc
from paper_1403_5524_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FLAG_FP64 = 32


@pytest.fixture(scope="module")
def rm():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1403_5524_gb300 import rm as _rm
    _rm.load_library()
    return _rm


def run(rm, w, E, prec, solve, sel=(0,)):
    n = w.n
    K = np.zeros((E.size, n, n))
    fl = np.zeros(E.size, np.uint8)
    no = np.zeros(E.size, np.int32)
    out = rm.host_outputs(E.size, n, len(sel))
    with rm.Plan([w], E, prec=prec, sel=sel, solve=solve) as p:
        p.kmatrix(0, 0, E.size, K=K, n_open=no, flags=fl)
        p.xsec(0, 0, E.size, eigsum=out["eigsum"], sig_tot=out["sig_tot"], sig_sel=out["sig_sel"])
    out.update(K=K, flags=fl, n_open=no)
    return out


def check(out, ref, tol_k, tol_sig):
    for t in range(ref["E"].shape[0]):
        assert out["n_open"][t] == ref["n_open"][t]
        if ref["flags"][t] & (orc.FLAG_ILLCOND | orc.FLAG_SINGULAR | orc.FLAG_NO_OPEN):
            continue
        no = ref["n_open"][t]
        Ko = ref["K"][t, :no, :no]
        assert np.abs(out["K"][t, :no, :no] - Ko).max() <= tol_k * np.abs(Ko).max(), t
        st = ref["sig_tot"][t, 0]
        if st > 0:
            assert np.abs(out["sig_sel"][t, 0] - ref["sig_sel"][t, 0]).max() <= tol_sig * st, t
        d = out["eigsum"][t] - ref["eta"][t]
        assert abs(np.mod(d + np.pi, 2 * np.pi) - np.pi) <= 1e-8, t


@pytest.mark.parametrize("seed,n,N", [(71, 6, 200), (72, 37, 1500), (73, 130, 5000)])
def test_mixed_fp64_against_oracle(rm, seed, n, N):
    wl = synth.small(seed, n, N, 1, pole_lo=-3.0, pole_hi=12.0, a=20.0)
    w = wl.waves[0]
    E = np.sort(np.concatenate([np.linspace(0.02, 3.3, 15), w.thresh[1:4] + 3e-5]))
    out = run(rm, w, E, "fp64", "mixed")
    ref = orc.sweep(w, E, keep_R=False)
    check(out, ref, 1e-9, 1e-9)
    assert np.count_nonzero(out["flags"] & FLAG_FP64) < E.size  # refinement converges on most energies


def test_mixed_equals_fp64_path_closely(rm):
    wl = synth.small(74, 48, 2000, 1, pole_lo=-3.0, pole_hi=12.0, a=20.0)
    w = wl.waves[0]
    E = np.linspace(0.03, 3.0, 120)
    a = run(rm, w, E, "split_bf16", "fp64")
    b = run(rm, w, E, "split_bf16", "mixed")
    for t in range(E.size):
        no = a["n_open"][t]
        if no == 0 or a["flags"][t] & (orc.FLAG_ILLCOND | orc.FLAG_SINGULAR):
            continue
        Ka = a["K"][t, :no, :no]
        assert np.abs(b["K"][t, :no, :no] - Ka).max() <= 1e-9 * np.abs(Ka).max(), t


def test_mixed_fallback_near_thresholds(rm):
    # energies just above thresholds (large |Lambda| columns, poorly conditioned M): whatever
    # path each energy takes, it agrees with the oracle
    wl = synth.small(75, 24, 900, 1, pole_lo=-3.0, pole_hi=12.0, a=20.0)
    w = wl.waves[0]
    E = np.sort(np.concatenate([w.thresh[1:] + 1e-7, w.thresh[1:] + 2e-9, np.linspace(0.05, 2.9, 10)]))
    out = run(rm, w, E, "fp64", "mixed")
    ref = orc.sweep(w, E, keep_R=False)
    check(out, ref, 1e-9, 1e-9)


def test_mixed_photo_and_grouped(rm):
    waves = [synth.small(80 + g, n, 40 * n, 1, pole_lo=-3.0, pole_hi=10.0, a=18.0, dipole=True).waves[0]
             for g, n in enumerate([9, 21])]
    E = np.linspace(0.04, 2.9, 80)
    with rm.Plan(waves, E, prec="split_bf16", delta=0.05, solve="mixed") as p:
        p.run()
        for g, w in enumerate(waves):
            tot = np.zeros(E.size)
            p.results_photo(g, 0, E.size, sig_pi=tot)
            idx = np.array([5, 40, 79])
            ref = orc.sweep(w, E, energy_idx=idx, keep_R=False, keep_K=False)
            for t, e in enumerate(idx):
                if ref["flags"][t] & orc.FLAG_ILLCOND:
                    continue
                assert abs(tot[e] - ref["sig_pi"][t]) <= 1e-8 * ref["sig_pi"][t]
