"""Photoionisation (bound-free dipole vector per wave) on the GPU against the
oracle (needs a GPU).

Tolerances: y_i is a pole sum like R (same kernels, the dipole vector as one
more row), so it carries R's accuracy; M^K adds one pass over the matching
solution (n multiply-adds per amplitude) and M^- one more right-hand side of
the complex LU, so sigma_PI inherits the K / sigma bounds of the same path:
1e-9 of the total in FP64, 1e-8 in the split-BF16 mode (the method's sigma
target), per energy and per final channel.
"""
import numpy as np
import pytest

from oracle import rmatrix as orc
from paper_1403_5524_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rm():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1403_5524_gb300 import rm as _rm
    _rm.load_library()
    return _rm


def check_photo(tot, ch, ref, tol):
    for t in range(ref["E"].shape[0]):
        if ref["flags"][t] & (orc.FLAG_ILLCOND | orc.FLAG_SINGULAR):
            continue
        st = ref["sig_pi"][t]
        if ref["n_open"][t] == 0:
            assert tot[t] == 0.0
            continue
        assert abs(tot[t] - st) <= tol * st, (t, tot[t], st)
        assert np.abs(ch[t] - ref["sig_pi_ch"][t]).max() <= tol * st, t


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-9), ("split_bf16", 1e-8)])
@pytest.mark.parametrize("seed,n,N", [(51, 5, 140), (52, 17, 700)])
def test_photo_against_oracle(rm, prec, tol, seed, n, N):
    wl = synth.small(seed, n, N, 1, pole_lo=-3.0, pole_hi=10.0, a=16.0, dipole=True)
    w = wl.waves[0]
    E = np.sort(np.concatenate([[-0.2], np.linspace(0.02, 3.1, 11), [w.thresh[1] + 2e-4]]))
    tot = np.zeros(E.size)
    ch = np.zeros((E.size, n))
    with rm.Plan([w], E, prec=prec, delta=0.05) as p:
        p.photo(0, 0, E.size, sig_pi=tot, sig_pi_ch=ch)
    ref = orc.sweep(w, E, keep_R=False, keep_K=False)
    assert tot[0] == 0.0  # below every threshold
    check_photo(tot, ch, ref, tol)


def test_coulomb_photo(rm):
    # photoionisation of an ion's bound state: final states around a z = 1 target
    wl = synth.small(53, 8, 300, 1, pole_lo=-3.0, pole_hi=10.0, a=16.0, z=1.0, dipole=True)
    w = wl.waves[0]
    E = np.linspace(0.03, 2.9, 9)
    tot = np.zeros(E.size)
    ch = np.zeros((E.size, w.n))
    with rm.Plan([w], E, prec="fp64") as p:
        p.photo(0, 0, E.size, sig_pi=tot, sig_pi_ch=ch)
    check_photo(tot, ch, orc.sweep(w, E, keep_R=False, keep_K=False), 1e-8)


def test_dipole_row_leaves_channel_results_alone(rm):
    wl = synth.small(54, 9, 400, 1, pole_lo=-3.0, pole_hi=10.0, a=16.0, dipole=True)
    w = wl.waves[0]
    w0 = synth.Wave(l=w.l, thresh=w.thresh, poles=w.poles, W=w.W, a=w.a)
    E = np.linspace(0.05, 2.5, 40)
    n, np_ = w.n, w.n * (w.n + 1) // 2
    for prec, tol in [("fp64", 0.0), ("split_bf16", 1e-12)]:
        outs = []
        for ww in (w, w0):
            R = np.zeros((E.size, np_))
            K = np.zeros((E.size, n, n))
            with rm.Plan([ww], E, prec=prec) as p:
                p.rmatrix(0, 0, E.size, R)
                p.kmatrix(0, 0, E.size, K=K)
            outs.append((R, K))
        scale = np.abs(outs[1][0]).max()
        assert np.abs(outs[0][0] - outs[1][0]).max() <= tol * scale, prec
        # without the photoionisation outputs the solve is the same program
        assert np.abs(outs[0][1] - outs[1][1]).max() <= max(tol, 1e-13) * np.abs(outs[1][1]).max(), prec


def test_grouped_photo_and_mixed_waves(rm):
    waves = [synth.small(60 + g, n, 40 * n, 1, pole_lo=-3.0, pole_hi=10.0, a=18.0, dipole=d).waves[0]
             for g, (n, d) in enumerate([(6, True), (13, False), (9, True)])]
    E = np.linspace(0.04, 3.0, 120)
    with rm.Plan(waves, E, prec="split_bf16", delta=0.05, sel=(0,)) as p:
        p.run()
        got = {}
        for g in (0, 2):
            tot = np.zeros(E.size)
            ch = np.zeros((E.size, waves[g].n))
            p.results_photo(g, 0, E.size, sig_pi=tot, sig_pi_ch=ch)
            got[g] = (tot, ch)
        with pytest.raises(rm.RMError):
            p.results_photo(1, 0, E.size, sig_pi=np.zeros(E.size))
        # the per-range call gives the same numbers as the grouped run
        tot2 = np.zeros(E.size)
        p.photo(2, 0, E.size, sig_pi=tot2)
        assert np.allclose(tot2, got[2][0], rtol=1e-12, atol=0)
    idx = np.array([3, 47, 90, 119])
    for g in (0, 2):
        ref = orc.sweep(waves[g], E, energy_idx=idx, keep_R=False, keep_K=False)
        check_photo(got[g][0][idx], got[g][1][idx], ref, 1e-8)


def test_photo_reproducible_in_any_call_order(rm):
    # every output is a function of the inputs only: repeated and reordered calls agree bit for bit
    wl = synth.small(55, 21, 900, 1, pole_lo=-3.0, pole_hi=10.0, a=16.0, dipole=True)
    w = wl.waves[0]
    E = np.linspace(0.03, 3.0, 64)
    runs = []
    with rm.Plan([w], E, prec="split_bf16", delta=0.05, sel=(0, 1)) as p:
        for order in range(3):
            tot = np.zeros(E.size)
            ch = np.zeros((E.size, w.n))
            K = np.zeros((E.size, w.n, w.n))
            if order == 1:
                p.kmatrix(0, 0, E.size, K=K)
            p.photo(0, 0, E.size, sig_pi=tot, sig_pi_ch=ch)
            if order != 1:
                p.kmatrix(0, 0, E.size, K=K)
            runs.append((tot, ch, K))
    for tot, ch, K in runs[1:]:
        assert np.array_equal(tot, runs[0][0]) and np.array_equal(ch, runs[0][1]) and np.array_equal(K, runs[0][2])
