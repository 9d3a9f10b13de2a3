"""Parity of the plain FP64 CUDA path with the FP64 CPU oracle (needs a GPU).

Tolerances (derived from the arithmetic, not fitted):
* R: both sides sum the same N products in FP64 in different orders; the
  rounding error of each element is below c sqrt(N) u sum_k |w_ik w_jk / (E_k - E)|
  (u = 2^-53).  The test checks |R - R*| <= 8 sqrt(N) u (1/2a) sum_k |...| per
  element, computed from the oracle's inputs.
* K: an LU solve perturbs K by about cond * n * u relative; energies the
  oracle flags ILLCOND (pivot ratio < 1e-12) are excluded, leaving
  cond <~ 1e12 worst case but typically < 1e6.  The normwise bound used is
  1e-9 (about n * u * 1e6 for n <= 256, with margin).
* sigma, eigenphase sum: T = 2i(I - iK)^-1 K is a Cayley map with
  ||d T|| <= 2 ||dK||, so they inherit the K bound (1e-9, sigma normalised by
  the total cross section of the initial channel; eta compared mod 2 pi).
"""
import math

import numpy as np
import pytest

from oracle import rmatrix as orc
from paper_1403_5524_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U = 2.0 ** -53


@pytest.fixture(scope="module")
def rm():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1403_5524_gb300 import rm as _rm
    _rm.load_library()
    return _rm


def r_bound(w, E, n_poles):
    d = np.abs(1.0 / (w.poles - E))
    S = (np.abs(w.W) * d[None, :]) @ np.abs(w.W).T / (2.0 * w.a)
    return 8.0 * math.sqrt(n_poles) * U * S + 1e-300


def gpu_sweep(rm, wl, sel=(0,), prec="fp64", chunk=0, idx=None):
    w = wl.waves[0]
    n, ne = w.n, wl.n_e
    with rm.Plan(wl.waves, wl.energies, prec=prec, sel=sel, chunk=chunk) as p:
        R = np.zeros((ne, n * (n + 1) // 2))
        K = np.zeros((ne, n, n))
        no = np.zeros(ne, np.int32)
        fl = np.zeros(ne, np.uint8)
        p.rmatrix(0, 0, ne, R)
        p.kmatrix(0, 0, ne, K=K, n_open=no, flags=fl)
        out = rm.host_outputs(ne, n, len(sel))
        p.xsec(0, 0, ne, eigsum=out["eigsum"], sig_tot=out["sig_tot"], sig_sel=out["sig_sel"])
    out.update(R=R, K=K, n_open=no, flags=fl)
    return out


def compare(wl, g, ref, idx=None, tolK=1e-9, tolS=1e-9, checkR=True):
    w = wl.waves[0]
    n = w.n
    idx = np.arange(wl.n_e) if idx is None else idx
    assert np.array_equal(g["n_open"][idx], ref["n_open"])
    nud = (ref["flags"] & orc.FLAG_NUDGED) != 0
    assert np.array_equal((g["flags"][idx] & orc.FLAG_NUDGED) != 0, nud)
    for t, e in enumerate(idx):
        if checkR:
            Rg = orc.unpack_upper(g["R"][e], n)
            Ro = orc.unpack_upper(ref["R"][t], n)
            bound = r_bound(w, ref["E"][t], w.N)
            assert np.all(np.abs(Rg - Ro) <= bound), (e, np.max(np.abs(Rg - Ro) / bound))
        if ref["flags"][t] & (orc.FLAG_ILLCOND | orc.FLAG_SINGULAR | orc.FLAG_NO_OPEN):
            continue
        no = ref["n_open"][t]
        Ko = ref["K"][t, :no, :no]
        Kg = g["K"][e, :no, :no]
        errK = np.abs(Kg - Ko).max() / max(np.abs(Ko).max(), 1e-300)
        assert errK <= tolK, (e, errK)
        assert np.all(g["K"][e, no:, :] == 0) and np.all(g["K"][e, :, no:] == 0)
        st = ref["sig_tot"][t]
        for q in range(st.shape[0]):
            if st[q] == 0:
                assert np.all(g["sig_sel"][e, q] == 0)
                continue
            errS = np.abs(g["sig_sel"][e, q] - ref["sig_sel"][t, q]).max() / st[q]
            assert errS <= tolS, (e, q, errS)
            assert abs(g["sig_tot"][e, q] - st[q]) <= tolS * st[q]
        assert abs(orc.wrap_angle(g["eigsum"][e] - ref["eta"][t])) <= tolS * 10


def test_config1_full_sweep(rm):
    wl = synth.config(1)
    sel = (0, 1, 2, 3)
    g = gpu_sweep(rm, wl, sel=sel)
    ref = orc.sweep(wl.waves[0], wl.energies, sel=sel)
    compare(wl, g, ref)


@pytest.mark.parametrize("n,N,ne", [(1, 1, 1), (2, 5, 7), (3, 63, 33), (17, 65, 130), (33, 200, 70),
                                    (16, 64, 64), (40, 129, 17)])
def test_ragged_sizes(rm, n, N, ne):
    wl = synth.small(100 + n, n, N, ne, e_lo=0.01, e_hi=3.0, pole_lo=-2.0, pole_hi=6.0, a=12.0)
    sel = tuple(range(min(n, 3)))
    g = gpu_sweep(rm, wl, sel=sel, chunk=5 if ne > 10 else 0)
    ref = orc.sweep(wl.waves[0], wl.energies, sel=sel)
    compare(wl, g, ref)


@pytest.mark.parametrize("prec", ["fp64", "split_bf16"])
def test_lmax15_zero_potential(rm, prec):
    # angular momenta up to 15 (the n_ch = 512 workload's range) in the zero-potential outer
    # region: open channels with x = k a < l take jhat_l from the downward (Miller) recurrence,
    # x > l from the upward one; closed channels of high l their khat_l log-derivative.  Energies
    # just above thresholds (x from 0.02 up), just below, and up to 6 Ry (x up to about 85).
    rng = np.random.default_rng(1515)
    l = np.array([0, 15, 8, 12, 3, 15, 9, 14, 1, 11, 10, 13, 2, 15, 7, 5], np.int32)
    w = synth.make_wave(rng, l.size, 1500, thr_hi=2.0, pole_lo=-10.0, pole_hi=80.0, a=35.0, l_fixed=l)
    E = list(np.linspace(0.01, 6.0, 40))
    for t in w.thresh[1:]:
        E += [t + 3e-7, t + (0.6 / w.a) ** 2, t + (4.0 / w.a) ** 2, t - 1e-4]
    E = np.unique(np.array([e for e in E if e > 0.005]))
    wl = synth.Workload("lmax15", [w], E, delta=0.05)
    sel = (0, 1, 5)
    g = gpu_sweep(rm, wl, sel=sel, prec=prec)
    ref = orc.sweep(w, E, sel=sel)
    if prec == "fp64":
        compare(wl, g, ref)
    else:
        compare(wl, g, ref, tolK=1e-6, tolS=1e-8, checkR=False)
        for t in range(E.size):
            Rg, Ro = g["R"][t], ref["R"][t]
            assert np.abs(Rg - Ro).max() <= 1e-6 * np.abs(Ro).max(), t


def test_config2_sampled(rm):
    wl = synth.config(2)
    w = wl.waves[0]
    e0, e1 = 9000, 9600   # a contiguous block (spans chunk and tile edges)
    sub = synth.Workload(wl.name, wl.waves, wl.energies[e0:e1])
    g = gpu_sweep(rm, sub, sel=(0, 5))
    idx = np.arange(0, e1 - e0, 7)
    ref = orc.sweep(w, sub.energies, sel=(0, 5), energy_idx=idx)
    compare(sub, g, ref, idx=idx)


def test_chunking_is_bit_exact(rm):
    wl = synth.small(3, 12, 150, 90)
    a = gpu_sweep(rm, wl, sel=(0, 2), chunk=0)
    b = gpu_sweep(rm, wl, sel=(0, 2), chunk=7)
    for k in ("R", "K", "eigsum", "sig_sel", "sig_tot", "n_open", "flags"):
        assert np.array_equal(a[k], b[k]), k


def test_run_results_equal_xsec(rm):
    wl = synth.small(4, 10, 120, 50)
    w = wl.waves[0]
    g = gpu_sweep(rm, wl, sel=(0, 1))
    with rm.Plan(wl.waves, wl.energies, sel=(0, 1)) as p:
        p.run()
        out = rm.host_outputs(wl.n_e, w.n, 2)
        p.results(0, 0, wl.n_e, **out)
    for k in ("eigsum", "sig_sel", "sig_tot", "n_open"):
        assert np.array_equal(out[k], g[k]), k


def test_device_tensors_match_host(rm):
    wl = synth.small(5, 8, 90, 40)
    w = wl.waves[0]
    g = gpu_sweep(rm, wl, sel=(0,))
    dev = torch.device("cuda:0")
    dw = synth.Wave(l=torch.from_numpy(w.l).to(dev), thresh=torch.from_numpy(w.thresh).to(dev),
                    poles=torch.from_numpy(w.poles).to(dev), W=torch.from_numpy(w.W).to(dev), a=w.a)
    E = torch.from_numpy(wl.energies).to(dev)
    with rm.Plan([dw], E, sel=(0,)) as p:
        R = torch.zeros((wl.n_e, w.n * (w.n + 1) // 2), dtype=torch.float64, device=dev)
        p.rmatrix(0, 0, wl.n_e, R)
        eta = torch.zeros(wl.n_e, dtype=torch.float64, device=dev)
        sig = torch.zeros((wl.n_e, 1, w.n), dtype=torch.float64, device=dev)
        p.xsec(0, 0, wl.n_e, eigsum=eta, sig_sel=sig)
        p.sync()
    assert np.array_equal(R.cpu().numpy(), g["R"])
    assert np.array_equal(eta.cpu().numpy(), g["eigsum"])
    assert np.array_equal(sig.cpu().numpy(), g["sig_sel"])


def test_nudge_and_no_open(rm):
    w = synth.small(6, 4, 40, 1, pole_lo=0.1, pole_hi=3.0).waves[0]
    on_pole, on_thr = w.poles[3], w.thresh[2] + 2e-10
    E = np.sort(np.array([-0.5, -0.1, on_pole, on_thr, 1.234]))
    wl = synth.Workload("edge", [w], E)
    g = gpu_sweep(rm, wl, sel=(0, 1))
    ref = orc.sweep(w, E, sel=(0, 1))
    assert g["flags"][0] & orc.FLAG_NO_OPEN and g["flags"][1] & orc.FLAG_NO_OPEN
    assert g["n_open"][0] == 0 and g["eigsum"][0] == 0.0 and np.all(g["sig_sel"][0] == 0)
    for e in range(E.size):
        if E[e] in (on_pole, on_thr):
            assert g["flags"][e] & orc.FLAG_NUDGED
    compare(wl, g, ref)


def test_error_paths(rm):
    wl = synth.small(8, 5, 30, 10)
    w = wl.waves[0]
    bad = synth.Wave(l=w.l, thresh=w.thresh, poles=w.poles[::-1].copy(), W=w.W, a=w.a)
    with pytest.raises(rm.RMError) as ei:
        rm.Plan([bad], wl.energies)
    assert ei.value.code == rm.RM_ERR_ORDER
    Wn = w.W.copy()
    Wn[1, 3] = np.nan
    with pytest.raises(rm.RMError) as ei:
        rm.Plan([synth.Wave(l=w.l, thresh=w.thresh, poles=w.poles, W=Wn, a=w.a)], wl.energies)
    assert ei.value.code == rm.RM_ERR_ARG
    lb = w.l.copy()
    lb[0] = 40
    with pytest.raises(rm.RMError) as ei:
        rm.Plan([synth.Wave(l=lb, thresh=w.thresh, poles=w.poles, W=w.W, a=w.a)], wl.energies)
    assert ei.value.code == rm.RM_ERR_ARG
    with pytest.raises(rm.RMError) as ei:
        rm.Plan(wl.waves, wl.energies[::-1].copy())
    assert ei.value.code == rm.RM_ERR_ORDER
    with rm.Plan(wl.waves, wl.energies) as p:
        with pytest.raises(rm.RMError) as ei:
            p.results(0, 0, 5, eigsum=np.zeros(5))
        assert ei.value.code == rm.RM_ERR_STATE
        with pytest.raises(rm.RMError) as ei:
            p.xsec(1, 0, 5, eigsum=np.zeros(5))
        assert ei.value.code == rm.RM_ERR_ARG
        with pytest.raises(rm.RMError) as ei:
            p.xsec(0, 3, 11, eigsum=np.zeros(8))
        assert ei.value.code == rm.RM_ERR_ARG


def test_plan_load_replaces_inputs(rm):
    a = synth.small(9, 6, 50, 20)
    b = synth.small(10, 6, 50, 20)
    ga = gpu_sweep(rm, a)
    gb = gpu_sweep(rm, b)
    with rm.Plan(a.waves, a.energies) as p:
        p.load(b.waves, b.energies)
        p.run()
        out = rm.host_outputs(b.n_e, 6, 1)
        p.results(0, 0, b.n_e, **out)
    assert np.array_equal(out["sig_sel"], gb["sig_sel"])
    assert not np.array_equal(ga["sig_sel"], gb["sig_sel"])
