"""Parity of the split-precision path (sliced BF16 tcgen05 pole sum + FP64
near-pole window + FP64 solves) with the FP64 CPU oracle (needs a GPU).

Tolerances:
* R per element (the default product set): P and D are formed in double-float
  (about 2^-46), and the slicing leaves at most 2^-31 of the product of the two
  scales per far term (test_split_product_sets bounds each set separately); the
  per-element check |R - R*| <= 4e-7 (1/2a) sum_k |w_ik w_jk / (E_k - E)| is the
  bound of an FP32 formation of every term, which all sets of 10 products or more
  stay far inside.
* R, K normwise <= 1e-6 and sigma <= 1e-8 (normalised by sigma_tot of the
  initial channel): the accuracy targets of the method's split form, on
  energies the oracle does not flag ILLCOND.
"""
import numpy as np
import pytest

from oracle import rmatrix as orc
from paper_1403_5524_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_R_NORM = 1e-6
TOL_K = 1e-6
TOL_SIG = 1e-8


@pytest.fixture(scope="module")
def rm():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1403_5524_gb300 import rm as _rm
    _rm.load_library()
    return _rm


def abs_sum(w, E):
    d = np.abs(1.0 / (w.poles - E))
    return (np.abs(w.W) * d[None, :]) @ np.abs(w.W).T / (2.0 * w.a)


def run_split(rm, wl, sel=(0,), idx=None, chunk=0, delta=None, slices=0, prec="split_bf16", run=False):
    w = wl.waves[0]
    n = w.n
    idx = np.arange(wl.n_e) if idx is None else np.asarray(idx)
    out = {"R": [], "K": [], "eta": [], "sig": [], "flags": [], "n_open": []}
    with rm.Plan(wl.waves, wl.energies, prec=prec, delta=wl.delta if delta is None else delta,
                 sel=sel, chunk=chunk, slices=slices) as p:
        if run:
            # the timed path too: rm_run (grouped tensor-core launch, D slices by TMA) and rm_results
            p.run()
            r = rm.host_outputs(wl.n_e, n, len(sel))
            p.results(0, 0, wl.n_e, **r)
            out["run_eta"] = r["eigsum"][idx]
            out["run_sig"] = r["sig_sel"][idx]
            out["run_flags"] = r["flags"][idx]
        for e in idx:
            e = int(e)
            R = np.zeros((1, n * (n + 1) // 2))
            p.rmatrix(0, e, e + 1, R)
            K = np.zeros((1, n, n))
            no = np.zeros(1, np.int32)
            fl = np.zeros(1, np.uint8)
            p.kmatrix(0, e, e + 1, K=K, n_open=no, flags=fl)
            eta = np.zeros(1)
            sig = np.zeros((1, len(sel), n))
            p.xsec(0, e, e + 1, eigsum=eta, sig_sel=sig)
            out["R"].append(R[0]); out["K"].append(K[0]); out["eta"].append(eta[0]); out["sig"].append(sig[0])
            out["flags"].append(fl[0]); out["n_open"].append(no[0])
    return {k: np.array(v) for k, v in out.items()}


# Slice-truncation error of one far term P_pk D_ke per product set, in units of the product of the
# two operands' power-of-two scales (each operand is scaled to [-256, 256] and cut into slices of
# 8 bits: integer, 2^-8, 2^-16 and a BF16-rounded rest; a set keeps the products with u + v below
# its order).  With x = s0 + s1 + s2 + s3, |s1| <= 2^-1, |s2| <= 2^-9, |s3| <= 2^-17 and the rest
# rounded to 8 bits (2^-25):  3 products (two slices): operand tails 2 * 2^8 * 2^-9 plus s1 t1 ->
# 1.25 of 2^16;  6: 2 * 2^8 * 2^-17 + s1 t2 + s2 t1 -> 2^-7.4;  10: 2 * 2^8 * 2^-25 + the order-4
# products -> 2^-15.2;  13: 2 * 2^8 * 2^-25 -> 2^-16;  15 (five slices, the fifth 2^-25 small and
# rounded to 2^-34): 2 * 2^8 * 2^-34 plus the order-5 products -> 2^-24.  Relative to 2^16, with
# margin:
SLICE_EPS = {3: 2.0 ** -15, 6: 2.0 ** -23, 10: 2.0 ** -31, 13: 2.0 ** -31.5, 15: 2.0 ** -39}


def slice_bound(w, E, eps, delta):
    # |R - R*| per element <= 4 eps (1/2a) sum over far poles of max_k |w_ik w_jk| max_far |1/(E_k - E)|
    # (the power-of-two scales are below twice the maxima), plus the double-float formation and FP64
    # near-window rounding (2^-40 of the absolute sum)
    d = np.abs(1.0 / (w.poles - E))
    far = np.abs(w.poles - E) >= delta
    n_far = int(far.sum())
    maxd = float(d[far].max()) if n_far else 0.0
    maxp = np.max(np.abs(w.W)[:, None, :] * np.abs(w.W)[None, :, :], axis=2)
    absum = (np.abs(w.W) * d[None, :]) @ np.abs(w.W).T
    return (4.0 * eps * n_far * maxp * maxd + 2.0 ** -40 * absum) / (2.0 * w.a) + 1e-300


def check(wl, g, ref, per_element=True):
    w = wl.waves[0]
    n = w.n
    worst = {"R": 0.0, "K": 0.0, "sig": 0.0}
    for t in range(ref["E"].shape[0]):
        Rg = orc.unpack_upper(g["R"][t], n)
        Ro = orc.unpack_upper(ref["R"][t], n)
        if per_element:
            bound = 4e-7 * abs_sum(w, ref["E"][t]) + 1e-300
            assert np.all(np.abs(Rg - Ro) <= bound), (t, float(np.max(np.abs(Rg - Ro) / bound)))
        eR = np.abs(Rg - Ro).max() / np.abs(Ro).max()
        worst["R"] = max(worst["R"], eR)
        assert eR <= TOL_R_NORM, (t, eR)
        assert g["n_open"][t] == ref["n_open"][t]
        if ref["flags"][t] & (orc.FLAG_ILLCOND | orc.FLAG_SINGULAR | orc.FLAG_NO_OPEN):
            continue
        no = ref["n_open"][t]
        Ko = ref["K"][t, :no, :no]
        eK = np.abs(g["K"][t, :no, :no] - Ko).max() / np.abs(Ko).max()
        worst["K"] = max(worst["K"], eK)
        assert eK <= TOL_K, (t, eK)
        for q in range(ref["sig_tot"].shape[1]):
            st = ref["sig_tot"][t, q]
            if st > 0:
                eS = np.abs(g["sig"][t, q] - ref["sig_sel"][t, q]).max() / st
                worst["sig"] = max(worst["sig"], eS)
                assert eS <= TOL_SIG, (t, q, eS)
    return worst


@pytest.mark.parametrize("seed,n,N,ne", [(1, 4, 200, 40), (2, 9, 513, 30), (3, 17, 1000, 25), (4, 33, 2049, 20),
                                         (5, 130, 700, 12)])
def test_split_small(rm, seed, n, N, ne):
    # ragged channel counts (not multiples of 8/16), poles not multiples of 32,
    # pole density high enough that every energy has a near window
    wl = synth.small(seed, n, N, ne, e_lo=0.05, e_hi=3.5, pole_lo=-3.0, pole_hi=12.0, a=20.0, delta=0.05)
    sel = (0, min(1, n - 1))
    g = run_split(rm, wl, sel=sel)
    ref = orc.sweep(wl.waves[0], wl.energies, sel=sel)
    check(wl, g, ref)


def test_split_window_edges(rm):
    # energies placed exactly delta away from poles, and on poles (nudged)
    wl = synth.small(11, 6, 300, 1, pole_lo=0.0, pole_hi=4.0, a=15.0)
    w = wl.waves[0]
    E = np.sort(np.array([w.poles[40] + 0.05, w.poles[80] - 0.05, w.poles[120], w.poles[160] + 0.0499999,
                          1.7, 2.2]))
    wl2 = synth.Workload("edges", [w], E, delta=0.05)
    g = run_split(rm, wl2, sel=(0,))
    ref = orc.sweep(w, E, sel=(0,))
    check(wl2, g, ref)


def test_split_chunk_tiles_and_run(rm):
    # energies across several 128-energy tiles and chunks; rm_run equals rm_xsec
    wl = synth.small(12, 20, 800, 300, e_lo=0.02, e_hi=3.0, pole_lo=-2.0, pole_hi=8.0, a=18.0)
    w = wl.waves[0]
    sel = (0, 3)
    with rm.Plan(wl.waves, wl.energies, prec="split_bf16", delta=0.05, sel=sel, chunk=256) as p:
        p.run()
        out = rm.host_outputs(wl.n_e, w.n, 2)
        p.results(0, 0, wl.n_e, **out)
        out2 = rm.host_outputs(wl.n_e, w.n, 2)
        p.xsec(0, 0, wl.n_e, eigsum=out2["eigsum"], sig_tot=out2["sig_tot"], sig_sel=out2["sig_sel"])
        p.sync()
    assert np.array_equal(out["sig_sel"], out2["sig_sel"])
    assert np.array_equal(out["eigsum"], out2["eigsum"])
    idx = np.arange(0, wl.n_e, 23)
    ref = orc.sweep(w, wl.energies, sel=sel, energy_idx=idx)
    for t, e in enumerate(idx):
        if ref["flags"][t] & orc.FLAG_ILLCOND:
            continue
        for q in range(2):
            st = ref["sig_tot"][t, q]
            if st > 0:
                assert np.abs(out["sig_sel"][e, q] - ref["sig_sel"][t, q]).max() / st <= TOL_SIG


def test_split_deterministic(rm):
    wl = synth.small(13, 24, 900, 16)
    a = run_split(rm, wl)
    b = run_split(rm, wl)
    for k in ("R", "K", "eta", "sig"):
        assert np.array_equal(a[k], b[k]), k


def test_split_config3_sampled(rm):
    # the full n_ch=256, N=20000 workload, checked on sampled energies of the mesh
    wl = synth.config(3)
    idx = np.linspace(0, wl.n_e - 1, 6).astype(int)
    g = run_split(rm, wl, sel=(0,), idx=idx)
    ref = orc.sweep(wl.waves[0], wl.energies, sel=(0,), energy_idx=idx)
    worst = check(wl, g, ref, per_element=False)
    print("config3 split worst normwise errors", worst)


@pytest.mark.parametrize("slices,prec", [(3, "split_bf16"), (6, "split_bf16"), (10, "split_bf16"),
                                         (13, "split_bf16"), (15, "split_bf16"), (10, "split_fp16")])
def test_split_product_sets(rm, slices, prec):
    # each product set of the tensor-core pole sum against the oracle, R per element within the
    # set's truncation bound; the sets that reach the method's targets here (10, 13, 15 products) are
    # also held to them for K, sigma and eta, through the per-range calls and through rm_run
    wl = synth.small(31, 24, 3000, 36, e_lo=0.05, e_hi=3.4, pole_lo=-3.0, pole_hi=12.0, a=20.0, delta=0.05)
    w = wl.waves[0]
    sel = (0, 3)
    g = run_split(rm, wl, sel=sel, slices=slices, prec=prec, run=True)
    ref = orc.sweep(w, wl.energies, sel=sel)
    worst = {"R": 0.0, "K": 0.0, "sig": 0.0, "eta": 0.0}
    for t in range(wl.n_e):
        Rg = orc.unpack_upper(g["R"][t], w.n)
        Ro = orc.unpack_upper(ref["R"][t], w.n)
        bound = slice_bound(w, ref["E"][t], SLICE_EPS[slices], wl.delta)
        assert np.all(np.abs(Rg - Ro) <= bound), (t, float(np.max(np.abs(Rg - Ro) / bound)))
        worst["R"] = max(worst["R"], float(np.abs(Rg - Ro).max() / np.abs(Ro).max()))
        if ref["flags"][t] & (orc.FLAG_ILLCOND | orc.FLAG_SINGULAR | orc.FLAG_NO_OPEN):
            continue
        no = ref["n_open"][t]
        Ko = ref["K"][t, :no, :no]
        worst["K"] = max(worst["K"], float(np.abs(g["K"][t, :no, :no] - Ko).max() / np.abs(Ko).max()))
        for q in range(len(sel)):
            st = ref["sig_tot"][t, q]
            if st > 0:
                for sg in (g["sig"][t, q], g["run_sig"][t, q]):
                    worst["sig"] = max(worst["sig"], float(np.abs(sg - ref["sig_sel"][t, q]).max() / st))
        for eta in (g["eta"][t], g["run_eta"][t]):
            worst["eta"] = max(worst["eta"], float(abs(orc.wrap_angle(eta - ref["eta"][t]))))
    print(f"{prec} {slices} products: worst normwise errors", worst)
    if slices >= 10:
        assert worst["R"] <= TOL_R_NORM and worst["K"] <= TOL_K
        assert worst["sig"] <= (TOL_SIG if prec == "split_bf16" else 5e-8)
        assert worst["eta"] <= 1e-7


def test_split_config5_sampled(rm):
    # the n_ch = 512, N = 25000 workload (l up to 15, a = 35): energies just above thresholds of
    # channels with l >= 8 (x = k a < l: the Miller downward recurrence of jhat_l) and high energies;
    # R per element, K and sigma normwise, sigma and eta also from the timed rm_run
    wl = synth.config(5)
    w = wl.waves[0]
    E = wl.energies
    low = []
    for i in np.argsort(w.thresh):
        if w.l[i] >= 8 and w.thresh[i] > 0.05:
            e = int(np.searchsorted(E, w.thresh[i], side="right"))
            k = np.sqrt(E[e] - w.thresh[i])
            if k * w.a < w.l[i] and e not in low:
                low.append(e)
        if len(low) == 4:
            break
    assert len(low) == 4
    idx = np.array(sorted(low + list(np.linspace(E.size // 2, E.size - 1, 4).astype(int))))
    sel = (0, 1)
    g = run_split(rm, wl, sel=sel, idx=idx, run=True)
    ref = orc.sweep(w, E, sel=sel, energy_idx=idx)
    worst = check(wl, g, ref, per_element=True)
    for t in range(idx.size):
        if ref["flags"][t] & (orc.FLAG_ILLCOND | orc.FLAG_SINGULAR | orc.FLAG_NO_OPEN):
            continue
        for q in range(len(sel)):
            st = ref["sig_tot"][t, q]
            if st > 0:
                eS = np.abs(g["run_sig"][t, q] - ref["sig_sel"][t, q]).max() / st
                assert eS <= TOL_SIG, (t, q, eS)
        assert abs(orc.wrap_angle(g["run_eta"][t] - ref["eta"][t])) <= 1e-7
    print("config5 split worst normwise errors", worst)


def test_split_multiwave(rm):
    # several partial waves of uneven size in one plan, one shared energy mesh
    rng_sizes = [(5, 200), (23, 900), (9, 360), (40, 1600)]
    waves = []
    for g, (n, N) in enumerate(rng_sizes):
        waves.append(synth.small(200 + g, n, N, 1, pole_lo=-3.0, pole_hi=10.0, a=18.0).waves[0])
    E = np.linspace(0.03, 3.2, 140)
    sel = (0, 1)
    with rm.Plan(waves, E, prec="split_bf16", delta=0.05, sel=sel, chunk=128) as p:
        p.run()
        outs = []
        for g, w in enumerate(waves):
            o = rm.host_outputs(E.size, w.n, 2)
            p.results(g, 0, E.size, **o)
            outs.append(o)
    idx = np.arange(0, E.size, 9)
    for g, w in enumerate(waves):
        ref = orc.sweep(w, E, sel=sel, energy_idx=idx, keep_R=False)
        for t, e in enumerate(idx):
            assert outs[g]["n_open"][e] == ref["n_open"][t]
            if ref["flags"][t] & orc.FLAG_ILLCOND:
                continue
            for q in range(2):
                st = ref["sig_tot"][t, q]
                if st > 0:
                    err = np.abs(outs[g]["sig_sel"][e, q] - ref["sig_sel"][t, q]).max() / st
                    assert err <= TOL_SIG, (g, e, q, err)
            d = outs[g]["eigsum"][e] - ref["eta"][t]
            assert abs(np.mod(d + np.pi, 2 * np.pi) - np.pi) <= 1e-7
