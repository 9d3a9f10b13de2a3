"""Grouped sweep (all partial waves per launch, CUDA-graph replay, autotuned
energy chunks) on the 40-wave workload (needs a GPU)."""
import os

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


def test_forty_waves_against_oracle(rm):
    # the 40-wave workload (n_ch 9..387, N = 40 n_ch) on a 600-energy mesh, through rm_run:
    # per wave five energies (spread over the mesh, one just above a threshold), sigma from two
    # initial channels and the totals, eta, the open-channel count and flags; and R per element of
    # one energy per wave through rm_rmatrix, within the split form's bound
    wl = synth.config(4)
    E = np.linspace(0.01, 5.0, 600)
    sel = (0, 1)
    with rm.Plan(wl.waves, E, prec="split_bf16", delta=0.05, sel=sel) as p:
        p.run()
        outs = []
        for g, w in enumerate(wl.waves):
            o = rm.host_outputs(E.size, w.n, len(sel))
            p.results(g, 0, E.size, **o)
            outs.append(o)
        Rs = []
        for g, w in enumerate(wl.waves):
            e = (37 * g + 11) % E.size
            R = np.zeros((1, w.n * (w.n + 1) // 2))
            p.rmatrix(g, e, e + 1, R)
            Rs.append((e, R[0]))
    checked = 0
    for g, w in enumerate(wl.waves):
        thr = w.thresh[min(3, w.n - 1)]
        e_thr = int(np.searchsorted(E, thr, side="right"))
        idx = np.unique(np.array([7 + 13 * g % 580, 599 - 7 * g % 300, 150 + 5 * g, 420 - 3 * g,
                                  min(e_thr, E.size - 1)]))
        ref = orc.sweep(w, E, sel=sel, energy_idx=idx, keep_R=False, keep_K=False)
        for t, e in enumerate(idx):
            assert outs[g]["n_open"][e] == ref["n_open"][t]
            assert (outs[g]["flags"][e] & orc.FLAG_NUDGED) == (ref["flags"][t] & orc.FLAG_NUDGED)
            if ref["flags"][t] & (orc.FLAG_ILLCOND | orc.FLAG_NO_OPEN):
                continue
            for q in range(len(sel)):
                st = ref["sig_tot"][t, q]
                if st == 0:
                    assert np.all(outs[g]["sig_sel"][e, q] == 0)
                    continue
                err = np.abs(outs[g]["sig_sel"][e, q] - ref["sig_sel"][t, q]).max() / st
                assert err <= 1e-8, (g, w.n, e, q, err)
                assert abs(outs[g]["sig_tot"][e, q] - st) <= 1e-8 * st
            d = outs[g]["eigsum"][e] - ref["eta"][t]
            assert abs(np.mod(d + np.pi, 2 * np.pi) - np.pi) <= 1e-7, (g, e)
            checked += 1
        e, Rg = Rs[g]
        Ro = orc.rmatrix(w.W, w.poles, orc.nudge_energies(E[e:e + 1], w.poles, w.thresh)[0][0], w.a)
        d = np.abs(1.0 / (w.poles - orc.nudge_energies(E[e:e + 1], w.poles, w.thresh)[0][0]))
        bound = 4e-7 * (np.abs(w.W) * d[None, :]) @ np.abs(w.W).T / (2.0 * w.a) + 1e-300
        assert np.all(np.abs(orc.unpack_upper(Rg, w.n) - Ro) <= bound), (g, e)
    assert checked >= 150


def test_graph_replay_and_launch_count(rm):
    waves = [synth.small(300 + g, n, 40 * n, 1, pole_lo=-3, pole_hi=12, a=20.0).waves[0]
             for g, n in enumerate([7, 30, 12])]
    E = np.linspace(0.05, 3.0, 300)
    with rm.Plan(waves, E, prec="split_bf16", delta=0.05, sel=(0, 1), chunk=128) as p:
        l0 = p.launches()
        p.run()
        l1 = p.launches()
        first = [rm.host_outputs(E.size, w.n, 2) for w in waves]
        for g in range(3):
            p.results(g, 0, E.size, **first[g])
        p.run()
        p.run()
        l3 = p.launches()
        for g in range(3):
            o = rm.host_outputs(E.size, waves[g].n, 2)
            p.results(g, 0, E.size, **o)
            for k in ("eigsum", "sig_sel", "sig_tot"):
                assert np.array_equal(o[k], first[g][k]), k
        # 3 chunks x ([D slices,] pole sum, near window, asymptotics, solve) per replay; the D-slice
        # kernel runs for shapes with cluster_x = 1
        per_chunk = 5 if p.cluster()[0] == 1 else 4
        assert l1 - l0 == 3 * per_chunk and l3 - l1 == 6 * per_chunk
        # profiled (direct) launches give the same numbers as the graph replay
        p.profile(True)
        p.run()
        prof = p.profile_read()
        p.profile(False)
        assert prof["solve"][1] == 3 and prof["polesum_split"][1] == 3
        assert prof["dslice"][1] == (3 if p.cluster()[0] == 1 else 0)
        for g in range(3):
            o = rm.host_outputs(E.size, waves[g].n, 2)
            p.results(g, 0, E.size, **o)
            assert np.array_equal(o["sig_sel"], first[g]["sig_sel"])


def test_autotune_and_cache(rm, tmp_path):
    wl = synth.small(41, 24, 900, 1500, e_lo=0.05, e_hi=3.0, pole_lo=-3, pole_hi=10, a=18.0)
    cache = str(tmp_path / "tune.txt")
    with rm.Plan(wl.waves, wl.energies, prec="split_bf16", delta=0.05, autotune=True, tune_cache=cache) as p:
        chunk = p.info(0)["chunk"]
        shape = p.cluster()
        p.run()
        o1 = rm.host_outputs(wl.n_e, 24, 1)
        p.results(0, 0, wl.n_e, **o1)
    # candidates: powers of two from 256 below the mesh size, and the whole mesh
    assert chunk in (256, 512, 1024, wl.n_e) and os.path.exists(cache)
    assert shape in [(1, 2), (1, 4), (2, 2), (1, 1), (4, 1), (2, 1)]
    line = open(cache).read().strip().splitlines()[-1]
    assert line.endswith("|%d %d %d" % (chunk, shape[0], shape[1]))
    with rm.Plan(wl.waves, wl.energies, prec="split_bf16", delta=0.05, autotune=True, tune_cache=cache) as p:
        assert p.info(0)["chunk"] == chunk and p.cluster() == shape
        p.run()
        o2 = rm.host_outputs(wl.n_e, 24, 1)
        p.results(0, 0, wl.n_e, **o2)
    assert np.array_equal(o1["sig_sel"], o2["sig_sel"])


CLUSTERS = [(1, 1), (2, 1), (4, 1), (1, 2), (2, 2), (1, 4), (4, 2), (2, 4)]


@pytest.fixture(scope="module", params=[0, 13], ids=["default-products", "13-products"])
def cluster_case(rm, request):
    # uneven waves (odd tile counts per wave, so clusters need padding), a mesh
    # that is not a multiple of 128 energies, two selected channels; the default
    # product set (five slices: a separate D ring with D by TMA, two stages with D
    # formed in the kernel) and the 13-product set (four slices, three stages)
    waves = [synth.small(500 + g, n, 40 * n, 1, pole_lo=-3, pole_hi=12, a=20.0).waves[0]
             for g, n in enumerate([5, 23, 9, 40, 17])]
    E = np.linspace(0.04, 3.3, 333)
    sel = (0, 1)
    slices = request.param
    with rm.Plan(waves, E, prec="split_bf16", delta=0.05, sel=sel, chunk=200, cluster=(1, 1), slices=slices) as p:
        assert p.cluster() == (1, 1)
        p.run()
        base = []
        for g, w in enumerate(waves):
            o = rm.host_outputs(E.size, w.n, 2)
            p.results(g, 0, E.size, **o)
            base.append(o)
    return waves, E, sel, base, slices


@pytest.mark.parametrize("shape", CLUSTERS, ids=["%dx%d" % c for c in CLUSTERS])
def test_cluster_shapes_identical(rm, cluster_case, shape):
    # every CTA forms the same slices whichever CTA of a cluster stores them, so
    # the sums (and everything after them) are bit-identical across cluster shapes
    waves, E, sel, base, slices = cluster_case
    try:
        p = rm.Plan(waves, E, prec="split_bf16", delta=0.05, sel=sel, chunk=200, cluster=shape, slices=slices)
    except rm.RMError as ex:
        pytest.skip(f"cluster shape {shape} not co-schedulable here: {ex}")
    with p:
        assert p.cluster() == shape
        p.run()
        for g, w in enumerate(waves):
            o = rm.host_outputs(E.size, w.n, 2)
            p.results(g, 0, E.size, **o)
            for k in ("eigsum", "sig_tot", "sig_sel", "n_open", "flags"):
                assert np.array_equal(o[k], base[g][k]), (shape, g, k)
    # and against the oracle on sampled energies
    for g, w in enumerate(waves):
        idx = np.array([3 + 31 * g, 332 - 17 * g])
        ref = orc.sweep(w, E, sel=sel, energy_idx=idx, keep_R=False, keep_K=False)
        for t, e in enumerate(idx):
            if ref["flags"][t] & orc.FLAG_ILLCOND:
                continue
            for q in range(2):
                st = ref["sig_tot"][t, q]
                if st > 0:
                    assert np.abs(base[g]["sig_sel"][e, q] - ref["sig_sel"][t, q]).max() / st <= 1e-8


@pytest.mark.parametrize("n_e", [333, 130, 1])
def test_mma_pair_matches_one_sm(rm, n_e):
    # the 2-SM form (tcgen05 cta_group::2, M = 256 energies over the CTA pair, each CTA holding the
    # P slices of the 64 pairs it forms) against the one-SM form of the same 1 x 2 cluster, on
    # uneven waves and meshes of 3, 2 and 1 energy tiles (odd counts leave the second CTA of the
    # last cluster past the mesh): the same slice products summed in the same order per
    # accumulator give the same bits; and against the oracle on sampled energies
    waves = [synth.small(700 + g, n, 40 * n, 1, pole_lo=-3, pole_hi=12, a=20.0).waves[0]
             for g, n in enumerate([5, 23, 9, 40, 17, 64])]
    E = np.linspace(0.04, 3.3, n_e)
    sel = (0, 2)
    outs = {}
    for pair in (0, -1):
        # both forms must be resident on a GB300: a kernel that cannot be (registers, shared
        # memory) would make the plan fall back to another shape silently, so this is a failure
        p = rm.Plan(waves, E, prec="split_bf16", delta=0.05, sel=sel, cluster=(1, 2), mma_pair=pair)
        with p:
            assert p.mma_pair() == (pair == 0)
            p.run()
            res = []
            for g, w in enumerate(waves):
                o = rm.host_outputs(E.size, w.n, 2)
                p.results(g, 0, E.size, **o)
                res.append(o)
            outs[pair] = res
    for g in range(len(waves)):
        for k in ("eigsum", "sig_tot", "sig_sel", "n_open", "flags"):
            assert np.array_equal(outs[0][g][k], outs[-1][g][k]), (n_e, g, k)
    for g, w in enumerate(waves):
        idx = np.unique(np.array([0, n_e // 2, n_e - 1]))
        ref = orc.sweep(w, E, sel=sel, energy_idx=idx, keep_R=False, keep_K=False)
        for t, e in enumerate(idx):
            if ref["flags"][t] & (orc.FLAG_ILLCOND | orc.FLAG_NO_OPEN):
                continue
            for q in range(2):
                st = ref["sig_tot"][t, q]
                if st > 0:
                    err = np.abs(outs[0][g]["sig_sel"][e, q] - ref["sig_sel"][t, q]).max() / st
                    assert err <= 1e-8, (g, e, q, err)
            d = outs[0][g]["eigsum"][e] - ref["eta"][t]
            assert abs(np.mod(d + np.pi, 2 * np.pi) - np.pi) <= 1e-7, (g, e)
