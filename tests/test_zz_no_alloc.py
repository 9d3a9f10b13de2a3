"""The allocation-free entry point rm_xsec_from_r_static (needs a GPU).

Some callers cannot call cudaMalloc: plug-ins bound to a host application's
fixed memory pool, real-time loops where an allocation may block or fail, code
running where the device allocator is off limits to it.  They get K, the
eigenphase sum and cross sections from R-matrices they already hold, with the
library's static scratch only.  Its results must equal those of the plan-based
rm_kmatrix / rm_xsec on the same R, and the oracle's, within the FP64 path's
tolerances, on two calls in a row (the second call reuses the scratch the first
one left behind), over several energy chunks with a ragged last one, and at the
largest channel count, where the scratch forces a smaller chunk.  This file is collected
last so that a run stopping at its first failure has run every other test.
"""
import ctypes as C

import numpy as np
import pytest

from oracle import rmatrix as orc
from paper_1403_5524_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1403_5524_gb300 import rm
    return rm.load_library()


def layout(lib, n, n_sel):
    c, s = C.c_int32(), C.c_int32()
    code = lib.rm_static_layout(n, n_sel, C.byref(c), C.byref(s))
    return code, c.value, s.value


def plan_reference(wl, sel, dev):
    from paper_1403_5524_gb300 import rm
    w = wl.waves[0]
    n, ne = w.n, wl.n_e
    with rm.Plan(wl.waves, wl.energies, prec="fp64", sel=tuple(sel)) as p:
        R = torch.zeros((ne, n * (n + 1) // 2), dtype=torch.float64, device=dev)
        p.rmatrix(0, 0, ne, R)
        K0 = np.zeros((ne, n, n))
        p.kmatrix(0, 0, ne, K=K0)
        ref = rm.host_outputs(ne, n, len(sel))
        p.xsec(0, 0, ne, eigsum=ref["eigsum"], sig_tot=ref["sig_tot"], sig_sel=ref["sig_sel"])
        p.sync()
    return R, K0, ref


def static_call(lib, R, w, E_dev, sel, dev, l_dev=None):
    n, ne = w.n, E_dev.shape[0]
    ns = len(sel)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    l = d(w.l) if l_dev is None else l_dev
    thr, poles = d(w.thresh), d(w.poles)
    out = {"K": torch.full((ne, n, n), np.nan, dtype=torch.float64, device=dev),
           "eta": torch.full((ne,), np.nan, dtype=torch.float64, device=dev),
           "st": torch.full((ne, ns), np.nan, dtype=torch.float64, device=dev),
           "ss": torch.full((ne, ns, n), np.nan, dtype=torch.float64, device=dev),
           "fl": torch.zeros(ne, dtype=torch.uint8, device=dev),
           "no": torch.zeros(ne, dtype=torch.int32, device=dev)}
    sel_h = np.ascontiguousarray(np.asarray(sel, np.int32))
    code = lib.rm_xsec_from_r_static(R.data_ptr(), n, w.N, w.a, l.data_ptr(), thr.data_ptr(), poles.data_ptr(),
                                     E_dev.data_ptr(), ne, sel_h.ctypes.data, ns, out["K"].data_ptr(),
                                     out["eta"].data_ptr(), out["st"].data_ptr(), out["ss"].data_ptr(),
                                     out["fl"].data_ptr(), out["no"].data_ptr(), None)
    assert code == 0, lib.rm_static_last_error()
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def check_against(g, K0, ref, tol=1e-9):
    ne = K0.shape[0]
    for e in range(ne):
        scale = max(np.abs(K0[e]).max(), 1e-300)
        assert np.abs(g["K"][e] - K0[e]).max() <= tol * scale, e
    for q in range(ref["sig_tot"].shape[1]):
        tot = np.maximum(ref["sig_tot"][:, q], 1e-300)
        err = np.abs(g["ss"][:, q, :] - ref["sig_sel"][:, q, :]).max(axis=1) / tot
        assert np.all(err <= tol), (q, err.max())
    assert np.allclose(g["st"], ref["sig_tot"], rtol=tol, atol=0)
    dd = g["eta"] - ref["eigsum"]
    assert np.all(np.abs(np.mod(dd + np.pi, 2 * np.pi) - np.pi) <= 10 * tol)


def check_oracle(g, w, E, sel, idx):
    ref = orc.sweep(w, E, sel=tuple(sel), energy_idx=idx, keep_R=False)
    for t, e in enumerate(idx):
        assert g["no"][e] == ref["n_open"][t]
        if ref["flags"][t] & (orc.FLAG_ILLCOND | orc.FLAG_SINGULAR | orc.FLAG_NO_OPEN):
            continue
        no = ref["n_open"][t]
        Ko = ref["K"][t, :no, :no]
        assert np.abs(g["K"][e, :no, :no] - Ko).max() <= 1e-9 * np.abs(Ko).max(), e
        for q in range(len(sel)):
            st = ref["sig_tot"][t, q]
            if st > 0:
                assert np.abs(g["ss"][e, q] - ref["sig_sel"][t, q]).max() <= 1e-9 * st, (e, q)
        assert abs(orc.wrap_angle(g["eta"][e] - ref["eta"][t])) <= 1e-8, e


def test_static_entry_matches_plan_and_oracle(lib):
    # 600 energies: with the 256-energy chunk of this size, three chunks, the last one ragged
    dev = torch.device("cuda:0")
    wl = synth.small(21, 13, 400, 600, e_lo=0.02, e_hi=3.0, pole_lo=-2.0, pole_hi=9.0, a=16.0)
    w = wl.waves[0]
    sel = [0, 2, 5]
    code, chunk, slots = layout(lib, w.n, len(sel))
    assert code == 0 and chunk == 256 and slots >= 1
    assert wl.n_e > 2 * chunk and wl.n_e % chunk != 0
    R, K0, ref = plan_reference(wl, sel, dev)
    E = torch.from_numpy(wl.energies).to(dev)
    for call in range(2):
        g = static_call(lib, R, w, E, sel, dev)
        check_against(g, K0, ref)
        assert not np.any(g["fl"] & 16)
    check_oracle(g, w, wl.energies, sel, np.arange(0, wl.n_e, 37))


def test_static_entry_largest_size_smaller_chunk(lib):
    # n_ch = 640, the largest channel count: one solve workspace is about 13 MB, so the 64 MiB
    # scratch holds five, and the asymptotic data of a 256-energy chunk would cost one of them;
    # the chunk shrinks (three chunks here, the last one ragged)
    dev = torch.device("cuda:0")
    wl = synth.small(22, 640, 1500, 150, e_lo=0.02, e_hi=3.0, pole_lo=-3.0, pole_hi=20.0, a=25.0)
    w = wl.waves[0]
    sel = [0, 7]
    code, chunk, slots = layout(lib, w.n, len(sel))
    assert code == 0 and chunk < 256 and 1 <= slots < 152
    assert wl.n_e > 2 * chunk and wl.n_e % chunk != 0
    R, K0, ref = plan_reference(wl, sel, dev)
    E = torch.from_numpy(wl.energies).to(dev)
    for call in range(2):
        g = static_call(lib, R, w, E, sel, dev)
        check_against(g, K0, ref)
    check_oracle(g, w, wl.energies, sel, np.arange(0, wl.n_e, 37))


def test_static_entry_flags_out_of_range_l(lib):
    # an angular momentum outside [0, RM_LMAX] is clamped for the asymptotic functions and flags
    # every energy RM_FLAG_ASYM; the call still completes with finite outputs
    dev = torch.device("cuda:0")
    wl = synth.small(23, 6, 200, 40)
    w = wl.waves[0]
    R, _, _ = plan_reference(wl, [0], dev)
    lb = w.l.copy()
    lb[2] = 1 << 30
    E = torch.from_numpy(wl.energies).to(dev)
    g = static_call(lib, R, w, E, [0], dev, l_dev=torch.from_numpy(lb).to(dev))
    assert np.all(g["fl"] & 16)
    g2 = static_call(lib, R, w, E, [0], dev)  # the flag word is per call
    assert not np.any(g2["fl"] & 16)


def test_static_entry_rejects_oversize(lib):
    # above the largest channel count: rejected with a message that says so, before any device
    # work; the layout query agrees
    dev = torch.device("cuda:0")
    z = torch.zeros(8, dtype=torch.float64, device=dev)
    zi = torch.zeros(8, dtype=torch.int32, device=dev)
    code = lib.rm_xsec_from_r_static(z.data_ptr(), 641, 10, 1.0, zi.data_ptr(), z.data_ptr(), z.data_ptr(),
                                     z.data_ptr(), 1, None, 1, None, None, None, None, None, None, None)
    assert code == 1
    assert b"640" in lib.rm_static_last_error()
    assert layout(lib, 641, 1)[0] == 1 and layout(lib, 640, 1)[0] == 0


def test_static_entry_survives_nan_r(lib):
    # the entry point does not validate the caller's R-matrices: an energy whose R is NaN must
    # come out as NaN (flagged ILLCOND by its LU), never as an index outside the workspace, and
    # the other energies of the call must be unaffected
    dev = torch.device("cuda:0")
    wl = synth.small(24, 11, 300, 60)
    w = wl.waves[0]
    sel = [0, 1]
    R, K0, ref = plan_reference(wl, sel, dev)
    bad = [3, 17, 41]
    Rn = R.clone()
    Rn[bad] = float("nan")
    E = torch.from_numpy(wl.energies).to(dev)
    g = static_call(lib, Rn, w, E, sel, dev)
    good = np.array([e for e in range(wl.n_e) if e not in bad])
    for e in bad:
        no = g["no"][e]
        if no > 0:
            assert np.isnan(g["eta"][e])
            for q, ch in enumerate(sel):  # a selected channel closed at e has no cross section
                assert np.isnan(g["st"][e, q]) if ch < no else g["st"][e, q] == 0.0
    keep = {"eigsum": ref["eigsum"][good], "sig_tot": ref["sig_tot"][good], "sig_sel": ref["sig_sel"][good]}
    check_against({k: v[good] for k, v in g.items()}, K0[good], keep)
    g2 = static_call(lib, R, w, E, sel, dev)  # and the next call is clean
    check_against(g2, K0, ref)
