"""The allocation-free entry point rm_xsec_from_r_static (needs a GPU).

Callers that may not allocate device memory (inside another library's stream
capture, under a fixed host-application memory pool, in real-time loops) get
K, the eigenphase sum and cross sections from R-matrices they already hold,
with the library's static scratch only.  Its results must equal those of the
plan-based rm_kmatrix / rm_xsec on the same R, within the FP64 path's
tolerances, on two calls in a row (the second call reuses the scratch the
first one left behind).
"""
import ctypes as C

import numpy as np
import pytest

from paper_1403_5524_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1403_5524_gb300 import rm
    lib = rm.load_library()
    P = C.c_void_p
    lib.rm_xsec_from_r_static.argtypes = [P, C.c_int32, C.c_int32, C.c_double, P, P, P, P, C.c_int64, P,
                                          C.c_int32, P, P, P, P, P, P, P]
    lib.rm_xsec_from_r_static.restype = C.c_int32
    lib.rm_static_last_error.restype = C.c_char_p
    return lib


def test_static_entry_matches_plan(lib):
    from paper_1403_5524_gb300 import rm
    dev = torch.device("cuda:0")
    wl = synth.small(21, 13, 400, 150, e_lo=0.02, e_hi=3.0, pole_lo=-2.0, pole_hi=9.0, a=16.0)
    w = wl.waves[0]
    n, ne = w.n, wl.n_e
    np_ = n * (n + 1) // 2
    sel = np.array([0, 2, 5], np.int32)
    ns = sel.size
    with rm.Plan(wl.waves, wl.energies, prec="fp64", sel=tuple(sel)) as p:
        R = torch.zeros((ne, np_), dtype=torch.float64, device=dev)
        p.rmatrix(0, 0, ne, R)
        K0 = np.zeros((ne, n, n))
        p.kmatrix(0, 0, ne, K=K0)
        ref = rm.host_outputs(ne, n, ns)
        p.xsec(0, 0, ne, eigsum=ref["eigsum"], sig_tot=ref["sig_tot"], sig_sel=ref["sig_sel"])
        p.sync()
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    l, thr, poles, E = d(w.l), d(w.thresh), d(w.poles), d(wl.energies)
    for call in range(2):
        K = torch.full((ne, n, n), np.nan, dtype=torch.float64, device=dev)
        eta = torch.full((ne,), np.nan, dtype=torch.float64, device=dev)
        st = torch.full((ne, ns), np.nan, dtype=torch.float64, device=dev)
        ss = torch.full((ne, ns, n), np.nan, dtype=torch.float64, device=dev)
        fl = torch.zeros(ne, dtype=torch.uint8, device=dev)
        no = torch.zeros(ne, dtype=torch.int32, device=dev)
        code = lib.rm_xsec_from_r_static(R.data_ptr(), n, w.N, w.a, l.data_ptr(), thr.data_ptr(), poles.data_ptr(),
                                         E.data_ptr(), ne, sel.ctypes.data, ns, K.data_ptr(), eta.data_ptr(),
                                         st.data_ptr(), ss.data_ptr(), fl.data_ptr(), no.data_ptr(), None)
        assert code == 0, lib.rm_static_last_error()
        torch.cuda.synchronize()
        Kg = K.cpu().numpy()
        for e in range(ne):
            scale = max(np.abs(K0[e]).max(), 1e-300)
            assert np.abs(Kg[e] - K0[e]).max() <= 1e-9 * scale, (call, e)
        for q in range(ns):
            tot = np.maximum(ref["sig_tot"][:, q], 1e-300)
            err = np.abs(ss.cpu().numpy()[:, q, :] - ref["sig_sel"][:, q, :]).max(axis=1) / tot
            assert np.all(err <= 1e-9), (call, q, err.max())
        assert np.allclose(st.cpu().numpy(), ref["sig_tot"], rtol=1e-9, atol=0)
        dd = eta.cpu().numpy() - ref["eigsum"]
        assert np.all(np.abs(np.mod(dd + np.pi, 2 * np.pi) - np.pi) <= 1e-8), call


def test_static_entry_rejects_oversize(lib):
    # a channel count whose single solve workspace exceeds the static scratch
    dev = torch.device("cuda:0")
    z = torch.zeros(8, dtype=torch.float64, device=dev)
    zi = torch.zeros(8, dtype=torch.int32, device=dev)
    code = lib.rm_xsec_from_r_static(z.data_ptr(), 4000, 10, 1.0, zi.data_ptr(), z.data_ptr(), z.data_ptr(),
                                     z.data_ptr(), 1, None, 1, None, None, None, None, None, None, None)
    assert code == 1
    assert lib.rm_static_last_error()
