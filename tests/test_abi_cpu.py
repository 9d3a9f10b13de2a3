"""Host-only checks of the C ABI: the library loads, exports every function
include/rm.h declares, and rejects bad arguments without touching a GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_1403_5524_gb300 import rm, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "rm.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(rm_[a-z_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    return rm.load_library()


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n
    assert set(rm.EXPORTS) <= set(names)


def test_status_strings(lib):
    for code in range(7):
        assert lib.rm_status_str(code)
    assert lib.rm_status_str(99) == b"unknown status"


def test_options_default(lib):
    o = rm.rm_options()
    lib.rm_options_default(C.byref(o))
    assert o.prec == rm.RM_PREC_FP64 and abs(o.delta - 0.05) < 1e-15 and o.mem == rm.RM_MEM_HOST
    assert o.chunk == 0 and o.n_sel == 0
    assert o.mma_pair == 0  # the 2-SM pole sum where it applies


def _create(lib, waves, energies, opt=None, n_waves=None):
    h = C.c_void_p()
    warr = (rm.rm_wave * max(1, len(waves)))()
    keep = []
    for g, w in enumerate(waves):
        keep += [w.l, w.thresh, w.poles, w.W]
        warr[g].n_ch, warr[g].n_poles, warr[g].a = w.l.shape[0], w.poles.shape[0], w.a
        warr[g].l, warr[g].thresh = w.l.ctypes.data, w.thresh.ctypes.data
        warr[g].pole_E, warr[g].W = w.poles.ctypes.data, w.W.ctypes.data
        warr[g].z = w.z
    code = lib.rm_plan_create(C.byref(h), warr, len(waves) if n_waves is None else n_waves,
                              energies.ctypes.data if energies is not None else None,
                              0 if energies is None else energies.shape[0],
                              C.byref(opt) if opt is not None else None, None)
    return code, h


def test_bad_arguments_rejected_before_device(lib):
    wl = synth.small(1, 4, 20, 5)
    w = wl.waves[0]
    assert lib.rm_plan_create(None, None, 0, None, 0, None, None) == rm.RM_ERR_ARG
    code, h = _create(lib, [w], wl.energies, n_waves=0)
    assert code == rm.RM_ERR_ARG and not h.value
    bad = synth.Wave(l=w.l, thresh=w.thresh, poles=w.poles, W=w.W, a=-1.0)
    assert _create(lib, [bad], wl.energies)[0] == rm.RM_ERR_ARG
    for z in (-1.0, float("nan"), float("inf")):  # repulsive or non-finite target charge
        badz = synth.Wave(l=w.l, thresh=w.thresh, poles=w.poles, W=w.W, a=w.a, z=z)
        assert _create(lib, [badz], wl.energies)[0] == rm.RM_ERR_ARG
    o = rm.rm_options()
    lib.rm_options_default(C.byref(o))
    o.prec = 7
    assert _create(lib, [w], wl.energies, o)[0] == rm.RM_ERR_ARG
    o.prec = rm.RM_PREC_FP64
    o.mem = 5
    assert _create(lib, [w], wl.energies, o)[0] == rm.RM_ERR_ARG
    o.mem = rm.RM_MEM_HOST
    sel = np.array([0, -1], np.int32)
    o.sel_init, o.n_sel = sel.ctypes.data, 2
    assert _create(lib, [w], wl.energies, o)[0] == rm.RM_ERR_ARG
    big = synth.Wave(l=np.zeros(700, np.int32), thresh=np.zeros(700), poles=w.poles,
                     W=np.zeros((700, w.N)), a=1.0)
    assert _create(lib, [big], wl.energies)[0] == rm.RM_ERR_ARG
    assert lib.rm_last_error()


def test_slices_option_checked_on_host(lib):
    # the product set of the tensor-core pole sum: 0 (default), 3, 6, 10 or 13, split modes only
    wl = synth.small(1, 4, 20, 5)
    o = rm.rm_options()
    lib.rm_options_default(C.byref(o))
    o.prec = rm.RM_PREC_SPLIT_BF16
    for bad in (1, 2, 4, 5, 7, 12, 14, -1):
        o.slices = bad
        assert _create(lib, wl.waves, wl.energies, o)[0] == rm.RM_ERR_ARG, bad
        assert b"slices" in lib.rm_last_error()
    for prec in (rm.RM_PREC_FP64, rm.RM_PREC_FP32_SIMT):
        o.prec, o.slices = prec, 6
        assert _create(lib, wl.waves, wl.energies, o)[0] == rm.RM_ERR_ARG
    o.prec, o.slices = rm.RM_PREC_SPLIT_FP16, 15  # the fifth slice is below FP16's range
    assert _create(lib, wl.waves, wl.energies, o)[0] == rm.RM_ERR_ARG
    assert b"15" in lib.rm_last_error()
    v = C.c_int32(-7)
    assert lib.rm_plan_slices(None, C.byref(v)) == rm.RM_ERR_ARG


def test_mma_pair_option_checked_on_host(lib):
    # mma_pair: -1 (one-SM MMAs), 0 or 1 (2-SM MMAs where they apply); anything else is rejected
    # before the device is touched
    wl = synth.small(1, 4, 20, 5)
    o = rm.rm_options()
    lib.rm_options_default(C.byref(o))
    o.prec = rm.RM_PREC_SPLIT_BF16
    for bad in (-2, 2, 7):
        o.mma_pair = bad
        assert _create(lib, wl.waves, wl.energies, o)[0] == rm.RM_ERR_ARG, bad
        assert b"mma_pair" in lib.rm_last_error()
    v = C.c_int32(-7)
    assert lib.rm_plan_mma_pair(None, C.byref(v)) == rm.RM_ERR_ARG


def test_static_entry_arguments_checked_on_host(lib):
    # the allocation-free entry point rejects bad sizes and null pointers before any CUDA call
    buf = np.zeros(64)
    ib = np.zeros(8, np.int32)
    d, i = buf.ctypes.data, ib.ctypes.data

    def call(R=d, n=4, N=10, a=1.0, l=i, thr=d, poles=d, E=d, ne=3, sel=None, ns=1):
        return lib.rm_xsec_from_r_static(R, n, N, a, l, thr, poles, E, ne, sel, ns,
                                         None, None, None, None, None, None, None)
    assert call(n=0) == rm.RM_ERR_ARG
    assert call(N=0) == rm.RM_ERR_ARG
    assert call(a=0.0) == rm.RM_ERR_ARG and call(a=float("nan")) == rm.RM_ERR_ARG
    assert call(ne=-1) == rm.RM_ERR_ARG
    assert call(ne=0) == rm.RM_OK  # nothing to do
    for k in ("R", "l", "thr", "poles", "E"):
        assert call(**{k: None}) == rm.RM_ERR_ARG, k
        assert b"null" in lib.rm_static_last_error()
    sel = np.array([0, -2], np.int32)
    assert call(sel=sel.ctypes.data, ns=2) == rm.RM_ERR_ARG
    assert call(sel=sel.ctypes.data, ns=0) == rm.RM_ERR_ARG
    assert call(sel=sel.ctypes.data, ns=65) == rm.RM_ERR_ARG
    c, sl = C.c_int32(), C.c_int32()
    assert lib.rm_static_layout(0, 1, C.byref(c), C.byref(sl)) == rm.RM_ERR_ARG
    assert lib.rm_static_layout(4, 0, C.byref(c), C.byref(sl)) == rm.RM_ERR_ARG


def test_checked_build_exports_and_normal_build_reports_state(lib):
    # the normal library has no bounds checks to report; the checked build (built beside it by
    # paper_1403_5524_gb300.build) loads and exports every declared function too
    u, l = C.c_int32(7), C.c_int32(7)
    assert lib.rm_checked_report(C.byref(u), C.byref(l)) == rm.RM_ERR_STATE
    assert u.value == -1 and l.value == 0
    path = os.path.join(ROOT, "paper_1403_5524_gb300", "librm_checked.so")
    if not os.path.exists(path):
        pytest.skip("checked library not built")
    chk = C.CDLL(path)
    for n in declared_functions():
        assert hasattr(chk, n), n


def test_no_gpu_is_an_error_not_a_crash(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    wl = synth.small(1, 4, 20, 5)
    code, h = _create(lib, wl.waves, wl.energies)
    assert code == rm.RM_ERR_CUDA and not h.value
    with pytest.raises(rm.RMError):
        rm.Plan(wl.waves, wl.energies)


def test_null_plan_calls(lib):
    assert lib.rm_run(None) == rm.RM_ERR_ARG
    assert lib.rm_sync(None) == rm.RM_ERR_ARG
    assert lib.rm_plan_destroy(None) == rm.RM_OK
    assert lib.rm_plan_launches(None) == -1


def test_convolve_arguments_checked_on_host(lib):
    E = np.linspace(0.0, 1.0, 11)
    sig = np.ones((2, 11))
    out = np.zeros(11)
    call = lambda E_, ns, fw, w=None: lib.rm_convolve(E_.ctypes.data, E_.shape[0], sig.ctypes.data, ns,
                                                      None if w is None else w.ctypes.data, fw, out.ctypes.data,
                                                      rm.RM_MEM_HOST, None)
    assert call(E, 0, 0.1) == rm.RM_ERR_ARG
    assert call(E, 17, 0.1) == rm.RM_ERR_ARG
    assert call(E, 2, -1.0) == rm.RM_ERR_ARG
    assert call(E, 2, float("nan")) == rm.RM_ERR_ARG
    assert call(E, 2, 0.1, np.array([0.5, float("inf")])) == rm.RM_ERR_ARG
    assert call(E[::-1].copy(), 2, 0.1) == rm.RM_ERR_ORDER


def test_binding_constants_match_the_header():
    # flag bits, kernel ids and solve-precision values of the binding are the header's
    txt = open(os.path.join(os.path.dirname(__file__), "..", "include", "rm.h")).read()
    defs = {m.group(1): int(m.group(2)) for m in re.finditer(r"#define (RM_\w+) (\d+)u?\b", txt)}
    flags = {"NUDGED": rm.FLAG_NUDGED, "ILLCOND": rm.FLAG_ILLCOND, "NO_OPEN": rm.FLAG_NO_OPEN,
             "SINGULAR": rm.FLAG_SINGULAR, "ASYM": rm.FLAG_ASYM, "FP64": rm.FLAG_FP64, "LU": rm.FLAG_LU,
             "NEAR_THRESHOLD": rm.FLAG_NEAR_THRESHOLD}
    for k, v in flags.items():
        assert defs["RM_FLAG_" + k] == v, k
    kern = {"polesum_fp64": "POLESUM_FP64", "polesum_split": "POLESUM_SPLIT", "near": "NEAR", "asym": "ASYM",
            "solve": "SOLVE", "dslice": "DSLICE"}
    for k, v in rm.KERNELS.items():
        assert defs["RM_KERNEL_" + kern[k]] == v, k
    assert defs["RM_KERNEL_COUNT"] == len(rm.KERNELS)
    assert defs["RM_DEFAULT_SLICES"] in (3, 6, 10, 13, 15)
    enum = re.search(r"typedef enum \{([^}]*)\} rm_solve_precision_t;", txt).group(1)
    vals = {m.group(1): int(m.group(2)) for m in re.finditer(r"RM_SOLVE_(\w+) = (\d+)", enum)}
    assert vals == {"FP64": rm.SOLVE["fp64"], "MIXED": rm.SOLVE["mixed"], "FP64_LU": rm.SOLVE["fp64_lu"]}
