"""ctypes binding of the C ABI in ``include/rm.h`` (argument marshalling only).

Every step of the path runs in the CUDA library ``librm.so``; this module
only converts NumPy arrays / torch tensors to pointers.  Loading fails loudly
when the library is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# RM_LIBRARY=checked selects the bounds-checked build (librm_checked.so)
LIB_PATH = os.path.join(_HERE, "librm_checked.so" if os.environ.get("RM_LIBRARY") == "checked" else "librm.so")

RM_OK, RM_ERR_ARG, RM_ERR_ORDER, RM_ERR_NOMEM, RM_ERR_CUDA, RM_ERR_TIMEOUT, RM_ERR_STATE = range(7)
RM_MEM_HOST, RM_MEM_DEVICE = 0, 1
RM_PREC_FP64, RM_PREC_SPLIT_BF16, RM_PREC_SPLIT_FP16, RM_PREC_FP32_SIMT = 0, 1, 2, 3
FLAG_NUDGED, FLAG_ILLCOND, FLAG_NO_OPEN, FLAG_SINGULAR, FLAG_ASYM, FLAG_FP64, FLAG_LU = 1, 2, 4, 8, 16, 32, 64
FLAG_NEAR_THRESHOLD = 128
SOLVE = {"fp64": 0, "mixed": 1, "fp64_lu": 2}

PREC = {"fp64": RM_PREC_FP64, "split_bf16": RM_PREC_SPLIT_BF16, "split_fp16": RM_PREC_SPLIT_FP16,
        "fp32_simt": RM_PREC_FP32_SIMT}

EXPORTS = ["rm_options_default", "rm_plan_create", "rm_plan_load", "rm_rmatrix", "rm_kmatrix",
           "rm_xsec", "rm_run", "rm_results", "rm_sync", "rm_plan_info", "rm_plan_launches",
           "rm_plan_destroy", "rm_status_str", "rm_last_error", "rm_profile_enable", "rm_profile_read",
           "rm_plan_cluster", "rm_plan_mma_pair", "rm_photo", "rm_results_photo", "rm_convolve", "rm_plan_slices",
           "rm_xsec_from_r_static", "rm_static_last_error", "rm_static_layout", "rm_checked_report"]

KERNELS = {"polesum_fp64": 0, "polesum_split": 1, "near": 2, "asym": 3, "solve": 4, "dslice": 5}


class rm_wave(C.Structure):
    _fields_ = [("n_ch", C.c_int32), ("n_poles", C.c_int32), ("a", C.c_double),
                ("l", C.c_void_p), ("thresh", C.c_void_p), ("pole_E", C.c_void_p), ("W", C.c_void_p),
                ("z", C.c_double), ("dip", C.c_void_p), ("e0", C.c_double)]


class rm_options(C.Structure):
    _fields_ = [("prec", C.c_int32), ("delta", C.c_double), ("slices", C.c_int32),
                ("sel_init", C.c_void_p), ("n_sel", C.c_int32), ("mem", C.c_int32),
                ("chunk", C.c_int32), ("autotune", C.c_int32), ("tune_cache", C.c_char_p),
                ("cluster_x", C.c_int32), ("cluster_y", C.c_int32), ("solve_prec", C.c_int32),
                ("mma_pair", C.c_int32)]


class RMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"rm status {code}: {msg}")
        self.code = code


_lib = None


def load_library(path: str = LIB_PATH):
    """Load librm.so (raises OSError if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError(f"{path} not found: build it with paper_1403_5524_gb300.build.build()")
    lib = C.CDLL(path)
    P = C.c_void_p
    i32, i64, dbl = C.c_int32, C.c_int64, C.c_double
    lib.rm_options_default.argtypes = [C.POINTER(rm_options)]
    lib.rm_options_default.restype = None
    lib.rm_plan_create.argtypes = [C.POINTER(P), C.POINTER(rm_wave), i32, P, i64, C.POINTER(rm_options), P]
    lib.rm_plan_load.argtypes = [P, C.POINTER(rm_wave), P, i32]
    lib.rm_rmatrix.argtypes = [P, i32, i64, i64, P, i32]
    lib.rm_kmatrix.argtypes = [P, i32, i64, i64, P, P, P, i32]
    lib.rm_xsec.argtypes = [P, i32, i64, i64, P, P, P, i32]
    lib.rm_run.argtypes = [P]
    lib.rm_results.argtypes = [P, i32, i64, i64, P, P, P, P, P, i32]
    lib.rm_sync.argtypes = [P]
    lib.rm_plan_info.argtypes = [P, i32, C.POINTER(i32), C.POINTER(i32), C.POINTER(i64), C.POINTER(i32),
                                 C.POINTER(i32), C.POINTER(i64)]
    lib.rm_plan_cluster.argtypes = [P, C.POINTER(i32), C.POINTER(i32)]
    lib.rm_plan_mma_pair.argtypes = [P, C.POINTER(i32)]
    lib.rm_photo.argtypes = [P, i32, i64, i64, P, P, i32]
    lib.rm_results_photo.argtypes = [P, i32, i64, i64, P, P, i32]
    lib.rm_convolve.argtypes = [P, i64, P, i32, P, dbl, P, i32, P]
    lib.rm_plan_slices.argtypes = [P, C.POINTER(i32)]
    lib.rm_xsec_from_r_static.argtypes = [P, i32, i32, dbl, P, P, P, P, i64, P, i32, P, P, P, P, P, P, P]
    lib.rm_static_last_error.argtypes = []
    lib.rm_static_last_error.restype = C.c_char_p
    lib.rm_static_layout.argtypes = [i32, i32, C.POINTER(i32), C.POINTER(i32)]
    lib.rm_checked_report.argtypes = [C.POINTER(i32), C.POINTER(i32)]
    lib.rm_plan_launches.argtypes = [P]
    lib.rm_plan_launches.restype = i64
    lib.rm_plan_destroy.argtypes = [P]
    lib.rm_profile_enable.argtypes = [P, i32]
    lib.rm_profile_read.argtypes = [P, i32, C.POINTER(dbl), C.POINTER(i64)]
    lib.rm_status_str.argtypes = [i32]
    lib.rm_status_str.restype = C.c_char_p
    lib.rm_last_error.argtypes = []
    lib.rm_last_error.restype = C.c_char_p
    for name in ["rm_plan_create", "rm_plan_load", "rm_rmatrix", "rm_kmatrix", "rm_xsec", "rm_run",
                 "rm_results", "rm_sync", "rm_plan_info", "rm_plan_destroy", "rm_profile_enable",
                 "rm_profile_read", "rm_plan_cluster", "rm_plan_mma_pair", "rm_photo", "rm_results_photo",
                 "rm_convolve",
                 "rm_plan_slices", "rm_xsec_from_r_static", "rm_static_layout", "rm_checked_report"]:
        getattr(lib, name).restype = C.c_int32
    _lib = lib
    return lib


def _check(code):
    if code != RM_OK:
        lib = load_library()
        raise RMError(code, lib.rm_last_error().decode())


def _ptr(x):
    """Pointer of a C-contiguous NumPy array or torch tensor (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"]
        return x.ctypes.data
    assert x.is_contiguous()
    return x.data_ptr()


def _is_dev(x):
    return x is not None and not isinstance(x, np.ndarray) and x.is_cuda


def convolve(energies, sigma, fwhm: float, weights: Optional[Sequence[float]] = None, out=None, stream=None):
    """Gaussian convolution (full width fwhm) and statistical average of cross-section series.

    ``sigma`` is (n_series, n_e) or (n_e,); NumPy (host) or CUDA torch tensors (device) like
    ``energies``; ``weights`` the statistical weights (default: equal).  Returns ``out``.
    """
    lib = load_library()
    dev = _is_dev(energies)
    n_e = int(energies.shape[0])
    n_series = 1 if len(sigma.shape) == 1 else int(sigma.shape[0])
    if out is None:
        if dev:
            import torch
            out = torch.empty(n_e, dtype=torch.float64, device=energies.device)
        else:
            out = np.zeros(n_e)
    w = None if weights is None else np.ascontiguousarray(np.asarray(weights, dtype=np.float64))
    stream_ptr = None if stream is None else int(stream.cuda_stream)
    _check(lib.rm_convolve(_ptr(energies), n_e, _ptr(sigma), n_series, None if w is None else w.ctypes.data,
                           float(fwhm), _ptr(out), RM_MEM_DEVICE if dev else RM_MEM_HOST, stream_ptr))
    return out


class Plan:
    """Owner of an ``rm_plan_t``.

    ``waves`` are :class:`synth.Wave`-like objects (l, thresh, poles, W, a) whose
    arrays are NumPy (host) or CUDA torch tensors (device); ``energies`` likewise.
    """

    def __init__(self, waves: Sequence, energies, prec: str = "fp64", delta: float = 0.05,
                 sel: Sequence[int] = (0,), chunk: int = 0, slices: int = 0, stream=None,
                 autotune: bool = False, tune_cache: Optional[str] = None,
                 cluster: Optional[Sequence[int]] = None, solve: str = "fp64", mma_pair: int = 0):
        self.lib = load_library()
        self._keep = []
        self.mem = RM_MEM_DEVICE if _is_dev(energies) else RM_MEM_HOST
        warr = self._waves(waves)
        self._sel = np.ascontiguousarray(np.asarray(sel, dtype=np.int32))
        opt = rm_options()
        self.lib.rm_options_default(C.byref(opt))
        opt.prec = PREC[prec]
        opt.delta = float(delta)
        opt.slices = int(slices)
        opt.sel_init = self._sel.ctypes.data
        opt.n_sel = int(self._sel.size)
        opt.mem = self.mem
        opt.chunk = int(chunk)
        opt.autotune = 1 if autotune else 0
        self._tune_cache = tune_cache.encode() if tune_cache else None
        opt.tune_cache = self._tune_cache
        if cluster is not None:
            opt.cluster_x, opt.cluster_y = int(cluster[0]), int(cluster[1])
        opt.solve_prec = SOLVE[solve]
        opt.mma_pair = int(mma_pair)
        h = C.c_void_p()
        self.n_e = int(energies.shape[0])
        self.n_waves = len(waves)
        self.n_ch = [int(w.l.shape[0]) for w in waves]
        self.n_sel = int(self._sel.size)
        stream_ptr = None if stream is None else int(stream.cuda_stream)
        _check(self.lib.rm_plan_create(C.byref(h), warr, len(waves), _ptr(energies), self.n_e,
                                       C.byref(opt), stream_ptr))
        self.h = h
        self._keep = []

    def _waves(self, waves):
        warr = (rm_wave * len(waves))()
        for g, w in enumerate(waves):
            arrs = []
            for name, dt in (("l", "int32"), ("thresh", "float64"), ("poles", "float64"), ("W", "float64")):
                a = getattr(w, name)
                if isinstance(a, np.ndarray):
                    a = np.ascontiguousarray(a, dtype=dt)
                arrs.append(a)
            self._keep.extend(arrs)
            warr[g].n_ch = int(arrs[0].shape[0])
            warr[g].n_poles = int(arrs[2].shape[0])
            warr[g].a = float(w.a)
            warr[g].z = float(getattr(w, "z", 0.0))
            warr[g].l, warr[g].thresh, warr[g].pole_E, warr[g].W = (_ptr(a) for a in arrs)
            dip = getattr(w, "dip", None)
            if dip is not None:
                if isinstance(dip, np.ndarray):
                    dip = np.ascontiguousarray(dip, dtype="float64")
                self._keep.append(dip)
                warr[g].dip = _ptr(dip)
                warr[g].e0 = float(getattr(w, "e0", 0.0))
        return warr

    def load(self, waves, energies):
        warr = self._waves(waves)
        mem = RM_MEM_DEVICE if _is_dev(energies) else RM_MEM_HOST
        _check(self.lib.rm_plan_load(self.h, warr, _ptr(energies), mem))
        self._keep = []

    def info(self, wave=0):
        n, N, ne, ns, ch = C.c_int32(), C.c_int32(), C.c_int64(), C.c_int32(), C.c_int32()
        ws = C.c_int64()
        _check(self.lib.rm_plan_info(self.h, wave, C.byref(n), C.byref(N), C.byref(ne), C.byref(ns),
                                     C.byref(ch), C.byref(ws)))
        return {"n_ch": n.value, "n_poles": N.value, "n_e": ne.value, "n_sel": ns.value,
                "chunk": ch.value, "workspace_bytes": ws.value}

    def cluster(self):
        """(cluster_x, cluster_y) of rm_run's tensor-core pole-sum launch."""
        cx, cy = C.c_int32(), C.c_int32()
        _check(self.lib.rm_plan_cluster(self.h, C.byref(cx), C.byref(cy)))
        return int(cx.value), int(cy.value)

    def mma_pair(self) -> bool:
        """True when rm_run's tensor-core pole sum runs as 2-SM (cta_group::2) MMAs."""
        v = C.c_int32()
        _check(self.lib.rm_plan_mma_pair(self.h, C.byref(v)))
        return bool(v.value)

    def slices(self) -> int:
        """Slice products per far term of the tensor-core pole sum (0 without one)."""
        v = C.c_int32()
        _check(self.lib.rm_plan_slices(self.h, C.byref(v)))
        return int(v.value)

    def launches(self) -> int:
        return int(self.lib.rm_plan_launches(self.h))

    def profile(self, on: bool = True):
        _check(self.lib.rm_profile_enable(self.h, 1 if on else 0))

    def profile_read(self):
        """{kernel name: (total ms, launches)} since the last read."""
        out = {}
        for name, k in KERNELS.items():
            ms, n = C.c_double(), C.c_int64()
            _check(self.lib.rm_profile_read(self.h, k, C.byref(ms), C.byref(n)))
            out[name] = (ms.value, n.value)
        return out

    @staticmethod
    def _mem(*outs):
        devs = {_is_dev(o) for o in outs if o is not None}
        assert len(devs) <= 1, "outputs must all be host or all be device"
        return RM_MEM_DEVICE if devs == {True} else RM_MEM_HOST

    def rmatrix(self, wave, e0, e1, out):
        _check(self.lib.rm_rmatrix(self.h, wave, e0, e1, _ptr(out), self._mem(out)))
        return out

    def kmatrix(self, wave, e0, e1, K=None, n_open=None, flags=None):
        _check(self.lib.rm_kmatrix(self.h, wave, e0, e1, _ptr(K), _ptr(n_open), _ptr(flags),
                                   self._mem(K, n_open, flags)))

    def xsec(self, wave, e0, e1, eigsum=None, sig_tot=None, sig_sel=None):
        _check(self.lib.rm_xsec(self.h, wave, e0, e1, _ptr(eigsum), _ptr(sig_tot), _ptr(sig_sel),
                                self._mem(eigsum, sig_tot, sig_sel)))

    def run(self):
        _check(self.lib.rm_run(self.h))

    def results(self, wave, e0, e1, eigsum=None, sig_tot=None, sig_sel=None, n_open=None, flags=None):
        _check(self.lib.rm_results(self.h, wave, e0, e1, _ptr(eigsum), _ptr(sig_tot), _ptr(sig_sel),
                                   _ptr(n_open), _ptr(flags), self._mem(eigsum, sig_tot, sig_sel, n_open, flags)))

    def photo(self, wave, e0, e1, sig_pi=None, sig_pi_ch=None):
        """Photoionisation cross sections of a wave with a dipole vector, energies [e0, e1)."""
        _check(self.lib.rm_photo(self.h, wave, e0, e1, _ptr(sig_pi), _ptr(sig_pi_ch), self._mem(sig_pi, sig_pi_ch)))

    def results_photo(self, wave, e0, e1, sig_pi=None, sig_pi_ch=None):
        """Photoionisation results of the last run()."""
        _check(self.lib.rm_results_photo(self.h, wave, e0, e1, _ptr(sig_pi), _ptr(sig_pi_ch),
                                         self._mem(sig_pi, sig_pi_ch)))

    def sync(self):
        _check(self.lib.rm_sync(self.h))

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.rm_plan_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def host_outputs(n_e, n_ch, n_sel):
    """Host output arrays for a full-range xsec / results call."""
    return {"eigsum": np.zeros(n_e), "sig_tot": np.zeros((n_e, n_sel)),
            "sig_sel": np.zeros((n_e, n_sel, n_ch)), "n_open": np.zeros(n_e, np.int32),
            "flags": np.zeros(n_e, np.uint8)}
