"""The comparison forms of the pole sum (needs a GPU): split slices held in
FP16, and plain FP32 on the CUDA cores; both keep the FP64 near window and
FP64 solves.

Tolerances: split-FP16 has the split form's R and K targets (<= 1e-6
normwise); its last slice is rounded on FP16's absolute 2^-24 subnormal grid
rather than to 8 relative bits as in BF16, about twice the last-slice error,
so its sigma bound is 5e-8 of sigma_tot (BF16 form: 1e-8).  FP32-SIMT rounds every term to FP32 and sums
N of them in FP32: about (2 + sqrt(N)) 2^-24 of sum_k |P D| per element,
checked as |R - R*| <= 8 (2 + sqrt(N)) 2^-24 (1/2a) sum_k |w_ik w_jk / (E_k - E)|.
"""
import math

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


def run(rm, wl, prec, sel, idx):
    w = wl.waves[0]
    n = w.n
    R = np.zeros((1, n * (n + 1) // 2))
    K = np.zeros((1, n, n))
    out = {"R": [], "K": [], "sig": []}
    with rm.Plan(wl.waves, wl.energies, prec=prec, delta=wl.delta, sel=sel) as p:
        for e in idx:
            e = int(e)
            p.rmatrix(0, e, e + 1, R)
            p.kmatrix(0, e, e + 1, K=K)
            sig = np.zeros((1, len(sel), n))
            p.xsec(0, e, e + 1, sig_sel=sig)
            out["R"].append(R[0].copy()); out["K"].append(K[0].copy()); out["sig"].append(sig[0])
    return out


@pytest.mark.parametrize("seed,n,N,ne", [(61, 7, 400, 20), (62, 33, 2000, 12), (63, 130, 900, 6)])
def test_split_fp16(rm, seed, n, N, ne):
    wl = synth.small(seed, n, N, ne, e_lo=0.05, e_hi=3.5, pole_lo=-3.0, pole_hi=12.0, a=20.0)
    idx = np.arange(ne)
    g = run(rm, wl, "split_fp16", (0,), idx)
    ref = orc.sweep(wl.waves[0], wl.energies, sel=(0,))
    for t in idx:
        Ro = ref["R"][t]
        assert np.abs(g["R"][t] - Ro).max() / np.abs(Ro).max() <= 1e-6
        if ref["flags"][t] & orc.FLAG_ILLCOND:
            continue
        no = ref["n_open"][t]
        Ko = ref["K"][t, :no, :no]
        assert np.abs(g["K"][t][:no, :no] - Ko).max() / np.abs(Ko).max() <= 1e-6
        st = ref["sig_tot"][t, 0]
        assert np.abs(g["sig"][t][0] - ref["sig_sel"][t, 0]).max() / st <= 5e-8


@pytest.mark.parametrize("seed,n,N,ne", [(71, 7, 400, 20), (72, 33, 2000, 12)])
def test_fp32_simt(rm, seed, n, N, ne):
    wl = synth.small(seed, n, N, ne, e_lo=0.05, e_hi=3.5, pole_lo=-3.0, pole_hi=12.0, a=20.0)
    w = wl.waves[0]
    idx = np.arange(ne)
    g = run(rm, wl, "fp32_simt", (0,), idx)
    ref = orc.sweep(w, wl.energies, sel=(0,))
    c = 8.0 * (2.0 + math.sqrt(N)) * 2.0 ** -24
    for t in idx:
        E = ref["E"][t]
        bound = c * ((np.abs(w.W) * np.abs(1.0 / (w.poles - E))[None, :]) @ np.abs(w.W).T) / (2 * w.a)
        Rg = orc.unpack_upper(g["R"][t], n)
        Ro = orc.unpack_upper(ref["R"][t], n)
        assert np.all(np.abs(Rg - Ro) <= bound + 1e-300), (t, float(np.max(np.abs(Rg - Ro) / bound)))
