"""Failure paths, exercised without any GPU fault (needs a GPU).

* Out of memory: the host-side hook RM_FAULT_ALLOC=k makes the k-th device
  allocation of rm_plan_create fail as cudaMalloc would.  The call must return
  RM_ERR_NOMEM, leave the plan handle NULL and give back every byte it had
  allocated (the device's free memory is unchanged), for every k up to the
  allocation count of a successful creation.
* A device-side wait that runs out: RM_FAULT_WAIT_CYCLES shortens every
  mbarrier wait of an unclustered tensor-core launch to a few cycles, so the
  pipeline's first wait gives up.  The tile then lets its own TMA copies (and
  any MMAs it issued) finish, frees its TMEM and raises the device error word;
  the host must read RM_ERR_TIMEOUT, and a fresh plan on the same device must
  run and match the oracle (the context is still usable).  No wait is ever
  unbounded and nothing traps.
"""
import ctypes as C
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


def free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


@pytest.mark.parametrize("prec", ["fp64", "split_bf16"])
def test_allocation_failure_frees_everything(rm, prec):
    wl = synth.small(41, 9, 300, 40)
    with rm.Plan(wl.waves, wl.energies, prec=prec) as p:  # warm the context and the module
        p.run()
        p.sync()
    base = free_bytes()
    failures = 0
    try:
        for k in range(1, 200):
            os.environ["RM_FAULT_ALLOC"] = str(k)
            try:
                p = rm.Plan(wl.waves, wl.energies, prec=prec)
            except rm.RMError as exc:
                assert exc.code == rm.RM_ERR_NOMEM, (k, str(exc))
                assert "RM_FAULT_ALLOC" in str(exc)
                assert free_bytes() == base, k
                failures += 1
                continue
            p.close()  # k is past the last allocation: creation succeeded
            break
        else:
            pytest.fail("the hook never let a plan through")
    finally:
        os.environ.pop("RM_FAULT_ALLOC", None)
    assert failures >= 10
    assert free_bytes() == base
    # and without the hook plans work again
    with rm.Plan(wl.waves, wl.energies, prec=prec) as p:
        p.run()
        p.sync()


def test_plan_create_hook_leaves_handle_null(rm):
    lib = rm.load_library()
    wl = synth.small(42, 4, 50, 5)
    w = wl.waves[0]
    warr = (rm.rm_wave * 1)()
    warr[0].n_ch, warr[0].n_poles, warr[0].a = w.n, w.N, w.a
    warr[0].l, warr[0].thresh, warr[0].pole_E, warr[0].W = (x.ctypes.data for x in (w.l, w.thresh, w.poles, w.W))
    h = C.c_void_p(12345)
    os.environ["RM_FAULT_ALLOC"] = "3"
    try:
        code = lib.rm_plan_create(C.byref(h), warr, 1, wl.energies.ctypes.data, wl.n_e, None, None)
    finally:
        os.environ.pop("RM_FAULT_ALLOC", None)
    assert code == rm.RM_ERR_NOMEM and not h.value


def test_wait_timeout_is_reported_and_context_survives(rm):
    wl = synth.small(43, 20, 900, 200, e_lo=0.05, e_hi=3.0, pole_lo=-2.0, pole_hi=9.0, a=18.0)
    w = wl.waves[0]
    os.environ["RM_FAULT_WAIT_CYCLES"] = "1"
    try:
        p = rm.Plan(wl.waves, wl.energies, prec="split_bf16", cluster=(1, 1))
    finally:
        os.environ.pop("RM_FAULT_WAIT_CYCLES", None)
    try:
        p.run()
        with pytest.raises(rm.RMError) as ei:
            p.sync()
        assert ei.value.code == rm.RM_ERR_TIMEOUT
        # the per-range path (unclustered kernel) reports it as well
        R = np.zeros((1, w.n * (w.n + 1) // 2))
        with pytest.raises(rm.RMError) as ei:
            p.rmatrix(0, 0, 1, R)
        assert ei.value.code == rm.RM_ERR_TIMEOUT
    finally:
        p.close()
    # the device still works: a new plan without the hook matches the oracle
    sel = (0,)
    with rm.Plan(wl.waves, wl.energies, prec="split_bf16", cluster=(1, 1), sel=sel) as p2:
        p2.run()
        out = rm.host_outputs(wl.n_e, w.n, 1)
        p2.results(0, 0, wl.n_e, **out)
    idx = np.arange(0, wl.n_e, 17)
    ref = orc.sweep(w, wl.energies, sel=sel, energy_idx=idx, keep_R=False)
    for t, e in enumerate(idx):
        if ref["flags"][t] & (orc.FLAG_ILLCOND | orc.FLAG_NO_OPEN):
            continue
        st = ref["sig_tot"][t, 0]
        assert np.abs(out["sig_sel"][e, 0] - ref["sig_sel"][t, 0]).max() <= 1e-8 * st
