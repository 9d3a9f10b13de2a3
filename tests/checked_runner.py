"""Ragged-size sweeps through the bounds-checked library (librm_checked.so).

Run as a child process with RM_LIBRARY=checked by tests/test_gpu_checked.py (the
binding loads one library per process).  Every case runs the per-range calls and
rm_run in the FP64 and split-BF16 forms, compares the cross sections with the
oracle, and then asks the library whether any kernel guard failed
(rm_checked_report).  Exits non-zero on the first problem.
"""
import ctypes as C
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle import rmatrix as orc  # noqa: E402
from paper_1403_5524_gb300 import rm, synth  # noqa: E402


def report(lib, what):
    unit, line = C.c_int32(), C.c_int32()
    code = lib.rm_checked_report(C.byref(unit), C.byref(line))
    if code != 0:
        raise SystemExit(f"{what}: rm_checked_report failed: {lib.rm_last_error().decode()}")
    if unit.value != -1:
        raise SystemExit(f"{what}: guard failed in unit {unit.value} at line {line.value}")


def sweep(lib, wl, prec, sel, chunk=0):
    w = wl.waves[0]
    n, ne = w.n, wl.n_e
    with rm.Plan(wl.waves, wl.energies, prec=prec, sel=sel, chunk=chunk, delta=0.05) as p:
        R = np.zeros((ne, n * (n + 1) // 2))
        p.rmatrix(0, 0, ne, R)
        K = np.zeros((ne, n, n))
        p.kmatrix(0, 0, ne, K=K)
        x = rm.host_outputs(ne, n, len(sel))
        p.xsec(0, 0, ne, eigsum=x["eigsum"], sig_tot=x["sig_tot"], sig_sel=x["sig_sel"])
        p.run()
        r = rm.host_outputs(ne, n, len(sel))
        p.results(0, 0, ne, **r)
    report(lib, f"{prec} n={n} N={w.N} n_e={ne}")
    idx = np.unique(np.linspace(0, ne - 1, min(ne, 12)).astype(int))
    ref = orc.sweep(w, wl.energies, sel=sel, energy_idx=idx, keep_R=False)
    tol = 1e-9 if prec == "fp64" else 1e-8
    for t, e in enumerate(idx):
        if ref["flags"][t] & (orc.FLAG_ILLCOND | orc.FLAG_NO_OPEN | orc.FLAG_SINGULAR):
            continue
        for q in range(len(sel)):
            st = ref["sig_tot"][t, q]
            if st > 0:
                for sg in (x["sig_sel"][e, q], r["sig_sel"][e, q]):
                    err = np.abs(sg - ref["sig_sel"][t, q]).max() / st
                    if not err <= tol:
                        raise SystemExit(f"{prec} n={n}: sigma error {err} at energy {e}")


def main():
    assert rm.LIB_PATH.endswith("librm_checked.so"), rm.LIB_PATH
    lib = rm.load_library()
    cases = [(1, 33, 1), (2, 65, 7), (3, 100, 33), (127, 1007, 9), (129, 1031, 130), (16, 64, 1)]
    for k, (n, N, ne) in enumerate(cases):
        wl = synth.small(500 + k, n, N, ne, e_lo=0.05, e_hi=3.2, pole_lo=-3.0, pole_hi=12.0, a=20.0)
        sel = tuple(range(min(n, 2)))
        for prec in ("fp64", "split_bf16"):
            sweep(lib, wl, prec, sel, chunk=5 if ne > 10 else 0)
        print(f"ok n={n} N={N} n_e={ne}", flush=True)
    # several uneven waves in one grouped launch
    waves = [synth.small(600 + g, n, N, 1, pole_lo=-3.0, pole_hi=10.0, a=18.0).waves[0]
             for g, (n, N) in enumerate([(5, 201), (23, 901), (9, 359), (129, 1601)])]
    E = np.linspace(0.03, 3.2, 140)
    for prec in ("fp64", "split_bf16"):
        with rm.Plan(waves, E, prec=prec, sel=(0, 1), chunk=64) as p:
            p.run()
            for g, w in enumerate(waves):
                o = rm.host_outputs(E.size, w.n, 2)
                p.results(g, 0, E.size, **o)
        report(lib, f"{prec} grouped")
    print("ok grouped", flush=True)
    # the allocation-free entry point, several chunks
    import torch
    dev = torch.device("cuda:0")
    wl = synth.small(700, 13, 300, 300, e_lo=0.02, e_hi=3.0, pole_lo=-2.0, pole_hi=9.0, a=16.0)
    w = wl.waves[0]
    with rm.Plan(wl.waves, wl.energies, prec="fp64", sel=(0,)) as p:
        Rd = torch.zeros((wl.n_e, w.n * (w.n + 1) // 2), dtype=torch.float64, device=dev)
        p.rmatrix(0, 0, wl.n_e, Rd)
        p.sync()
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    l, thr, poles, Ed = d(w.l), d(w.thresh), d(w.poles), d(wl.energies)
    eta = torch.zeros(wl.n_e, dtype=torch.float64, device=dev)
    code = lib.rm_xsec_from_r_static(Rd.data_ptr(), w.n, w.N, w.a, l.data_ptr(), thr.data_ptr(), poles.data_ptr(),
                                     Ed.data_ptr(), wl.n_e, None, 1, None, eta.data_ptr(), None, None, None, None,
                                     None)
    if code != 0:
        raise SystemExit("static entry failed: " + lib.rm_static_last_error().decode())
    report(lib, "static entry")
    print("ok static entry", flush=True)
    print("CHECKED OK")


if __name__ == "__main__":
    main()
