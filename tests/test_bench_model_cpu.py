"""The benchmark's flop model of the solve (host logic, no GPU): which work it counts on the FP64
pipe and which in double-float, per energy path, against counts written out by hand."""
import importlib.util
import os

import numpy as np

from paper_1403_5524_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def one_wave(n, N, n_e, dip=False):
    wl = synth.small(5, n, N, n_e, dipole=dip)
    return wl


def test_outgoing_wave_split_per_path():
    b = bench()
    n, r = 12, 2
    wl = one_wave(n, 60, 4)
    no = np.array([12, 5, 0, 7])                    # all open, some closed, none open, some closed
    fl = np.array([0, 32, 0, 64], dtype=np.uint8)   # plain, S'' redone in FP64, NO_OPEN-like, LU path
    pole, f64, df = b.algorithmic_flops(wl, [no], [fl], r, "fp64")
    assert pole == 2.0 * (n * (n + 1) / 2) * 60 * 4
    closed = lambda o: (n ** 3 - o ** 3) / 3.0
    lu = lambda o: (2.0 / 3.0) * n ** 3 + 2.0 * n * n * o + (4.0 / 3.0) * o ** 3 + 8.0 * o * o * r
    zdf = lambda o: (4.0 / 3.0) * o ** 3 + 16.0 * o * o * r
    # energy 0: closed elimination (none here) and the refinement residual in FP64; S'' and Z in
    # double-float.  Energy 1: S'' in FP64.  Energy 2: no open channel, nothing.  Energy 3: the LU
    # path in FP64 after the outgoing-wave attempt (closed elimination and S'' paid)
    want64 = (closed(12) + 4.0 * 144 * r) + (closed(5) + 5 ** 3 / 3.0 + 4.0 * 25 * r) + (closed(7) + lu(7))
    wantdf = (12 ** 3 / 3.0 + zdf(12)) + zdf(5) + 7 ** 3 / 3.0
    assert np.isclose(f64, want64, rtol=1e-12), (f64, want64)
    assert np.isclose(df, wantdf, rtol=1e-12), (df, wantdf)


def test_dipole_waves_factor_z_in_fp64():
    b = bench()
    n, r = 9, 1
    wl = one_wave(n, 40, 1, dip=True)
    assert wl.waves[0].dip is not None
    no = np.array([6])
    _, f64, df = b.algorithmic_flops(wl, [no], [np.zeros(1, np.uint8)], r, "fp64")
    assert np.isclose(f64, (n ** 3 - 6 ** 3) / 3.0 + (4.0 / 3.0) * 6 ** 3 + 8.0 * 36 * (r + 1))
    assert np.isclose(df, 6 ** 3 / 3.0)


def test_lu_forms_count_fp64_only():
    b = bench()
    n, r = 10, 1
    wl = one_wave(n, 30, 2)
    no = np.array([4, 10])
    for solve in ("fp64_lu", "mixed"):
        _, f64, df = b.algorithmic_flops(wl, [no], [np.zeros(2, np.uint8)], r, solve)
        want = sum((2.0 / 3.0) * n ** 3 + 2.0 * n * n * o + (4.0 / 3.0) * o ** 3 + 8.0 * o * o * r for o in no)
        assert np.isclose(f64, want) and df == 0.0
