"""Seeded synthetic inputs for the outer-region energy sweep.

This module only draws random numbers and lays them out; it holds none of the
method's arithmetic, so both the CUDA path and the CPU oracle may read it.

A *wave* (one partial wave, J-pi symmetry) is the tuple the method consumes:
channel angular momenta ``l`` (int32, n), channel thresholds ``thresh``
(float64, n, sorted, first = 0 Ry), pole energies ``poles`` (float64, N,
sorted, Ry), surface amplitudes ``W`` (float64, n x N row-major, w_ik) and the
R-matrix radius ``a`` (bohr).  Energies are a float64 mesh in Ry.

The pole energies E_k and amplitudes w_ik stand in for the inner-region
eigenvalues and boundary amplitudes of the paper's Eq. 1; the paper's own
atomic data (B II, Ca II, Fe III) are not available, so their sizes are
bracketed by the named workloads below (poles per channel 40-78, against
m/n ~ 62 in the paper's Table 3).

Draw order per wave (documented reading): thresholds, l, poles, W.
Thresholds: n draws of U[0, thr_hi], sorted, first set to 0.
l: c1 uses l_i = i; the others draw integers U{0..lmax}.
Poles: N draws of U[lo, hi], sorted.  W: N(0, 1/N) entries.
Energy meshes are inclusive linspace; nudging of energies that sit on a pole
or a threshold is part of the method, not of the input, and is done by each
implementation itself.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional, List

import numpy as np


@dataclass
class Wave:
    l: np.ndarray          # int32 (n,)
    thresh: np.ndarray     # float64 (n,), sorted, thresh[0] == 0
    poles: np.ndarray      # float64 (N,), sorted
    W: np.ndarray          # float64 (n, N), C-contiguous
    a: float               # R-matrix radius, bohr
    z: float = 0.0         # residual charge of the target (0 neutral, > 0 ion)
    dip: Optional[np.ndarray] = None  # float64 (N,) bound-free dipole vector d_k, or None
    e0: float = 0.0        # initial bound-state energy (Ry) of the photoionisation

    @property
    def n(self) -> int:
        return int(self.l.shape[0])

    @property
    def N(self) -> int:
        return int(self.poles.shape[0])


@dataclass
class Workload:
    name: str
    waves: List[Wave]
    energies: np.ndarray   # float64 (n_e,)
    delta: float = 0.05    # near-pole window half width, Ry
    meta: dict = field(default_factory=dict)

    @property
    def n_e(self) -> int:
        return int(self.energies.shape[0])


def make_wave(rng: np.random.Generator, n: int, N: int, *, lmax: int = 7,
              thr_hi: float = 2.0, pole_lo: float = -5.0, pole_hi: float = 60.0,
              a: float = 30.0, l_fixed=None, z: float = 0.0, dipole: bool = False,
              e0: float = -0.5) -> Wave:
    """Draw one wave in the documented order (thresholds, l, poles, W, then the
    dipole vector d_k ~ N(0, 1/N) when asked for)."""
    thr = np.sort(rng.uniform(0.0, thr_hi, size=n))
    if n > 0:
        thr[0] = 0.0
    if l_fixed is not None:
        l = np.asarray(l_fixed, dtype=np.int32).copy()
    else:
        l = rng.integers(0, lmax + 1, size=n).astype(np.int32)
    poles = np.sort(rng.uniform(pole_lo, pole_hi, size=N))
    W = rng.normal(0.0, 1.0 / np.sqrt(max(N, 1)), size=(n, N))
    dip = rng.normal(0.0, 1.0 / np.sqrt(max(N, 1)), size=N).astype(np.float64) if dipole else None
    return Wave(l=l, thresh=thr.astype(np.float64), poles=poles.astype(np.float64),
                W=np.ascontiguousarray(W, dtype=np.float64), a=float(a), z=float(z), dip=dip,
                e0=float(e0))


def config(idx: int, seed: int = 0) -> Workload:
    """The five named workloads (1-based index).

    1 single wave n=4, N=200, 1000 energies on [0.01, 3] Ry, a=20
    2 n=64, N=4000, 20000 energies on [0.01, 4] Ry, a=25
    3 n=256, N=20000, 50000 energies on [0.01, 5] Ry, a=30, delta=0.05
    4 40 waves, n log-uniform in [8, 400], N=40 n, 10000 energies, a=30
    5 n=512, N=25000, 8192 energies on [0.01, 6] Ry, a=35
    """
    if idx == 1:
        rng = np.random.default_rng(seed)
        w = make_wave(rng, 4, 200, thr_hi=1.0, pole_lo=-2.0, pole_hi=20.0, a=20.0,
                      l_fixed=[0, 1, 2, 3])
        return Workload("n_ch=4 N=200 n_e=1000", [w], np.linspace(0.01, 3.0, 1000))
    if idx == 2:
        rng = np.random.default_rng(seed)
        w = make_wave(rng, 64, 4000, lmax=7, thr_hi=2.0, pole_lo=-5.0, pole_hi=40.0, a=25.0)
        return Workload("n_ch=64 N=4000 n_e=20000", [w], np.linspace(0.01, 4.0, 20000))
    if idx == 3:
        rng = np.random.default_rng(seed)
        w = make_wave(rng, 256, 20000, lmax=7, thr_hi=2.0, pole_lo=-5.0, pole_hi=60.0, a=30.0)
        return Workload("n_ch=256 N=20000 n_e=50000", [w], np.linspace(0.01, 5.0, 50000),
                        delta=0.05)
    if idx == 4:
        nrng = np.random.default_rng([seed, 999])
        ns = np.rint(np.exp(nrng.uniform(np.log(8.0), np.log(400.0), size=40))).astype(int)
        waves = []
        for g, n in enumerate(ns):
            rng = np.random.default_rng([seed, g])
            waves.append(make_wave(rng, int(n), 40 * int(n), lmax=7, thr_hi=2.0,
                                   pole_lo=-5.0, pole_hi=60.0, a=30.0))
        return Workload("40 waves n_ch in [8,400] N=40n n_e=10000", waves,
                        np.linspace(0.01, 5.0, 10000), delta=0.05, meta={"n_ch": ns.tolist()})
    if idx == 5:
        rng = np.random.default_rng(seed)
        w = make_wave(rng, 512, 25000, lmax=15, thr_hi=2.0, pole_lo=-10.0, pole_hi=80.0, a=35.0)
        return Workload("n_ch=512 N=25000 n_e=8192", [w], np.linspace(0.01, 6.0, 8192),
                        delta=0.05)
    raise ValueError(f"unknown workload {idx}")


def small(seed: int, n: int, N: int, n_e: int, *, e_lo: float = 0.01, e_hi: float = 3.0,
          lmax: int = 7, thr_hi: float = 2.0, pole_lo: float = -5.0, pole_hi: float = 40.0,
          a: float = 25.0, delta: float = 0.05, z: float = 0.0, dipole: bool = False) -> Workload:
    """A small seeded single-wave workload with the distributions of the named ones."""
    rng = np.random.default_rng(seed)
    w = make_wave(rng, n, N, lmax=lmax, thr_hi=thr_hi, pole_lo=pole_lo, pole_hi=pole_hi, a=a, z=z,
                  dipole=dipole)
    return Workload(f"small n={n} N={N} n_e={n_e} seed={seed}", [w],
                    np.linspace(e_lo, e_hi, n_e), delta=delta)
