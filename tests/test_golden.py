"""Stored values under tests/golden/ (no GPU).

* table3_matrix_sizes.txt: the R-matrix formation sizes n x m the paper prints (Table 3).  The
  seeded workloads stand in for the paper's atomic data, so their shapes must bracket the paper's:
  poles per channel N/n around the paper's m/n, channel counts inside its range.
* oracle_config1_sample.txt: the oracle's outputs on eight energies of the n_ch = 4 workload,
  written by tests/golden/make_oracle_golden.py (which calls only the oracle and the seeded
  inputs); recomputed here so that any change to the oracle's arithmetic shows.
"""
import os

import numpy as np

from paper_1403_5524_gb300 import synth

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    return np.loadtxt(os.path.join(HERE, name), comments="#", ndmin=2)


def test_workloads_bracket_the_papers_matrix_sizes():
    t = load("table3_matrix_sizes.txt")
    n, m = t[:, 0], t[:, 1]
    ratio = m / n
    assert 60.0 < ratio.min() and ratio.max() < 64.0  # the paper's waves carry about 62 poles per channel
    ours = []
    for c in (2, 3, 5):
        w = synth.config(c).waves[0]
        ours.append(w.N / w.n)
    ours += [w.N / w.n for w in synth.config(4).waves]
    assert min(ours) <= ratio.min() and max(ours) >= ratio.max()
    # the benchmark workload's 256 and the large workload's 512 channels lie inside the paper's range
    assert n.min() <= 256 <= n.max() and n.min() <= 512 <= n.max()


def test_oracle_matches_its_stored_sample():
    import sys
    sys.path.insert(0, HERE)
    import make_oracle_golden as g
    stored = load("oracle_config1_sample.txt")
    fresh = np.array(g.rows(), dtype=np.float64)
    assert stored.shape == fresh.shape
    assert np.array_equal(stored[:, [0, 2, 3]], fresh[:, [0, 2, 3]])  # index, n_open, flags
    assert np.allclose(stored[:, 1], fresh[:, 1], rtol=0, atol=0)
    scale = np.maximum(np.abs(stored[:, 4:]), 1.0)
    assert np.all(np.abs(stored[:, 4:] - fresh[:, 4:]) <= 1e-12 * scale)
