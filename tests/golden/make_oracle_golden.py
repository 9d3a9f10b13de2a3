"""Write tests/golden/oracle_config1_sample.txt: the FP64 oracle's outputs on eight energies of
the n_ch = 4 workload (seed 0).  Calls only oracle/ and the seeded input generator; the stored
values guard the oracle against accidental change (tests/test_golden.py recomputes them)."""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import rmatrix as orc  # noqa: E402
from paper_1403_5524_gb300 import synth  # noqa: E402

IDX = [0, 95, 230, 333, 512, 640, 811, 999]
SEL = (0, 1, 2, 3)


def rows():
    wl = synth.config(1)
    ref = orc.sweep(wl.waves[0], wl.energies, sel=SEL, energy_idx=np.array(IDX))
    out = []
    for t, e in enumerate(IDX):
        no = int(ref["n_open"][t])
        kd = [float(ref["K"][t, i, i]) for i in range(4)]
        out.append([e, float(ref["E"][t]), no, int(ref["flags"][t]), float(ref["eta"][t])]
                   + [float(x) for x in ref["sig_tot"][t]] + kd)
    return out


def main():
    path = os.path.join(HERE, "oracle_config1_sample.txt")
    with open(path, "w") as f:
        f.write("# FP64 oracle on the n_ch = 4, N = 200 workload (seed 0), written by make_oracle_golden.py\n")
        f.write("# columns: mesh index, nudged E (Ry), n_open, flags, eta, sig_tot for initial channels 0..3, "
                "K_ii for i = 0..3\n")
        for r in rows():
            f.write(" ".join(repr(x) for x in r) + "\n")
    print("wrote", path)


if __name__ == "__main__":
    main()
