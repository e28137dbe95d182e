"""Writes tests/golden/c4_target.txt: the target reflection spectrum |R_t(f)| of the adjoint
workload, computed by the FP64 oracle alone (no CUDA code involved).

Target profile: workloads.c4_profile(C4_TARGET_OFFSET) -- the smooth random plasma of seed
0x17090000 + 1000 on cells [2048, 6144) of a 65536-cell line, 30000 steps, probe at 1024,
source at 512, 256 frequencies to 100 GHz. R = (X_tot - X_inc)/X_inc at the probe.
Only cells within one cell per step of the source can be non-zero after 30000 steps, so the
line is cut at 512 + 30000 + 2 cells: the result is bitwise that of the full line.
Run: python tests/golden/make_c4_target.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1709_00821_gb300 import workloads as wl  # noqa: E402


def main():
    full = wl.c4_profile(wl.C4_TARGET_OFFSET)
    cut = full.src_cell + full.steps + 2
    s = wl.c4_profile(wl.C4_TARGET_OFFSET, nz=cut)
    assert np.array_equal(s.wp2, full.wp2[:cut]) and np.array_equal(s.nu, full.nu[:cut])
    tot, _ = oracle.run1d(s, omp=True)
    inc, _ = oracle.run1d(s.vacuum(), omp=True)
    R = (tot.X[0] - inc.X[0]) / inc.X[0]
    out = os.path.join(HERE, "c4_target.txt")
    with open(out, "w") as f:
        f.write("# |R_t(f)| of the adjoint workload's target profile (FP64 oracle); columns: f_hz abs_R\n")
        for fq, r in zip(s.freq_hz, np.abs(R)):
            f.write(f"{fq:.6e} {r:.17e}\n")
    print(out)


if __name__ == "__main__":
    main()
