"""Write the oracle's IIF2 step of the 3D cubic workload (level 6, degree 2).

Calls only ``oracle/`` (plus the seeded input generator): projects the seeded
8-mode initial datum, takes one IIF2 step (f = -100 u^3, diffusion
diag(1, 0.5, 0.1), M = 30, dt = 0.005) and stores U^0 and U^1 in
cubic3d_step1.npz next to this script.  Run: python tests/golden/make_cubic3d_step.py
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle.iif import IIF2Solver  # noqa: E402
from oracle.index_set import IndexSet  # noqa: E402
from oracle.operator import sipg_1d  # noqa: E402
from oracle.projection import project_separable  # noqa: E402
from paper_1810_11111_gb300.workloads import cubic3d  # noqa: E402


def main():
    cfg = cubic3d()
    idx = IndexSet(cfg["d"], cfg["n"], cfg["k"])
    init = cfg["init"][0]
    U0 = project_separable(idx, init["amp"], init["wavenum"], init["kind"], init["const"])
    sol = IIF2Solver(idx, sipg_1d(cfg["n"], cfg["k"]), cfg["kappas"], cfg["reaction"], cfg["dt"], cfg["M"])
    t = time.time()
    U1 = sol.run([U0], 1)[0]
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "cubic3d_step1.npz")
    np.savez_compressed(out, U0=U0, U1=U1, newton=np.array(sol.stats["newton"]),
                        inner=np.array(sol.stats["inner"]))
    print("wrote", out, "in %.1f s" % (time.time() - t), sol.stats)


if __name__ == "__main__":
    main()
