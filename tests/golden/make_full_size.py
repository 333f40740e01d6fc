"""Write the oracle's full-size multi-step runs used by the GPU parity tests.

Calls only ``oracle/`` (plus the seeded input generators, which hold none of
the method's arithmetic):

* cubic3d_steps.npz -- the 3D cubic workload (d = 3, level 6, degree 2,
  f = -100 u^3, diffusion diag(1, 0.5, 0.1), IIF2, M = 30, dt = 0.005): the
  projected seeded initial state U0 and the states after steps 1, 5, 10 and
  20 (U1, U5, U10, U20; 20 steps is the whole configured solve).
* cubic3d_interp_steps.npz -- the same 3D cubic workload with the
  sparse-grid interpolation form of the reaction term (oracle.interp, a
  labelled deviation from the paper's F): states after steps 1, 5, 10, 20.
* schnak2d_steps.npz -- the two-species Schnakenberg workload at its stated
  size (d = 2, level 8, degree 2, kappa 0.01 / 0.5, IIF2 with GMRES, M = 40,
  dt = 0.05): the seeded noisy initial states of both species and the states
  after steps 1, 5 and 10.

Run: python tests/golden/make_full_size.py [cubic3d|cubic3d_interp|schnak2d]
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
from paper_1810_11111_gb300.workloads import coefficient_noise, cubic3d, schnak2d  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def run(cfg, U0, keep, reaction_form="quadrature"):
    idx = IndexSet(cfg["d"], cfg["n"], cfg["k"])
    sol = IIF2Solver(idx, sipg_1d(cfg["n"], cfg["k"]), cfg["kappas"], cfg["reaction"], cfg["dt"], cfg["M"],
                     reaction_form=reaction_form)
    out, U, t0 = {}, U0, time.time()
    for step in range(1, max(keep) + 1):
        U = sol.run(U, 1)
        if step in keep:
            out["U%d" % step] = np.stack(U)
        print("%s step %d (%.1f s) %s" % (cfg["name"], step, time.time() - t0, sol.stats), flush=True)
    return out, sol.stats


def cubic(reaction_form="quadrature"):
    cfg = cubic3d()
    idx = IndexSet(cfg["d"], cfg["n"], cfg["k"])
    init = cfg["init"][0]
    U0 = project_separable(idx, init["amp"], init["wavenum"], init["kind"], init["const"])
    out, stats = run(cfg, [U0], (1, 5, 10, 20), reaction_form)
    name = "cubic3d_steps.npz" if reaction_form == "quadrature" else "cubic3d_interp_steps.npz"
    np.savez_compressed(os.path.join(HERE, name), U0=np.stack([U0]), **out,
                        newton=np.array(stats["newton"]), inner=np.array(stats["inner"]))


def schnak():
    cfg = schnak2d()
    idx = IndexSet(cfg["d"], cfg["n"], cfg["k"])
    init = cfg["init"]
    U0 = coefficient_noise(init[0]["noise_seed"], idx.dof, 2, [init[0]["base"], init[1]["base"]])
    out, stats = run(cfg, U0, (1, 5, 10))
    np.savez_compressed(os.path.join(HERE, "schnak2d_steps.npz"), U0=np.stack(U0), **out,
                        newton=np.array(stats["newton"]), inner=np.array(stats["inner"]))


if __name__ == "__main__":
    which = sys.argv[1:] or ["cubic3d", "schnak2d"]
    if "cubic3d" in which:
        cubic()
    if "cubic3d_interp" in which:
        cubic("interp")
    if "schnak2d" in which:
        schnak()
