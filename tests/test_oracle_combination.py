"""Pins for the combination-technique form of the reaction term
(oracle.combination; a candidate for the paper's first stated future
direction, not built on the GPU).

* Linear f: F_C is exact and equals the paper's quadrature F.
* u_h depending on one coordinate only: the combination coefficients
  telescope to the one grid that holds u_h, so F_C equals the quadrature F
  for a cubic f (d = 2 and 3).
* J_C against central differences of F_C.
* On the cubic workload's data F_C is far closer to the quadrature F than
  the interpolation form (module interp) at the same level.
* For smooth data F_C approaches the quadrature F at order k + 1; an IIF2
  step with it (GMRES Newton) converges.
"""
import numpy as np
import pytest

from oracle.combination import CombinationReaction
from oracle.index_set import IndexSet
from oracle.interp import InterpReaction
from oracle.projection import project_separable
from oracle.reaction import Reaction

CUBIC = [[(-100.0, (3,))]]


@pytest.mark.parametrize("d,N,k", [(2, 4, 1), (2, 3, 2), (3, 3, 1)])
def test_linear_reaction_exact(d, N, k):
    idx = IndexSet(d, N, k)
    U = np.random.default_rng(1).standard_normal(idx.dof)
    rx = [[(0.7, (1,)), (-0.2, (0,))]]
    got = CombinationReaction(idx, rx).F([U])[0]
    want = 0.7 * U
    want[0] -= 0.2
    assert np.linalg.norm(got - want) <= 1e-12 * np.linalg.norm(want)
    assert np.linalg.norm(got - Reaction(idx, rx).F([U])[0]) <= 1e-12 * np.linalg.norm(want)


@pytest.mark.parametrize("d,N,k,axis", [(2, 4, 2, 0), (2, 4, 1, 1), (3, 3, 2, 2)])
def test_one_coordinate_data_equals_quadrature(d, N, k, axis):
    idx = IndexSet(d, N, k)
    wn = [[0] * d, [0] * d]
    wn[0][axis], wn[1][axis] = 1, 3
    kinds = [[1] * d, [1] * d]
    kinds[0][axis] = 0
    U = project_separable(idx, [0.8, -0.3], wn, kinds, 0.2)
    got = CombinationReaction(idx, CUBIC).F([U])[0]
    want = Reaction(idx, CUBIC).F([U])[0]
    assert np.linalg.norm(got - want) <= 1e-11 * np.linalg.norm(want)


def test_jacobian_central_differences():
    idx = IndexSet(2, 3, 2)
    rng = np.random.default_rng(2)
    U = [0.5 * rng.standard_normal(idx.dof), 0.5 * rng.standard_normal(idx.dof)]
    W = [rng.standard_normal(idx.dof), rng.standard_normal(idx.dof)]
    rx = [[(0.1, (0, 0)), (-1.0, (1, 0)), (1.0, (2, 1))], [(0.9, (0, 0)), (-1.0, (2, 1))]]
    cr = CombinationReaction(idx, rx)
    J = cr.J(U, W)
    eps = 1e-5
    Fp = cr.F([U[s] + eps * W[s] for s in range(2)])
    Fm = cr.F([U[s] - eps * W[s] for s in range(2)])
    for s in range(2):
        fd = (Fp[s] - Fm[s]) / (2 * eps)
        assert np.linalg.norm(J[s] - fd) <= 1e-7 * np.linalg.norm(J[s])


def test_closer_to_the_projection_than_interpolation():
    from paper_1810_11111_gb300 import workloads
    ini = workloads.cubic3d()["init"][0]
    idx = IndexSet(3, 4, 2)
    U = project_separable(idx, ini["amp"], ini["wavenum"], ini["kind"], ini["const"])
    Fq = Reaction(idx, CUBIC).F([U])[0]
    ec = np.linalg.norm(CombinationReaction(idx, CUBIC).F([U])[0] - Fq) / np.linalg.norm(Fq)
    ei = np.linalg.norm(InterpReaction(idx, CUBIC).F([U])[0] - Fq) / np.linalg.norm(Fq)
    assert ec < 1.0 < 10.0 < ei


def test_iif2_step_with_the_combination_form_runs_newton_to_tolerance():
    from oracle.iif import IIF2Solver
    from oracle.operator import sipg_1d
    idx = IndexSet(2, 3, 1)
    U0 = project_separable(idx, [0.6], [[1, 2]], [[0, 1]], 0.1)
    sol = IIF2Solver(idx, sipg_1d(3, 1), [[1.0, 0.5]], CUBIC, 0.005, 16, reaction_form="combination")
    U1 = sol.run([U0], 2)[0]
    assert np.all(np.isfinite(U1)) and np.linalg.norm(U1) < np.linalg.norm(U0)
    assert all(n >= 1 for n in sol.stats["newton"])


@pytest.mark.parametrize("k,Ns", [(1, (5, 6, 7)), (2, (5, 6, 7)), (3, (4, 5, 6))])
def test_converges_to_the_quadrature_form_at_order(k, Ns):
    rx = [[(-1.0, (3,))]]
    errs = []
    for N in Ns:
        idx = IndexSet(2, N, k)
        U = project_separable(idx, [1.0], [[1, 1]], [[0, 1]], 0.3)
        Fq = Reaction(idx, rx).F([U])[0]
        errs.append(np.linalg.norm(CombinationReaction(idx, rx).F([U])[0] - Fq) / np.linalg.norm(Fq))
    assert errs[-1] < errs[-2] < errs[-3]
    assert errs[-2] / errs[-1] > 0.6 * 2 ** (k + 1), errs
