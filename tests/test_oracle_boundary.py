"""Pins for the Dirichlet load of non-zero boundary data (oracle/boundary.py).

* Consistency (Galerkin orthogonality): for u_p a polynomial of degree <= k
  in each direction, A P(u_p) + b(u_p|boundary) = P(div(k grad u_p)) exactly,
  because SIPG with the consistent boundary term is satisfied by smooth
  solutions and P is exact on the space.  A dropped term, a wrong sign of
  the flux or penalty part, a wrong trace or a wrong normal fails it.
"""
import numpy as np

from oracle.boundary import dirichlet_load, project_product
from oracle.index_set import IndexSet
from oracle.operator import DIRICHLET0, sipg_1d, sparse_matvec


def test_load_is_consistent_for_polynomials():
    rng = np.random.default_rng(11)
    for d, N, k in ((1, 3, 1), (2, 3, 1), (2, 3, 2), (3, 2, 2)):
        idx = IndexSet(d, N, k)
        S = sipg_1d(N, k, DIRICHLET0)
        kappa = rng.uniform(0.3, 1.5, d)
        coef = rng.standard_normal((d, k + 1))  # u_p = prod_m sum_j coef[m, j] x^j
        gs = [np.polynomial.Polynomial(coef[m]) for m in range(d)]
        U = project_product(idx, [(1.0, gs)])
        b = dirichlet_load(idx, kappa, [(1.0, gs)])
        # div(k grad u_p) = sum_i k_i g_i'' prod_{m != i} g_m
        lap = [(kappa[i], [gs[m].deriv(2) if m == i else gs[m] for m in range(d)]) for i in range(d)]
        want = project_product(idx, lap)
        got = sparse_matvec(idx, S, kappa, U) + b
        scale = np.linalg.norm(b) + np.linalg.norm(want)
        assert np.linalg.norm(got - want) < 1e-11 * scale, (d, N, k, np.linalg.norm(got - want) / scale)
