"""Pins for the SIPG operator with a full constant SPD diffusion tensor K
(oracle/operator.py: cross_blocks_1d, dense_sparse_operator_general; the
bilinear form of Section 2 with off-diagonal K_ij).

* The sparse-grid matrix is symmetric and negative semidefinite (constant
  mode in the kernel for periodic boundaries), and a diagonal K gives the
  operator of the diagonal case exactly.
* Consistency, exactly: u = prod_m x_m (1 - x_m) is continuous, vanishes on
  the boundary and lies in the space for k >= 2, so the SIPG form with zero
  Dirichlet data satisfies A P(u) = P(div(K grad u)) up to rounding.  The
  mixed derivative u_xy tests the cross terms; dropping a face term,
  swapping a transpose or flipping a sign breaks the identity.
* Periodic: the Rayleigh quotient of the projected mode cos(2 pi m.x)
  converges to -4 pi^2 m^T K m at the rate of the diagonal case.
"""
import numpy as np

from oracle.boundary import project_product
from oracle.index_set import IndexSet
from oracle.operator import (DIRICHLET0, PERIODIC, cross_blocks_1d, dense_sparse_operator,
                             dense_sparse_operator_general, sipg_1d)
from oracle.projection import project_separable


def _spd(d, rng):
    Q, _ = np.linalg.qr(rng.standard_normal((d, d)))
    return Q @ np.diag(rng.uniform(0.3, 1.5, d)) @ Q.T


def _operator(d, N, k, K, bc):
    idx = IndexSet(d, N, k)
    P, E = cross_blocks_1d(N, k, bc)
    return idx, dense_sparse_operator_general(idx, sipg_1d(N, k, bc), P, E, K)


def test_symmetric_negative_semidefinite():
    rng = np.random.default_rng(12)
    for d, N, k in ((2, 3, 1), (2, 3, 2), (3, 2, 2)):
        for bc in (PERIODIC, DIRICHLET0):
            _, A = _operator(d, N, k, _spd(d, rng), bc)
            scale = np.abs(A).max()
            assert np.abs(A - A.T).max() <= 1e-13 * scale
            assert np.linalg.eigvalsh(0.5 * (A + A.T)).max() <= 1e-11 * scale, (d, N, k, bc)


def test_diagonal_tensor_reduces_to_the_diagonal_operator():
    K = np.diag([0.7, 0.2, 1.1])
    for bc in (PERIODIC, DIRICHLET0):
        idx, A = _operator(3, 2, 1, K, bc)
        assert np.array_equal(A, dense_sparse_operator(idx, sipg_1d(2, 1, bc), np.diag(K)))


def test_exact_for_the_bubble_polynomial():
    rng = np.random.default_rng(13)
    bubble = np.polynomial.Polynomial([0.0, 1.0, -1.0])  # x (1 - x)
    for d, N, k in ((2, 3, 2), (2, 4, 3), (3, 2, 2)):
        K = _spd(d, rng)
        idx, A = _operator(d, N, k, K, DIRICHLET0)
        U = project_product(idx, [(1.0, [bubble] * d)])
        terms = []
        for i in range(d):
            for j in range(d):
                gs = [bubble] * d
                if i == j:
                    gs = [bubble.deriv(2) if m == i else bubble for m in range(d)]
                else:
                    gs = [bubble.deriv(1) if m in (i, j) else bubble for m in range(d)]
                terms.append((K[i, j], gs))
        want = project_product(idx, terms)
        assert np.linalg.norm(A @ U - want) <= 1e-10 * np.linalg.norm(want), (d, N, k)


def test_periodic_rayleigh_quotient_converges():
    K = np.array([[1.0, 0.4], [0.4, 0.6]])
    m = np.array([1, 1])
    lam = 4 * np.pi ** 2 * m @ K @ m
    errs = []
    for N in (3, 4, 5):
        idx, A = _operator(2, N, 2, K, PERIODIC)
        # cos(2 pi (x + y)) = cos cos - sin sin
        U = project_separable(idx, [1.0, -1.0], [[1, 1], [1, 1]], [[1, 1], [0, 0]])
        errs.append(abs(U @ A @ U / (U @ U) + lam) / lam)
    assert errs[-1] < 2e-4, errs
    for e0, e1 in zip(errs, errs[1:]):
        assert np.log2(e0 / e1) > 3.0, errs


def test_matrix_free_matvec_equals_the_restricted_matrix():
    # two implementations of the same definition: the dense full-tensor
    # matrix restricted to the index set, and the per-pair triangle form
    from oracle.operator import sparse_matvec_general
    rng = np.random.default_rng(17)
    for d, N, k, bc in ((2, 4, 1, PERIODIC), (2, 3, 2, DIRICHLET0), (3, 3, 1, PERIODIC), (3, 2, 2, DIRICHLET0)):
        K = _spd(d, rng)
        idx, A = _operator(d, N, k, K, bc)
        P, E = cross_blocks_1d(N, k, bc)
        x = rng.standard_normal(idx.dof)
        y = sparse_matvec_general(idx, sipg_1d(N, k, bc), P, E, K, x)
        assert np.linalg.norm(y - A @ x) <= 1e-12 * np.linalg.norm(A @ x), (d, N, k, bc)
