"""Pins for the oracle's inner linear solvers (oracle/iif.py), against dense
LAPACK solves: conjugate gradients on SPD systems, restarted GMRES (CGS2
Arnoldi, Givens rotations) on nonsymmetric ones, with and without restarts,
and the exact-solution early exit of GMRES (happy breakdown)."""
import numpy as np

from oracle.iif import cg, gmres


def test_cg_solves_spd_systems():
    rng = np.random.default_rng(14)
    for n in (1, 7, 40):
        B = rng.standard_normal((n, n))
        A = B @ B.T + n * np.eye(n)
        b = rng.standard_normal(n)
        x, it = cg(lambda v: A @ v, b)
        assert np.linalg.norm(x - np.linalg.solve(A, b)) <= 1e-11 * np.linalg.norm(np.linalg.solve(A, b))
        assert it <= n + 2


def test_gmres_solves_nonsymmetric_systems():
    rng = np.random.default_rng(15)
    for n, restart in ((6, 50), (30, 50), (30, 8)):
        A = np.eye(n) + 0.3 * rng.standard_normal((n, n)) / np.sqrt(n)
        b = rng.standard_normal(n)
        x, it = gmres(lambda v: A @ v, b, restart=restart, maxit=500)
        want = np.linalg.solve(A, b)
        assert np.linalg.norm(x - want) <= 1e-11 * np.linalg.norm(want), (n, restart)
        if restart >= n:
            assert it <= n


def test_gmres_exits_on_an_invariant_subspace():
    # b in a 3-dimensional invariant subspace of A: the Krylov space is
    # exhausted after 3 steps and the solution is exact
    rng = np.random.default_rng(16)
    Q, _ = np.linalg.qr(rng.standard_normal((12, 12)))
    D = np.diag(np.r_[[2.0, 3.0, 5.0], rng.uniform(1, 2, 9)])
    A = Q @ D @ Q.T
    b = Q[:, :3] @ np.array([1.0, -2.0, 0.5])
    x, it = gmres(lambda v: A @ v, b)
    assert it == 3
    assert np.linalg.norm(A @ x - b) <= 1e-12 * np.linalg.norm(b)
    assert np.array_equal(gmres(lambda v: A @ v, np.zeros(12))[0], np.zeros(12))
