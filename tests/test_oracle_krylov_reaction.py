"""Pins for the oracle's projection, reaction term, Krylov exponential and expm.

* expm_pade13 against scipy.linalg.expm and against the eigendecomposition of
  symmetric matrices (Section 3 cites scaling and squaring with Pade).
* Arnoldi (eq. krylov7): V orthonormal, A V_M = V_{M+1} H; with M equal to the
  dimension of the space the Krylov formula (eq. krylov8) is exact, so it must
  match scipy's dense expm(dt A) v; a constant vector is an eigenvector of the
  periodic operator (happy breakdown at M_eff = 1).
* Projection: the coefficient norm converges to ||u_0||_L2 (orthonormal basis)
  and the reconstruction converges at order k+1.
* Reaction: constant f touches only the constant mode; linear f gives F = a U
  exactly; cubic and two-species products match an independent quadrature
  that evaluates the hierarchical functions directly at a finer Gauss rule;
  the Jacobian matches central differences of F and is symmetric (scalar f).
"""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle.basis import alpert_coefficients, gauss_legendre, hier_eval
from oracle.index_set import IndexSet
from oracle.krylov import (arnoldi_cgs2, expm_pade13, krylov_error_estimate, krylov_expv, krylov_expv_substeps,
                           pade_coefficients)
from oracle.operator import dense_sparse_operator, sipg_1d, sparse_matvec
from oracle.projection import project_separable
from oracle.reaction import Reaction


def test_pade_coefficients():
    c = pade_coefficients(13)
    assert c[0] == 1.0 and abs(c[1] - 0.5) < 1e-16
    # the [13/13] approximant reproduces e to full precision at x = 1
    p = sum(cj for cj in c)
    q = sum(cj * (-1) ** j for j, cj in enumerate(c))
    assert abs(p / q - np.e) < 4e-16 * np.e


@pytest.mark.parametrize("scale", [1e-3, 0.5, 3.0, 40.0, 2000.0])
def test_expm_matches_scipy(scale):
    rng = np.random.default_rng(3)
    X = rng.standard_normal((12, 12)) * scale / 12
    E = expm_pade13(X)
    R = sla.expm(X)
    assert np.abs(E - R).max() <= 1e-12 * max(1.0, np.abs(R).max())


def test_expm_symmetric_negative_matches_eigendecomposition():
    # stiff symmetric negative definite, as dt H is for the diffusion operator
    rng = np.random.default_rng(4)
    Q, _ = np.linalg.qr(rng.standard_normal((20, 20)))
    lam = -np.logspace(-2, 4, 20)
    X = (Q * lam) @ Q.T
    E = expm_pade13(X)
    R = (Q * np.exp(lam)) @ Q.T
    # squaring s ~ log2(||X||/theta) times leaves a forward error of order
    # u ||X||; require no worse than scipy's own implementation
    err_scipy = np.abs(sla.expm(X) - R).max()
    assert np.abs(E - R).max() < max(4 * err_scipy, 1e-14)


def _heat_setup(d=2, N=2, k=1, kap=(1.0, 0.7)):
    idx = IndexSet(d, N, k)
    S = sipg_1d(N, k)
    A = dense_sparse_operator(idx, S, kap)
    return idx, S, A, list(kap)


def test_arnoldi_relations():
    idx, S, A, kap = _heat_setup(2, 3, 1)
    v = np.random.default_rng(5).standard_normal(idx.dof)
    M = 15
    V, H, gamma, m_eff = arnoldi_cgs2(lambda x: A @ x, v, M)
    assert m_eff == M
    assert np.abs(V.T @ V - np.eye(M + 1)).max() < 1e-12
    assert np.abs(A @ V[:, :M] - V @ H).max() < 1e-10 * np.abs(A).max()
    assert abs(gamma - np.linalg.norm(v)) < 1e-14 * gamma


def test_krylov_full_dimension_is_exact():
    idx, S, A, kap = _heat_setup(2, 2, 1)
    assert idx.dof == 32
    v = np.random.default_rng(6).standard_normal(idx.dof)
    dt = 0.01
    w, m_eff = krylov_expv(lambda x: sparse_matvec(idx, S, kap, x), v, dt, idx.dof)
    ref = sla.expm(dt * A) @ v
    assert np.linalg.norm(w - ref) <= 1e-11 * np.linalg.norm(ref)


def test_krylov_substeps_converge_to_the_exponential():
    # exp(dt A) = exp((dt/s) A)^s: with M = 8 fixed, one projection at
    # dt rho(A) ~ 16 is off by ~1e-2 while 64 sub-projections of dt/64 reach
    # the dense exponential to rounding; the error falls with every
    # refinement (each sub-span's projection converges superlinearly)
    idx, S, A, kap = _heat_setup(2, 3, 1)
    assert idx.dof == 80
    mv = lambda x: sparse_matvec(idx, S, kap, x)  # noqa: E731
    v = np.random.default_rng(3).standard_normal(idx.dof)
    dt = 1e-3
    ref = sla.expm(dt * A) @ v
    w1, m1 = krylov_expv(mv, v, dt, 8)
    ws, ms = krylov_expv_substeps(mv, v, dt, 8, 1)
    assert np.array_equal(w1, ws) and m1 == ms == 8
    errs = [np.linalg.norm(krylov_expv_substeps(mv, v, dt, 8, s)[0] - ref) / np.linalg.norm(ref)
            for s in (1, 4, 16, 64)]
    assert errs[0] > 1e-3
    assert all(b < a / 10 for a, b in zip(errs, errs[1:]))
    assert errs[-1] <= 1e-12


@pytest.mark.parametrize("dt,M", [(1e-3, 8), (1e-3, 20), (1e-2, 30), (5e-3, 30), (2e-4, 12)])
def test_krylov_error_estimate_bounds_the_error(dt, M):
    # on this dissipative operator the estimate lies above the true error of
    # the projection against the dense exponential, by less than two orders
    # of magnitude, across converged and unconverged spans
    idx, S, A, kap = _heat_setup(2, 4, 1, (1.0, 1.0))
    mv = lambda x: sparse_matvec(idx, S, kap, x)  # noqa: E731
    v = np.random.default_rng(12).standard_normal(idx.dof)
    V, H, gamma, m = arnoldi_cgs2(mv, v, M)
    w, _ = krylov_expv(mv, v, dt, M)
    ref = sla.expm(dt * A) @ v
    err = np.linalg.norm(w - ref) / np.linalg.norm(ref)
    est = krylov_error_estimate(H, m, dt)
    assert err > 1e-9  # every case here is short of convergence
    assert err <= est <= 100 * err


def test_krylov_error_estimate_vanishes_on_breakdown_and_converges():
    idx, S, A, kap = _heat_setup(2, 3, 2)
    mv = lambda x: sparse_matvec(idx, S, kap, x)  # noqa: E731
    v = np.zeros(idx.dof)
    v[0] = 2.5
    V, H, gamma, m = arnoldi_cgs2(mv, v, 20)
    assert m == 1 and krylov_error_estimate(H, m, 0.1) <= 1e-12
    v = np.random.default_rng(4).standard_normal(idx.dof)
    ests = []
    for M in (4, 8, 16, 32):
        V, H, gamma, m = arnoldi_cgs2(mv, v, M)
        ests.append(krylov_error_estimate(H, m, 1e-4))
    assert all(b < a for a, b in zip(ests, ests[1:]))
    assert ests[-1] < 1e-12


def test_krylov_breakdown_on_constant_mode():
    idx, S, A, kap = _heat_setup(2, 3, 2)
    v = np.zeros(idx.dof)
    v[0] = 2.5
    w, m_eff = krylov_expv(lambda x: sparse_matvec(idx, S, kap, x), v, 0.1, 20)
    assert m_eff == 1
    assert np.abs(w - v).max() < 1e-12


def test_projection_norm_and_order():
    errs = []
    for N in (3, 4, 5):
        idx = IndexSet(2, N, 1)
        U = project_separable(idx, [1.0], [[1, 1]], [[0, 0]])
        # ||P u||^2 <= ||u||^2 = 1/4, with the gap the squared L2 error (O9)
        gap = 0.25 - U @ U
        assert gap > 0
        errs.append(np.sqrt(gap))
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0


def test_projection_constant_term():
    idx = IndexSet(3, 3, 2)
    U = project_separable(idx, [], np.zeros((0, 3), int), np.zeros((0, 3), int), const_term=0.9)
    assert U[0] == 0.9 and np.count_nonzero(U) == 1


def _direct_quadrature_F(idx, U, f, q):
    """Independent F: evaluate every hierarchical function directly at a
    q-point Gauss rule on each finest cell (no change of basis), apply f and
    integrate against each basis function."""
    d, N, k = idx.d, idx.N, idx.k
    alpert = alpert_coefficients(k)
    nc = 1 << N
    xi, w = gauss_legendre(q)
    cells = np.repeat(np.arange(nc), q)
    vals, _ = hier_eval(N, k, cells, np.tile(xi, nc), alpert)
    w1 = np.tile(w / 2 * 2.0 ** (-N), nc)
    a = idx.hier_indices()
    npts = nc * q
    # u at all tensor points
    us = []
    for Us in U:
        u = np.zeros((npts,) * d)
        for i in range(idx.dof):
            term = Us[i]
            prod = term
            for m in range(d):
                shape = [1] * d
                shape[m] = npts
                prod = prod * vals[:, a[i, m]].reshape(shape)
            u = u + prod
        us.append(u)
    fs = f(us)
    out = []
    W = np.ones((npts,) * d)
    for m in range(d):
        shape = [1] * d
        shape[m] = npts
        W = W * w1.reshape(shape)
    for g in fs:
        Fs = np.zeros(idx.dof)
        for i in range(idx.dof):
            prod = g * W
            for m in range(d):
                prod = np.tensordot(vals[:, a[i, m]], prod, axes=([0], [0]))
            Fs[i] = prod
        out.append(Fs)
    return out


def test_reaction_constant_and_linear():
    idx = IndexSet(2, 3, 2)
    U = np.random.default_rng(8).standard_normal(idx.dof)
    Fc = Reaction(idx, [[(3.0, (0,))]]).F([U])[0]
    assert abs(Fc[0] - 3.0) < 1e-13 and np.abs(Fc[1:]).max() < 1e-13
    Fl = Reaction(idx, [[(-2.5, (1,))]]).F([U])[0]
    assert np.abs(Fl + 2.5 * U).max() < 1e-12 * np.abs(U).max()


@pytest.mark.parametrize("k", [1, 2])
def test_reaction_cubic_matches_direct_quadrature(k):
    idx = IndexSet(2, 2, k)
    U = np.random.default_rng(9).standard_normal(idx.dof) * 0.5
    F = Reaction(idx, [[(-100.0, (3,))]]).F([U])[0]
    ref = _direct_quadrature_F(idx, [U], lambda u: [-100.0 * u[0] ** 3], 2 * k + 4)[0]
    assert np.abs(F - ref).max() < 1e-11 * np.abs(ref).max()


def test_reaction_two_species_matches_direct_quadrature():
    idx = IndexSet(2, 2, 1)
    rng = np.random.default_rng(10)
    U = [1.0 + 0.1 * rng.standard_normal(idx.dof), 0.9 + 0.1 * rng.standard_normal(idx.dof)]
    rx = [[(0.1, (0, 0)), (-1.0, (1, 0)), (1.0, (2, 1))], [(0.9, (0, 0)), (-1.0, (2, 1))]]
    F = Reaction(idx, rx).F(U)
    ref = _direct_quadrature_F(idx, U, lambda u: [0.1 - u[0] + u[0] ** 2 * u[1], 0.9 - u[0] ** 2 * u[1]], 5)
    for s in range(2):
        assert np.abs(F[s] - ref[s]).max() < 1e-12 * np.abs(ref[s]).max()


def test_jacobian_matches_central_difference_and_is_symmetric():
    idx = IndexSet(3, 2, 1)
    rng = np.random.default_rng(11)
    U = rng.standard_normal(idx.dof)
    w1, w2 = rng.standard_normal(idx.dof), rng.standard_normal(idx.dof)
    R = Reaction(idx, [[(-100.0, (3,))]])
    eps = 1e-5
    fd = (R.F([U + eps * w1])[0] - R.F([U - eps * w1])[0]) / (2 * eps)
    J1 = R.J([U], [w1])[0]
    assert np.abs(J1 - fd).max() < 1e-7 * np.abs(J1).max()
    J2 = R.J([U], [w2])[0]
    assert abs(J1 @ w2 - J2 @ w1) < 1e-10 * abs(J1 @ w2)


def test_two_species_jacobian_central_difference():
    idx = IndexSet(2, 3, 1)
    rng = np.random.default_rng(12)
    U = [1 + 0.1 * rng.standard_normal(idx.dof), 0.9 + 0.1 * rng.standard_normal(idx.dof)]
    W = [rng.standard_normal(idx.dof), rng.standard_normal(idx.dof)]
    rx = [[(0.1, (0, 0)), (-1.0, (1, 0)), (1.0, (2, 1))], [(0.9, (0, 0)), (-1.0, (2, 1))]]
    R = Reaction(idx, rx)
    eps = 1e-6
    Fp = R.F([U[s] + eps * W[s] for s in range(2)])
    Fm = R.F([U[s] - eps * W[s] for s in range(2)])
    J = R.J(U, W)
    for s in range(2):
        fd = (Fp[s] - Fm[s]) / (2 * eps)
        assert np.abs(J[s] - fd).max() < 1e-7 * np.abs(J[s]).max()
