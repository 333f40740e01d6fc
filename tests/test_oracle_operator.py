"""Pins for the oracle's SIPG operator (Section 2.1) and sparse-grid matvec.

* The hierarchical 1D matrix equals T^T S_L T, where S_L is the finest-mesh
  SIPG matrix assembled independently in the local Legendre basis from the
  closed-form Legendre traces P_r(+-1) = (+-1)^r, P_r'(+-1) = (+-1)^{r+1}
  r(r+1)/2 and int P_r' P_s' = min(r,s)(min(r,s)+1) for r+s even.
* Spectrum: symmetric positive semidefinite; periodic kernel = constants;
  the smallest nonzero eigenvalues approach (2 pi m)^2 and the smallest
  zero-Dirichlet eigenvalue approaches pi^2.
* Sparse matvec = the full Kronecker-sum operator restricted to the index set
  (tiny grids); A symmetric negative semidefinite; A 1 = 0 (periodic).
"""
import numpy as np
import pytest

from oracle.basis import finest_legendre_transform
from oracle.index_set import IndexSet
from oracle.operator import DIRICHLET0, PERIODIC, dense_sparse_operator, sipg_1d, sparse_matvec


def legendre_sipg(N, k, bc, sigma=20.0):
    """Finest-mesh SIPG in the cell-local orthonormal Legendre basis, closed form."""
    h = 2.0 ** (-N)
    nc = 1 << N
    r = np.arange(k + 1)
    s2 = np.sqrt(2 * r + 1)
    val_r = s2 / np.sqrt(h)                     # L_r at the right end
    val_l = s2 * (-1.0) ** r / np.sqrt(h)       # L_r at the left end
    der_r = (2 / h) * s2 * r * (r + 1) / 2 / np.sqrt(h)
    der_l = (2 / h) * s2 * (-1.0) ** (r + 1) * r * (r + 1) / 2 / np.sqrt(h)
    vol = np.zeros((k + 1, k + 1))
    for a in r:
        for b in r:
            if (a + b) % 2 == 0:
                m = min(a, b)
                vol[a, b] = (2 / h ** 2) * s2[a] * s2[b] * m * (m + 1)
    n = nc * (k + 1)
    S = np.zeros((n, n))
    for c in range(nc):
        S[c * (k + 1):(c + 1) * (k + 1), c * (k + 1):(c + 1) * (k + 1)] += vol
    faces = range(nc) if bc == PERIODIC else range(nc + 1)
    for f in faces:
        J = np.zeros(n)
        G = np.zeros(n)
        left = (f - 1) % nc if bc == PERIODIC else f - 1
        right = f % nc if bc == PERIODIC else f
        if bc == PERIODIC or 0 < f < nc:
            J[left * (k + 1):(left + 1) * (k + 1)] += val_r
            J[right * (k + 1):(right + 1) * (k + 1)] -= val_l
            G[left * (k + 1):(left + 1) * (k + 1)] += 0.5 * der_r
            G[right * (k + 1):(right + 1) * (k + 1)] += 0.5 * der_l
        elif f == 0:
            J[0:k + 1] -= val_l
            G[0:k + 1] += der_l
        else:
            J[left * (k + 1):(left + 1) * (k + 1)] += val_r
            G[left * (k + 1):(left + 1) * (k + 1)] += der_r
        S += -(np.outer(G, J) + np.outer(J, G)) + (sigma / h) * np.outer(J, J)
    return S


@pytest.mark.parametrize("k", [1, 2, 3])
@pytest.mark.parametrize("bc", [PERIODIC, DIRICHLET0])
def test_hier_operator_equals_rotated_legendre_operator(k, bc):
    N = 4
    S = sipg_1d(N, k, bc)
    T = finest_legendre_transform(N, k)
    SL = legendre_sipg(N, k, bc)
    assert np.allclose(S, T.T @ SL @ T, rtol=0, atol=1e-9 * np.abs(S).max())


@pytest.mark.parametrize("k", [1, 2, 3])
def test_periodic_spectrum(k):
    N = 5
    S = sipg_1d(N, k)
    assert np.abs(S - S.T).max() <= 1e-12 * np.abs(S).max()
    ev = np.linalg.eigvalsh(0.5 * (S + S.T))
    assert ev[0] > -1e-9 * ev[-1]
    assert ev[1] > 1.0                      # kernel is one-dimensional
    assert np.abs(S[:, 0]).max() < 1e-9 * np.abs(S).max()   # constants in the kernel
    tol = {1: 0.05, 2: 1e-3, 3: 1e-4}[k]
    for m, pair in ((1, ev[1:3]), (2, ev[3:5])):
        assert np.allclose(pair / (2 * np.pi * m) ** 2, 1.0, atol=tol)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_dirichlet_lowest_eigenvalue(k):
    S = sipg_1d(5, k, DIRICHLET0)
    ev = np.linalg.eigvalsh(0.5 * (S + S.T))
    assert ev[0] > 0
    assert abs(ev[0] / np.pi ** 2 - 1) < {1: 5e-3, 2: 1e-4, 3: 1e-5}[k]


@pytest.mark.parametrize("d,N,k", [(2, 3, 1), (2, 4, 2), (3, 3, 1), (3, 2, 2), (2, 3, 3)])
@pytest.mark.parametrize("bc", [PERIODIC, DIRICHLET0])
def test_sparse_matvec_is_restricted_kronecker_sum(d, N, k, bc):
    idx = IndexSet(d, N, k)
    S = sipg_1d(N, k, bc)
    kap = [1.0, 0.5, 0.1][:d]
    A = dense_sparse_operator(idx, S, kap)
    x = np.random.default_rng(7).standard_normal(idx.dof)
    y = sparse_matvec(idx, S, kap, x)
    assert np.abs(y - A @ x).max() <= 1e-12 * np.abs(A).max() * np.abs(x).max() * 10
    assert np.abs(A - A.T).max() <= 1e-12 * np.abs(A).max()
    ev = np.linalg.eigvalsh(0.5 * (A + A.T))
    assert ev[-1] <= 1e-9 * abs(ev[0])
    if bc == PERIODIC:
        e0 = np.zeros(idx.dof)
        e0[0] = 1.0
        assert np.abs(sparse_matvec(idx, S, kap, e0)).max() < 1e-9 * np.abs(A).max()


def test_energy_of_smooth_mode():
    # x^T S x = int u'^2 + O(h^{2k}) for u = sqrt(2) sin(2 pi x): 4 pi^2
    from oracle.projection import project_1d
    N, k = 6, 2
    u = np.sqrt(2) * project_1d(N, k, 1, 0)
    S = sipg_1d(N, k)
    assert abs(u @ S @ u / (4 * np.pi ** 2) - 1) < 1e-6
