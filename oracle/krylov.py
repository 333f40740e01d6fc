"""Krylov approximation of exp(dt A) v (oracle; test infrastructure only).

Section 3, eqs. krylov7-krylov8: an orthonormal basis V_M of
K_M = span{v, A v, .., A^{M-1} v} and the Hessenberg projection H_M come from
the Arnoldi process; exp(dt A) v ~ gamma V_M exp(dt H_M) e_1, gamma = ||v||_2.

Readings where the paper is silent:
  * orthogonalisation is classical Gram-Schmidt applied twice (CGS2);
  * happy breakdown: when h_{j+1,j} <= 1e-12 ||H_{0:j+1,0:j+1}||_F the basis
    is truncated to M_eff = j + 1 columns (no error);
  * exp of the small matrix is the scaling-and-squaring method with the
    [13/13] Pade approximant (the paper cites Higham for scaling and squaring
    with Pade; Higham, SIAM J. Matrix Anal. Appl. 26 (2005), Algorithm 2.3
    with the degree fixed at 13): s = max(0, ceil(log2(||X||_1 / theta_13))),
    theta_13 = 5.371920351148152 (Higham 2005, Table 2.3).
"""
import math

import numpy as np

THETA_13 = 5.371920351148152
BREAKDOWN_TOL = 1e-12


def pade_coefficients(m):
    """Coefficients c_j of the numerator of the [m/m] Pade approximant of e^x:
    c_j = (2m - j)! m! / ((2m)! j! (m - j)!)."""
    f = math.factorial
    return [f(2 * m - j) * f(m) / (f(2 * m) * f(j) * f(m - j)) for j in range(m + 1)]


def expm_pade13(X):
    """exp(X) for a small dense matrix by Pade(13) scaling and squaring."""
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    norm1 = np.abs(X).sum(axis=0).max() if n else 0.0
    s = max(0, int(math.ceil(math.log2(norm1 / THETA_13)))) if norm1 > 0 else 0
    A = X / (2.0 ** s)
    b = pade_coefficients(13)
    I = np.eye(n)
    A2 = A @ A
    A4 = A2 @ A2
    A6 = A4 @ A2
    U = A @ (A6 @ (b[13] * A6 + b[11] * A4 + b[9] * A2) + b[7] * A6 + b[5] * A4 + b[3] * A2 + b[1] * I)
    V = A6 @ (b[12] * A6 + b[10] * A4 + b[8] * A2) + b[6] * A6 + b[4] * A4 + b[2] * A2 + b[0] * I
    R = np.linalg.solve(V - U, V + U)
    for _ in range(s):
        R = R @ R
    return R


def arnoldi_cgs2(matvec, v, M):
    """Arnoldi with classical Gram-Schmidt applied twice (eq. krylov7).

    Returns (V, H, gamma, m_eff): V has m_eff + 1 columns (the last one is
    only meaningful when no breakdown occurred), H is (M+1) x M.
    """
    n = v.size
    gamma = float(np.linalg.norm(v))
    V = np.zeros((n, M + 1))
    H = np.zeros((M + 1, M))
    if gamma == 0.0:
        return V, H, gamma, 0
    V[:, 0] = v / gamma
    m_eff = M
    for j in range(M):
        w = matvec(V[:, j])
        h1 = V[:, : j + 1].T @ w
        w = w - V[:, : j + 1] @ h1
        h2 = V[:, : j + 1].T @ w
        w = w - V[:, : j + 1] @ h2
        H[: j + 1, j] = h1 + h2
        beta = float(np.linalg.norm(w))
        H[j + 1, j] = beta
        if beta <= BREAKDOWN_TOL * np.linalg.norm(H[: j + 1, : j + 1]):
            m_eff = j + 1
            break
        V[:, j + 1] = w / beta
    return V, H, gamma, m_eff


def krylov_expv(matvec, v, dt, M):
    """gamma V_M exp(dt H_M) e_1 (eq. krylov8); returns (w, m_eff)."""
    V, H, gamma, m_eff = arnoldi_cgs2(matvec, v, M)
    if m_eff == 0:
        return np.zeros_like(v), 0
    E = expm_pade13(dt * H[:m_eff, :m_eff])
    return gamma * (V[:, :m_eff] @ E[:, 0]), m_eff


def krylov_error_estimate(H, m_eff, dt):
    """A-posteriori estimate of the relative error of gamma V_m exp(dt H_m)
    e_1 (an extension: the paper takes M fixed with no error control).

    Saad, SIAM J. Numer. Anal. 29 (1992), Section 5: the projected solution
    w_m(t) = gamma V_m exp(t H_m) e_1 satisfies w_m' = A w_m - r(t) with the
    residual r(t) = gamma h_{m+1,m} [exp(t H_m) e_1]_m v_{m+1}; the span dt
    times the residual at its end, relative to the result, is
        dt h_{m+1,m} |[exp(dt H_m) e_1]_m| / ||exp(dt H_m) e_1||.
    0 when nothing was projected; 1 when the projected result underflowed to
    zero (the projection lost it)."""
    if m_eff == 0:
        return 0.0
    y = expm_pade13(dt * H[:m_eff, :m_eff])[:, 0]
    ny = float(np.linalg.norm(y))
    if ny == 0.0:
        return 1.0
    return abs(dt * H[m_eff, m_eff - 1] * y[m_eff - 1]) / ny


def krylov_expv_substeps(matvec, v, dt, M, substeps):
    """exp(dt A) v as `substeps` successive projections (eq. krylov8) over
    dt / substeps each: the semigroup property exp(dt A) = exp((dt/s) A)^s.
    An extension, not in the paper (which takes one projection per
    exponential); substeps = 1 is krylov_expv.  Returns (w, m_eff of the
    last projection)."""
    w, m_eff = v, 0
    for _ in range(substeps):
        w, m_eff = krylov_expv(matvec, w, dt / substeps, M)
    return w, m_eff
