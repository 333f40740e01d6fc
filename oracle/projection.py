"""L2 projection of separable initial data (oracle; test infrastructure only).

Theorem 2.4 starts the scheme from u_h(0) = P u_0, the L2 projection onto the
sparse-grid space.  Every initial datum used here is
    u_0(x) = c_0 + sum_t amp_t prod_m g_{t,m}(2 pi w_{t,m} x_m),
g in {sin, cos} (kind 0 = sin, 1 = cos).  Because the basis is an
orthonormal tensor product (eqs. sp9, sp14), the coefficient of
prod_m v_{a_m} is sum_t amp_t prod_m int_0^1 g_{t,m}(2 pi w x) v_{a_m}(x) dx,
and the constant c_0 lands on the single level-0, degree-0 function
(phi_0 = 1).  The 1D integrals use 12-point Gauss quadrature per finest cell.
"""
import numpy as np

from .basis import alpert_coefficients, gauss_legendre, hier_eval

NQ_PROJECT = 12


def project_1d(N, k, wavenumber, kind, alpert=None):
    """int_0^1 g(2 pi w x) v_a(x) dx for all 1D hierarchical indices a."""
    if alpert is None:
        alpert = alpert_coefficients(k)
    ncell = 1 << N
    h = 2.0 ** (-N)
    xi, w = gauss_legendre(NQ_PROJECT)
    cells = np.repeat(np.arange(ncell), NQ_PROJECT)
    xis = np.tile(xi, ncell)
    vals, _ = hier_eval(N, k, cells, xis, alpert)
    x = (cells + (xis + 1.0) / 2.0) * h
    g = np.sin(2.0 * np.pi * wavenumber * x) if kind == 0 else np.cos(2.0 * np.pi * wavenumber * x)
    return (g * np.tile(h * w / 2.0, ncell)) @ vals


def project_separable(idx, amp, wavenum, kind, const_term=0.0):
    """Coefficients of P u_0 in the sparse-grid layout of ``idx``.

    amp: (T,), wavenum: (T, d) ints, kind: (T, d) ints (0 sin, 1 cos).
    """
    alpert = alpert_coefficients(idx.k)
    a = idx.hier_indices()
    U = np.zeros(idx.dof)
    cache = {}
    for t in range(len(amp)):
        term = np.full(idx.dof, float(amp[t]))
        for m in range(idx.d):
            key = (int(wavenum[t][m]), int(kind[t][m]))
            if key not in cache:
                cache[key] = project_1d(idx.N, idx.k, key[0], key[1], alpert)
            term *= cache[key][a[:, m]]
        U += term
    U[0] += const_term
    return U
