"""Load vector of non-zero Dirichlet data (oracle; test infrastructure only).

Section 2's scheme with Dirichlet boundary condition u = g puts the boundary
data on the right-hand side, L(v) = int f v - int_{dOmega} (...) g ds.  The
printed integrand reads (k grad v . n + sigma/h v); the reading taken here is
the consistent one, in which the penalty term enters with the opposite sign
to the flux term:
    L_g(v) = - int_{dOmega} (k grad v . n - sigma/h v) g ds,
which follows from the bilinear form B when the exterior trace on a boundary
face is g (jump (u - g) n, one-sided average).  With it, the exact solution
satisfies the scheme; with the printed sign it would not.  The penalty is
scaled like the rest of the operator (k_i sigma / h_N on faces normal to
direction i, h_N the finest mesh size), as in the zero-Dirichlet operator of
operator.py.  In the ODE dU/dt = A U + F(U) + b, b_a = L_g(v_a).

For a face x_i = c (c = 0 with outward normal -1, c = 1 with +1) and a
tensor-product basis function v_a = prod_m v_{a_m}(x_m):
    int_{x_i = c} (k grad v_a . n - sigma/h v_a) g ds
        = k_i (n_c v'_{a_i}(c) - sigma/h v_{a_i}(c)) int g(x)|_{x_i = c} prod_{m != i} v_{a_m}(x_m),
with the one-sided traces from inside [0, 1].  For g the restriction of a
sum of products G(x) = sum_t amp_t prod_m g_{t,m}(x_m) the face integral is a
product of 1D projections, so b is a sum of separable terms.
"""
import numpy as np

from .basis import alpert_coefficients, gauss_legendre, hier_eval

NQ = 12


def boundary_traces(N, k, alpert=None):
    """v(0+), v'(0+), v(1-), v'(1-) of all 1D hierarchical functions."""
    v0, d0 = hier_eval(N, k, [0], [-1.0], alpert)
    v1, d1 = hier_eval(N, k, [(1 << N) - 1], [1.0], alpert)
    return v0[0], d0[0], v1[0], d1[0]


def project_1d(N, k, g, alpert=None):
    """int_0^1 g(x) v_a(x) dx for a vectorised callable g, NQ-point Gauss per finest cell."""
    ncell = 1 << N
    h = 2.0 ** (-N)
    xi, w = gauss_legendre(NQ)
    cells = np.repeat(np.arange(ncell), NQ)
    xis = np.tile(xi, ncell)
    vals, _ = hier_eval(N, k, cells, xis, alpert)
    x = (cells + (xis + 1.0) / 2.0) * h
    return (g(x) * np.tile(h * w / 2.0, ncell)) @ vals


def project_product(idx, terms):
    """Coefficients of sum_t amp_t prod_m g_{t,m}(x_m); terms = [(amp, [g_1, .., g_d])]."""
    alpert = alpert_coefficients(idx.k)
    a = idx.hier_indices()
    U = np.zeros(idx.dof)
    for amp, gs in terms:
        term = np.full(idx.dof, float(amp))
        for m in range(idx.d):
            term *= project_1d(idx.N, idx.k, gs[m], alpert)[a[:, m]]
        U += term
    return U


def dirichlet_load(idx, kappa, terms, sigma=20.0):
    """b_a = L_g(v_a) for g = G restricted to the boundary, G given as terms
    [(amp, [g_1, .., g_d])] of vectorised callables; kappa: the diagonal."""
    alpert = alpert_coefficients(idx.k)
    a = idx.hier_indices()
    h = 2.0 ** (-idx.N)
    v0, d0, v1, d1 = boundary_traces(idx.N, idx.k, alpert)
    b = np.zeros(idx.dof)
    for amp, gs in terms:
        proj = [project_1d(idx.N, idx.k, g, alpert) for g in gs]
        for i in range(idx.d):
            for c, n_c, v, dv in ((0.0, -1.0, v0, d0), (1.0, 1.0, v1, d1)):
                # - k_i (n_c v' - sigma/h v) g_i(c): the face-normal factor
                beta = -kappa[i] * (n_c * dv - sigma / h * v) * float(gs[i](np.array([c]))[0])
                term = np.full(idx.dof, float(amp))
                for m in range(idx.d):
                    term *= (beta if m == i else proj[m])[a[:, m]]
                b += term
    return b


def trig_terms(d, amp, wavenum, kind, const_term=0.0):
    """The separable family of projection.py as callables: const_term plus
    sum_t amp_t prod_m g_{t,m}(2 pi w x_m), g = sin (kind 0) or cos (kind 1).
    At the boundary points 0 and 1 the factors are evaluated exactly for
    integer w (sin 0, cos 1)."""
    def factor(w, kd):
        def g(x):
            x = np.asarray(x, dtype=np.float64)
            exact = np.isin(x, (0.0, 1.0))
            val = np.sin(2 * np.pi * w * x) if kd == 0 else np.cos(2 * np.pi * w * x)
            return np.where(exact, 0.0 if kd == 0 else 1.0, val)
        return g
    terms = [(amp[t], [factor(int(wavenum[t][m]), int(kind[t][m])) for m in range(d)]) for t in range(len(amp))]
    if const_term != 0.0:
        terms.append((const_term, [lambda x: np.ones_like(np.asarray(x, dtype=np.float64))] * d))
    return terms
