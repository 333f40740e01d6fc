"""Reaction term F(U) and its Jacobian (oracle; test infrastructure only).

Section 4 (implementation remarks) and Section 5: F(U)_a = int f(u_h) v_a dx
is evaluated by reconstructing u_h at the Gauss points of the finest-level
mesh and integrating by the quadrature rule.  The oracle does exactly that:

  1. u_h lies in the full-grid space V_N^k on the finest mesh, so its
     coefficients in the finest-cell Legendre basis are obtained by applying
     the 1D change of basis T (basis.finest_legendre_transform) along every
     axis of the hierarchical coefficient tensor (zero off the sparse set);
  2. u_h is evaluated at the q^d tensor Gauss points of every finest cell;
  3. f is evaluated pointwise (species are coupled pointwise) and multiplied
     by the quadrature weights;
  4. the Legendre moments of each cell are formed and T^T maps them back to
     hierarchical indices, of which the sparse set is kept.

Reading of the unspecified quadrature order: q is the smallest Gauss rule
that integrates f(u_h) v exactly for a polynomial f of total degree p,
q = ceil((p k + k + 1) / 2); F is then the exact L2 projection of f(u_h) onto
the sparse-grid space.  The Jacobian product J_F(U) w = P(f'(u_h) w_h) uses
the same quadrature (its integrand has the same degree).

A reaction is a list per species of monomials (coef, exponents), exponents
indexed by species: f_s(u) = sum coef prod_r u_r^{e_r}.
"""
import math

import numpy as np

from .basis import finest_legendre_transform, gauss_legendre, legendre_table


def reaction_degree(reaction):
    return max((sum(e) for terms in reaction for _, e in terms), default=0)


def quadrature_points(reaction, k):
    p = reaction_degree(reaction)
    return max(1, math.ceil((p * k + k + 1) / 2))


def eval_reaction(reaction, u):
    """f_s(u) at points; u is a list of arrays (one per species)."""
    out = []
    for terms in reaction:
        acc = np.zeros_like(u[0])
        for coef, exps in terms:
            t = np.full_like(u[0], coef)
            for r, e in enumerate(exps):
                if e:
                    t = t * u[r] ** e
            acc = acc + t
        out.append(acc)
    return out


def eval_reaction_jacobian(reaction, u, w):
    """sum_r df_s/du_r (u) w_r at points, per species s."""
    out = []
    for terms in reaction:
        acc = np.zeros_like(u[0])
        for coef, exps in terms:
            for r, e in enumerate(exps):
                if e == 0:
                    continue
                t = np.full_like(u[0], coef * e) * w[r]
                for r2, e2 in enumerate(exps):
                    ee = e2 - 1 if r2 == r else e2
                    if ee:
                        t = t * u[r2] ** ee
                acc = acc + t
        out.append(acc)
    return out


class FinestGridQuadrature:
    """Reconstruction on the finest mesh and projection back (Section 4)."""

    def __init__(self, idx, q):
        self.idx, self.q = idx, q
        N, k, d = idx.N, idx.k, idx.d
        self.H = (k + 1) << N
        self.ncell = 1 << N
        self.T = finest_legendre_transform(N, k)
        h = 2.0 ** (-N)
        xi, w = gauss_legendre(q)
        self.B = legendre_table(k, xi) * np.sqrt(2.0 * np.arange(k + 1) + 1.0) / np.sqrt(h)
        self.w1 = h * w / 2.0
        self.full = idx.flat_full_indices()

    def _mode(self, X, M, axis):
        return np.moveaxis(np.tensordot(M, X, axes=([1], [axis])), 0, axis)

    def to_points(self, U):
        """u_h at all finest-cell Gauss points; shape (ncell q,)*d."""
        d, k, q, nc = self.idx.d, self.idx.k, self.q, self.ncell
        X = np.zeros(self.H ** d)
        X[self.full] = U
        X = X.reshape((self.H,) * d)
        for m in range(d):
            X = self._mode(X, self.T, m)
        for m in range(d):
            sh = X.shape
            pre, post = int(np.prod(sh[:m])), int(np.prod(sh[m + 1:]))
            X = X.reshape(pre, nc, k + 1, post)
            X = np.einsum("gr,icrj->icgj", self.B, X).reshape(sh[:m] + (nc * q,) + sh[m + 1:])
        return X

    def project(self, P):
        """int g v_a for g given at all finest-cell Gauss points; sparse layout."""
        d, k, q, nc = self.idx.d, self.idx.k, self.q, self.ncell
        wq = np.tile(self.w1, nc)
        X = P
        for m in range(d):
            shape = [1] * d
            shape[m] = nc * q
            X = X * wq.reshape(shape)
        for m in range(d):
            sh = X.shape
            pre, post = int(np.prod(sh[:m])), int(np.prod(sh[m + 1:]))
            X = X.reshape(pre, nc, q, post)
            X = np.einsum("gr,icgj->icrj", self.B, X).reshape(sh[:m] + (nc * (k + 1),) + sh[m + 1:])
        for m in range(d):
            X = self._mode(X, self.T.T, m)
        return X.reshape(-1)[self.full]


class Reaction:
    """F(U) and J_F(U) w for a polynomial reaction on one index set."""

    def __init__(self, idx, reaction):
        self.idx = idx
        self.reaction = reaction
        self.nspecies = len(reaction)
        self.quad = FinestGridQuadrature(idx, quadrature_points(reaction, idx.k))

    def F(self, U):
        """U: list of coefficient vectors (one per species)."""
        u = [self.quad.to_points(Us) for Us in U]
        return [self.quad.project(fs) for fs in eval_reaction(self.reaction, u)]

    def J(self, U, W):
        u = [self.quad.to_points(Us) for Us in U]
        w = [self.quad.to_points(Ws) for Ws in W]
        return [self.quad.project(js) for js in eval_reaction_jacobian(self.reaction, u, w)]
