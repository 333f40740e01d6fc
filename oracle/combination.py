"""Combination-technique form of the reaction term (oracle; test
infrastructure only).

NOT THE PAPER'S F, and not built on the GPU: a second candidate for the
paper's first stated future direction (Section 5, an evaluation of the
reaction integral that does not reconstruct u_h on the finest full grid),
kept here with its pins as the definition a future kernel must match.

The L2 projection onto the sparse-grid space satisfies the combination
identity P_N = sum_{q=0}^{d-1} (-1)^q C(d-1, q) sum_{|l|_1 = N-q} P_l, P_l the
L2 projection onto the anisotropic full-grid space V_{l_1} x ... x V_{l_d}
(the nested 1D projections telescope).  The form replaces P_l f(u_h) by
P_l f(P_l u_h):

    F_C(U) = sum_q (-1)^q C(d-1, q) sum_{|l|_1 = N-q} P_l f(P_l u_h),

so every term needs u_h only on one anisotropic grid of 2^{N-q} cells, where
the finest-grid form needs (2^N)^d cells.  P_l u_h keeps the hierarchical
blocks of u_h whose level tuple lies below l (the Alpert basis is orthonormal
and hierarchical); f(P_l u_h) is projected by the q-point Gauss rule of
module reaction on every anisotropic cell (exact for polynomial f), and the
result enters F_C with the term's coefficient on the blocks below l.

F_C equals the paper's F where f(u_h) is unchanged by the truncations: linear
f, and u_h that depends on one coordinate only (the coefficients telescope to
the single grid that holds it).  Its Jacobian is
J_C(U) w = sum_q c_q sum_l P_l (f'(P_l u_h) P_l w); with coefficients of both
signs it need not be definite, so a solver using it takes GMRES.
"""
import itertools
from math import comb

import numpy as np

from .basis import finest_legendre_transform, gauss_legendre, hier_level_count, legendre_table
from .reaction import eval_reaction, eval_reaction_jacobian, quadrature_points


def _slices(t, k, d):
    out = []
    for m in range(d):
        o = 0 if t[m] == 0 else (k + 1) << (t[m] - 1)
        out.append(slice(o, o + hier_level_count(t[m], k)))
    return tuple(out)


class AnisotropicGrid:
    """One anisotropic full grid V_l: cell Gauss points and projection."""

    def __init__(self, l, k, q):
        self.l, self.k, self.q = tuple(l), k, q
        xi, w = gauss_legendre(q)
        self.T, self.B, self.wq = [], [], []
        for lm in l:
            h = 2.0 ** (-lm)
            self.T.append(finest_legendre_transform(lm, k))
            self.B.append(legendre_table(k, xi) * np.sqrt(2.0 * np.arange(k + 1) + 1.0) / np.sqrt(h))
            self.wq.append(np.tile(h * w / 2.0, 1 << lm))

    @staticmethod
    def _mode(X, M, axis):
        return np.moveaxis(np.tensordot(M, X, axes=([1], [axis])), 0, axis)

    def to_points(self, X):
        """Hierarchical coefficients of V_l (dense tensor) -> values at the
        Gauss points of every cell."""
        d, k, q = len(self.l), self.k, self.q
        for m in range(d):
            X = self._mode(X, self.T[m], m)
        for m in range(d):
            nc, sh = 1 << self.l[m], X.shape
            pre, post = int(np.prod(sh[:m])), int(np.prod(sh[m + 1:]))
            X = np.einsum("gr,icrj->icgj", self.B[m], X.reshape(pre, nc, k + 1, post))
            X = X.reshape(sh[:m] + (nc * q,) + sh[m + 1:])
        return X

    def project(self, G):
        """Values at the Gauss points -> hierarchical coefficients of the L2
        projection onto V_l."""
        d, k, q = len(self.l), self.k, self.q
        for m in range(d):
            shape = [1] * d
            shape[m] = G.shape[m]
            G = G * self.wq[m].reshape(shape)
        for m in range(d):
            nc, sh = 1 << self.l[m], G.shape
            pre, post = int(np.prod(sh[:m])), int(np.prod(sh[m + 1:]))
            G = np.einsum("gr,icgj->icrj", self.B[m], G.reshape(pre, nc, q, post))
            G = G.reshape(sh[:m] + (nc * (k + 1),) + sh[m + 1:])
        for m in range(d):
            G = self._mode(G, self.T[m].T, m)
        return G


class CombinationReaction:
    """F_C(U) and J_C(U) w for a polynomial reaction on one index set (the
    reaction description of module reaction)."""

    symmetric = False

    def __init__(self, idx, reaction):
        self.idx, self.reaction = idx, reaction
        self.nspecies = len(reaction)
        d, N, k = idx.d, idx.N, idx.k
        q = quadrature_points(reaction, k)
        self.terms = []
        for qq in range(d):
            c = (-1) ** qq * comb(d - 1, qq)
            for l in itertools.product(range(N + 1), repeat=d):
                if sum(l) == N - qq:
                    below = [t for t in idx.tuples if all(t[m] <= l[m] for m in range(d))]
                    self.terms.append((c, AnisotropicGrid(l, k, q), below))

    def _restrict(self, U, grid, below):
        k, d = self.idx.k, self.idx.d
        X = np.zeros(tuple((k + 1) << lm for lm in grid.l))
        for t in below:
            X[_slices(t, k, d)] = self.idx.block(U, t)
        return X

    def _accumulate(self, out, G, c, below):
        k, d = self.idx.k, self.idx.d
        for t in below:
            self.idx.block(out, t)[...] += c * G[_slices(t, k, d)]

    def F(self, U):
        out = [np.zeros(self.idx.dof) for _ in range(self.nspecies)]
        for c, grid, below in self.terms:
            u = [grid.to_points(self._restrict(Us, grid, below)) for Us in U]
            for s, fs in enumerate(eval_reaction(self.reaction, u)):
                self._accumulate(out[s], grid.project(fs), c, below)
        return out

    def J(self, U, W):
        out = [np.zeros(self.idx.dof) for _ in range(self.nspecies)]
        for c, grid, below in self.terms:
            u = [grid.to_points(self._restrict(Us, grid, below)) for Us in U]
            w = [grid.to_points(self._restrict(Ws, grid, below)) for Ws in W]
            for s, js in enumerate(eval_reaction_jacobian(self.reaction, u, w)):
                self._accumulate(out[s], grid.project(js), c, below)
        return out
