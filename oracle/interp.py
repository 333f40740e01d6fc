"""Sparse-grid interpolation form of the reaction term (oracle; test
infrastructure only).

NOT THE PAPER'S F.  The paper evaluates F(U)_a = int f(u_h) v_a dx by
reconstructing u_h at the Gauss points of the finest full grid (Section 4;
module ``reaction``), and names as its first future direction (Section 5) an
evaluation of that integral that uses the structure of the multiwavelet basis
instead.  This module defines such a form, a labelled deviation from the
paper's discretisation:

    F_I(U) = coefficients, in the orthonormal Alpert basis, of the unique
             w in the sparse-grid space V_N^k with w(x_p) = f(u_h(x_p)) at
             every sparse-grid collocation point x_p.

F_I equals the paper's F whenever f(u_h) lies in the sparse-grid space
(linear f) and otherwise differs from it by an interpolation error of the
same order as the scheme's; it never touches the finest full grid.

Collocation points.  Degree k uses k+1 points X_0 in [0, 1):
    k = 1: {1/3, 2/3}    k = 2: {0, 1/3, 2/3}    k = 3: {1/5, 2/5, 3/5, 4/5}.
Each set is mapped into itself by x -> 2x mod 1, so the sets of level n,
X_n = {(c + x)/2^n : c < 2^n, x in X_0} (X_0 copied into every level-n cell),
are nested: X_{n-1} is a subset of X_n.  The k+1 points of X_n \\ X_{n-1}
inside the level-(n-1) cell j, sorted, carry the 1D hierarchical indices
(n, j, p = 0..k) of the Alpert functions v^j_{p,n} (eq. sp9); level 0 carries
X_0 itself.  A point c/2^n on a cell edge (k = 2) is a point of the cell to
its right, where a discontinuous u_h is taken from the right.  The sparse
point of the d-dimensional index (l, j, p) is the tensor point of its 1D
indices, so there is one point per coefficient.

Interpolatory hierarchical basis.  ell_q for the point q of level n is the
degree-k Lagrange polynomial on the level-n cell of q through the k+1 points
of X_n in that cell (1 at q), zero elsewhere.  It vanishes at every point of
a coarser level, and {ell_q : level <= n} spans V_n^k.

Computation by directions.  With E[p, a] = v_a(x_p) and B[p, q] = ell_q(x_p)
in 1D, E = B A, where A (Alpert coefficients to interpolation surpluses)
only maps a level to the same or coarser levels and B (surpluses to point
values) only to the same or finer levels.  On a sparse index set (closed
under lowering any level) a Kronecker product of such factors restricted to
the set is the product of its 1D factors applied direction by direction,
each on the fibers of the set truncated to their own maximum level (the
unidirectional principle of Section 4).  So the collocation matrix of the
sparse set is C = (x_m B)(x_m A), and
    u_h at the points = C U  (A along every direction, then B),
    F_I(U) = C^{-1} f(C U)   (B^{-1} along every direction, then A^{-1}).
``SparseInterpolation.dense`` forms C entry by entry from the basis
definitions (tiny grids); the tests pin the directional route to it.

Jacobian: J_I(U) w = C^{-1} (f'(C U) * (C w)).  It is not symmetric, so the
Newton stage of a solver that uses F_I solves its linear systems by GMRES.
In point values the implicit stage U - c F_I(U) = W is the set of decoupled
pointwise equations u_p - c f(u_p) = (C W)_p, which is how the CUDA path
solves it; the oracle keeps the coefficient-space Newton of module ``iif``.
"""
import numpy as np

from .basis import alpert_coefficients, hier_decode, hier_eval, hier_level_count, hier_level_offset, hier_size
from .reaction import eval_reaction, eval_reaction_jacobian

BASE_POINTS = {1: (1.0 / 3.0, 2.0 / 3.0), 2: (0.0, 1.0 / 3.0, 2.0 / 3.0), 3: (0.2, 0.4, 0.6, 0.8)}


def base_points(k):
    """X_0 for degree k (sorted)."""
    return np.array(BASE_POINTS[k], dtype=np.float64)


def new_points_local(k):
    """Local coordinates in (0, 1) of the level-n points of a level-(n-1)
    cell that are not level-(n-1) points (sorted): both halves' copies of X_0
    minus X_0 itself."""
    x0 = base_points(k)
    both = np.concatenate([x0 / 2.0, 0.5 + x0 / 2.0])
    new = np.array(sorted(y for y in both if np.min(np.abs(x0 - y)) > 1e-12))
    assert new.size == k + 1
    return new


def hier_points(N, k):
    """Coordinate of the collocation point of every 1D hierarchical index."""
    H = hier_size(N, k)
    x = np.zeros(H)
    x[: k + 1] = base_points(k)
    new = new_points_local(k)
    for n in range(1, N + 1):
        o, c = hier_level_offset(n, k), hier_level_count(n, k)
        t = np.arange(c)
        j, p = t // (k + 1), t % (k + 1)
        x[o:o + c] = (j + new[p]) * 2.0 ** (1 - n)
    return x


def alpert_at(N, k, x, alpert=None):
    """E[i, a] = v_a(x_i) for all 1D hierarchical indices a < (k+1) 2^N, each
    function taken from the finest cell that contains x_i (from the right at
    a cell edge)."""
    x = np.asarray(x, dtype=np.float64)
    scaled = x * (1 << N)
    cell = np.minimum(np.floor(scaled).astype(np.int64), (1 << N) - 1)
    xi = 2.0 * (scaled - cell) - 1.0
    vals, _ = hier_eval(N, k, cell, xi, alpert)
    return vals


def lagrange_hier_at(N, k, x):
    """B[i, q] = ell_q(x_i) for all 1D hierarchical indices q (module doc)."""
    x = np.asarray(x, dtype=np.float64)
    H = hier_size(N, k)
    level, _, _ = hier_decode(N, k)
    xq = hier_points(N, k)
    x0 = base_points(k)
    out = np.zeros((x.size, H))
    for q in range(H):
        h = 2.0 ** (-int(level[q]))
        c = np.floor(xq[q] / h + 1e-9)
        nodes = (c + x0) * h
        me = int(np.argmin(np.abs(nodes - xq[q])))
        inside = (x >= c * h - 1e-15) & (x < (c + 1) * h - 1e-15)
        val = np.ones(x.size)
        for t in range(k + 1):
            if t != me:
                val *= (x - nodes[t]) / (nodes[me] - nodes[t])
        out[:, q] = np.where(inside, val, 0.0)
    return out


def one_dim_factors(N, k):
    """The 1D factors of the collocation matrix at level N: A (Alpert ->
    surpluses), B (surpluses -> values) and their inverses.  A = B^{-1} E by a
    dense solve; the entries that the level structure makes zero (A, A^{-1}:
    a finer row level than column level; B, B^{-1}: a coarser one) are
    rounding residue and set to zero."""
    x = hier_points(N, k)
    E = alpert_at(N, k, x)
    B = lagrange_hier_at(N, k, x)
    level, _, _ = hier_decode(N, k)
    finer_row = level[:, None] > level[None, :]
    coarser_row = level[:, None] < level[None, :]
    A = np.linalg.solve(B, E)
    A[finer_row] = 0.0
    Ainv = np.linalg.inv(A)
    Ainv[finer_row] = 0.0
    B = B.copy()
    B[coarser_row] = 0.0
    Binv = np.linalg.inv(B)
    Binv[coarser_row] = 0.0
    return A, B, Binv, Ainv


def apply_direction(idx, T, i, x):
    """y = (I x .. x T x .. x I) x on the sparse set, T along direction i,
    each fiber multiplied by the leading principal block of T of its length
    (exact for factors that only map levels one way, module doc)."""
    d, k = idx.d, idx.k
    y = np.zeros_like(x)
    groups = {}
    for l in idx.tuples:
        groups.setdefault(l[:i] + l[i + 1:], []).append(l)
    for blocks in groups.values():
        blocks = sorted(blocks, key=lambda l: l[i])
        assert [l[i] for l in blocks] == list(range(len(blocks)))
        stacked = np.concatenate([idx.block(x, l) for l in blocks], axis=i)
        nf = stacked.shape[i]
        res = np.moveaxis(np.tensordot(T[:nf, :nf], stacked, axes=([1], [i])), 0, i)
        start = 0
        for l in blocks:
            c = hier_level_count(l[i], k)
            sl = [slice(None)] * d
            sl[i] = slice(start, start + c)
            idx.block(y, l)[...] = res[tuple(sl)]
            start += c
    return y


class SparseInterpolation:
    """Point values at the sparse collocation points and interpolation back."""

    def __init__(self, idx):
        self.idx = idx
        self.A, self.B, self.Binv, self.Ainv = one_dim_factors(idx.N, idx.k)

    def _chain(self, x, first, second):
        for i in range(self.idx.d):
            x = apply_direction(self.idx, first, i, x)
        for i in range(self.idx.d):
            x = apply_direction(self.idx, second, i, x)
        return x

    def to_points(self, U):
        """u_h at the collocation points (C U), in the coefficient layout."""
        return self._chain(np.asarray(U, dtype=np.float64), self.A, self.B)

    def from_points(self, g):
        """Alpert coefficients of the sparse interpolant of point values g
        (C^{-1} g)."""
        return self._chain(np.asarray(g, dtype=np.float64), self.Binv, self.Ainv)

    def points(self):
        """(dof, d) coordinates of the collocation point of every coefficient."""
        x = hier_points(self.idx.N, self.idx.k)
        return x[self.idx.hier_indices()]

    def dense(self):
        """C[p, a] = prod_m v_{a_m}(x_{p_m}) over the sparse set, from the
        basis functions at the points (tiny grids only)."""
        idx = self.idx
        E = alpert_at(idx.N, idx.k, hier_points(idx.N, idx.k), alpert_coefficients(idx.k))
        ha = idx.hier_indices()
        C = np.ones((idx.dof, idx.dof))
        for m in range(idx.d):
            C *= E[ha[:, m]][:, ha[:, m]]
        return C


class InterpReaction:
    """F_I(U) and J_I(U) w for a polynomial reaction on one index set (the
    same reaction description as module ``reaction``)."""

    symmetric = False

    def __init__(self, idx, reaction):
        self.idx = idx
        self.reaction = reaction
        self.nspecies = len(reaction)
        self.interp = SparseInterpolation(idx)

    def F(self, U):
        u = [self.interp.to_points(Us) for Us in U]
        return [self.interp.from_points(fs) for fs in eval_reaction(self.reaction, u)]

    def J(self, U, W):
        u = [self.interp.to_points(Us) for Us in U]
        w = [self.interp.to_points(Ws) for Ws in W]
        return [self.interp.from_points(js) for js in eval_reaction_jacobian(self.reaction, u, w)]
