"""Sparse-grid index set and coefficient layout (oracle; test infrastructure only).

Section 2.1, eqs. sp10-sp13: the sparse-grid space is the direct sum of the
tensor spaces W_l = W_{l_1} x ... x W_{l_d} over level tuples with
|l|_1 <= N; W_l has basis functions prod_m v^{j_m}_{p_m, l_m}(x_m) with
j_m = 0 .. max(0, 2^{l_m - 1} - 1) and p_m = 0 .. k (eq. sp14).

Coefficient layout (shared by definition with the CUDA path, not by code):
  * level tuples in lexicographic order, l_1 varying slowest;
  * one contiguous block per tuple, row-major over the local 1D indices
    t_m = j_m (k+1) + p_m, dimension d fastest.
"""
import itertools

import numpy as np

from .basis import hier_level_count, hier_level_offset


def level_tuples(d, N):
    """All l in N^d with |l|_1 <= N, lexicographic with l_1 slowest."""
    return [l for l in itertools.product(range(N + 1), repeat=d) if sum(l) <= N]


def block_shape(l, k):
    return tuple(hier_level_count(n, k) for n in l)


def dof_formula(d, N, k):
    """(k+1)^d sum_{|l|_1<=N} prod_m max(1, 2^{l_m - 1}) (eq. sp13, sp14)."""
    return sum((k + 1) ** d * int(np.prod([max(1, 1 << (n - 1)) if n > 0 else 1 for n in l]))
               for l in level_tuples(d, N))


class IndexSet:
    """Level tuples, block offsets and the map to 1D hierarchical indices."""

    def __init__(self, d, N, k):
        self.d, self.N, self.k = d, N, k
        self.tuples = level_tuples(d, N)
        self.rank = {l: i for i, l in enumerate(self.tuples)}
        self.shapes = [block_shape(l, k) for l in self.tuples]
        sizes = [int(np.prod(s)) for s in self.shapes]
        self.offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        self.dof = int(self.offsets[-1])

    def levels_array(self):
        return np.array(self.tuples, dtype=np.int32).reshape(len(self.tuples), self.d)

    def block(self, x, l):
        """View of block l of a coefficient vector, shaped by the block."""
        i = self.rank[l]
        return x[self.offsets[i]:self.offsets[i + 1]].reshape(self.shapes[i])

    def hier_indices(self):
        """(dof, d) array of 1D hierarchical indices a_m of every coefficient."""
        out = np.zeros((self.dof, self.d), dtype=np.int64)
        for i, l in enumerate(self.tuples):
            grids = np.meshgrid(*[hier_level_offset(n, self.k) + np.arange(hier_level_count(n, self.k))
                                  for n in l], indexing="ij")
            out[self.offsets[i]:self.offsets[i + 1]] = np.stack([g.ravel() for g in grids], axis=1)
        return out

    def flat_full_indices(self):
        """Row-major index of each coefficient in the full (H,)*d tensor."""
        H = hier_level_offset(self.N, self.k) + hier_level_count(self.N, self.k)
        a = self.hier_indices()
        return np.ravel_multi_index(tuple(a.T), (H,) * self.d)
