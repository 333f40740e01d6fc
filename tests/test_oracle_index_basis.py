"""Pins for the oracle's index set and bases against what the paper fixes.

Index set: the closed-form DOF count must equal every DOF printed in the
paper's Tables 1-4, and the number of level tuples is C(N+d, d).  Bases: the
hierarchical functions must be orthonormal (Section 2.1), the wavelets must
have Alpert's vanishing moments, and the hierarchical basis must span the
full piecewise-polynomial space V_N^k (the change of basis T is orthogonal).
"""
import math
import os

import numpy as np
import pytest

from oracle.basis import (alpert_coefficients, alpert_eval, finest_legendre_transform, gauss_legendre,
                          hier_eval, hier_size)
from oracle.index_set import IndexSet, dof_formula, level_tuples

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        return [ln.split() for ln in fh if ln.strip() and not ln.startswith("#")]


@pytest.mark.parametrize("row", _rows("paper_dof.txt"))
def test_dof_matches_paper_tables(row):
    d, k, N, dof = map(int, row[:4])
    assert dof_formula(d, N, k) == dof
    if dof < 200000:
        assert IndexSet(d, N, k).dof == dof


@pytest.mark.parametrize("row", _rows("paper_dof_full.txt"))
def test_full_grid_dof_matches_table2(row):
    d, k, N, dof = map(int, row[:4])
    assert ((k + 1) * 2 ** N) ** d == dof


@pytest.mark.parametrize("d,N", [(1, 5), (2, 6), (3, 4), (4, 3), (6, 2)])
def test_tuple_count_and_layout(d, N):
    k = 1
    t = level_tuples(d, N)
    assert len(t) == math.comb(N + d, d)
    assert t == sorted(t)
    idx = IndexSet(d, N, k)
    a = idx.hier_indices()
    # every coefficient maps to a distinct full-tensor position
    assert len(np.unique(idx.flat_full_indices())) == idx.dof
    lev = np.zeros_like(a)
    for m in range(d):
        lev[:, m] = np.where(a[:, m] < k + 1, 0, np.floor(np.log2(np.maximum(a[:, m], 1) / (k + 1))).astype(int) + 1)
    assert (lev.sum(axis=1) <= N).all()


@pytest.mark.parametrize("k", [1, 2, 3])
def test_alpert_vanishing_moments_and_orthonormality(k):
    c = alpert_coefficients(k)
    assert np.allclose(c @ c.T, np.eye(k + 1), atol=1e-13)
    xi, w = gauss_legendre(3 * k + 4)
    for p in range(k + 1):
        for i in range(p + k + 1):
            mom = 0.0
            for half, y in ((0, (xi - 1) / 2), (1, (xi + 1) / 2)):
                v, _ = alpert_eval(k, c, y, half)
                mom += (w / 2) @ (y ** i * v[:, p])
            assert abs(mom) < 1e-13, (p, i, mom)
        # the next moment does not vanish (otherwise the order would be wrong)
        i = p + k + 1
        mom = 0.0
        for half, y in ((0, (xi - 1) / 2), (1, (xi + 1) / 2)):
            v, _ = alpert_eval(k, c, y, half)
            mom += (w / 2) @ (y ** i * v[:, p])
        assert abs(mom) > 1e-6


@pytest.mark.parametrize("k", [1, 2, 3])
def test_hierarchical_basis_orthonormal(k):
    N = 4
    ncell = 1 << N
    xi, w = gauss_legendre(k + 2)
    cells = np.repeat(np.arange(ncell), xi.size)
    vals, _ = hier_eval(N, k, cells, np.tile(xi, ncell))
    wq = np.tile(w / 2 * 2.0 ** (-N), ncell)
    G = vals.T @ (vals * wq[:, None])
    assert np.allclose(G, np.eye(hier_size(N, k)), atol=1e-12)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_hierarchical_basis_spans_full_space(k):
    T = finest_legendre_transform(4, k)
    assert np.allclose(T.T @ T, np.eye(T.shape[0]), atol=1e-12)
    assert np.allclose(T @ T.T, np.eye(T.shape[0]), atol=1e-12)


def test_level0_is_scaled_legendre():
    # level-0 functions: sqrt(2p+1) P_p(2x-1); at x = 1 they equal sqrt(2p+1)
    k = 3
    vals, ders = hier_eval(3, k, [7], [1.0])
    assert np.allclose(vals[0, :k + 1], np.sqrt(2 * np.arange(k + 1) + 1))
    # P_p'(1) = p(p+1)/2, times the chain factor 2
    assert np.allclose(ders[0, :k + 1], np.sqrt(2 * np.arange(k + 1) + 1) * np.arange(k + 1) * (np.arange(k + 1) + 1))


def test_wavelet_support_and_scaling():
    # level n, cell j lives on (j 2^{1-n}, (j+1) 2^{1-n}) and is zero elsewhere
    N, k = 4, 1
    ncell = 1 << N
    vals, _ = hier_eval(N, k, np.arange(ncell), np.zeros(ncell))
    n, j = 3, 2
    col = (k + 1) * (1 << (n - 1)) + j * (k + 1)
    support = (np.arange(ncell) >> (N - n + 1)) == j
    assert np.all(vals[~support, col] == 0.0)
    assert np.any(vals[support, col] != 0.0)
