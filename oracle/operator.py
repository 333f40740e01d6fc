"""Sparse-grid SIPG diffusion operator (oracle; test infrastructure only).

Section 2.1, bilinear form B and eq. sp3, restricted to a constant diagonal
diffusion tensor k = diag(kappa_1 .. kappa_d):

  B(u, v) = sum_i kappa_i [ int d_i u d_i v
                            - sum_{faces _|_ e_i} ({d_i u}[v] + {d_i v}[u])
                            + (sigma / h) sum_{faces _|_ e_i} [u][v] ]

with sigma = 20 and h = h_N = 2^-N on every face of the finest mesh (the
penalty reading follows the energy norm of Section 2.2, which weights the
faces by h_N).  Every sparse-grid function is a tensor product, the 1D basis
is orthonormal (mass matrix I, eq. sp9) and the face integrals split into a
1D trace term times 1D L2 products, so B is a Kronecker sum of one 1D matrix
S per direction (the unidirectional principle of Section 4).  The
semi-discrete system is dU/dt = A U + F(U) with A = -B (eq. krylov1).

Jump and average in 1D (eq. sp3): at an interior face, [q] = q(x^-) - q(x^+)
and {q} = (q(x^-) + q(x^+))/2.  Periodic: the face at x = 0 ~ 1 has x^- the
trace from the last cell.  Zero Dirichlet: at x = 0, [q] = -q(0^+) and
{q'} = q'(0^+); at x = 1, [q] = q(1^-) and {q'} = q'(1^-).
"""
import numpy as np

from .basis import alpert_coefficients, gauss_legendre, hier_eval, hier_level_count, hier_level_offset, hier_size

PERIODIC = 0
DIRICHLET0 = 1


def sipg_1d(N, k, bc=PERIODIC, sigma=20.0):
    """1D SIPG matrix S[a, b] = b(v_b, v_a) in the hierarchical basis of V_N^k."""
    alpert = alpert_coefficients(k)
    H = hier_size(N, k)
    ncell = 1 << N
    h = 2.0 ** (-N)
    # volume term: sum over finest cells of int v_a' v_b', (k+1)-point Gauss
    xi, w = gauss_legendre(k + 1)
    cells = np.repeat(np.arange(ncell), k + 1)
    _, D = hier_eval(N, k, cells, np.tile(xi, ncell), alpert)
    wq = np.tile(h * w / 2.0, ncell)
    S = D.T @ (D * wq[:, None])
    # face terms: jumps J_f(a) and derivative averages G_f(a) per face
    if bc == PERIODIC:
        faces = list(range(ncell))          # face f at x = f h; face 0 wraps
    else:
        faces = list(range(ncell + 1))
    J = np.zeros((len(faces), H))
    G = np.zeros((len(faces), H))
    for i, f in enumerate(faces):
        left_cell = (f - 1) % ncell if bc == PERIODIC else f - 1
        right_cell = f % ncell if bc == PERIODIC else f
        has_left = bc == PERIODIC or f > 0
        has_right = bc == PERIODIC or f < ncell
        vl = dl = vr = dr = np.zeros(H)
        if has_left:
            v, dv = hier_eval(N, k, [left_cell], [1.0], alpert)
            vl, dl = v[0], dv[0]
        if has_right:
            v, dv = hier_eval(N, k, [right_cell], [-1.0], alpert)
            vr, dr = v[0], dv[0]
        if has_left and has_right:
            J[i] = vl - vr
            G[i] = 0.5 * (dl + dr)
        elif has_right:                      # boundary x = 0, outward normal -1
            J[i] = -vr
            G[i] = dr
        else:                                # boundary x = 1, outward normal +1
            J[i] = vl
            G[i] = dl
    S = S - (G.T @ J + J.T @ G) + (sigma / h) * (J.T @ J)
    return S


def sparse_matvec(idx, S, kappa, x):
    """y = A x with A = -sum_i kappa_i (S along direction i), restricted to the
    sparse index set (Section 4, unidirectional principle).

    For direction i and each tuple of the other levels l_{-i}, the blocks with
    l_i = 0 .. N - |l_{-i}| stacked along axis i form fibers in the 1D
    hierarchical index a_i < (k+1) 2^{N'}; S restricted to that leading
    principal submatrix is applied along axis i.
    """
    d, N, k = idx.d, idx.N, idx.k
    y = np.zeros_like(x)
    for i in range(d):
        groups = {}
        for l in idx.tuples:
            rest = l[:i] + l[i + 1:]
            groups.setdefault(rest, []).append(l)
        for rest, blocks in groups.items():
            blocks = sorted(blocks, key=lambda l: l[i])
            assert [l[i] for l in blocks] == list(range(len(blocks)))
            stacked = np.concatenate([idx.block(x, l) for l in blocks], axis=i)
            nf = stacked.shape[i]
            res = np.moveaxis(np.tensordot(S[:nf, :nf], stacked, axes=([1], [i])), 0, i)
            start = 0
            for l in blocks:
                c = hier_level_count(l[i], k)
                sl = [slice(None)] * d
                sl[i] = slice(start, start + c)
                yb = idx.block(y, l)
                yb -= kappa[i] * res[tuple(sl)]
                start += c
    return y


def dense_full_operator(d, S, kappa):
    """-sum_i kappa_i I x .. x S x .. x I on the full tensor space (tiny grids)."""
    H = S.shape[0]
    A = np.zeros((H ** d, H ** d))
    for i in range(d):
        term = np.ones((1, 1))
        for m in range(d):
            term = np.kron(term, S if m == i else np.eye(H))
        A -= kappa[i] * term
    return A


def dense_sparse_operator(idx, S, kappa):
    """The full tensor operator restricted to the sparse index set (tiny grids)."""
    A = dense_full_operator(idx.d, S, kappa)
    f = idx.flat_full_indices()
    return A[np.ix_(f, f)]


# ------------------------------------------- full diffusion tensor (NEXT) ---

def cross_blocks_1d(N, k, bc=PERIODIC):
    """1D pieces of the mixed-derivative part of the SIPG form of Section 2
    for a constant SPD tensor K, in the hierarchical basis of V_N^k:
        P[a, b] = sum over finest cells of int v_a' v_b dx
                  (derivative of the test function, value of the trial one),
        E[a, b] = sum over faces of [v_a] {v_b}
                  (jump of the test function, average of the trial values),
    with [v] = v(x-) - v(x+) on interior faces and, for zero Dirichlet, the
    one-sided trace times the outward normal on the two boundary faces (and
    the one-sided trace as the average)."""
    alpert = alpert_coefficients(k)
    H = hier_size(N, k)
    ncell = 1 << N
    h = 2.0 ** (-N)
    xi, w = gauss_legendre(k + 1)
    cells = np.repeat(np.arange(ncell), k + 1)
    V, D = hier_eval(N, k, cells, np.tile(xi, ncell), alpert)
    wq = np.tile(h * w / 2.0, ncell)
    P = D.T @ (V * wq[:, None])
    faces = list(range(ncell)) if bc == PERIODIC else list(range(ncell + 1))
    E = np.zeros((H, H))
    for f in faces:
        left_cell = (f - 1) % ncell if bc == PERIODIC else f - 1
        right_cell = f % ncell if bc == PERIODIC else f
        has_left = bc == PERIODIC or f > 0
        has_right = bc == PERIODIC or f < ncell
        vl = vr = np.zeros(H)
        if has_left:
            vl = hier_eval(N, k, [left_cell], [1.0], alpert)[0][0]
        if has_right:
            vr = hier_eval(N, k, [right_cell], [-1.0], alpert)[0][0]
        if has_left and has_right:
            J, A = vl - vr, 0.5 * (vl + vr)
        elif has_right:
            J, A = -vr, vr
        else:
            J, A = vl, vl
        E += np.outer(J, A)
    return P, E


def dense_full_operator_general(d, S, P, E, K):
    """A = -(sum_i K_ii S_i + sum_{i<j} K_ij B_ij) on the full tensor space
    (tiny grids), with B_ij the mixed terms of the form: the volume integrals
    K_ij int (d_j u d_i v + d_i u d_j v), the face integrals of the averaged
    tangential derivative of u against the normal jump of v, and their
    symmetric counterparts.  In 1D factors (test index first, direction i
    then j):
        B_ij = P x P^T + P^T x P - E x P^T - P^T x E - E^T x P - P x E^T."""
    K = np.asarray(K, dtype=np.float64)
    H = S.shape[0]
    A = dense_full_operator(d, S, np.diag(K))
    pairs = [(P, P.T), (P.T, P), (-E, P.T), (-P.T, E), (-E.T, P), (-P, E.T)]
    for i in range(d):
        for j in range(i + 1, d):
            if K[i, j] == 0.0:
                continue
            for X, Y in pairs:
                term = np.ones((1, 1))
                for m in range(d):
                    term = np.kron(term, X if m == i else (Y if m == j else np.eye(H)))
                A -= K[i, j] * term
    return A


def dense_sparse_operator_general(idx, S, P, E, K):
    """The full-tensor operator of dense_full_operator_general restricted to
    the sparse index set (the Galerkin matrix of the sparse space)."""
    A = dense_full_operator_general(idx.d, S, P, E, K)
    f = idx.flat_full_indices()
    return A[np.ix_(f, f)]


def sparse_matvec_general(idx, S, P, E, K, x):
    """y = A x for the full-tensor operator of dense_full_operator_general,
    restricted to the sparse index set, without forming it.  The diagonal
    part is sparse_matvec.  For a pair i < j and each tuple of the other
    levels, the blocks with l_i + l_j <= N - |rest| form a triangle of the 2D
    hierarchical index space (a_i, a_j); x is placed on the full square
    (zero outside the triangle), the six Kronecker products act along the
    two axes, and the result is read back on the triangle: the Galerkin
    matrix of the sparse space is the full one restricted to its indices."""
    K = np.asarray(K, dtype=np.float64)
    d, N, k = idx.d, idx.N, idx.k
    y = sparse_matvec(idx, S, np.diag(K), x)
    pairs = [(P, P.T), (P.T, P), (-E, P.T), (-P.T, E), (-E.T, P), (-P, E.T)]
    for i in range(d):
        for j in range(i + 1, d):
            if K[i, j] == 0.0:
                continue
            groups = {}
            for l in idx.tuples:
                rest = tuple(l[m] for m in range(d) if m not in (i, j))
                groups.setdefault(rest, []).append(l)
            for rest, blocks in groups.items():
                L = N - sum(rest)
                Hs = hier_level_offset(L, k) + hier_level_count(L, k)
                shape = [idx.block(x, blocks[0]).shape[m] for m in range(d)]
                shape[i] = shape[j] = Hs
                full = np.zeros(shape)
                for l in blocks:
                    o_i, o_j = hier_level_offset(l[i], k), hier_level_offset(l[j], k)
                    c_i, c_j = hier_level_count(l[i], k), hier_level_count(l[j], k)
                    sl = [slice(None)] * d
                    sl[i] = slice(o_i, o_i + c_i)
                    sl[j] = slice(o_j, o_j + c_j)
                    full[tuple(sl)] = idx.block(x, l)
                res = np.zeros_like(full)
                for X, Y in pairs:
                    t = np.moveaxis(np.tensordot(X[:Hs, :Hs], full, axes=([1], [i])), 0, i)
                    res += np.moveaxis(np.tensordot(Y[:Hs, :Hs], t, axes=([1], [j])), 0, j)
                for l in blocks:
                    o_i, o_j = hier_level_offset(l[i], k), hier_level_offset(l[j], k)
                    c_i, c_j = hier_level_count(l[i], k), hier_level_count(l[j], k)
                    sl = [slice(None)] * d
                    sl[i] = slice(o_i, o_i + c_i)
                    sl[j] = slice(o_j, o_j + c_j)
                    yb = idx.block(y, l)
                    yb -= K[i, j] * res[tuple(sl)]
    return y
