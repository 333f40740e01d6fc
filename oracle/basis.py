"""1D bases of the sparse-grid DG space (oracle; test infrastructure only).

Section 2.1 of the paper:
  * nested partition I_n^j = (2^-n j, 2^-n (j+1)]                    (eq. sp4)
  * V_n^k piecewise polynomials of degree <= k on level n            (eq. sp5)
  * W_n^k = orthogonal complement of V_{n-1}^k in V_n^k              (eq. sp7)
  * level 0 basis: scaled Legendre polynomials on [0, 1]
  * level n >= 1:  v^j_{p,n}(x) = 2^{n/2} f_p(2^n x - (2j+1)),
    j = 0 .. 2^{n-1}-1, with f_p Alpert's orthonormal multiwavelets on (-1, 1)
                                                                     (eq. sp9)
Eq. sp9 as printed has "2^l x"; the only reading under which the printed
prefactor 2^{n/2} makes the functions orthonormal and the supports match
j = 0 .. 2^{n-1}-1 is 2^n x, which is used here.

Alpert's wavelets are fixed by their vanishing moments: f_p (p = 0 .. k) is
orthogonal to x^i for i = 0 .. p+k and to f_{p+1} .. f_k, which leaves one
direction; the sign is chosen so that the first right-half Legendre
coefficient of magnitude above 1e-8, scanned from degree k down, is positive.

One-dimensional hierarchical index a in [0, (k+1) 2^N): level 0 occupies
a in [0, k+1) (a = p); level n >= 1 occupies [(k+1) 2^{n-1}, (k+1) 2^n) with
a = (k+1) 2^{n-1} + j (k+1) + p.
"""
import numpy as np
from numpy.polynomial import legendre as npleg


def gauss_legendre(q):
    """q-point Gauss-Legendre nodes and weights on [-1, 1] (weights sum to 2)."""
    return npleg.leggauss(q)


def legendre_table(k, t):
    """P_r(t) for r = 0..k; shape (len(t), k+1)."""
    return npleg.legvander(np.asarray(t, dtype=np.float64), k)


def legendre_deriv_table(k, t):
    """P_r'(t) for r = 0..k; shape (len(t), k+1)."""
    t = np.asarray(t, dtype=np.float64)
    out = np.zeros((t.size, k + 1))
    for r in range(k + 1):
        c = np.zeros(k + 1)
        c[r] = 1.0
        out[:, r] = npleg.legval(t, npleg.legder(c)) if r > 0 else 0.0
    return out


def alpert_coefficients(k):
    """Alpert multiwavelets f_0..f_k on (-1, 1) (Section 2.1, eq. sp9).

    Returns an array c of shape (k+1, 2(k+1)).  Row p holds the coefficients
    of f_p in the orthonormal basis of piecewise polynomials on (-1, 1):
      columns 0..k    : sqrt(2r+1) P_r(2y+1) on (-1, 0), zero on (0, 1)
      columns k+1..2k+1: sqrt(2r+1) P_r(2y-1) on (0, 1), zero on (-1, 0)
    Because that basis is orthonormal on (-1, 1), inner products of wavelets
    are dot products of these rows.
    """
    nq = 2 * k + 6
    xi, w = gauss_legendre(nq)
    y_left, y_right, wh = (xi - 1.0) / 2.0, (xi + 1.0) / 2.0, w / 2.0
    scale = np.sqrt(2.0 * np.arange(k + 1) + 1.0)
    psi_left = legendre_table(k, 2.0 * y_left + 1.0) * scale
    psi_right = legendre_table(k, 2.0 * y_right - 1.0) * scale
    # moments m_i(psi_b) = int_{-1}^{1} y^i psi_b(y) dy, exact by quadrature
    mom = np.zeros((2 * k + 2, 2 * (k + 1)))
    for i in range(2 * k + 2):
        mom[i, : k + 1] = (wh * y_left ** i) @ psi_left
        mom[i, k + 1:] = (wh * y_right ** i) @ psi_right
    f = np.zeros((k + 1, 2 * (k + 1)))
    for p in range(k, -1, -1):
        constraints = np.vstack([mom[: p + k + 1]] + [f[pp][None, :] for pp in range(p + 1, k + 1)])
        _, _, vt = np.linalg.svd(constraints)
        c = vt[-1].copy()
        for r in range(k, -1, -1):
            if abs(c[k + 1 + r]) > 1e-8:
                if c[k + 1 + r] < 0:
                    c = -c
                break
        f[p] = c
    return f


def alpert_eval(k, coeffs, y, half):
    """Values and derivatives of f_0..f_k at y on the given half.

    half = 0 selects the (-1, 0) piece, half = 1 the (0, 1) piece (so one-sided
    limits at y = 0 are well defined).  Returns (values, derivs), each of shape
    (len(y), k+1).
    """
    y = np.asarray(y, dtype=np.float64)
    half = np.broadcast_to(np.asarray(half), y.shape)
    scale = np.sqrt(2.0 * np.arange(k + 1) + 1.0)
    t = np.where(half == 0, 2.0 * y + 1.0, 2.0 * y - 1.0)
    P = legendre_table(k, t) * scale
    dP = legendre_deriv_table(k, t) * scale * 2.0
    cl, cr = coeffs[:, : k + 1], coeffs[:, k + 1:]
    vals = np.where(half[:, None] == 0, P @ cl.T, P @ cr.T)
    ders = np.where(half[:, None] == 0, dP @ cl.T, dP @ cr.T)
    return vals, ders


def hier_size(N, k):
    """Dimension of V_N^k in 1D: (k+1) 2^N (eq. sp8)."""
    return (k + 1) * (1 << N)


def hier_level_offset(n, k):
    """First 1D hierarchical index of level n."""
    return 0 if n == 0 else (k + 1) * (1 << (n - 1))


def hier_level_count(n, k):
    """Number of 1D functions on level n: (k+1) max(1, 2^{n-1})."""
    return (k + 1) * (1 if n == 0 else (1 << (n - 1)))


def hier_decode(N, k):
    """Arrays (level, j, p) for every 1D hierarchical index a < (k+1) 2^N."""
    H = hier_size(N, k)
    level = np.zeros(H, dtype=np.int64)
    j = np.zeros(H, dtype=np.int64)
    p = np.zeros(H, dtype=np.int64)
    for n in range(N + 1):
        o, c = hier_level_offset(n, k), hier_level_count(n, k)
        t = np.arange(c)
        level[o:o + c] = n
        j[o:o + c] = t // (k + 1)
        p[o:o + c] = t % (k + 1)
    return level, j, p


def hier_eval(N, k, cell, xi, alpert=None):
    """Evaluate all 1D hierarchical basis functions of V_N^k.

    Points are given per finest cell: x = (cell + (xi + 1)/2) h, h = 2^-N, with
    xi in [-1, 1]; the function pieces are those of the given finest cell, so
    xi = -1 / +1 yield the one-sided traces from inside that cell.
    Returns (values, derivatives), shape (len(cell), (k+1) 2^N).
    """
    if alpert is None:
        alpert = alpert_coefficients(k)
    cell = np.asarray(cell, dtype=np.int64)
    xi = np.asarray(xi, dtype=np.float64)
    h = 2.0 ** (-N)
    x = (cell + (xi + 1.0) / 2.0) * h
    H = hier_size(N, k)
    vals = np.zeros((cell.size, H))
    ders = np.zeros((cell.size, H))
    # level 0: phi_p(x) = sqrt(2p+1) P_p(2x - 1)
    scale = np.sqrt(2.0 * np.arange(k + 1) + 1.0)
    vals[:, : k + 1] = legendre_table(k, 2.0 * x - 1.0) * scale
    ders[:, : k + 1] = legendre_deriv_table(k, 2.0 * x - 1.0) * scale * 2.0
    for n in range(1, N + 1):
        o = hier_level_offset(n, k)
        j = cell >> (N - n + 1)                 # support cell at level n-1
        half = (cell >> (N - n)) & 1            # which level-n half of it
        y = (2.0 ** n) * x - (2 * j + 1)
        fv, fd = alpert_eval(k, alpert, y, half)
        amp = 2.0 ** (n / 2.0)
        rows = np.arange(cell.size)
        for p in range(k + 1):
            cols = o + j * (k + 1) + p
            vals[rows, cols] = amp * fv[:, p]
            ders[rows, cols] = amp * (2.0 ** n) * fd[:, p]
    return vals, ders


def finest_legendre_transform(N, k, alpert=None):
    """Matrix T with T[c(k+1)+r, a] = int_{I_N^c} v_a(x) L_{c,r}(x) dx.

    L_{c,r} is the orthonormal Legendre basis of the finest cell c,
    h^{-1/2} sqrt(2r+1) P_r(2(x - x_c)/h - 1).  Every v_a lies in V_N^k, so
    T maps hierarchical coefficients to finest-mesh Legendre coefficients
    exactly; (k+1)-point Gauss quadrature integrates the degree-2k product.
    """
    H = hier_size(N, k)
    ncell = 1 << N
    h = 2.0 ** (-N)
    xi, w = gauss_legendre(k + 1)
    cells = np.repeat(np.arange(ncell), k + 1)
    xis = np.tile(xi, ncell)
    vals, _ = hier_eval(N, k, cells, xis, alpert)
    scale = np.sqrt(2.0 * np.arange(k + 1) + 1.0)
    Lg = legendre_table(k, xi) * scale / np.sqrt(h)          # (q, k+1)
    T = np.zeros((H, H))
    for c in range(ncell):
        rows = slice(c * (k + 1), (c + 1) * (k + 1))
        pts = slice(c * (k + 1), (c + 1) * (k + 1))
        T[rows, :] = (Lg * (h * w / 2.0)[:, None]).T @ vals[pts, :]
    return T
