// One-time host construction of the 1D tables of the sparse-grid DG method:
// Gauss-Legendre rules, Alpert multiwavelets, the change of basis T from the
// 1D hierarchical basis of V_N^k to the finest-cell Legendre basis, and the
// 1D SIPG matrix in the hierarchical basis (Section 2.1).  These run once per
// index set / operator, before the time loop (Section 4: the 1D integrals are
// computed once before the time evolution).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "sgk_internal.h"

typedef long double ld;

namespace {

// P_0..P_k and P_0'..P_k' at t by the three-term recurrence.
void legendre_eval(int k, ld t, ld* P, ld* dP) {
    P[0] = 1;
    dP[0] = 0;
    if (k >= 1) {
        P[1] = t;
        dP[1] = 1;
    }
    for (int r = 1; r < k; ++r) {
        P[r + 1] = ((2 * r + 1) * t * P[r] - r * P[r - 1]) / (r + 1);
        dP[r + 1] = dP[r - 1] + (2 * r + 1) * P[r];
    }
}

void gauss_legendre_ld(int q, std::vector<ld>& x, std::vector<ld>& w) {
    x.assign(q, 0);
    w.assign(q, 0);
    const ld pi = 3.141592653589793238462643383279502884L;
    for (int i = 0; i < q; ++i) {
        ld z = std::cos(pi * (i + 0.75L) / (q + 0.5L));
        for (int it = 0; it < 100; ++it) {
            ld p0 = 1, p1 = z;
            for (int r = 1; r < q; ++r) {
                ld p2 = ((2 * r + 1) * z * p1 - r * p0) / (r + 1);
                p0 = p1;
                p1 = p2;
            }
            ld pq = (q == 0) ? 1 : (q == 1 ? z : p1);
            if (q == 1) p0 = 1;
            ld dp = q * (z * pq - p0) / (z * z - 1);
            ld dz = pq / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-19L) break;
        }
        ld p0 = 1, p1 = z;
        for (int r = 1; r < q; ++r) {
            ld p2 = ((2 * r + 1) * z * p1 - r * p0) / (r + 1);
            p0 = p1;
            p1 = p2;
        }
        ld pq = (q == 1) ? z : p1;
        if (q == 1) p0 = 1;
        ld dp = q * (z * pq - p0) / (z * z - 1);
        x[q - 1 - i] = z;
        w[q - 1 - i] = 2 / ((1 - z * z) * dp * dp);
    }
}

// Value of the hierarchical function (level n, cell j, degree p) of V_N^k at
// x = (cell + (xi+1)/2) h on the piece belonging to finest cell `cell`.
ld hier_value(int N, int k, const std::vector<ld>& alp, int n, int j, int p, int cell, ld xi) {
    std::vector<ld> P(k + 1), dP(k + 1);
    ld h = std::ldexp((ld)1, -N);
    ld x = (cell + (xi + 1) / 2) * h;
    if (n == 0) {
        legendre_eval(k, 2 * x - 1, P.data(), dP.data());
        return std::sqrt((ld)(2 * p + 1)) * P[p];
    }
    int half = (cell >> (N - n)) & 1;
    ld y = std::ldexp(x, n) - (2 * j + 1);
    ld t = half == 0 ? 2 * y + 1 : 2 * y - 1;
    legendre_eval(k, t, P.data(), dP.data());
    ld v = 0;
    for (int r = 0; r <= k; ++r) v += alp[p * 2 * (k + 1) + half * (k + 1) + r] * std::sqrt((ld)(2 * r + 1)) * P[r];
    return std::ldexp(v, 0) * std::pow((ld)2, (ld)n / 2);
}

std::vector<ld> alpert_ld(int k) {
    const int m = 2 * (k + 1);
    const int nq = 2 * k + 6;
    std::vector<ld> xi, w;
    gauss_legendre_ld(nq, xi, w);
    // moments of the piecewise Legendre basis: mom[i][b] = int y^i psi_b
    std::vector<ld> mom((2 * k + 2) * m, 0);
    std::vector<ld> P(k + 1), dP(k + 1);
    for (int g = 0; g < nq; ++g) {
        for (int half = 0; half < 2; ++half) {
            ld y = half == 0 ? (xi[g] - 1) / 2 : (xi[g] + 1) / 2;
            ld t = half == 0 ? 2 * y + 1 : 2 * y - 1;
            legendre_eval(k, t, P.data(), dP.data());
            ld yi = 1;
            for (int i = 0; i < 2 * k + 2; ++i) {
                for (int r = 0; r <= k; ++r)
                    mom[i * m + half * (k + 1) + r] += w[g] / 2 * yi * std::sqrt((ld)(2 * r + 1)) * P[r];
                yi *= y;
            }
        }
    }
    std::vector<ld> f((k + 1) * m, 0);
    for (int p = k; p >= 0; --p) {
        // constraints: moments 0..p+k and the wavelets already fixed
        std::vector<std::vector<ld>> rows;
        for (int i = 0; i <= p + k; ++i) rows.emplace_back(mom.begin() + i * m, mom.begin() + (i + 1) * m);
        for (int pp = p + 1; pp <= k; ++pp) rows.emplace_back(f.begin() + pp * m, f.begin() + (pp + 1) * m);
        // orthonormalise the constraint rows (modified Gram-Schmidt, twice)
        std::vector<std::vector<ld>> Q;
        for (auto r : rows) {
            for (int pass = 0; pass < 2; ++pass)
                for (auto& q : Q) {
                    ld dot = 0;
                    for (int b = 0; b < m; ++b) dot += q[b] * r[b];
                    for (int b = 0; b < m; ++b) r[b] -= dot * q[b];
                }
            ld nrm = 0;
            for (int b = 0; b < m; ++b) nrm += r[b] * r[b];
            nrm = std::sqrt(nrm);
            if (nrm > 1e-14L) {
                for (int b = 0; b < m; ++b) r[b] /= nrm;
                Q.push_back(r);
            }
        }
        // the null direction: the unit vector with the largest remainder
        std::vector<ld> best;
        ld best_norm = -1;
        for (int e = 0; e < m; ++e) {
            std::vector<ld> v(m, 0);
            v[e] = 1;
            for (int pass = 0; pass < 2; ++pass)
                for (auto& q : Q) {
                    ld dot = 0;
                    for (int b = 0; b < m; ++b) dot += q[b] * v[b];
                    for (int b = 0; b < m; ++b) v[b] -= dot * q[b];
                }
            ld nrm = 0;
            for (int b = 0; b < m; ++b) nrm += v[b] * v[b];
            if (nrm > best_norm) {
                best_norm = nrm;
                best = v;
            }
        }
        ld nrm = std::sqrt(best_norm);
        for (int b = 0; b < m; ++b) best[b] /= nrm;
        for (int r = k; r >= 0; --r) {
            ld c = best[(k + 1) + r];
            if (std::fabs(c) > 1e-8L) {
                if (c < 0)
                    for (int b = 0; b < m; ++b) best[b] = -best[b];
                break;
            }
        }
        std::copy(best.begin(), best.end(), f.begin() + p * m);
    }
    return f;
}

}  // namespace

void gauss_legendre(int q, std::vector<double>& x, std::vector<double>& w) {
    std::vector<ld> xl, wl;
    gauss_legendre_ld(q, xl, wl);
    x.assign(xl.begin(), xl.end());
    w.assign(wl.begin(), wl.end());
}

std::vector<double> alpert_coefficients(int k) {
    std::vector<ld> f = alpert_ld(k);
    return std::vector<double>(f.begin(), f.end());
}

void Csr::upload(cudaStream_t s) {
    d_ptr.upload(ptr, s);
    d_col.upload(col, s);
    d_val.upload(val, s);
    std::vector<float> vf(val.begin(), val.end());
    d_valf.alloc(vf.size());
    d_valf.upload(vf.data(), vf.size(), s);
    // vf must outlive the async copy
    SGK_CUDA_CHECK(cudaStreamSynchronize(s));
}

void build_transform_tables(int N, int k, Tables1D& out) {
    const int kp1 = k + 1;
    const int ncell = 1 << N;
    const int H = kp1 * ncell;
    out.N = N;
    out.k = k;
    out.H = H;
    std::vector<ld> alp = alpert_ld(k);
    out.alpert.assign(alp.begin(), alp.end());
    std::vector<ld> xi, w;
    gauss_legendre_ld(kp1, xi, w);
    const ld h = std::ldexp((ld)1, -N);
    // Legendre basis of a finest cell at the Gauss points: h^{-1/2} sqrt(2r+1) P_r(xi)
    std::vector<ld> Lg(kp1 * kp1), P(kp1), dP(kp1);
    for (int g = 0; g < kp1; ++g) {
        legendre_eval(k, xi[g], P.data(), dP.data());
        for (int r = 0; r < kp1; ++r) Lg[g * kp1 + r] = std::sqrt((ld)(2 * r + 1)) * P[r] / std::sqrt(h);
    }
    Csr& T = out.T;
    T.rows = T.cols = H;
    T.ptr.assign(H + 1, 0);
    T.col.clear();
    T.val.clear();
    for (int c = 0; c < ncell; ++c) {
        for (int r = 0; r < kp1; ++r) {
            for (int n = 0; n <= N; ++n) {
                int j = n == 0 ? 0 : (c >> (N - n + 1));
                for (int p = 0; p < kp1; ++p) {
                    int a = level_offset(n, kp1) + j * kp1 + p;
                    ld acc = 0;
                    for (int g = 0; g < kp1; ++g)
                        acc += h * w[g] / 2 * hier_value(N, k, alp, n, j, p, c, xi[g]) * Lg[g * kp1 + r];
                    T.col.push_back(a);
                    T.val.push_back((double)acc);
                }
            }
            T.ptr[c * kp1 + r + 1] = (int)T.col.size();
        }
    }
    // two-scale filters on the reference parent [0,1] with children [0,1/2],
    // [1/2,1]: parent phi_r(x) = sqrt(2r+1) P_r(2x-1), child h phi^h_s(x) =
    // sqrt(2) sqrt(2s+1) P_s(4x-1-2h); the wavelets psi_p restricted to child
    // h have Legendre coefficients alpert[p][h (k+1) + s] (dilation invariance)
    {
        std::vector<ld> gx, gw;
        gauss_legendre_ld(kp1 + 1, gx, gw);
        out.two_scale.assign(4 * kp1 * kp1, 0.0);
        std::vector<ld> Pp(kp1), dPp(kp1), Pc(kp1), dPc(kp1);
        for (int h = 0; h < 2; ++h) {
            std::vector<ld> acc(kp1 * kp1, 0);
            for (int g = 0; g < kp1 + 1; ++g) {
                const ld x = (h + (gx[g] + 1) / 2) / 2;  // point in child h
                legendre_eval(k, 2 * x - 1, Pp.data(), dPp.data());
                legendre_eval(k, gx[g], Pc.data(), dPc.data());
                for (int r = 0; r < kp1; ++r)
                    for (int s = 0; s < kp1; ++s)
                        acc[r * kp1 + s] += gw[g] / 4 * std::sqrt((ld)(2 * r + 1)) * Pp[r] * std::sqrt((ld)2) *
                                            std::sqrt((ld)(2 * s + 1)) * Pc[s];
            }
            for (int i = 0; i < kp1 * kp1; ++i) out.two_scale[h * kp1 * kp1 + i] = (double)acc[i];
            for (int p = 0; p < kp1; ++p)
                for (int s = 0; s < kp1; ++s)
                    out.two_scale[(2 + h) * kp1 * kp1 + p * kp1 + s] = (double)alp[p * 2 * kp1 + h * kp1 + s];
        }
    }
    // transpose (columns stay sorted because rows are visited in order)
    Csr& Tt = out.Tt;
    Tt.rows = Tt.cols = H;
    Tt.ptr.assign(H + 1, 0);
    for (int e = 0; e < (int)T.col.size(); ++e) Tt.ptr[T.col[e] + 1]++;
    for (int a = 0; a < H; ++a) Tt.ptr[a + 1] += Tt.ptr[a];
    Tt.col.assign(T.col.size(), 0);
    Tt.val.assign(T.col.size(), 0);
    std::vector<int> fill(Tt.ptr.begin(), Tt.ptr.end() - 1);
    for (int y = 0; y < H; ++y)
        for (int e = T.ptr[y]; e < T.ptr[y + 1]; ++e) {
            int a = T.col[e];
            Tt.col[fill[a]] = y;
            Tt.val[fill[a]] = T.val[e];
            fill[a]++;
        }
}

std::vector<double> build_sipg_hier(const Tables1D& tab, int bc, double sigma) {
    // SIPG on the finest mesh in the cell-local orthonormal Legendre basis
    // (closed form), then rotated: S = T^T S_L T.
    const int k = tab.k, kp1 = k + 1, N = tab.N, H = tab.H;
    const int nc = 1 << N;
    const ld h = std::ldexp((ld)1, -N);
    std::vector<ld> vr(kp1), vl(kp1), dr(kp1), dl(kp1), vol(kp1 * kp1, 0);
    for (int r = 0; r < kp1; ++r) {
        ld s = std::sqrt((ld)(2 * r + 1)) / std::sqrt(h);
        ld sgn = (r % 2 == 0) ? 1 : -1;
        vr[r] = s;
        vl[r] = s * sgn;
        dr[r] = (2 / h) * s * r * (r + 1) / 2;
        dl[r] = -(2 / h) * s * sgn * r * (r + 1) / 2;
    }
    for (int a = 0; a < kp1; ++a)
        for (int b = 0; b < kp1; ++b)
            if ((a + b) % 2 == 0) {
                int m = std::min(a, b);
                vol[a * kp1 + b] = (2 / (h * h)) * std::sqrt((ld)(2 * a + 1)) * std::sqrt((ld)(2 * b + 1)) * m * (m + 1);
            }
    // S_L as a dense-row map: rows y, entries among 3 neighbouring cells
    std::vector<std::vector<std::pair<int, ld>>> SL(H);
    auto add = [&](int y, int y2, ld v) {
        for (auto& e : SL[y])
            if (e.first == y2) { e.second += v; return; }
        SL[y].push_back({y2, v});
    };
    for (int c = 0; c < nc; ++c)
        for (int a = 0; a < kp1; ++a)
            for (int b = 0; b < kp1; ++b)
                if (vol[a * kp1 + b] != 0) add(c * kp1 + a, c * kp1 + b, vol[a * kp1 + b]);
    const int nfaces = bc == SGK_PERIODIC ? nc : nc + 1;
    for (int f = 0; f < nfaces; ++f) {
        std::vector<std::pair<int, ld>> J, G;
        bool interior = bc == SGK_PERIODIC || (f > 0 && f < nc);
        if (interior) {
            int L = (f - 1 + nc) % nc, R = f % nc;
            for (int r = 0; r < kp1; ++r) {
                J.push_back({L * kp1 + r, vr[r]});
                G.push_back({L * kp1 + r, dr[r] / 2});
            }
            for (int r = 0; r < kp1; ++r) {
                J.push_back({R * kp1 + r, -vl[r]});
                G.push_back({R * kp1 + r, dl[r] / 2});
            }
        } else if (f == 0) {
            for (int r = 0; r < kp1; ++r) {
                J.push_back({r, -vl[r]});
                G.push_back({r, dl[r]});
            }
        } else {
            int L = nc - 1;
            for (int r = 0; r < kp1; ++r) {
                J.push_back({L * kp1 + r, vr[r]});
                G.push_back({L * kp1 + r, dr[r]});
            }
        }
        // periodic with nc == 1: both traces belong to the same cell; merge
        for (auto& a : J)
            for (auto& b : J) add(a.first, b.first, (ld)sigma / h * a.second * b.second);
        for (auto& a : G)
            for (auto& b : J) {
                add(a.first, b.first, -a.second * b.second);
                add(b.first, a.first, -a.second * b.second);
            }
    }
    // Z = S_L T (rows y), then S = T^T Z accumulated row by row
    const Csr& T = tab.T;
    const Csr& Tt = tab.Tt;
    std::vector<std::vector<std::pair<int, ld>>> Z(H);
    std::vector<ld> acc(H, 0);
    std::vector<int> touched;
    std::vector<char> mark(H, 0);
    for (int y = 0; y < H; ++y) {
        touched.clear();
        for (auto& e : SL[y])
            for (int q = T.ptr[e.first]; q < T.ptr[e.first + 1]; ++q) {
                int b = T.col[q];
                if (!mark[b]) { mark[b] = 1; touched.push_back(b); }
                acc[b] += e.second * (ld)T.val[q];
            }
        for (int b : touched) {
            Z[y].push_back({b, acc[b]});
            acc[b] = 0;
            mark[b] = 0;
        }
    }
    std::vector<double> S((size_t)H * H, 0.0);
    for (int a = 0; a < H; ++a) {
        touched.clear();
        for (int q = Tt.ptr[a]; q < Tt.ptr[a + 1]; ++q) {
            int y = Tt.col[q];
            ld t = Tt.val[q];
            for (auto& e : Z[y]) {
                if (!mark[e.first]) { mark[e.first] = 1; touched.push_back(e.first); }
                acc[e.first] += t * e.second;
            }
        }
        for (int b : touched) {
            S[(size_t)a * H + b] = (double)acc[b];
            acc[b] = 0;
            mark[b] = 0;
        }
    }
    // symmetrise (exact in exact arithmetic) and drop entries that vanish by
    // orthogonality but carry rounding residue
    for (int a = 0; a < H; ++a)
        for (int b = a + 1; b < H; ++b) {
            double m = 0.5 * (S[(size_t)a * H + b] + S[(size_t)b * H + a]);
            S[(size_t)a * H + b] = S[(size_t)b * H + a] = m;
        }
    // (relative to the two diagonal entries, with a floor of 1e-14 of the
    // largest diagonal entry for rows whose own diagonal vanishes: the
    // constant mode under periodic conditions)
    double dmax = 0.0;
    for (int a = 0; a < H; ++a) dmax = std::max(dmax, std::fabs(S[(size_t)a * H + a]));
    for (int a = 0; a < H; ++a)
        for (int b = 0; b < H; ++b) {
            double scale = std::sqrt(std::fabs(S[(size_t)a * H + a]) * std::fabs(S[(size_t)b * H + b]));
            if (std::fabs(S[(size_t)a * H + b]) <= std::max(1e-12 * scale, 1e-14 * dmax)) S[(size_t)a * H + b] = 0.0;
        }
    return S;
}

namespace {

// A = T^T A_L T for a matrix A_L given by rows over the finest-cell Legendre
// index (dense H x H output, rows and columns hierarchical).
std::vector<double> rotate_dense(const Tables1D& tab, const std::vector<std::vector<std::pair<int, ld>>>& AL) {
    const int H = tab.H;
    std::vector<ld> Z((size_t)H * H, 0);  // A_L T
    for (int y = 0; y < H; ++y)
        for (auto& e : AL[y])
            for (int q = tab.T.ptr[e.first]; q < tab.T.ptr[e.first + 1]; ++q)
                Z[(size_t)y * H + tab.T.col[q]] += e.second * (ld)tab.T.val[q];
    std::vector<double> out((size_t)H * H, 0.0);
    std::vector<ld> acc(H);
    for (int a = 0; a < H; ++a) {
        std::fill(acc.begin(), acc.end(), (ld)0);
        for (int q = tab.Tt.ptr[a]; q < tab.Tt.ptr[a + 1]; ++q) {
            const ld t = tab.Tt.val[q];
            const ld* z = &Z[(size_t)tab.Tt.col[q] * H];
            for (int b = 0; b < H; ++b) acc[b] += t * z[b];
        }
        for (int b = 0; b < H; ++b) out[(size_t)a * H + b] = (double)acc[b];
    }
    return out;
}

}  // namespace

void build_cross_hier(const Tables1D& tab, int bc, std::vector<double>& P, std::vector<double>& E) {
    // Finest-cell Legendre basis L_r = h^{-1/2} sqrt(2r+1) P_r(xi):
    // int L_a' L_b over a cell = 2 sqrt((2a+1)(2b+1)) / h for b < a with a + b
    // odd (int_{-1}^{1} P_a' P_b = 2 there, 0 otherwise); traces at the right
    // and left cell ends h^{-1/2} sqrt(2r+1) and (-1)^r times that.
    const int k = tab.k, kp1 = k + 1, N = tab.N, H = tab.H;
    const int nc = 1 << N;
    const ld h = std::ldexp((ld)1, -N);
    std::vector<ld> vr(kp1), vl(kp1);
    for (int r = 0; r < kp1; ++r) {
        vr[r] = std::sqrt((ld)(2 * r + 1)) / std::sqrt(h);
        vl[r] = (r % 2 == 0) ? vr[r] : -vr[r];
    }
    std::vector<std::vector<std::pair<int, ld>>> PL(H), EL(H);
    for (int c = 0; c < nc; ++c)
        for (int a = 0; a < kp1; ++a)
            for (int b = 0; b < a; ++b)
                if ((a + b) % 2 == 1)
                    PL[c * kp1 + a].push_back(
                        {c * kp1 + b, 2 * std::sqrt((ld)(2 * a + 1)) * std::sqrt((ld)(2 * b + 1)) / h});
    // faces: jump of the test function (left trace minus right trace) against
    // the average of the trial traces; one-sided with the outward normal on
    // zero-Dirichlet boundary faces
    const int nfaces = bc == SGK_PERIODIC ? nc : nc + 1;
    for (int f = 0; f < nfaces; ++f) {
        std::vector<std::pair<int, ld>> J, A;
        const bool interior = bc == SGK_PERIODIC || (f > 0 && f < nc);
        if (interior) {
            const int L = (f - 1 + nc) % nc, R = f % nc;
            for (int r = 0; r < kp1; ++r) {
                J.push_back({L * kp1 + r, vr[r]});
                A.push_back({L * kp1 + r, vr[r] / 2});
            }
            for (int r = 0; r < kp1; ++r) {
                J.push_back({R * kp1 + r, -vl[r]});
                A.push_back({R * kp1 + r, vl[r] / 2});
            }
        } else if (f == 0) {
            for (int r = 0; r < kp1; ++r) {
                J.push_back({r, -vl[r]});
                A.push_back({r, vl[r]});
            }
        } else {
            for (int r = 0; r < kp1; ++r) {
                J.push_back({(nc - 1) * kp1 + r, vr[r]});
                A.push_back({(nc - 1) * kp1 + r, vr[r]});
            }
        }
        // periodic with nc == 1: both sides are the same cell, so entries add
        for (auto& a : J)
            for (auto& b : A) {
                bool merged = false;
                for (auto& e : EL[a.first])
                    if (e.first == b.first) {
                        e.second += a.second * b.second;
                        merged = true;
                        break;
                    }
                if (!merged) EL[a.first].push_back({b.first, a.second * b.second});
            }
    }
    P = rotate_dense(tab, PL);
    E = rotate_dense(tab, EL);
}

// ------------------------------------------------------------------------
// 1D factors of the collocation matrix of the sparse-grid interpolation form
// of the reaction term.  This form is not the paper's F: it serves its first
// stated future direction (Section 5, evaluating the reaction integral with
// the structure of the basis instead of at the finest-mesh Gauss points).
//
// Degree k uses the k+1 points X_0 = {1/3, 2/3}, {0, 1/3, 2/3} or
// {1/5, 2/5, 3/5, 4/5} of [0, 1); each set is mapped into itself by
// x -> 2x mod 1, so the point sets X_n of the levels (X_0 copied into every
// level-n cell) are nested.  The 1D hierarchical index (n, j, p) of level
// n >= 1 carries the p-th (sorted) point of X_n \ X_{n-1} inside the
// level-(n-1) cell j; level 0 carries X_0.  A point on a cell edge belongs to
// the cell on its right.  ell_q is the degree-k Lagrange polynomial through
// the X_n points of the level-n cell of q (n = level of q), 1 at q, zero
// outside that cell.  With E[p][a] = v_a(x_p) and B[p][q] = ell_q(x_p):
//   A    = B^{-1} E : Alpert coefficients -> interpolation surpluses,
//                     A[p][a] = v_a(x_p) - (I_{n-1} v_a)(x_p) for p on level
//                     n >= 1 (I_{n-1}: interpolation on the level-(n-1)
//                     cell of x_p), v_a(x_p) on level 0;
//   B             : surpluses -> point values;
//   B^{-1}        : s_p = g_p - sum_t L_t(x_p) g(z_t), z_t the X_{n-1}
//                     points of the level-(n-1) cell of x_p;
//   A^{-1}        : surpluses -> Alpert coefficients, A^{-1}[a][q] =
//                     int ell_q v_a (the Alpert basis is orthonormal).
// Every entry is formed from these local formulas in long double (not by
// inverting matrices); only the entries the supports and levels allow are
// stored.  A and A^{-1} map a level to the same or coarser levels, B and
// B^{-1} to the same or finer ones.
// ------------------------------------------------------------------------

namespace {

struct InterpGeometry {
    int N = 0, k = 0, kp1 = 0, H = 0;
    int den = 1, D = 2;           // X_0 = {num_t / den}; integer point keys over D 2^N
    std::vector<int> x0num;       // numerators of X_0 over den
    std::vector<int> newnum;      // numerators of the new points of a level over D (local to the parent cell)
    std::vector<int> lev, jj, pp;  // per 1D index
    std::vector<int64_t> key;     // x 2^N D (an integer for every point of level <= N)
    std::vector<int> of_key;      // inverse of key, -1 where no point
    std::vector<ld> alp;

    void build(int N_, int k_) {
        N = N_;
        k = k_;
        kp1 = k + 1;
        H = kp1 << N;
        static const int nums[4][4] = {{0}, {1, 2}, {0, 1, 2}, {1, 2, 3, 4}};
        static const int dens[4] = {1, 3, 3, 5};
        den = dens[k];
        D = 2 * den;
        x0num.assign(nums[k], nums[k] + kp1);
        // both halves' copies of X_0, over D: x/2 -> num, 1/2 + x/2 -> den + num
        newnum.clear();
        for (int h = 0; h < 2; ++h)
            for (int t = 0; t < kp1; ++t) {
                const int c = h * den + x0num[t];
                bool old = false;
                for (int r = 0; r < kp1; ++r) old = old || c == 2 * x0num[r];
                if (!old) newnum.push_back(c);
            }
        std::sort(newnum.begin(), newnum.end());
        SGK_REQUIRE((int)newnum.size() == kp1, SGK_EINVAL, "interp: collocation points are not nested");
        lev.assign(H, 0);
        jj.assign(H, 0);
        pp.assign(H, 0);
        key.assign(H, 0);
        of_key.assign((size_t)D << N, -1);
        for (int a = 0; a < H; ++a) {
            int n = 0;
            while (a >= level_offset(n, kp1) + level_count(n, kp1)) ++n;
            const int t = a - level_offset(n, kp1);
            lev[a] = n;
            jj[a] = t / kp1;
            pp[a] = t % kp1;
            key[a] = n == 0 ? (int64_t)(2 * x0num[pp[a]]) << N
                            : ((int64_t)jj[a] * D + newnum[pp[a]]) << (N + 1 - n);
            SGK_REQUIRE(key[a] >= 0 && key[a] < ((int64_t)D << N), SGK_EINVAL, "interp: point outside [0, 1)");
            SGK_REQUIRE(of_key[key[a]] < 0, SGK_EINVAL, "interp: two indices share a point");
            of_key[key[a]] = a;
        }
        alp = alpert_ld(k);
    }
    // level-m cell of the point with key X (the cell on the right at an edge)
    int64_t cell(int64_t X, int m) const { return X / ((int64_t)D << (N - m)); }
    // key of the t-th X_0 point of the level-m cell c
    int64_t node(int m, int64_t c, int t) const { return (c * D + 2 * x0num[t]) << (N - m); }
    // L_t at the local coordinate s in [0, 1) of a cell (nodes: X_0)
    ld lagrange_local(int t, ld s) const {
        ld v = 1;
        for (int r = 0; r < kp1; ++r)
            if (r != t) v *= (s - (ld)(2 * x0num[r]) / D) / ((ld)(2 * x0num[t] - 2 * x0num[r]) / D);
        return v;
    }
    // L_t(x) of the level-m cell c, x given by its key
    ld lagrange(int m, int64_t c, int t, int64_t X) const {
        const ld scale = std::ldexp((ld)D, N - m);
        return lagrange_local(t, ((ld)X - (ld)c * scale) / scale);
    }
    // index of the X_0 node of a point's own cell
    int node_index(int a) const {
        const int m = lev[a];
        const int64_t c = cell(key[a], m);
        for (int t = 0; t < kp1; ++t)
            if (node(m, c, t) == key[a]) return t;
        throw SgkError{SGK_EINVAL, "interp: point is not a node of its cell"};
    }
    // v_a at a point given by its key (zero outside the support)
    ld alpert_at_key(int a, int64_t X) const {
        const int64_t fc = X / D;
        if (lev[a] > 0 && (fc >> (N - lev[a] + 1)) != jj[a]) return 0;
        const ld xi = 2 * (ld)(X - fc * D) / D - 1;
        return hier_value(N, k, alp, lev[a], jj[a], pp[a], (int)fc, xi);
    }
    // v_a at an interior point x (long double coordinate)
    ld alpert_at_x(int a, ld x) const {
        const ld s = std::ldexp(x, N);
        const int fc = std::min((int)std::floor(s), (1 << N) - 1);
        if (lev[a] > 0 && (fc >> (N - lev[a] + 1)) != jj[a]) return 0;
        return hier_value(N, k, alp, lev[a], jj[a], pp[a], fc, 2 * (s - fc) - 1);
    }
};

void finish_csr(int H, std::vector<std::vector<std::pair<int, ld>>>& rows, Csr& out) {
    out.rows = out.cols = H;
    out.ptr.assign(1, 0);
    out.col.clear();
    out.val.clear();
    for (int r = 0; r < H; ++r) {
        std::sort(rows[r].begin(), rows[r].end(),
                  [](const std::pair<int, ld>& a, const std::pair<int, ld>& b) { return a.first < b.first; });
        for (size_t e = 0; e < rows[r].size(); ++e) {
            SGK_REQUIRE(e == 0 || rows[r][e].first != rows[r][e - 1].first, SGK_EINVAL, "interp: duplicate entry");
            out.col.push_back(rows[r][e].first);
            out.val.push_back((double)rows[r][e].second);
        }
        out.ptr.push_back((int)out.col.size());
    }
}

}  // namespace

void build_interp_factors(int N, int k, InterpFactors1D& out) {
    InterpGeometry g;
    g.build(N, k);
    const int H = g.H, kp1 = g.kp1;
    std::vector<std::vector<std::pair<int, ld>>> rA(H), rB(H), rBi(H), rAi(H);
    // the new points of level m inside the level-(m-1) cell J (m >= 1), or
    // the points of level 0
    auto level_points = [&](int m, int64_t J, std::vector<int>& q) {
        q.clear();
        for (int r = 0; r < kp1; ++r) q.push_back(m == 0 ? r : level_offset(m, kp1) + (int)J * kp1 + r);
    };
    std::vector<int> qs;
    for (int p = 0; p < H; ++p) {
        const int mp = g.lev[p];
        const int64_t X = g.key[p];
        // B and B^{-1}
        rB[p].push_back({p, 1});
        rBi[p].push_back({p, 1});
        for (int m = 0; m < mp; ++m) {
            const int64_t c = g.cell(X, m);
            level_points(m, m == 0 ? 0 : c >> 1, qs);
            for (int q : qs)
                if (g.cell(g.key[q], m) == c) rB[p].push_back({q, g.lagrange(m, c, g.node_index(q), X)});
        }
        if (mp >= 1) {
            const int64_t J = g.cell(X, mp - 1);
            for (int t = 0; t < kp1; ++t) {
                const int64_t Z = g.node(mp - 1, J, t);
                const int z = g.of_key[Z];
                SGK_REQUIRE(z >= 0 && g.lev[z] <= mp - 1, SGK_EINVAL, "interp: coarse node missing");
                rBi[p].push_back({z, -g.lagrange(mp - 1, J, t, X)});
            }
        }
        // A: v_a(x_p) - (I_{mp-1} v_a)(x_p) over the functions a of level >=
        // mp whose support lies in the level-(mp-1) cell of x_p
        if (mp == 0) {
            for (int a = 0; a < H; ++a)
                if (g.lev[a] == 0 || (X / g.D >> (N - g.lev[a] + 1)) == g.jj[a])
                    rA[p].push_back({a, g.alpert_at_key(a, X)});
        } else {
            const int64_t J = g.cell(X, mp - 1);
            ld Lt[4];
            int64_t Zt[4];
            for (int t = 0; t < kp1; ++t) {
                Zt[t] = g.node(mp - 1, J, t);
                Lt[t] = g.lagrange(mp - 1, J, t, X);
            }
            for (int l = mp; l <= N; ++l)
                for (int64_t ja = J << (l - mp); ja < (J + 1) << (l - mp); ++ja)
                    for (int r = 0; r < kp1; ++r) {
                        const int a = level_offset(l, kp1) + (int)ja * kp1 + r;
                        ld v = g.alpert_at_key(a, X);
                        for (int t = 0; t < kp1; ++t) v -= Lt[t] * g.alpert_at_key(a, Zt[t]);
                        rA[p].push_back({a, v});
                    }
        }
    }
    // A^{-1}[a][q] = int ell_q v_a over the cell of q, for q of level >=
    // level(a) inside the support of v_a (Gauss rule with k + 2 points:
    // exact for the degree-2k product)
    std::vector<ld> gx, gw;
    gauss_legendre_ld(kp1 + 1, gx, gw);
    for (int a = 0; a < H; ++a) {
        const int l = g.lev[a];
        for (int m = l; m <= N; ++m) {
            // parents (level m - 1) of the level-m points inside the support
            int64_t J0 = 0, J1 = 1;
            if (m >= 1) {
                if (l == 0) {
                    J0 = 0;
                    J1 = (int64_t)1 << (m - 1);
                } else {
                    J0 = (int64_t)g.jj[a] << (m - l);
                    J1 = (int64_t)(g.jj[a] + 1) << (m - l);
                }
            }
            for (int64_t J = J0; J < J1; ++J) {
                level_points(m, J, qs);
                for (int q : qs) {
                    const int64_t c = g.cell(g.key[q], m);
                    const int t = g.node_index(q);
                    const ld h = std::ldexp((ld)1, -m);
                    ld acc = 0;
                    for (size_t e = 0; e < gx.size(); ++e) {
                        const ld s = (gx[e] + 1) / 2;
                        acc += gw[e] * g.lagrange_local(t, s) * g.alpert_at_x(a, (c + s) * h);
                    }
                    rAi[a].push_back({q, acc * h / 2});
                }
            }
        }
    }
    finish_csr(H, rA, out.A);
    finish_csr(H, rB, out.B);
    finish_csr(H, rBi, out.Binv);
    finish_csr(H, rAi, out.Ainv);
}
