// Gather form of the sparse-grid matvec (Section 4, unidirectional
// principle): the per-output device routine shared by the matvec kernel and
// the persistent Arnoldi kernel.
//
// A group of G lanes owns one coefficient y_g of block l (local multi-index
// c, 1D hierarchical index a_i = off(l_i) + c_i along direction i).  For
// each direction i the group walks row a_i of the 1D hierarchical SIPG
// matrix truncated to the levels lb <= N' = N - sum_{m!=i} l_m, and gathers
// x at the coefficient of block (l with l_i = lb) that shares the other
// local indices c_m (m != i).  The entries of a row are stored sorted by
// column, each packed as (lb, position within level lb), so the source block
// offset comes from a small per-(tuple, direction) table and the address is
// base + (o n_lb + p) I + in, with o the row-major index of c_0..c_{i-1} and
// in that of c_{i+1}..c_{d-1} (I their extent).  Lane r of the group takes
// entries r, r + G, ... of every row; the caller combines the lanes.
#pragma once
#include "sgk_df64.h"
#include "sgk_internal.h"

template <typename T, int D>
struct GmvArgs {
    int64_t n;
    int N;
    const int64_t* __restrict__ offsets;  // ntuples + 1
    const int32_t* __restrict__ levels;   // ntuples x D
    const int32_t* __restrict__ chunk;    // tuple holding element c * 256, c <= ceil(n / 256)
    const int64_t* __restrict__ cb;       // ntuples x D x (N + 1) block offsets
    const int32_t* __restrict__ rp;       // H + 1
    const int32_t* __restrict__ rlen;     // H x (N + 1)
    const int32_t* __restrict__ ce;       // packed (lb << 16) | p
    const T* __restrict__ cvk;  // -kappa_i S_q, direction i at cvk + i nnz
    int64_t nnz;
};

// Where output g's rows live: per direction the row range [q0, qe) of the
// 1D matrix and the terms of the source address base[lb] + (oI << (lb-1))
// + p I + in (oI = o I (k+1), lb >= 1; oI itself for lb = 0).
template <int D>
struct GmvLoc {
    int cbrow[D];  // offset of the (tuple, direction) row of the block-offset table
    int q0[D], qe[D];
    int64_t oI[D], I[D], in[D];
};

template <typename T, int D, int KP1>
__device__ __forceinline__ void gmv_locate(const GmvArgs<T, D>& a, int64_t g, GmvLoc<D>& L) {
    const int nl = a.N + 1;
    // tuple of g: binary search between the tuples of the chunk's ends
    int lo = a.chunk[g >> 8], hi = a.chunk[(g >> 8) + 1];
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.offsets[mid] <= g) lo = mid;
        else hi = mid - 1;
    }
    const int t = lo;
    int64_t e = g - a.offsets[t];
    int lv[D], sh[D], c[D], cnt[D];
    int sum = 0;
#pragma unroll
    for (int m = 0; m < D; ++m) {
        lv[m] = a.levels[t * D + m];
        sum += lv[m];
        sh[m] = lv[m] > 0 ? lv[m] - 1 : 0;
        cnt[m] = KP1 << sh[m];
    }
    // local multi-index, last direction fastest; cnt[m] = KP1 2^sh[m]
#pragma unroll
    for (int m = D - 1; m >= 0; --m) {
        const int64_t q = (e >> sh[m]) / KP1;
        c[m] = (int)(e - q * cnt[m]);
        e = q;
    }
#pragma unroll
    for (int i = 0; i < D; ++i) {
        int64_t o = 0, in = 0, I = 1;
#pragma unroll
        for (int m = 0; m < i; ++m) o = o * cnt[m] + c[m];
#pragma unroll
        for (int m = D - 1; m > i; --m) {
            in += (int64_t)c[m] * I;
            I *= cnt[m];
        }
        const int np = a.N - (sum - lv[i]);
        const int ai = (lv[i] ? (KP1 << (lv[i] - 1)) : 0) + c[i];
        L.cbrow[i] = (t * D + i) * nl;
        L.q0[i] = a.rp[ai];
        L.qe[i] = L.q0[i] + a.rlen[ai * nl + np];
        L.oI[i] = o * I * KP1;
        L.I[i] = I;
        L.in[i] = in;
    }
}

// y_g for a located output, computed by the G lanes of a group (lane r of
// G; G divides 8, the group is G consecutive lanes of a warp, every lane of
// the warp calls this).  The sum does not depend on G: the entries of every
// row are dealt to 8 virtual lanes (entry q to virtual lane q mod 8, two
// chains each, directions in order), optionally minus a correction
// sum_c h_c z_c whose columns are dealt the same way, and the 8 virtual sums
// are added in one fixed binary tree -- physical lanes hold 8/G virtual
// lanes, the lower tree levels are shuffles, the upper ones local.  The
// result is returned in every lane of the group.  LD selects the loads of
// x: 0 plain (read-only for the kernel), 1 L2 only, 2 cached in L1 through
// the coherent path (for vectors written by other CTAs of the same
// persistent kernel and published by a barrier whose acquire made L1
// current).
template <typename T, int D, int G, int LD>
__device__ __forceinline__ T gmv_accumulate(const GmvArgs<T, D>& a, const T* __restrict__ x, const GmvLoc<D>& L,
                                            int r, bool live, int ncorr = 0, const T* hc = nullptr,
                                            const T* zc = nullptr, int64_t zld = 0) {
    constexpr int VL = 8, PER = VL / G;
    T b[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) b[k] = T(0);
    if (live) {
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int v = r + k * G;
            T s0 = T(0), s1 = T(0);
#pragma unroll
            for (int i = 0; i < D; ++i) {
                const int64_t* __restrict__ base = a.cb + L.cbrow[i];
                const T* __restrict__ cv = a.cvk + i * a.nnz;
                const int64_t oI = L.oI[i], I = L.I[i], in = L.in[i];
                auto ld = [&](int pk) {
                    const int lb = pk >> 16, p = pk & 0xffff;
                    const int64_t ob = lb ? (oI << (lb - 1)) : oI;
                    const T* px = x + base[lb] + ob + (int64_t)p * I + in;
                    if constexpr (LD == 1) return __ldcg(px);
                    else if constexpr (LD == 2) return __ldca(px);
                    else return *px;
                };
                const int qe = L.qe[i];
                int q = L.q0[i] + v;
#pragma unroll 2
                for (; q + VL < qe; q += 2 * VL) {
                    const int p0 = a.ce[q], p1 = a.ce[q + VL];
                    const T v0 = cv[q], v1 = cv[q + VL];
                    s0 += v0 * ld(p0);
                    s1 += v1 * ld(p1);
                }
                if (q < qe) s0 += cv[q] * ld(a.ce[q]);
            }
            T c0 = T(0);
            for (int c = v; c < ncorr; c += VL) c0 += hc[c] * zc[c * zld];
            b[k] = (s0 + s1) - c0;
        }
    }
#pragma unroll
    for (int o = 1; o < G; o <<= 1)
#pragma unroll
        for (int k = 0; k < PER; ++k) b[k] += __shfl_xor_sync(0xffffffffu, b[k], o);
#pragma unroll
    for (int m = 1; m < PER; m <<= 1)
#pragma unroll
        for (int k = 0; k + m < PER; k += 2 * m) b[k] += b[k + m];
    return b[0];
}

// The same sum from a pre-located entry list (shared memory): eo[i] ..
// eo[i + 1] are direction i's entries {index of x, index into cvk} of this
// output in row order, dealt to the virtual lanes exactly as above, so the
// result is bitwise that of gmv_accumulate.  x is read through L1 on the
// coherent path (written by other CTAs, published by a barrier).
template <int D, int G>
__device__ __forceinline__ double gmv_accumulate_list(const int* eo, const int2* ent,
                                                      const double* __restrict__ cvk, const double* x, int r,
                                                      bool live, int ncorr, const double* hc, const double* zc,
                                                      int64_t zld) {
    constexpr int VL = 8, PER = VL / G;
    double b[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) b[k] = 0.0;
    if (live) {
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int v = r + k * G;
            double s0 = 0.0, s1 = 0.0;
#pragma unroll
            for (int i = 0; i < D; ++i) {
                const int qe = eo[i + 1];
                int q = eo[i] + v;
#pragma unroll 2
                for (; q + VL < qe; q += 2 * VL) {
                    const int2 e0 = ent[q], e1 = ent[q + VL];
                    s0 += __ldg(cvk + e0.y) * __ldca(x + e0.x);
                    s1 += __ldg(cvk + e1.y) * __ldca(x + e1.x);
                }
                if (q < qe) {
                    const int2 e0 = ent[q];
                    s0 += __ldg(cvk + e0.y) * __ldca(x + e0.x);
                }
            }
            double c0 = 0.0;
            for (int c = v; c < ncorr; c += VL) c0 += hc[c] * zc[c * zld];
            b[k] = (s0 + s1) - c0;
        }
    }
#pragma unroll
    for (int o = 1; o < G; o <<= 1)
#pragma unroll
        for (int k = 0; k < PER; ++k) b[k] += __shfl_xor_sync(0xffffffffu, b[k], o);
#pragma unroll
    for (int m = 1; m < PER; m <<= 1)
#pragma unroll
        for (int k = 0; k + m < PER; k += 2 * m) b[k] += b[k + m];
    return b[0];
}

// The same sum in double-float arithmetic (sgk_df64.h) from double-float
// copies of the values (cvk2), of x and of the correction's columns and
// coefficients: the same entries in the same virtual lanes and order, each
// product and sum with ~48-bit significands instead of FP64 operations.
template <int D, int G>
__device__ __forceinline__ df64 gmv_accumulate_list_df(const int* eo, const int2* ent, const float2* __restrict__ cvk2,
                                                       const float2* x, int r, bool live, int ncorr,
                                                       const float2* hc, const float2* zc, int64_t zld) {
    constexpr int VL = 8, PER = VL / G;
    df64 b[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) b[k] = df_make(0.f, 0.f);
    if (live) {
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int v = r + k * G;
            df64 s0 = df_make(0.f, 0.f), s1 = df_make(0.f, 0.f);
#pragma unroll
            for (int i = 0; i < D; ++i) {
                const int qe = eo[i + 1];
                int q = eo[i] + v;
#pragma unroll 2
                for (; q + VL < qe; q += 2 * VL) {
                    const int2 e0 = ent[q], e1 = ent[q + VL];
                    s0 = df_add(s0, df_mul(df_from_float2(__ldg(cvk2 + e0.y)), df_from_float2(__ldca(x + e0.x))));
                    s1 = df_add(s1, df_mul(df_from_float2(__ldg(cvk2 + e1.y)), df_from_float2(__ldca(x + e1.x))));
                }
                if (q < qe) {
                    const int2 e0 = ent[q];
                    s0 = df_add(s0, df_mul(df_from_float2(__ldg(cvk2 + e0.y)), df_from_float2(__ldca(x + e0.x))));
                }
            }
            df64 c0 = df_make(0.f, 0.f);
            for (int c = v; c < ncorr; c += VL) c0 = df_add(c0, df_mul(df_from_float2(hc[c]), df_from_float2(zc[c * zld])));
            b[k] = df_add(df_add(s0, s1), df_neg(c0));
        }
    }
#pragma unroll
    for (int o = 1; o < G; o <<= 1)
#pragma unroll
        for (int k = 0; k < PER; ++k) b[k] = df_add(b[k], df_shfl_xor(b[k], o));
#pragma unroll
    for (int m = 1; m < PER; m <<= 1)
#pragma unroll
        for (int k = 0; k + m < PER; k += 2 * m) b[k] = df_add(b[k], b[k + m]);
    return b[0];
}

template <typename T, int D>
GmvArgs<T, D> make_gmv_args(const sgk_op* op) {
    const sgk_index* idx = op->idx;
    GmvArgs<T, D> a;
    a.n = idx->dof;
    a.N = idx->n;
    a.offsets = idx->d_offsets.p;
    a.levels = idx->d_levels.p;
    a.chunk = op->gmv_chunk.p;
    a.cb = op->gmv_cb.p;
    a.rp = op->S.d_ptr.p;
    a.rlen = op->rlen.p;
    a.ce = op->gmv_ce.p;
    a.cvk = sizeof(T) == 8 ? reinterpret_cast<const T*>(op->gmv_cvk.p) : reinterpret_cast<const T*>(op->gmv_cvkf.p);
    a.nnz = (int64_t)op->S.col.size();
    return a;
}
