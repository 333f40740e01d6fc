// Sparse-grid matvec y = A x, A = -sum_i kappa_i (S along direction i),
// all directions in one launch (Section 4, unidirectional principle), in the
// gather form of sgk_gmv.h.
//
// y is written once; x is gathered through L2 (the 1D rows overlap, so
// neighbouring outputs share most of their loads).  The sums are taken in a
// fixed order (per lane two accumulators per direction, directions in order,
// then a fixed xor tree over the group), so results are deterministic.
#include <algorithm>
#include <cmath>

#include "sgk_gmv.h"

namespace {

template <typename T, int D, int KP1, int G>
__global__ void __launch_bounds__(256) gmv_kernel(const GmvArgs<T, D> a, const T* __restrict__ x,
                                                  T* __restrict__ y) {
    // G consecutive lanes share one output coefficient (more loads in flight
    // for small vectors, whose cost is latency)
    const int r = threadIdx.x & (G - 1), lane = threadIdx.x & 31;
    const int64_t total = a.n * G;
    // the trip count is uniform over the warp (the shuffles below need every
    // lane); lanes past the end carry zeros
    for (int64_t gg = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gg - lane < total;
         gg += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = gg / G;
        const bool live = g < a.n;
        GmvLoc<D> L;
        if (live) gmv_locate<T, D, KP1>(a, g, L);
        const T acc = gmv_accumulate<T, D, G, 0>(a, x, L, r, live);
        if (live && r == 0) y[g] = acc;
    }
}

template <typename T, int D>
void gmv_dispatch(const sgk_op* op, const T* x, T* y) {
    const sgk_index* idx = op->idx;
    const GmvArgs<T, D> a = make_gmv_args<T, D>(op);
    sgk_ctx* ctx = op->ctx;
    const int threads = 256;
    // lanes per output: enough threads to fill the GPU when the vector is
    // small (latency-bound), one lane per output when it is large
    int G = 1;
    while (G < 8 && idx->dof * G < (int64_t)ctx->num_sms * 1024) G *= 2;
    const int64_t blocks = (idx->dof * G + threads - 1) / threads;
    const int grid = (int)std::min<int64_t>(blocks, (int64_t)ctx->num_sms * 8);
    KTimer kt(ctx, KC_MATVEC);
#define SGK_GMV(K, GG) gmv_kernel<T, D, K, GG><<<grid, threads, 0, ctx->stream>>>(a, x, y)
#define SGK_GMV_K(K)                         \
    switch (G) {                             \
        case 1: SGK_GMV(K, 1); break;        \
        case 2: SGK_GMV(K, 2); break;        \
        case 4: SGK_GMV(K, 4); break;        \
        default: SGK_GMV(K, 8); break;       \
    }
    switch (idx->k + 1) {
        case 2: SGK_GMV_K(2) break;
        case 3: SGK_GMV_K(3) break;
        case 4: SGK_GMV_K(4) break;
        default: throw SgkError{SGK_EUNSUPPORTED, "matvec: degree must be 1..3"};
    }
#undef SGK_GMV_K
#undef SGK_GMV
    check_launch("gmv_kernel");
    count_launch(ctx);
}

}  // namespace

// Host tables of the gather matvec, with every address the kernel can form
// checked against the vector length.
void build_gmv_tables(sgk_op* op) {
    const sgk_index* idx = op->idx;
    const int d = idx->d, N = idx->n, kp1 = idx->k + 1, nl = N + 1;
    const Csr& S = op->S;
    std::vector<int32_t> ce(S.col.size());
    for (int a = 0; a < S.rows; ++a)
        for (int q = S.ptr[a]; q < S.ptr[a + 1]; ++q) {
            const int b = S.col[q];
            int lb = 0;
            while (b >= level_offset(lb, kp1) + level_count(lb, kp1)) ++lb;
            SGK_REQUIRE(lb <= N, SGK_EINVAL, "matvec: column outside the 1D space");
            const int p = b - level_offset(lb, kp1);
            ce[q] = (lb << 16) | p;
        }
    // truncated row lengths, as uploaded: rl[a (N+1) + L]
    std::vector<int> rl((size_t)S.rows * nl, 0);
    for (int a = 0; a < S.rows; ++a)
        for (int L = 0; L < nl; ++L) {
            int c = 0;
            for (int q = S.ptr[a]; q < S.ptr[a + 1] && S.col[q] < (kp1 << L); ++q) ++c;
            rl[(size_t)a * nl + L] = c;
        }
    op->rlen_host = rl;
    int64_t madds = 0;
    std::vector<int64_t> cb((size_t)idx->ntuples * d * nl, -1);
    for (int64_t t = 0; t < idx->ntuples; ++t) {
        const int32_t* l = &idx->levels[t * d];
        int sum = 0;
        for (int m = 0; m < d; ++m) sum += l[m];
        for (int i = 0; i < d; ++i) {
            std::vector<int> lv(l, l + d);
            const int np = N - (sum - l[i]);
            int64_t blk = 1;  // block size without direction i
            for (int m = 0; m < d; ++m)
                if (m != i) blk *= level_count(l[m], kp1);
            int64_t rows = 0;  // entries of the rows of this block's direction-i positions
            for (int c = 0; c < level_count(l[i], kp1); ++c)
                rows += rl[(size_t)(level_offset(l[i], kp1) + c) * nl + np];
            madds += rows * blk;
            for (int lb = 0; lb <= np; ++lb) {
                lv[i] = lb;
                const long long r = tuple_rank(lv, N);
                SGK_REQUIRE(r >= 0 && r < idx->ntuples, SGK_EINVAL, "matvec: tuple rank out of range");
                const int64_t off = idx->offsets[r];
                SGK_REQUIRE(idx->offsets[r + 1] - off == blk * level_count(lb, kp1), SGK_EINVAL,
                            "matvec: block size mismatch");
                SGK_REQUIRE(off + blk * level_count(lb, kp1) <= idx->dof, SGK_EINVAL, "matvec: block outside x");
                cb[((size_t)t * d + i) * nl + lb] = off;
            }
        }
    }
    const int64_t nchunk = (idx->dof + 255) / 256;
    std::vector<int32_t> chunk(nchunk + 1);
    int64_t t = 0;
    for (int64_t c = 0; c <= nchunk; ++c) {
        const int64_t g = std::min<int64_t>(c * 256, idx->dof - 1);
        while (idx->offsets[t + 1] <= g) ++t;
        chunk[c] = (int32_t)t;
    }
    op->madds = madds;
    // ||A||_2 <= sum_i |kappa_i| ||S||_2 (A restricted from the full tensor
    // operator to a subspace spanned by orthonormal basis functions), and
    // ||S||_2 <= max(||S||_1, ||S||_inf)
    {
        std::vector<double> rs(S.rows, 0.0), cs(S.rows, 0.0);
        for (int a = 0; a < S.rows; ++a)
            for (int q = S.ptr[a]; q < S.ptr[a + 1]; ++q) {
                rs[a] += std::fabs(S.val[q]);
                if (S.col[q] < S.rows) cs[S.col[q]] += std::fabs(S.val[q]);
            }
        double sn = 0.0;
        for (int a = 0; a < S.rows; ++a) sn = std::max(sn, std::max(rs[a], cs[a]));
        double ks = 0.0;
        for (int i = 0; i < d; ++i) ks += std::fabs(op->kappa[i]);
        op->anorm = ks * sn;
    }
    const size_t nnz = S.val.size();
    std::vector<double> cvk(nnz * d);
    std::vector<float> cvkf(nnz * d);
    std::vector<float2> cvk2(nnz * d);
    for (int i = 0; i < d; ++i)
        for (size_t q = 0; q < nnz; ++q) {
            const double v = -op->kappa[i] * S.val[q];
            cvk[i * nnz + q] = v;
            cvkf[i * nnz + q] = (float)v;
            const float hi = (float)v;
            cvk2[i * nnz + q] = make_float2(hi, (float)(v - (double)hi));
        }
    // pre-located gathers: the host mirror of gmv_locate and of the address
    // formed per entry in gmv_accumulate
    op->gmv_ecnt_host.clear();
    std::vector<int32_t> eoff;  // alive until the stream synchronisation below
    std::vector<int2> ent;
    if (madds <= GMV_LIST_MAX && idx->dof * d < (int64_t(1) << 31) && (int64_t)nnz * d < (int64_t(1) << 31)) {
        eoff.resize((size_t)idx->dof * d + 1);
        ent.reserve((size_t)madds);
        op->gmv_ecnt_host.resize(idx->dof);
        for (int64_t t = 0; t < idx->ntuples; ++t) {
            const int32_t* lv = &idx->levels[t * d];
            int sum = 0;
            std::vector<int> sh(d), cnt(d), c(d);
            for (int m = 0; m < d; ++m) {
                sum += lv[m];
                sh[m] = lv[m] > 0 ? lv[m] - 1 : 0;
                cnt[m] = kp1 << sh[m];
            }
            for (int64_t g = idx->offsets[t]; g < idx->offsets[t + 1]; ++g) {
                int64_t e = g - idx->offsets[t];
                for (int m = d - 1; m >= 0; --m) {
                    const int64_t q = (e >> sh[m]) / kp1;
                    c[m] = (int)(e - q * cnt[m]);
                    e = q;
                }
                const size_t first = ent.size();
                for (int i = 0; i < d; ++i) {
                    eoff[(size_t)g * d + i] = (int32_t)ent.size();
                    int64_t o = 0, in = 0, I = 1;
                    for (int m = 0; m < i; ++m) o = o * cnt[m] + c[m];
                    for (int m = d - 1; m > i; --m) {
                        in += (int64_t)c[m] * I;
                        I *= cnt[m];
                    }
                    const int np = N - (sum - lv[i]);
                    const int ai = (lv[i] ? (kp1 << (lv[i] - 1)) : 0) + c[i];
                    const int q0 = S.ptr[ai], qe = q0 + rl[(size_t)ai * nl + np];
                    const int64_t oI = o * I * kp1;
                    for (int q = q0; q < qe; ++q) {
                        const int lb = ce[q] >> 16, pp = ce[q] & 0xffff;
                        const int64_t ob = lb ? (oI << (lb - 1)) : oI;
                        const int64_t xi = cb[((size_t)t * d + i) * nl + lb] + ob + (int64_t)pp * I + in;
                        SGK_REQUIRE(xi >= 0 && xi < idx->dof, SGK_EINVAL, "matvec: gather outside x");
                        ent.push_back(make_int2((int)xi, (int)((int64_t)i * nnz + q)));
                    }
                }
                op->gmv_ecnt_host[g] = (int32_t)(ent.size() - first);
            }
        }
        eoff[(size_t)idx->dof * d] = (int32_t)ent.size();
        SGK_REQUIRE((int64_t)ent.size() == madds, SGK_EINVAL, "matvec: entry list size mismatch");
        op->gmv_eoff.upload(eoff, op->ctx->stream);
        op->gmv_ent.upload(ent, op->ctx->stream);
    }
    op->gmv_cvk.upload(cvk, op->ctx->stream);
    op->gmv_cvkf.upload(cvkf, op->ctx->stream);
    op->gmv_cvk2.upload(cvk2, op->ctx->stream);
    op->gmv_ce.upload(ce, op->ctx->stream);
    op->gmv_cb.upload(cb, op->ctx->stream);
    op->gmv_chunk.upload(chunk, op->ctx->stream);
    SGK_CUDA_CHECK(cudaStreamSynchronize(op->ctx->stream));
}

std::vector<int64_t> arnoldi_slice_bounds(const sgk_op* op, int nb, int extra, int64_t cap_len, int64_t cap_ent) {
    const sgk_index* idx = op->idx;
    const int d = idx->d, N = idx->n, kp1 = idx->k + 1, nl = N + 1;
    const int64_t n = idx->dof;
    // entries of every output (the per-output matvec work)
    std::vector<int32_t> ecnt = op->gmv_ecnt_host;
    if ((int64_t)ecnt.size() != n) {
        const std::vector<int>& rl = op->rlen_host;
        ecnt.assign(n, 0);
        std::vector<int> c(d), sh(d), cnt(d);
        for (int64_t t = 0; t < idx->ntuples; ++t) {
            const int32_t* lv = &idx->levels[t * d];
            int sum = 0;
            for (int m = 0; m < d; ++m) {
                sum += lv[m];
                sh[m] = lv[m] > 0 ? lv[m] - 1 : 0;
                cnt[m] = kp1 << sh[m];
            }
            std::fill(c.begin(), c.end(), 0);
            for (int64_t g = idx->offsets[t]; g < idx->offsets[t + 1]; ++g) {
                int e = 0;
                for (int i = 0; i < d; ++i)
                    e += rl[(size_t)((lv[i] ? (kp1 << (lv[i] - 1)) : 0) + c[i]) * nl + N - (sum - lv[i])];
                ecnt[g] = e;
                for (int m = d - 1; m >= 0; --m) {  // row-major odometer, last direction fastest
                    if (++c[m] < cnt[m]) break;
                    c[m] = 0;
                }
            }
        }
    }
    // contiguous slices minimising the largest cost (entries + extra per
    // output) under the caps: the greedy cut is optimal for a given bound,
    // and the least feasible bound is found by bisection
    auto fits = [&](int64_t C, std::vector<int64_t>* out) {
        int k = 0;
        int64_t cc = 0, cl = 0, ce = 0;
        if (out) (*out)[0] = 0;
        for (int64_t g = 0; g < n; ++g) {
            const int64_t w = ecnt[g] + extra;
            if (ecnt[g] > cap_ent || w > C) return false;
            if (cl > 0 && (cc + w > C || cl + 1 > cap_len || ce + ecnt[g] > cap_ent)) {
                if (++k >= nb) return false;
                if (out) (*out)[k] = g;
                cc = cl = ce = 0;
            }
            cc += w;
            ++cl;
            ce += ecnt[g];
        }
        if (out)
            for (int j = k + 1; j <= nb; ++j) (*out)[j] = n;
        return true;
    };
    int64_t lo = 0, hi = 0;
    for (int64_t g = 0; g < n; ++g) hi += ecnt[g] + extra;
    if (n == 0 || !fits(hi, nullptr)) return {};
    while (hi - lo > 1) {
        const int64_t mid = lo + (hi - lo) / 2;
        if (fits(mid, nullptr)) hi = mid;
        else lo = mid;
    }
    std::vector<int64_t> b(nb + 1, n);
    fits(hi, &b);
    return b;
}

template <typename T>
void op_matvec(const sgk_op* op, const T* x, T* y) {
    if (op->idx->dof == 0) return;
    switch (op->idx->d) {
        case 1: gmv_dispatch<T, 1>(op, x, y); break;
        case 2: gmv_dispatch<T, 2>(op, x, y); break;
        case 3: gmv_dispatch<T, 3>(op, x, y); break;
        case 4: gmv_dispatch<T, 4>(op, x, y); break;
        case 5: gmv_dispatch<T, 5>(op, x, y); break;
        case 6: gmv_dispatch<T, 6>(op, x, y); break;
        default: throw SgkError{SGK_EUNSUPPORTED, "matvec: d must be 1..6"};
    }
    op_cross_matvec<T>(op, x, y);
}

template void op_matvec<double>(const sgk_op*, const double*, double*);
template void op_matvec<float>(const sgk_op*, const float*, float*);
