// Persistent Arnoldi process for the Krylov approximation of exp(dt A) v
// (Section 3, eqs. krylov1-krylov3): gamma = ||v||, then M steps of matvec,
// classical Gram-Schmidt twice (CGS2) and normalisation, all in one
// cooperative launch.
//
// Each CTA owns a contiguous slice of the coefficient vector.  It computes
// the matvec outputs of its slice (gather form, sgk_gmv.h) and at once the
// partial inner products of that slice with the basis columns, so the
// matvec and the first projection need no barrier between them.  Three grid
// barriers per step publish (1) the partials of V^T w, (2) those of the
// second pass, (3) those of ||w||^2; after each, every CTA sums the partials
// of all CTAs itself, in a fixed order, so all CTAs hold bitwise equal
// h1, h2 and beta and take the same breakdown decision without another
// barrier.  The next matvec gathers the unnormalised w (final after barrier
// 3) and scales its outputs by 1 / beta; the two w buffers alternate so that
// those gathers never race with the writes of the next step.  Partial sums go
// to three rotating buffers for the same reason.
//
// Barriers are counters in global memory with a bounded wait: a CTA that
// waits longer than the limit sets an error flag and returns, and every
// other CTA sees the flag in its own wait and returns too; the host reports
// SGK_ETIMEOUT.  The cooperative launch makes every CTA resident at once.
#include <algorithm>

#include "sgk_gmv.h"
#include "sgk_krylov.h"

namespace {

constexpr int PT = 1024;                       // threads per CTA, one CTA per SM
constexpr int PNW = PT / 32;                   // warps per CTA
constexpr unsigned BAR_SPIN_LIMIT = 1u << 21;  // polls of ~0.1-0.5 us each

struct ArnArgs {
    int64_t n;
    int M;
    int ldp;  // row stride of the partial-sum buffers (>= M + 1)
    const double* v;
    double* V;  // column c at V + c n
    double* w0;
    double* w1;
    double* H;     // (M + 1) x M row-major
    double* pbuf;  // 3 buffers of gridDim.x x ldp
    unsigned* bar;  // [0] barrier arrivals (zero at launch), [1] error flag
    KrylovScalars* ks;
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// All CTAs arrive; returns false if the wait ran out or another CTA failed.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned target, int* s_ok) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(bar, 1u);
        int ok = 1;
        for (unsigned it = 0;; ++it) {
            if (ld_acquire(bar) >= target) break;
            if (it >= BAR_SPIN_LIMIT || ld_acquire(bar + 1) != 0u) {
                ok = 0;
                break;
            }
            __nanosleep(100);
        }
        if (!ok) atomicExch(bar + 1, 1u);
        __threadfence();
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

// out[c] = sum over CTAs b of P[b ldp + c], c < ncols: a warp per column,
// lanes over b in a fixed order, then a fixed shuffle tree.  Identical in
// every CTA.  P was written by other CTAs during this launch: L2 loads.
__device__ __forceinline__ void colsum(const double* P, int nb, int ldp, int ncols, double* out) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int c = wid; c < ncols; c += PNW) {
        double a = 0.0, b = 0.0;
        int k = lane;
        for (; k + 32 < nb; k += 64) {
            a += __ldcg(P + (int64_t)k * ldp + c);
            b += __ldcg(P + (int64_t)(k + 32) * ldp + c);
        }
        if (k < nb) a += __ldcg(P + (int64_t)k * ldp + c);
        a += b;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0) out[c] = a;
    }
}

// out[c] = sum_{u < ne} V[c n + lo + u] ws[u], c < ncols (this CTA's slice)
__device__ __forceinline__ void slice_dots(const double* V, int64_t n, int ncols, const double* ws, int64_t lo,
                                           int ne, double* out) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int c = wid; c < ncols; c += PNW) {
        const double* vc = V + c * n + lo;
        double a = 0.0, b = 0.0;
        int u = lane;
        for (; u + 32 < ne; u += 64) {
            a += vc[u] * ws[u];
            b += vc[u + 32] * ws[u + 32];
        }
        if (u < ne) a += vc[u] * ws[u];
        a += b;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0) out[c] = a;
    }
}

// w -= V[:, :ncols] h on this CTA's slice (global and staged copies)
__device__ __forceinline__ void slice_update(const double* V, int64_t n, int ncols, const double* h, double* w,
                                             double* ws, int64_t lo, int ne) {
    for (int u = threadIdx.x; u < ne; u += PT) {
        const double* vi = V + lo + u;
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
        int c = 0;
        for (; c + 3 < ncols; c += 4) {
            a0 += vi[c * n] * h[c];
            a1 += vi[(c + 1) * n] * h[c + 1];
            a2 += vi[(c + 2) * n] * h[c + 2];
            a3 += vi[(c + 3) * n] * h[c + 3];
        }
        for (; c < ncols; ++c) a0 += vi[c * n] * h[c];
        const double x = ws[u] - ((a0 + a1) + (a2 + a3));
        ws[u] = x;
        w[lo + u] = x;
    }
}

// sum of x^2 over the staged slice, written by thread 0 to *out
__device__ __forceinline__ void slice_norm2(const double* ws, int ne, double* red, double* out) {
    double a = 0.0;
    for (int u = threadIdx.x; u < ne; u += PT) a += ws[u] * ws[u];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < PNW; ++k) t += red[k];
        *out = t;
    }
}

template <int D, int KP1, int G>
__global__ void __launch_bounds__(PT, 1) arnoldi_kernel(const GmvArgs<double, D> ga, const ArnArgs a) {
    extern __shared__ __align__(16) double ws[];  // this CTA's slice of w
    __shared__ double h1[SGK_MAX_KRYLOV + 1];
    __shared__ double h2[SGK_MAX_KRYLOV + 1];
    __shared__ double red[PNW];
    __shared__ double s_scal[2];
    __shared__ int s_ok;
    const int nb = gridDim.x, b = blockIdx.x;
    const int64_t n = a.n;
    const int64_t E = (n + nb - 1) / nb;
    const int64_t lo = std::min<int64_t>(n, (int64_t)b * E);
    const int ne = (int)(std::min<int64_t>(n, lo + E) - lo);
    double* const P0 = a.pbuf;                       // V^T w, first pass
    double* const P1 = a.pbuf + (int64_t)nb * a.ldp;  // second pass
    double* const P2 = a.pbuf + (int64_t)2 * nb * a.ldp;  // norms
    unsigned epoch = 0;
    auto barrier = [&]() {
        ++epoch;
        return grid_barrier(a.bar, epoch * (unsigned)nb, &s_ok);
    };
    const int r = threadIdx.x & (G - 1);
    KrylovScalars* ks = a.ks;

    // gamma = ||v||
    for (int u = threadIdx.x; u < ne; u += PT) ws[u] = a.v[lo + u];
    __syncthreads();
    slice_norm2(ws, ne, red, P2 + (int64_t)b * a.ldp);
    if (!barrier()) return;
    colsum(P2, nb, a.ldp, 1, s_scal);
    __syncthreads();
    // scalar FP64 work (square roots, reciprocals, the Frobenius norm of H)
    // runs on one thread per CTA and is broadcast through shared memory: FP64
    // issue is about two operations per clock per SM on this part
    if (threadIdx.x == 0) {
        const double gamma = sqrt(s_scal[0]);
        s_scal[1] = gamma > 0.0 ? 1.0 / gamma : 0.0;
        if (b == 0) {
            ks->gamma = gamma;
            ks->inv_gamma = s_scal[1];
            ks->fro2 = 0.0;
            ks->stop = gamma > 0.0 ? 0 : 1;
            ks->m_eff = 0;
            ks->breakdown = 0;
        }
    }
    __syncthreads();
    if (!(s_scal[1] > 0.0)) return;  // gamma = 0: the same decision in every CTA
    double scale = s_scal[1];
    for (int u = threadIdx.x; u < ne; u += PT) a.V[lo + u] = ws[u] * scale;
    const double* x = a.v;
    double fro2 = 0.0, sub = 0.0;  // used by thread 0
    for (int j = 0; j < a.M; ++j) {
        double* w = (j & 1) ? a.w1 : a.w0;
        const int nc = j + 1;
        // w = A v_j on this slice (v_j = scale * x), staged in shared memory
        for (int base = 0; base < ne; base += PT / G) {
            const int u = base + (int)threadIdx.x / G;
            double acc = u < ne ? gmv_lane<double, D, KP1, G, true>(ga, x, lo + u, r) : 0.0;
#pragma unroll
            for (int o = 1; o < G; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (u < ne && r == 0) {
                acc *= scale;
                ws[u] = acc;
                w[lo + u] = acc;
            }
        }
        __syncthreads();
        slice_dots(a.V, n, nc, ws, lo, ne, P0 + (int64_t)b * a.ldp);
        if (!barrier()) return;
        colsum(P0, nb, a.ldp, nc, h1);
        __syncthreads();
        slice_update(a.V, n, nc, h1, w, ws, lo, ne);
        __syncthreads();
        slice_dots(a.V, n, nc, ws, lo, ne, P1 + (int64_t)b * a.ldp);
        if (!barrier()) return;
        colsum(P1, nb, a.ldp, nc, h2);
        __syncthreads();
        slice_update(a.V, n, nc, h2, w, ws, lo, ne);
        __syncthreads();
        slice_norm2(ws, ne, red, P2 + (int64_t)b * a.ldp);
        if (!barrier()) return;
        colsum(P2, nb, a.ldp, 1, s_scal);
        __syncthreads();
        // column j of H and the breakdown test: thread 0 of every CTA, alike
        if (threadIdx.x == 0) {
            double f = fro2 + sub * sub;
            for (int i = 0; i < nc; ++i) {
                const double hv = h1[i] + h2[i];
                f += hv * hv;
                if (b == 0) a.H[(int64_t)i * a.M + j] = hv;
            }
            fro2 = f;
            const double beta = sqrt(s_scal[0]);
            sub = beta;
            const bool brk = beta <= 1e-12 * sqrt(f);
            s_scal[1] = brk ? 0.0 : 1.0 / beta;
            if (b == 0) {
                a.H[(int64_t)(j + 1) * a.M + j] = beta;
                ks->fro2 = f;
                ks->m_eff = j + 1;
                if (brk) {
                    ks->stop = 1;
                    ks->breakdown = 1;
                }
            }
        }
        __syncthreads();
        if (!(s_scal[1] > 0.0)) return;  // breakdown: the same decision in every CTA
        scale = s_scal[1];
        for (int u = threadIdx.x; u < ne; u += PT) a.V[(int64_t)(j + 1) * n + lo + u] = ws[u] * scale;
        x = w;
        // the next step overwrites ws only after its matvec has read nothing
        // from it; V and w of this slice were written by this CTA
        __syncthreads();
    }
}

template <int D, int KP1, int G>
void arn_launch(sgk_ctx* ctx, const sgk_op* op, const ArnArgs& a, int nb, size_t smem) {
    auto kern = arnoldi_kernel<D, KP1, G>;
    const GmvArgs<double, D> ga = make_gmv_args<double, D>(op);
    SGK_CUDA_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int occ = 0;
    SGK_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, PT, smem));
    SGK_REQUIRE(occ >= 1 && nb <= occ * ctx->num_sms, SGK_EUNSUPPORTED, "persistent Arnoldi grid does not fit");
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nb);
    cfg.blockDim = dim3(PT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = ctx->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    SGK_CUDA_CHECK(cudaLaunchKernelEx(&cfg, kern, ga, a));
}

template <int D, int KP1>
void arn_launch_g(sgk_ctx* ctx, const sgk_op* op, const ArnArgs& a, int nb, size_t smem, int G) {
    switch (G) {
        case 1: arn_launch<D, KP1, 1>(ctx, op, a, nb, smem); break;
        case 2: arn_launch<D, KP1, 2>(ctx, op, a, nb, smem); break;
        case 4: arn_launch<D, KP1, 4>(ctx, op, a, nb, smem); break;
        default: arn_launch<D, KP1, 8>(ctx, op, a, nb, smem); break;
    }
}

template <int D>
void arn_launch_k(sgk_ctx* ctx, const sgk_op* op, const ArnArgs& a, int nb, size_t smem, int G) {
    switch (op->idx->k + 1) {
        case 2: arn_launch_g<D, 2>(ctx, op, a, nb, smem, G); break;
        case 3: arn_launch_g<D, 3>(ctx, op, a, nb, smem, G); break;
        case 4: arn_launch_g<D, 4>(ctx, op, a, nb, smem, G); break;
        default: throw SgkError{SGK_EUNSUPPORTED, "persistent Arnoldi: degree must be 1..3"};
    }
}

}  // namespace

static int persistent_ctas(const sgk_ctx* ctx) {
    return ctx->persist_ctas > 0 ? std::min(ctx->persist_ctas, ctx->num_sms) : ctx->num_sms;
}

int64_t arnoldi_persistent_max_n(const sgk_ctx* ctx) {
    // the slice of w is staged in shared memory: at most 24 K doubles per CTA
    return (int64_t)persistent_ctas(ctx) * 24 * 1024;
}

size_t arnoldi_persistent_pbuf_size(const sgk_ctx* ctx, int M) { return (size_t)3 * ctx->num_sms * (M + 1); }

void arnoldi_persistent(sgk_ctx* ctx, const sgk_op* op, const PersistentWork& pw, const KrylovWork<double>& kw,
                        const double* v, int64_t n, int M) {
    SGK_REQUIRE(n >= 1 && n <= arnoldi_persistent_max_n(ctx), SGK_EUNSUPPORTED, "persistent Arnoldi: n too large");
    SGK_REQUIRE(M >= 1 && M <= SGK_MAX_KRYLOV, SGK_EINVAL, "persistent Arnoldi: bad M");
    const int nb = persistent_ctas(ctx);
    const int64_t E = (n + nb - 1) / nb;
    int G = 1;
    while (G < 8 && E * G * 2 <= PT) G *= 2;
    ArnArgs a;
    a.n = n;
    a.M = M;
    a.ldp = M + 1;
    a.v = v;
    a.V = kw.V;
    a.w0 = kw.w;
    a.w1 = pw.w_alt;
    a.H = kw.H;
    a.pbuf = pw.pbuf;
    a.bar = pw.bar;
    a.ks = kw.ks;
    const size_t smem = sizeof(double) * (size_t)E;
    KTimer kt(ctx, KC_KRYLOV);
    SGK_CUDA_CHECK(cudaMemsetAsync(pw.bar, 0, sizeof(unsigned), ctx->stream));
    switch (op->idx->d) {
        case 1: arn_launch_k<1>(ctx, op, a, nb, smem, G); break;
        case 2: arn_launch_k<2>(ctx, op, a, nb, smem, G); break;
        case 3: arn_launch_k<3>(ctx, op, a, nb, smem, G); break;
        case 4: arn_launch_k<4>(ctx, op, a, nb, smem, G); break;
        case 5: arn_launch_k<5>(ctx, op, a, nb, smem, G); break;
        case 6: arn_launch_k<6>(ctx, op, a, nb, smem, G); break;
        default: throw SgkError{SGK_EUNSUPPORTED, "persistent Arnoldi: d must be 1..6"};
    }
    check_launch("arnoldi_kernel");
    count_launch(ctx);
}
