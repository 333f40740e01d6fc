// Krylov approximation of exp(dt A) v (Section 3, eqs. krylov7-krylov8) and
// the vector kernels of the Newton solve.
//
// Arnoldi uses classical Gram-Schmidt applied twice.  Inner products and
// norms are accumulated in FP64 with deterministic two-stage reductions
// (per-block partials, then one block summing them in a fixed order), so a
// run is bitwise reproducible on a given device.  Every Arnoldi step runs
// without a host round trip: breakdown (h_{j+1,j} <= 1e-12 ||H_{0:j+1,0:j+1}||_F)
// sets a device flag that makes the remaining steps' kernels return at once.
//
// exp(tau H) e_1 is computed by one CTA with scaling and squaring and the
// [13/13] Pade approximant (Higham, SIAM J. Matrix Anal. Appl. 26 (2005),
// with the degree fixed at 13): s = max(0, ceil(log2(||tau H||_1 / theta_13))),
// then (V - U) R = (V + U) by LU with partial pivoting, then R <- R^2 s times.
#include <atomic>
#include <cmath>
#include <mutex>

#include "sgk_dfloat.h"
#include "sgk_krylov.h"

namespace {

constexpr double THETA13 = 5.371920351148152;  // Higham (2005), Table 2.3

__device__ __forceinline__ double block_sum(double v, double* sh) { return block_sum_f64(v, sh); }

template <typename TA, typename TB>
__global__ void dot_partial_kernel(const TA* __restrict__ a, const TB* __restrict__ b, long long n,
                                   double* __restrict__ partials, const int* __restrict__ stop) {
    if (stop && *stop) return;
    __shared__ double sh[32];
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        acc += (double)a[i] * (double)b[i];
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// out = sum(partials) (mode 0), sqrt(sum) (mode 1)
__global__ void reduce_final_kernel(const double* __restrict__ partials, int nb, double* __restrict__ out, int mode,
                                    const int* __restrict__ stop) {
    if (stop && *stop) return;
    __shared__ double sh[32];
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) acc += partials[i];
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) out[0] = mode == 1 ? sqrt(acc) : acc;
}

// partials[block][c] = sum_e V[c][e] w[e] over the block's elements, c < ncols
template <typename T>
__global__ void mdot_partial_kernel(const T* __restrict__ V, long long ldv, int ncols, const T* __restrict__ w,
                                    long long n, double* __restrict__ partials, const int* __restrict__ stop) {
    if (stop && *stop) return;
    __shared__ double sh[32];
    constexpr int CH = 8;
    for (int c0 = 0; c0 < ncols; c0 += CH) {
        double acc[CH];
#pragma unroll
        for (int c = 0; c < CH; ++c) acc[c] = 0.0;
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
             i += (long long)gridDim.x * blockDim.x) {
            const double wv = (double)w[i];
#pragma unroll
            for (int c = 0; c < CH; ++c)
                if (c0 + c < ncols) acc[c] += (double)V[(c0 + c) * ldv + i] * wv;
        }
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            if (c0 + c >= ncols) break;
            const double s = block_sum(acc[c], sh);
            if (threadIdx.x == 0) partials[(long long)blockIdx.x * ncols + c0 + c] = s;
        }
    }
}

__global__ void mdot_final_kernel(const double* __restrict__ partials, int nb, int ncols, double* __restrict__ out,
                                  const int* __restrict__ stop) {
    if (stop && *stop) return;
    for (int c = threadIdx.x; c < ncols; c += blockDim.x) {
        double acc = 0.0;
        for (int b = 0; b < nb; ++b) acc += partials[(long long)b * ncols + c];
        out[c] = acc;
    }
}

// w -= V[:, :ncols] h  (arithmetic in T)
template <typename T>
__global__ void gs_update_kernel(const T* __restrict__ V, long long ldv, int ncols, const double* __restrict__ h,
                                 T* __restrict__ w, long long n, const int* __restrict__ stop) {
    if (stop && *stop) return;
    __shared__ T hs[SGK_MAX_KRYLOV + 1];
    for (int c = threadIdx.x; c < ncols; c += blockDim.x) hs[c] = (T)h[c];
    __syncthreads();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        T acc = T(0);
        for (int c = 0; c < ncols; ++c) acc += V[c * ldv + i] * hs[c];
        w[i] -= acc;
    }
}

// Start of an Arnoldi process: gamma = ||v||, flags reset, breakdown if v = 0.
__global__ void krylov_init_kernel(const double* __restrict__ gamma2, KrylovScalars* __restrict__ ks) {
    const double g = sqrt(*gamma2);
    ks->gamma = g;
    ks->inv_gamma = g > 0.0 ? 1.0 / g : 0.0;
    ks->fro2 = 0.0;
    ks->stop = g > 0.0 ? 0 : 1;
    ks->m_eff = 0;
    ks->breakdown = 0;
}

template <typename T>
__global__ void scale_to_kernel(const double* __restrict__ x, T* __restrict__ y, long long n,
                                const double* __restrict__ s, const int* __restrict__ stop) {
    if (stop && *stop) return;
    const double a = *s;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = (T)(x[i] * a);
}

template <typename T>
__global__ void scale_vec_kernel(const T* __restrict__ x, T* __restrict__ y, long long n,
                                 const double* __restrict__ s, const int* __restrict__ stop) {
    if (stop && *stop) return;
    const T a = (T)(*s);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = x[i] * a;
}

// ------------------------------------------- fused Gram-Schmidt kernels ---
//
// FP64 adds have a long dependent latency on this GPU, so reductions keep
// several independent chains per thread.  Each kernel ends its grid-wide
// reduction in the last block to finish (a counter in global memory); that
// block sums the per-block partials in a fixed order, so the result is
// deterministic.

// Each block owns GS_E consecutive elements (one per thread), stages the
// (updated) vector slice in shared memory, and gives every warp whole
// columns: a lane sums GS_E / 32 products and the warp reduces once per
// column, so the reduction adds stay a small fraction of the FP64 work.
constexpr int GS_E = 128;

// partials[block][c] = sum_{t < GS_E} V[c][i0 + t] ws[t].  A warp takes four
// columns at a time (c, c + nw, c + 2 nw, c + 3 nw) so that their loads,
// FMAs and shuffle reductions interleave instead of waiting on one another.
template <typename T>
__device__ __forceinline__ void warp_column_dots(const T* __restrict__ V, long long ldv, int ncols, const T* ws,
                                                 long long i0, double* __restrict__ partials) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double wl[GS_E / 32];
#pragma unroll
    for (int k = 0; k < GS_E / 32; ++k) wl[k] = (double)ws[lane + 32 * k];
    for (int c0 = wid; c0 < ncols; c0 += 4 * nw) {
        double a[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int c = c0 + u * nw;
            a[u] = 0.0;
            if (c < ncols) {
                const T* vc = V + c * ldv + i0;
#pragma unroll
                for (int k = 0; k < GS_E / 32; ++k) a[u] += (double)vc[lane + 32 * k] * wl[k];
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int u = 0; u < 4; ++u) a[u] += __shfl_down_sync(0xffffffffu, a[u], o);
        if (lane == 0)
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (c0 + u * nw < ncols) partials[(long long)blockIdx.x * ncols + c0 + u * nw] = a[u];
    }
}

// True in the last block to arrive; that block resets the counter.
__device__ __forceinline__ bool last_block(unsigned* counter) {
    __shared__ bool is_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned t = atomicAdd(counter, 1u);
        is_last = (t == gridDim.x - 1);
        if (is_last) *counter = 0u;
    }
    __syncthreads();
    return is_last;
}

// out[c] = sum_b partials[b][c] in a fixed order (a warp per column, four
// columns interleaved)
__device__ void final_columns(const double* partials, int nb, int ncols, double* out) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    for (int c0 = wid; c0 < ncols; c0 += 4 * nw) {
        double a[4] = {0.0, 0.0, 0.0, 0.0};
        for (int b = lane; b < nb; b += 32)
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (c0 + u * nw < ncols) a[u] += __ldcg(partials + (long long)b * ncols + c0 + u * nw);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int u = 0; u < 4; ++u) a[u] += __shfl_down_sync(0xffffffffu, a[u], o);
        if (lane == 0)
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (c0 + u * nw < ncols) out[c0 + u * nw] = a[u];
    }
}

// ws[t] = w[i0 + t] after w -= V[:, :ncols] h on this block's slice (zero
// beyond n); four independent FMA chains per element
template <typename T>
__device__ __forceinline__ void slice_update(const T* __restrict__ V, long long ldv, int ncols, const T* hs, T* w,
                                             long long n, long long i0, T* ws, bool update) {
    const long long i = i0 + threadIdx.x;
    T v = T(0);
    if (i < n) {
        v = w[i];
        if (update) {
            T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
            int c = 0;
            for (; c + 3 < ncols; c += 4) {
                a0 += V[c * ldv + i] * hs[c];
                a1 += V[(c + 1) * ldv + i] * hs[c + 1];
                a2 += V[(c + 2) * ldv + i] * hs[c + 2];
                a3 += V[(c + 3) * ldv + i] * hs[c + 3];
            }
            for (; c < ncols; ++c) a0 += V[c * ldv + i] * hs[c];
            v -= (a0 + a1) + (a2 + a3);
            w[i] = v;
        }
    }
    ws[threadIdx.x] = v;
    __syncthreads();
}

// h1 = V^T w
template <typename T>
__global__ void __launch_bounds__(GS_E) arn_dots_kernel(const T* __restrict__ V, long long ldv, int ncols, T* w,
                                                        long long n, double* __restrict__ partials, unsigned* counter,
                                                        double* __restrict__ h, const int* __restrict__ stop) {
    if (*stop) return;
    __shared__ T ws[GS_E];
    const long long i0 = (long long)blockIdx.x * GS_E;
    slice_update<T>(V, ldv, ncols, nullptr, w, n, i0, ws, false);
    // the last slice reads V beyond n only where ws is zero; V has M + 1
    // full columns, so the reads stay inside the basis allocation
    warp_column_dots<T>(V, ldv, ncols, ws, i0, partials);
    if (last_block(counter)) final_columns(partials, gridDim.x, ncols, h);
}

// w -= V h1, then h2 = V^T w
template <typename T>
__global__ void __launch_bounds__(GS_E) arn_update_dots_kernel(const T* __restrict__ V, long long ldv, int ncols,
                                                               const double* __restrict__ h1, T* w, long long n,
                                                               double* __restrict__ partials, unsigned* counter,
                                                               double* __restrict__ h2, const int* __restrict__ stop) {
    if (*stop) return;
    __shared__ T ws[GS_E];
    __shared__ T hs[SGK_MAX_KRYLOV + 1];
    for (int c = threadIdx.x; c < ncols; c += blockDim.x) hs[c] = (T)h1[c];
    __syncthreads();
    const long long i0 = (long long)blockIdx.x * GS_E;
    slice_update<T>(V, ldv, ncols, hs, w, n, i0, ws, true);
    warp_column_dots<T>(V, ldv, ncols, ws, i0, partials);
    if (last_block(counter)) final_columns(partials, gridDim.x, ncols, h2);
}

// w -= V h2, ||w||^2, and in the last block: column j of H, the breakdown
// test and 1 / h_{j+1,j}
template <typename T>
__global__ void __launch_bounds__(GS_E) arn_update_norm_kernel(const T* __restrict__ V, long long ldv, int ncols,
                                                               const double* __restrict__ h1,
                                                               const double* __restrict__ h2, T* w, long long n,
                                                               double* __restrict__ partials, unsigned* counter,
                                                               double* __restrict__ H, int j, int M,
                                                               KrylovScalars* __restrict__ ks) {
    if (ks->stop) return;
    __shared__ T ws[GS_E];
    __shared__ T hs[SGK_MAX_KRYLOV + 1];
    __shared__ double wsum[GS_E / 32];
    for (int c = threadIdx.x; c < ncols; c += blockDim.x) hs[c] = (T)h2[c];
    __syncthreads();
    const long long i0 = (long long)blockIdx.x * GS_E;
    slice_update<T>(V, ldv, ncols, hs, w, n, i0, ws, true);
    double a = (double)ws[threadIdx.x] * (double)ws[threadIdx.x];
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < GS_E / 32; ++k) t += wsum[k];
        partials[blockIdx.x] = t;
    }
    if (!last_block(counter)) return;
    __shared__ double beta2;
    final_columns(partials, gridDim.x, 1, &beta2);
    __syncthreads();
    if (threadIdx.x != 0) return;
    double f = ks->fro2;
    if (j >= 1) {
        const double sub = H[(long long)j * M + (j - 1)];
        f += sub * sub;
    }
    for (int i = 0; i <= j; ++i) {
        const double v = h1[i] + h2[i];
        H[(long long)i * M + j] = v;
        f += v * v;
    }
    ks->fro2 = f;
    const double beta = sqrt(beta2);
    H[(long long)(j + 1) * M + j] = beta;
    ks->m_eff = j + 1;
    if (beta <= 1e-12 * sqrt(f)) {
        ks->stop = 1;
        ks->breakdown = 1;
    } else {
        ks->inv_beta = 1.0 / beta;
    }
}

// ---------------------------------------------------------- expm kernel ---

__device__ void blk_matmul(const double* A, const double* B, double* C, int m) {
    for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
        const int i = idx / m, j = idx - (idx / m) * m;
        double acc = 0.0;
        for (int k = 0; k < m; ++k) acc += A[i * m + k] * B[k * m + j];
        C[idx] = acc;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(512) expm_e1_kernel(const double* __restrict__ Hh, int M, const int* __restrict__ m_p,
                                                       int m_fixed, double tau, PadeCoef pc, double* __restrict__ ws,
                                                       double* __restrict__ y) {
    __shared__ double sh[32];
    __shared__ int s_piv;
    __shared__ int s_scale;
    const int m = m_p ? *m_p : m_fixed;
    for (int i = threadIdx.x; i < M; i += blockDim.x) y[i] = 0.0;
    __syncthreads();
    if (m <= 0) return;
    const int mm = m * m;
    double* X = ws;
    double* A2 = ws + 1 * mm;
    double* A4 = ws + 2 * mm;
    double* A6 = ws + 3 * mm;
    double* U = ws + 4 * mm;
    double* V = ws + 5 * mm;
    double* T1 = ws + 6 * mm;
    double* T2 = ws + 7 * mm;
    for (int idx = threadIdx.x; idx < mm; idx += blockDim.x) {
        const int i = idx / m, j = idx - (idx / m) * m;
        X[idx] = tau * Hh[(long long)i * M + j];
    }
    __syncthreads();
    // 1-norm: maximum absolute column sum
    double colmax = 0.0;
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
        double s = 0.0;
        for (int i = 0; i < m; ++i) s += fabs(X[i * m + j]);
        colmax = fmax(colmax, s);
    }
    for (int o = 16; o > 0; o >>= 1) colmax = fmax(colmax, __shfl_down_sync(0xffffffffu, colmax, o));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = colmax;
    __syncthreads();
    if (threadIdx.x == 0) {
        double nm = 0.0;
        for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) nm = fmax(nm, sh[w]);
        int s = 0;
        if (nm > 0.0) s = max(0, (int)ceil(log2(nm / THETA13)));
        s_scale = s;
    }
    __syncthreads();
    const int s = s_scale;
    for (int idx = threadIdx.x; idx < mm; idx += blockDim.x) X[idx] = ldexp(X[idx], -s);
    __syncthreads();
    blk_matmul(X, X, A2, m);
    blk_matmul(A2, A2, A4, m);
    blk_matmul(A4, A2, A6, m);
    const double* b = pc.c;
    for (int idx = threadIdx.x; idx < mm; idx += blockDim.x) T1[idx] = b[13] * A6[idx] + b[11] * A4[idx] + b[9] * A2[idx];
    __syncthreads();
    blk_matmul(A6, T1, T2, m);
    for (int idx = threadIdx.x; idx < mm; idx += blockDim.x) {
        const int i = idx / m, j = idx - (idx / m) * m;
        T2[idx] += b[7] * A6[idx] + b[5] * A4[idx] + b[3] * A2[idx] + (i == j ? b[1] : 0.0);
    }
    __syncthreads();
    blk_matmul(X, T2, U, m);
    for (int idx = threadIdx.x; idx < mm; idx += blockDim.x) T1[idx] = b[12] * A6[idx] + b[10] * A4[idx] + b[8] * A2[idx];
    __syncthreads();
    blk_matmul(A6, T1, V, m);
    for (int idx = threadIdx.x; idx < mm; idx += blockDim.x) {
        const int i = idx / m, j = idx - (idx / m) * m;
        const double v = V[idx] + b[6] * A6[idx] + b[4] * A4[idx] + b[2] * A2[idx] + (i == j ? b[0] : 0.0);
        const double u = U[idx];
        T1[idx] = v - u;  // P
        T2[idx] = v + u;  // Q (right-hand sides)
    }
    __syncthreads();
    double* P = T1;
    double* Q = T2;
    // LU with partial pivoting of P, applied to Q
    for (int k = 0; k < m; ++k) {
        if (threadIdx.x == 0) {
            int piv = k;
            double best = fabs(P[k * m + k]);
            for (int i = k + 1; i < m; ++i)
                if (fabs(P[i * m + k]) > best) {
                    best = fabs(P[i * m + k]);
                    piv = i;
                }
            s_piv = piv;
        }
        __syncthreads();
        const int piv = s_piv;
        if (piv != k) {
            for (int j = threadIdx.x; j < m; j += blockDim.x) {
                double t = P[k * m + j];
                P[k * m + j] = P[piv * m + j];
                P[piv * m + j] = t;
                t = Q[k * m + j];
                Q[k * m + j] = Q[piv * m + j];
                Q[piv * m + j] = t;
            }
            __syncthreads();
        }
        const double pkk = P[k * m + k];
        for (int i = k + 1 + threadIdx.x; i < m; i += blockDim.x) P[i * m + k] /= pkk;
        __syncthreads();
        const int rows = m - k - 1;
        for (int idx = threadIdx.x; idx < rows * m; idx += blockDim.x) {
            const int i = k + 1 + idx / m, j = idx - (idx / m) * m;
            const double l = P[i * m + k];
            Q[i * m + j] -= l * Q[k * m + j];
            if (j > k) P[i * m + j] -= l * P[k * m + j];
        }
        __syncthreads();
    }
    // back substitution, all right-hand sides at once
    for (int k = m - 1; k >= 0; --k) {
        const double pkk = P[k * m + k];
        for (int j = threadIdx.x; j < m; j += blockDim.x) Q[k * m + j] /= pkk;
        __syncthreads();
        for (int idx = threadIdx.x; idx < k * m; idx += blockDim.x) {
            const int i = idx / m, j = idx - (idx / m) * m;
            Q[i * m + j] -= P[i * m + k] * Q[k * m + j];
        }
        __syncthreads();
    }
    // squaring
    double* R = Q;
    double* Rn = U;
    for (int t = 0; t < s; ++t) {
        blk_matmul(R, R, Rn, m);
        double* tmp = R;
        R = Rn;
        Rn = tmp;
    }
    for (int i = threadIdx.x; i < m; i += blockDim.x) y[i] = R[i * m];
}

// Cluster version of the same computation for m <= EXPM_CLUSTER_MAX_M: eight
// CTAs on eight SMs (one thread-block cluster), each holding full copies of
// the work matrices in its shared memory.  A product C = A B is split by
// rows; each CTA writes its rows into every CTA's copy of C through
// distributed shared memory and the cluster barrier (a hardware barrier, no
// spin loop) publishes them.  The elementwise Pade combinations and the LU
// factorisation of the denominator run redundantly in every CTA (identical
// operations in identical order, so the copies stay bitwise equal); the
// right-hand sides of the solve are split by columns.  FP64 throughput per SM
// is what bounds the single-CTA kernel; eight SMs share the products.
constexpr int XCL = 8;
constexpr int XTH = 256;
constexpr int EXPM_CLUSTER_MAX_M = 56;  // 8 m^2 doubles per CTA within 227 KB

// Cluster primitives (PTX ISA: barrier.cluster, mapa, %cluster_ctarank).
// The barrier is the hardware cluster barrier with release/acquire
// semantics for shared::cluster memory; every thread of every CTA executes
// each one, uniformly.
__device__ __forceinline__ void cluster_barrier() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ double* cluster_map(double* p, int rank) {
    unsigned long long out;
    asm volatile("mapa.u64 %0, %1, %2;" : "=l"(out) : "l"(reinterpret_cast<unsigned long long>(p)), "r"(rank));
    return reinterpret_cast<double*>(out);
}
__device__ __forceinline__ int cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return (int)r;
}

__device__ __forceinline__ void xcl_matmul(double* xs, const double* A, const double* B, int coff, int m, int rank) {
    const int r0 = rank * m / XCL, r1 = (rank + 1) * m / XCL;
    for (int idx = threadIdx.x; idx < (r1 - r0) * m; idx += XTH) {
        const int i = r0 + idx / m, j = idx - (idx / m) * m;
        const double* a = A + i * m;
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        int k = 0;
        for (; k + 3 < m; k += 4) {
            s0 += a[k] * B[k * m + j];
            s1 += a[k + 1] * B[(k + 1) * m + j];
            s2 += a[k + 2] * B[(k + 2) * m + j];
            s3 += a[k + 3] * B[(k + 3) * m + j];
        }
        for (; k < m; ++k) s0 += a[k] * B[k * m + j];
        const double v = (s0 + s1) + (s2 + s3);
        double* dst = xs + coff + i * m + j;
#pragma unroll
        for (int p = 0; p < XCL; ++p) *cluster_map(dst, p) = v;
    }
    cluster_barrier();
}

__global__ void __cluster_dims__(XCL, 1, 1) __launch_bounds__(XTH, 1)
    expm_cluster_kernel(const double* __restrict__ Hh, int M, const int* __restrict__ m_p, int m_fixed, double tau,
                        PadeCoef pc, double* __restrict__ y) {
    extern __shared__ __align__(16) double xs[];
    __shared__ double red[XTH / 32];
    __shared__ int s_piv;
    __shared__ double s_inv;
    __shared__ int s_perm[2][EXPM_CLUSTER_MAX_M];
    __shared__ int s_lpiv[2];
    __shared__ double s_linv[2];
    const int rank = cluster_rank();
    const int m = m_p ? *m_p : m_fixed;
    if (rank == 0)
        for (int i = threadIdx.x; i < M; i += XTH) y[i] = 0.0;
    if (m <= 0) return;  // uniform over the cluster: no CTA touches another's memory
    const int mm = m * m;
    enum { X_ = 0, A2_ = 1, A4_ = 2, A6_ = 3, U_ = 4, V_ = 5, T1_ = 6, T2_ = 7 };
    double* X = xs + X_ * mm;
    double* A2 = xs + A2_ * mm;
    double* A4 = xs + A4_ * mm;
    double* A6 = xs + A6_ * mm;
    double* U = xs + U_ * mm;
    double* V = xs + V_ * mm;
    double* T1 = xs + T1_ * mm;
    double* T2 = xs + T2_ * mm;
    for (int idx = threadIdx.x; idx < mm; idx += XTH) {
        const int i = idx / m, j = idx - (idx / m) * m;
        X[idx] = tau * Hh[(long long)i * M + j];
    }
    __syncthreads();
    // ||X||_1: eight threads per column (consecutive lanes) sum strided
    // rows, then xor shuffles within the eight and a maximum over columns
    double colmax = 0.0;
    for (int base = 0; base < m * 8; base += XTH) {
        const int t = base + threadIdx.x, j = t >> 3, part = t & 7;
        double cs = 0.0;
        if (j < m)
            for (int i = part; i < m; i += 8) cs += fabs(X[i * m + j]);
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) cs += __shfl_xor_sync(0xffffffffu, cs, o);
        colmax = fmax(colmax, cs);
    }
    for (int o = 8; o < 32; o <<= 1) colmax = fmax(colmax, __shfl_xor_sync(0xffffffffu, colmax, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = colmax;
    __syncthreads();
    // the scaling exponent s = ceil(log2(||X||_1 / theta_13)), read off the
    // binary exponent of the ratio (exact: x = f 2^e with f in [1/2, 1) has
    // ceil(log2 x) = e, or e - 1 when f = 1/2), and the factor 2^-s
    if (threadIdx.x == 0) {
        double nm = 0.0;
        for (int w = 0; w < XTH / 32; ++w) nm = fmax(nm, red[w]);
        int sc = 0;
        const double ratio = nm / THETA13;
        if (ratio > 1.0) {
            int e = 0;
            const double f = frexp(ratio, &e);
            sc = f == 0.5 ? e - 1 : e;
        }
        s_piv = sc;
        s_inv = ldexp(1.0, -sc);
    }
    __syncthreads();
    const int s = s_piv;
    const double s_fac = s_inv;
    for (int idx = threadIdx.x; idx < mm; idx += XTH) X[idx] *= s_fac;
    // every CTA of the cluster must be running before its shared memory is
    // written by a peer
    __syncthreads();
    cluster_barrier();
    xcl_matmul(xs, X, X, A2_ * mm, m, rank);
    xcl_matmul(xs, A2, A2, A4_ * mm, m, rank);
    xcl_matmul(xs, A4, A2, A6_ * mm, m, rank);
    const double* b = pc.c;
    for (int idx = threadIdx.x; idx < mm; idx += XTH) T1[idx] = b[13] * A6[idx] + b[11] * A4[idx] + b[9] * A2[idx];
    __syncthreads();
    xcl_matmul(xs, A6, T1, T2_ * mm, m, rank);
    for (int idx = threadIdx.x; idx < mm; idx += XTH) {
        const int i = idx / m, j = idx - (idx / m) * m;
        T2[idx] += b[7] * A6[idx] + b[5] * A4[idx] + b[3] * A2[idx] + (i == j ? b[1] : 0.0);
    }
    __syncthreads();
    xcl_matmul(xs, X, T2, U_ * mm, m, rank);
    for (int idx = threadIdx.x; idx < mm; idx += XTH) T1[idx] = b[12] * A6[idx] + b[10] * A4[idx] + b[8] * A2[idx];
    __syncthreads();
    xcl_matmul(xs, A6, T1, V_ * mm, m, rank);
    for (int idx = threadIdx.x; idx < mm; idx += XTH) {
        const int i = idx / m, j = idx - (idx / m) * m;
        const double v = V[idx] + b[6] * A6[idx] + b[4] * A4[idx] + b[2] * A2[idx] + (i == j ? b[0] : 0.0);
        const double u = U[idx];
        T1[idx] = v - u;  // P
        T2[idx] = v + u;  // Q
    }
    __syncthreads();
    double* P = T1;
    double* Q = T2;
    double* Dinv = A4;  // reciprocals of the pivots, by position
    // LU with partial pivoting of P (redundant in every CTA, identical
    // operations in identical order), applied to this CTA's columns [c0, c1)
    // of Q.  Rows are not moved: perm maps a position to its row (two
    // buffers, the step's mapping read from one and the next written to the
    // other).  Each step is one CTA barrier: warp 0 first eliminates column
    // k + 1 and finds its pivot and reciprocal (look-ahead) while the other
    // warps eliminate the remaining columns and the right-hand sides.
    const int c0 = rank * m / XCL, c1 = (rank + 1) * m / XCL, nc = c1 - c0;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    // multipliers by position, two buffers (the step's and the next one's)
    double* const Lbuf = A2;
    // On warp 0: the pivot of column kk over positions i >= kk under the map
    // rowof (largest |P|, compared as the bit patterns of |x|, which order
    // like the values; NaN never wins, ties go to the lowest position), its
    // reciprocal, and the multipliers P[row(i)][kk] / pivot of the positions
    // below it; the position and reciprocal go to slot sl, the multipliers to
    // buffer sl.
    auto pivot = [&](int kk, auto&& rowof, int sl) {
        // per lane its best position (first of its rows), keys as 32-bit
        // halves for the warp max-reductions; key 0 with has = false for a
        // lane without a comparable entry
        unsigned long long best = 0ull;
        int pos = m;
        for (int i = kk + lane; i < m; i += 32) {
            const unsigned long long bits =
                (unsigned long long)__double_as_longlong(P[rowof(i) * m + kk]) & 0x7fffffffffffffffull;
            if (bits <= 0x7ff0000000000000ull && (pos == m || bits > best)) {
                best = bits;
                pos = i;
            }
        }
        const bool has = pos < m;
        const unsigned hi = has ? (unsigned)(best >> 32) + 1u : 0u;  // +1: below every real key
        const unsigned hmax = __reduce_max_sync(0xffffffffu, hi);
        const unsigned lo = hi == hmax ? (unsigned)best : 0u;
        const unsigned lmax = __reduce_max_sync(0xffffffffu, hi == hmax ? lo : 0u);
        // the winners hold (hmax, lmax); positions grow with the lane within
        // a round of 32 rows and each lane keeps its first, so the lowest
        // winning lane holds the lowest winning position... unless a lane's
        // own first row is in a later round than another winner's: take the
        // minimum position over the winners
        const bool win = hmax != 0u && hi == hmax && lo == lmax;
        pos = (int)__reduce_min_sync(0xffffffffu, win ? (unsigned)pos : 0xffffffffu);
        if (hmax == 0u || pos >= m) pos = kk;  // no comparable entry (NaN column)
        const int rp = rowof(pos), rkk = rowof(kk);
        const double pv = P[rp * m + kk];
        // 1 / pv: an FP32 seed refined by two Newton steps r <- r + r (1 - pv r)
        // (quadratic convergence, 2^-24 -> 2^-48 -> below one ulp); the
        // division when pv is outside the FP32 range
        double inv;
        const double apv = fabs(pv);
        if (apv > 1e-30 && apv < 1e30) {
            double r = (double)__frcp_rn((float)pv);
            r = fma(r, fma(-pv, r, 1.0), r);
            r = fma(r, fma(-pv, r, 1.0), r);
            inv = r;
        } else {
            inv = 1.0 / pv;
        }
        if (lane == 0) {
            s_lpiv[sl] = pos;
            s_linv[sl] = inv;
        }
        // positions below kk after exchanging kk and pos
        double* const Lm = Lbuf + sl * m;
        for (int i = kk + 1 + lane; i < m; i += 32) {
            const int ri = i == pos ? rkk : rowof(i);
            Lm[i] = P[ri * m + kk] * inv;
        }
    };
    for (int i = threadIdx.x; i < m; i += XTH) s_perm[0][i] = i;
    __syncthreads();
    if (wid == 0) pivot(0, [&](int i) { return i; }, 0);
    __syncthreads();
    for (int k = 0; k < m; ++k) {
        const int cur_b = k & 1;
        const int* perm = s_perm[cur_b];
        const int piv = s_lpiv[cur_b];
        const double inv = s_linv[cur_b];
        const int rowk = perm[piv], rowp = perm[k];
        // position -> row for this step (positions k and piv exchanged)
        auto rowof = [&](int i) { return i == k ? rowk : (i == piv ? rowp : perm[i]); };
        if (threadIdx.x == 0) Dinv[k] = inv;
        for (int i = threadIdx.x; i < m; i += XTH) s_perm[cur_b ^ 1][i] = rowof(i);
        const double* pk = P + rowk * m;  // the pivot row
        const int rows = m - k - 1;
        const int wcols = m - k - 2 > 0 ? m - k - 2 : 0;
        // multipliers of this step (written by warp 0 in the previous one)
        const double* const Lcur = Lbuf + cur_b * m;
        double lreg[(EXPM_CLUSTER_MAX_M + 31) / 32];
        if (wid == 0) {
            // column k + 1, then its pivot and the next multipliers
#pragma unroll
            for (int q = 0; q < (EXPM_CLUSTER_MAX_M + 31) / 32; ++q) {
                const int i = k + 1 + lane + 32 * q;
                lreg[q] = i < m ? Lcur[i] : 0.0;
            }
#pragma unroll
            for (int q = 0; q < (EXPM_CLUSTER_MAX_M + 31) / 32; ++q) {
                const int i = k + 1 + lane + 32 * q;
                if (i < m && k + 1 < m) P[rowof(i) * m + k + 1] -= lreg[q] * pk[k + 1];
            }
            __syncwarp();
            if (k + 1 < m) pivot(k + 1, rowof, cur_b ^ 1);
        } else if ((wid & 3) != 0) {
            // columns k + 2 .. m - 1 of P and the c1 - c0 right-hand sides,
            // (rows x w) items over the warps that do not share warp 0's
            // sub-partition (warp w runs on sub-partition w mod 4), so that
            // warp 0's FP64 chain does not queue behind their FP64 work
            const int w = wcols + nc;
            const int wk = wid - 1 - wid / 4, nthr = (XTH / 32 - XTH / 128) * 32;
            for (int idx = wk * 32 + lane; idx < rows * w; idx += nthr) {
                const int i = k + 1 + idx / w, jj = idx - (idx / w) * w;
                const int ri = rowof(i);
                const double l = Lcur[i];
                if (jj < wcols) {
                    const int j = k + 2 + jj;
                    P[ri * m + j] -= l * pk[j];
                } else {
                    const int j = c0 + jj - wcols;
                    Q[ri * m + j] -= l * Q[rowk * m + j];
                }
            }
        }
        __syncthreads();
    }
    // back substitution U x = Q' for each own column: one warp per column,
    // lanes over positions (x in registers), the solved entry broadcast by
    // shuffle; perm holds the final position -> row map
    {
        const int* perm = s_perm[m & 1];
        constexpr int PL = (EXPM_CLUSTER_MAX_M + 31) / 32;  // positions per lane
        for (int cc = wid; cc < nc; cc += XTH / 32) {
            const int j = c0 + cc;
            double x[PL];
#pragma unroll
            for (int q = 0; q < PL; ++q) {
                const int i = lane + 32 * q;
                x[q] = i < m ? Q[perm[i] * m + j] : 0.0;
            }
            for (int k = m - 1; k >= 0; --k) {
                const int ql = k >> 5, kl = k & 31;
                double xk = 0.0;
#pragma unroll
                for (int q = 0; q < PL; ++q)
                    if (q == ql) xk = x[q];
                xk = __shfl_sync(0xffffffffu, xk, kl) * Dinv[k];
#pragma unroll
                for (int q = 0; q < PL; ++q) {
                    const int i = lane + 32 * q;
                    if (i < k) x[q] -= P[perm[i] * m + k] * xk;
                    else if (i == k) x[q] = xk;
                }
            }
            // publish this column of R = P^{-1} Q into every CTA's copy of Q
#pragma unroll
            for (int q = 0; q < PL; ++q) {
                const int i = lane + 32 * q;
                if (i < m)
#pragma unroll
                    for (int pr = 0; pr < XCL; ++pr) *cluster_map(xs + T2_ * mm + i * m + j, pr) = x[q];
            }
        }
    }
    cluster_barrier();
    int cur = T2_, nxt = U_;
    for (int t = 0; t < s; ++t) {
        // the barrier closing this product also ends every CTA's reads of
        // cur, which the next product overwrites
        xcl_matmul(xs, xs + cur * mm, xs + cur * mm, nxt * mm, m, rank);
        const int tmp = cur;
        cur = nxt;
        nxt = tmp;
    }
    if (rank == 0)
        for (int i = threadIdx.x; i < m; i += XTH) y[i] = xs[cur * mm + i * m];
}

// W = gamma V[:, :m_eff] y  (FP64 accumulation, four chains over the
// columns: FP64 dependent latency is long on this part)
template <typename T>
__global__ void combine_kernel(const T* __restrict__ V, long long ldv, KrylovScalars* __restrict__ ks,
                               const double* __restrict__ y, double* __restrict__ W, long long n,
                               const double* __restrict__ H, int M, double tau) {
    __shared__ double ys[SGK_MAX_KRYLOV + 1];
    const int m = ks->m_eff;
    const double g = ks->gamma;
    for (int c = threadIdx.x; c < m; c += blockDim.x) ys[c] = y[c] * g;
    // a-posteriori error estimate of the Krylov approximation, relative to
    // the result: tau h_{m+1,m} |[exp(tau H_m) e_1]_m| / ||exp(tau H_m) e_1||
    // (Saad, SIAM J. Numer. Anal. 29 (1992), Section 5: the residual of the
    // projected ODE at the end of the span, times the span).  A projection
    // whose result underflowed to zero without a breakdown has lost it: 1
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        double est = 0.0;
        if (m >= 1 && !ks->breakdown && ks->gamma > 0.0) {
            double yy = 0.0;
            for (int c = 0; c < m; ++c) yy += y[c] * y[c];
            const double beta = H[(long long)m * M + (m - 1)];
            est = yy > 0.0 ? fabs(tau * beta * y[m - 1]) / sqrt(yy) : 1.0;
        }
        ks->err_est = est;
        ks->err_max = fmax(ks->err_max, est);
    }
    __syncthreads();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
        int c = 0;
        for (; c + 3 < m; c += 4) {
            a0 += (double)V[c * ldv + i] * ys[c];
            a1 += (double)V[(c + 1) * ldv + i] * ys[c + 1];
            a2 += (double)V[(c + 2) * ldv + i] * ys[c + 2];
            a3 += (double)V[(c + 3) * ldv + i] * ys[c + 3];
        }
        for (; c < m; ++c) a0 += (double)V[c * ldv + i] * ys[c];
        W[i] = (a0 + a1) + (a2 + a3);
    }
}

// blocks of 128 threads for the combination: at least one per SM
int combine_grid(const sgk_ctx* ctx, long long n) {
    const long long b = (n + 127) / 128;
    return (int)std::max(1LL, std::min<long long>(b, (long long)ctx->num_sms * 8));
}

// ------------------------------------------------------ vector kernels ---

template <typename TS, typename TD>
__global__ void convert_kernel(const TS* __restrict__ x, TD* __restrict__ y, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = (TD)x[i];
}

// z = a x + b y, scalars from the host
__global__ void axpby_kernel(double a, const double* __restrict__ x, double b, const double* __restrict__ y,
                             double* __restrict__ z, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        z[i] = a * x[i] + b * y[i];
}

// G = U - c F - W
__global__ void residual_kernel(const double* __restrict__ U, const double* __restrict__ F,
                                const double* __restrict__ W, double c, double* __restrict__ G, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        G[i] = U[i] - c * F[i] - W[i];
}

// q = p - c Jp
template <typename T>
__global__ void jac_finish_kernel(const double* __restrict__ p, const T* __restrict__ Jp, double c,
                                  double* __restrict__ q, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        q[i] = p[i] - c * (double)Jp[i];
}

// CG: alpha = rr / pq; x += alpha p; r -= alpha q
__global__ void cg_update_kernel(double* __restrict__ x, double* __restrict__ r, const double* __restrict__ p,
                                 const double* __restrict__ q, const double* __restrict__ rr,
                                 const double* __restrict__ pq, long long n) {
    const double alpha = *rr / *pq;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        x[i] += alpha * p[i];
        r[i] -= alpha * q[i];
    }
}

// CG: p = r + (rr_new / rr_old) p
__global__ void cg_direction_kernel(double* __restrict__ p, const double* __restrict__ r,
                                    const double* __restrict__ rr_new, const double* __restrict__ rr_old, long long n) {
    const double beta = *rr_new / *rr_old;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        p[i] = r[i] + beta * p[i];
}

__global__ void copy_scalar_kernel(double* __restrict__ dst, const double* __restrict__ src) { *dst = *src; }

// x += V[:, :m] y with y on the device
__global__ void basis_accumulate_kernel(const double* __restrict__ V, long long ldv, int m,
                                        const double* __restrict__ y, double* __restrict__ x, long long n) {
    __shared__ double ys[SGK_MAX_KRYLOV + 1];
    for (int c = threadIdx.x; c < m; c += blockDim.x) ys[c] = y[c];
    __syncthreads();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int c = 0; c < m; ++c) acc += V[c * ldv + i] * ys[c];
        x[i] += acc;
    }
}

// GMRES: Givens rotations on column j of the (restart+1) x restart matrix
// Hg (row-major, ld = restart), update of g; reports |g_{j+1}|, h_{j+1,j}
// and the rotated diagonal to the host.
__global__ void gmres_givens_kernel(int j, int ld, double* __restrict__ Hg, double* __restrict__ cs,
                                    double* __restrict__ sn, double* __restrict__ g, const double* __restrict__ h1,
                                    const double* __restrict__ h2, const double* __restrict__ hn2,
                                    double* __restrict__ report) {
    if (threadIdx.x != 0) return;
    for (int i = 0; i <= j; ++i) Hg[i * ld + j] = h1[i] + h2[i];
    const double hn = sqrt(*hn2);
    Hg[(j + 1) * ld + j] = hn;
    for (int i = 0; i < j; ++i) {
        const double t = cs[i] * Hg[i * ld + j] + sn[i] * Hg[(i + 1) * ld + j];
        Hg[(i + 1) * ld + j] = -sn[i] * Hg[i * ld + j] + cs[i] * Hg[(i + 1) * ld + j];
        Hg[i * ld + j] = t;
    }
    const double den = hypot(Hg[j * ld + j], Hg[(j + 1) * ld + j]);
    cs[j] = Hg[j * ld + j] / den;
    sn[j] = Hg[(j + 1) * ld + j] / den;
    Hg[j * ld + j] = den;
    Hg[(j + 1) * ld + j] = 0.0;
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    report[0] = fabs(g[j + 1]);
    report[1] = hn;
    report[2] = den;
    report[3] = hn > 0.0 ? 1.0 / hn : 0.0;
}

// GMRES: solve the triangular system H[:m,:m] y = g[:m]
__global__ void gmres_solve_kernel(int m, int ld, const double* __restrict__ Hg, const double* __restrict__ g,
                                   double* __restrict__ y) {
    if (threadIdx.x != 0) return;
    for (int i = m - 1; i >= 0; --i) {
        double acc = g[i];
        for (int c = i + 1; c < m; ++c) acc -= Hg[i * ld + c] * y[c];
        y[i] = acc / Hg[i * ld + i];
    }
}

__global__ void gmres_init_kernel(double* __restrict__ g, int len, const double* __restrict__ beta,
                                  double* __restrict__ inv_beta) {
    for (int i = threadIdx.x; i < len; i += blockDim.x) g[i] = 0.0;
    __syncthreads();
    if (threadIdx.x == 0) {
        g[0] = *beta;
        *inv_beta = 1.0 / *beta;
    }
}

int grid_for(const sgk_ctx* ctx, long long n) {
    long long b = (n + 255) / 256;
    return (int)std::max(1LL, std::min<long long>(b, (long long)ctx->num_sms * 4));
}

}  // namespace

int reduction_blocks(const sgk_ctx* ctx, int64_t n) {
    // about one block per SM: FP64 throughput is per SM
    long long b = (n + 127) / 128;
    return (int)std::max(1LL, std::min<long long>(b, (long long)ctx->num_sms));
}

// ------------------------------------------------------------ host API ---

PadeCoef pade13_coefficients() {
    // numerator coefficients of the [m/m] Pade approximant of e^x:
    // c_j = (2m - j)! m! / ((2m)! j! (m - j)!)
    PadeCoef pc;
    const int m = 13;
    long double f[27];
    f[0] = 1;
    for (int i = 1; i <= 26; ++i) f[i] = f[i - 1] * i;
    for (int j = 0; j <= m; ++j) pc.c[j] = (double)(f[2 * m - j] * f[m] / (f[2 * m] * f[j] * f[m - j]));
    return pc;
}

void vk_dot(sgk_ctx* ctx, const double* a, const double* b, long long n, double* partials, double* out, int mode,
            const int* stop) {
    KTimer kt(ctx, KC_REDUCE);
    const int nb = reduction_blocks(ctx, n);
    dot_partial_kernel<double, double><<<nb, RED_THREADS, 0, ctx->stream>>>(a, b, n, partials, stop);
    reduce_final_kernel<<<1, RED_THREADS, 0, ctx->stream>>>(partials, nb, out, mode, stop);
    check_launch("dot");
    count_launch(ctx, 2);
}

template <typename T>
void vk_dotT(sgk_ctx* ctx, const T* a, const T* b, long long n, double* partials, double* out, int mode,
             const int* stop) {
    KTimer kt(ctx, KC_REDUCE);
    const int nb = reduction_blocks(ctx, n);
    dot_partial_kernel<T, T><<<nb, RED_THREADS, 0, ctx->stream>>>(a, b, n, partials, stop);
    reduce_final_kernel<<<1, RED_THREADS, 0, ctx->stream>>>(partials, nb, out, mode, stop);
    check_launch("dotT");
    count_launch(ctx, 2);
}

template <typename T>
void vk_mdot(sgk_ctx* ctx, const T* V, long long ldv, int ncols, const T* w, long long n, double* partials,
             double* out, const int* stop) {
    KTimer kt(ctx, KC_REDUCE);
    const int nb = reduction_blocks(ctx, n);
    mdot_partial_kernel<T><<<nb, RED_THREADS, 0, ctx->stream>>>(V, ldv, ncols, w, n, partials, stop);
    mdot_final_kernel<<<1, 256, 0, ctx->stream>>>(partials, nb, ncols, out, stop);
    check_launch("mdot");
    count_launch(ctx, 2);
}

template <typename T>
void vk_gs_update(sgk_ctx* ctx, const T* V, long long ldv, int ncols, const double* h, T* w, long long n,
                  const int* stop) {
    KTimer kt(ctx, KC_REDUCE);
    gs_update_kernel<T><<<grid_for(ctx, n), 256, 0, ctx->stream>>>(V, ldv, ncols, h, w, n, stop);
    check_launch("gs_update");
    count_launch(ctx);
}

void vk_convert(sgk_ctx* ctx, const double* x, float* y, long long n) {
    KTimer kt(ctx, KC_VECTOR);
    convert_kernel<double, float><<<grid_for(ctx, n), 256, 0, ctx->stream>>>(x, y, n);
    check_launch("convert");
    count_launch(ctx);
}
void vk_convert(sgk_ctx* ctx, const float* x, double* y, long long n) {
    KTimer kt(ctx, KC_VECTOR);
    convert_kernel<float, double><<<grid_for(ctx, n), 256, 0, ctx->stream>>>(x, y, n);
    check_launch("convert");
    count_launch(ctx);
}
// double-float conversions (split, pair sum in FP64, pair sum in FP32)
__global__ void df_split_kernel(const double* __restrict__ x, dfloat* __restrict__ y, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = df_split(x[i]);
}
__global__ void df_value_kernel(const dfloat* __restrict__ x, double* __restrict__ y, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = df_value(x[i]);
}
__global__ void df_float_kernel(const dfloat* __restrict__ x, float* __restrict__ y, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = df_float(x[i]);
}
void vk_convert(sgk_ctx* ctx, const double* x, dfloat* y, long long n) {
    KTimer kt(ctx, KC_VECTOR);
    df_split_kernel<<<grid_for(ctx, n), 256, 0, ctx->stream>>>(x, y, n);
    check_launch("df_split");
    count_launch(ctx);
}
void vk_convert(sgk_ctx* ctx, const dfloat* x, double* y, long long n) {
    KTimer kt(ctx, KC_VECTOR);
    df_value_kernel<<<grid_for(ctx, n), 256, 0, ctx->stream>>>(x, y, n);
    check_launch("df_value");
    count_launch(ctx);
}
void vk_convert(sgk_ctx* ctx, const dfloat* x, float* y, long long n) {
    KTimer kt(ctx, KC_VECTOR);
    df_float_kernel<<<grid_for(ctx, n), 256, 0, ctx->stream>>>(x, y, n);
    check_launch("df_float");
    count_launch(ctx);
}
void vk_axpby(sgk_ctx* ctx, double a, const double* x, double b, const double* y, double* z, long long n) {
    KTimer kt(ctx, KC_VECTOR);
    axpby_kernel<<<grid_for(ctx, n), 256, 0, ctx->stream>>>(a, x, b, y, z, n);
    check_launch("axpby");
    count_launch(ctx);
}
void vk_residual(sgk_ctx* ctx, const double* U, const double* F, const double* W, double c, double* G, long long n) {
    KTimer kt(ctx, KC_VECTOR);
    residual_kernel<<<grid_for(ctx, n), 256, 0, ctx->stream>>>(U, F, W, c, G, n);
    check_launch("residual");
    count_launch(ctx);
}
template <typename T>
void vk_jac_finish(sgk_ctx* ctx, const double* p, const T* Jp, double c, double* q, long long n) {
    KTimer kt(ctx, KC_VECTOR);
    jac_finish_kernel<T><<<grid_for(ctx, n), 256, 0, ctx->stream>>>(p, Jp, c, q, n);
    check_launch("jac_finish");
    count_launch(ctx);
}
void vk_cg_update(sgk_ctx* ctx, double* x, double* r, const double* p, const double* q, const double* rr,
                  const double* pq, long long n) {
    KTimer kt(ctx, KC_VECTOR);
    cg_update_kernel<<<grid_for(ctx, n), 256, 0, ctx->stream>>>(x, r, p, q, rr, pq, n);
    check_launch("cg_update");
    count_launch(ctx);
}
void vk_cg_direction(sgk_ctx* ctx, double* p, const double* r, const double* rr_new, const double* rr_old,
                     long long n) {
    KTimer kt(ctx, KC_VECTOR);
    cg_direction_kernel<<<grid_for(ctx, n), 256, 0, ctx->stream>>>(p, r, rr_new, rr_old, n);
    check_launch("cg_direction");
    count_launch(ctx);
}
void vk_copy_scalar(sgk_ctx* ctx, double* dst, const double* src) {
    KTimer kt(ctx, KC_VECTOR);
    copy_scalar_kernel<<<1, 1, 0, ctx->stream>>>(dst, src);
    check_launch("copy_scalar");
    count_launch(ctx);
}
void vk_basis_accumulate(sgk_ctx* ctx, const double* V, long long ldv, int m, const double* y, double* x,
                         long long n) {
    KTimer kt(ctx, KC_VECTOR);
    basis_accumulate_kernel<<<grid_for(ctx, n), 256, 0, ctx->stream>>>(V, ldv, m, y, x, n);
    check_launch("basis_accumulate");
    count_launch(ctx);
}
void vk_scale_from(sgk_ctx* ctx, const double* x, double* y, long long n, const double* s, const int* stop) {
    KTimer kt(ctx, KC_VECTOR);
    scale_to_kernel<double><<<grid_for(ctx, n), 256, 0, ctx->stream>>>(x, y, n, s, stop);
    check_launch("scale");
    count_launch(ctx);
}
void gmres_givens(sgk_ctx* ctx, int j, int ld, double* Hg, double* cs, double* sn, double* g, const double* h1,
                  const double* h2, const double* hn2, double* report) {
    KTimer kt(ctx, KC_VECTOR);
    gmres_givens_kernel<<<1, 32, 0, ctx->stream>>>(j, ld, Hg, cs, sn, g, h1, h2, hn2, report);
    check_launch("gmres_givens");
    count_launch(ctx);
}
void gmres_solve(sgk_ctx* ctx, int m, int ld, const double* Hg, const double* g, double* y) {
    KTimer kt(ctx, KC_VECTOR);
    gmres_solve_kernel<<<1, 32, 0, ctx->stream>>>(m, ld, Hg, g, y);
    check_launch("gmres_solve");
    count_launch(ctx);
}
void gmres_init(sgk_ctx* ctx, double* g, int len, const double* beta, double* inv_beta) {
    KTimer kt(ctx, KC_VECTOR);
    gmres_init_kernel<<<1, 64, 0, ctx->stream>>>(g, len, beta, inv_beta);
    check_launch("gmres_init");
    count_launch(ctx);
}

void expm_e1(sgk_ctx* ctx, const double* H, int M, const int* m_dev, int m_fixed, double tau, double* ws, double* y) {
    KTimer kt(ctx, KC_EXPM);
    if (M <= EXPM_CLUSTER_MAX_M) {
        const size_t smem = sizeof(double) * 8 * M * M;
        allow_max_dynamic_smem(ctx->smem_optin, expm_cluster_kernel);
        expm_cluster_kernel<<<XCL, XTH, smem, ctx->stream>>>(H, M, m_dev, m_fixed, tau, pade13_coefficients(), y);
        check_launch("expm_cluster");
    } else {
        expm_e1_kernel<<<1, 512, 0, ctx->stream>>>(H, M, m_dev, m_fixed, tau, pade13_coefficients(), ws, y);
        check_launch("expm_e1");
    }
    count_launch(ctx);
}

// ------------------------------------------- allocation-free expm entry ---
//
// Scratch of sgk_expm_e1_noalloc for m above EXPM_CLUSTER_MAX_M (smaller m
// run the cluster kernel, whose work matrices live in shared memory): eight
// m x m work matrices for m up to SGK_EXPM_NOALLOC_MAX_M, compiled into the
// library (every GPU that loads it
// holds the 256 KB until the process exits).  The kernel writes every work
// entry before reading it, so nothing has to start at zero; concurrent calls
// share it and must not overlap on the GPU.
static __device__ __align__(256) double g_expm_scratch[8 * SGK_EXPM_NOALLOC_MAX_M * SGK_EXPM_NOALLOC_MAX_M];

// Per-device set-up of sgk_expm_e1_noalloc, made by the first call on a
// device and again whenever that device's context is not the one the set-up
// was made in (after a cudaDeviceReset the runtime creates a new primary
// context, in which the symbol may live at another address and function
// attributes start over).  Host code cannot pass g_expm_scratch itself (its
// name there is a host-side stand-in), so the set-up looks up the device
// address with cudaGetSymbolAddress; it also raises the cluster kernel's
// dynamic shared-memory limit once instead of on every call.
struct NoallocSetup {
    std::mutex mu;
    unsigned long long ctx_id = 0;  // context of the set-up (0: none yet, or ids unavailable)
    bool done = false;
    double* scratch = nullptr;
};
static NoallocSetup g_noalloc_setup[256];

// Unique id of the calling thread's current context (cuCtxGetCurrent and
// cuCtxGetId through the runtime's driver entry points, so that the library
// does not link the driver library itself); 0 when the driver does not
// provide them.
static unsigned long long current_context_id() {
    using GetCurrent = int (*)(void**);
    using GetId = int (*)(void*, unsigned long long*);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<GetCurrent>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetId>(f);
        (void)cudaGetLastError();
    });
    void* ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
    return id;
}

extern "C" int sgk_expm_e1_noalloc(int m, const double* X_dev, double tau, double* y_dev, void* cuda_stream) {
    if (m < 1 || m > SGK_EXPM_NOALLOC_MAX_M || !X_dev || !y_dev) return SGK_EINVAL;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) {
        (void)cudaGetLastError();
        return SGK_ECUDA;
    }
    // 0 when this thread has not used the device through the runtime yet:
    // the set-up below binds the context, and its id is stored after it
    const unsigned long long ctx_id = current_context_id();
    NoallocSetup& su = g_noalloc_setup[dev];
    double* ws = nullptr;
    {
        std::lock_guard<std::mutex> lock(su.mu);
        if (!su.done || su.ctx_id != ctx_id) {
            su.done = false;
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_expm_scratch) != cudaSuccess || !p) {
                (void)cudaGetLastError();
                return SGK_ECUDA;
            }
            su.scratch = static_cast<double*>(p);
            int optin = 0;
            cudaFuncAttributes fa;
            if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
                cudaFuncGetAttributes(&fa, reinterpret_cast<const void*>(expm_cluster_kernel)) != cudaSuccess ||
                cudaFuncSetAttribute(expm_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     optin - (int)fa.sharedSizeBytes) != cudaSuccess) {
                (void)cudaGetLastError();
                return SGK_ECUDA;
            }
            su.ctx_id = current_context_id();
            su.done = true;
        }
        ws = su.scratch;
    }
    if (m <= EXPM_CLUSTER_MAX_M) {
        // the cluster kernel keeps its work matrices in shared memory
        const size_t smem = sizeof(double) * 8 * m * m;
        expm_cluster_kernel<<<XCL, XTH, smem, static_cast<cudaStream_t>(cuda_stream)>>>(X_dev, m, nullptr, m, tau,
                                                                                     pade13_coefficients(), y_dev);
        return cudaGetLastError() == cudaSuccess ? SGK_OK : SGK_ECUDA;
    }
    expm_e1_kernel<<<1, 512, 0, static_cast<cudaStream_t>(cuda_stream)>>>(X_dev, m, nullptr, m, tau,
                                                                          pade13_coefficients(), ws, y_dev);
    if (cudaGetLastError() != cudaSuccess) return SGK_ECUDA;
    return SGK_OK;
}

void krylov_finish(sgk_ctx* ctx, const KrylovWork<double>& kw, double* W, long long n, int M, double dt) {
    expm_e1(ctx, kw.H, M, &kw.ks->m_eff, 0, dt, kw.expm_ws, kw.y);
    {
        KTimer kt(ctx, KC_VECTOR);
        combine_kernel<double><<<combine_grid(ctx, n), 128, 0, ctx->stream>>>(kw.V, n, kw.ks, kw.y, W, n, kw.H, M, dt);
    }
    check_launch("combine");
    count_launch(ctx);
}

void krylov_expv_persistent(sgk_ctx* ctx, const sgk_op* op, const PersistentWork& pw, const KrylovWork<double>& kw,
                            const double* v, double* W, long long n, int M, double dt) {
    arnoldi_persistent(ctx, op, pw, kw, v, n, M);
    expm_e1(ctx, kw.H, M, &kw.ks->m_eff, 0, dt, kw.expm_ws, kw.y);
    {
        KTimer kt(ctx, KC_VECTOR);
        combine_kernel<double><<<combine_grid(ctx, n), 128, 0, ctx->stream>>>(kw.V, n, kw.ks, kw.y, W, n, kw.H, M, dt);
    }
    check_launch("combine");
    count_launch(ctx);
}

template <typename T>
void krylov_expv_dev(sgk_ctx* ctx, const KrylovWork<T>& kw, const std::function<void(const T*, T*)>& matvec,
                     const double* v, double* W, long long n, int M, double dt) {
    KrylovScalars* ks = kw.ks;
    const int* stop = &ks->stop;
    // gamma = ||v||
    vk_dot(ctx, v, v, n, kw.partials, kw.scal, 0, nullptr);
    {
        KTimer kt(ctx, KC_VECTOR);
        krylov_init_kernel<<<1, 1, 0, ctx->stream>>>(kw.scal, ks);
    }
    check_launch("krylov_init");
    count_launch(ctx);
    {
        KTimer kt(ctx, KC_VECTOR);
        scale_to_kernel<T><<<grid_for(ctx, n), 256, 0, ctx->stream>>>(v, kw.V, n, &ks->inv_gamma, stop);
    }
    check_launch("scale_to");
    count_launch(ctx);
    for (int j = 0; j < M; ++j) {
        T* vj = kw.V + (long long)j * n;
        matvec(vj, kw.w);
        {
            // classical Gram-Schmidt twice and the norm, three fused kernels
            KTimer kt(ctx, KC_REDUCE);
            const int nb = (int)((n + GS_E - 1) / GS_E);
            arn_dots_kernel<T><<<nb, GS_E, 0, ctx->stream>>>(kw.V, n, j + 1, kw.w, n, kw.partials, kw.counter, kw.h1,
                                                            stop);
            arn_update_dots_kernel<T><<<nb, GS_E, 0, ctx->stream>>>(kw.V, n, j + 1, kw.h1, kw.w, n, kw.partials,
                                                                   kw.counter, kw.h2, stop);
            arn_update_norm_kernel<T><<<nb, GS_E, 0, ctx->stream>>>(kw.V, n, j + 1, kw.h1, kw.h2, kw.w, n, kw.partials,
                                                                   kw.counter, kw.H, j, M, ks);
        }
        check_launch("arnoldi_cgs2");
        count_launch(ctx, 3);
        {
            KTimer kt(ctx, KC_VECTOR);
            scale_vec_kernel<T><<<grid_for(ctx, n), 256, 0, ctx->stream>>>(kw.w, kw.V + (long long)(j + 1) * n, n,
                                                                            &ks->inv_beta, stop);
        }
        check_launch("scale_vec");
        count_launch(ctx);
    }
    expm_e1(ctx, kw.H, M, &ks->m_eff, 0, dt, kw.expm_ws, kw.y);
    {
        KTimer kt(ctx, KC_VECTOR);
        combine_kernel<T><<<combine_grid(ctx, n), 128, 0, ctx->stream>>>(kw.V, n, ks, kw.y, W, n, kw.H, M, dt);
    }
    check_launch("combine");
    count_launch(ctx);
}

template void krylov_expv_dev<double>(sgk_ctx*, const KrylovWork<double>&,
                                      const std::function<void(const double*, double*)>&, const double*, double*,
                                      long long, int, double);
template void krylov_expv_dev<float>(sgk_ctx*, const KrylovWork<float>&,
                                     const std::function<void(const float*, float*)>&, const double*, double*,
                                     long long, int, double);
template void vk_mdot<double>(sgk_ctx*, const double*, long long, int, const double*, long long, double*, double*,
                              const int*);
template void vk_gs_update<double>(sgk_ctx*, const double*, long long, int, const double*, double*, long long,
                                   const int*);
template void vk_jac_finish<double>(sgk_ctx*, const double*, const double*, double, double*, long long);
template void vk_jac_finish<float>(sgk_ctx*, const double*, const float*, double, double*, long long);
