// Measured arithmetic peaks for the ALU-bound rooflines (no counterpart in
// the paper): the FMA rate of the FP32 and FP64 pipes on this device, from a
// kernel whose every thread runs eight independent FMA chains.
//
// Eight chains per thread and eight resident CTAs of 256 threads per SM keep
// each pipe's dependent-issue latency covered many times over, so the rate
// is the issue rate of the FMA instruction.  The multiplier and addend are
// kernel arguments (not constants the compiler could fold), chosen so that
// the values stay finite and normal for any trip count: x <- x m + c with
// m = 1 - 2^-20 and c = 2^-20 converges to 1 from any start in [0, 2].
#include <algorithm>
#include <vector>

#include "sgk_internal.h"

namespace {

constexpr int CHAINS = 8;
constexpr int PROBE_THREADS = 256;

template <typename T>
__global__ void __launch_bounds__(PROBE_THREADS) fma_probe_kernel(int iters, T m, T c, T* __restrict__ sink) {
    T x[CHAINS];
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) x[k] = T(1) + T(k) * T(0.0625);
#pragma unroll 1
    for (int it = 0; it < iters; it += 8) {
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int k = 0; k < CHAINS; ++k) x[k] = fma(x[k], m, c);
    }
    T s = T(0);
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) s += x[k];
    sink[blockIdx.x * (size_t)PROBE_THREADS + threadIdx.x] = s;
}

template <typename T>
double probe(int device, int iters) {
    int sms = 0;
    SGK_CUDA_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    const int grid = sms * 8;
    T* sink = nullptr;
    SGK_CUDA_CHECK(cudaMalloc(&sink, sizeof(T) * (size_t)grid * PROBE_THREADS));
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double best = 0.0;
    try {
        SGK_CUDA_CHECK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        SGK_CUDA_CHECK(cudaEventCreate(&e0));
        SGK_CUDA_CHECK(cudaEventCreate(&e1));
        const T m = T(1) - T(1.0 / 1048576.0), c = T(1.0 / 1048576.0);
        // three untimed launches (clock ramp, module load), then the best of
        // five timed ones
        for (int rep = 0; rep < 8; ++rep) {
            SGK_CUDA_CHECK(cudaEventRecord(e0, s));
            fma_probe_kernel<T><<<grid, PROBE_THREADS, 0, s>>>(iters, m, c, sink);
            check_launch("fma_probe_kernel");
            SGK_CUDA_CHECK(cudaEventRecord(e1, s));
            SGK_CUDA_CHECK(cudaEventSynchronize(e1));
            float ms = 0.f;
            SGK_CUDA_CHECK(cudaEventElapsedTime(&ms, e0, e1));
            if (rep >= 3 && ms > 0.f) {
                const double flops = 2.0 * CHAINS * (double)iters * grid * PROBE_THREADS;
                best = std::max(best, flops / (ms * 1e-3));
            }
        }
    } catch (...) {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (s) cudaStreamDestroy(s);
        cudaFree(sink);
        throw;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(s);
    cudaFree(sink);
    return best;
}

}  // namespace

int sgk_alu_peak(int device, int kind, double* flops_per_s) {
    if (!flops_per_s || (kind != SGK_PEAK_FP32_FMA && kind != SGK_PEAK_FP64_FMA)) return SGK_EINVAL;
    try {
        int ndev = 0;
        SGK_CUDA_CHECK(cudaGetDeviceCount(&ndev));
        if (device < 0 || device >= ndev) return SGK_EINVAL;
        SGK_CUDA_CHECK(cudaSetDevice(device));
        // about 20 ms per launch on a part of this class: 2^18 FP32 or 2^12
        // FP64 iterations of the 8 chains
        *flops_per_s = kind == SGK_PEAK_FP32_FMA ? probe<float>(device, 1 << 18) : probe<double>(device, 1 << 12);
        return SGK_OK;
    } catch (const SgkError& e) {
        return e.code;
    }
}
