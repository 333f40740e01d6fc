// Sparse-grid index set on the device (Section 2.1, eqs. sp10-sp14).
//
// Level tuples |l|_1 <= n are enumerated in lexicographic order (l_1
// slowest).  The order is a combinatorial number system: the rank of l is
//   sum_m sum_{v < l_m} C(B_m - v + d - m - 1, d - m - 1),  B_m = n - sum_{m'<m} l_m',
// i.e. the number of admissible tuples that precede l.  That rank is the
// level hash: a minimal, order-preserving perfect hash of the level tuples,
// computed in O(d n) without a table.  Block sizes are
// (k+1)^d prod_m max(1, 2^{l_m - 1}); offsets are their exclusive prefix sum.
#include "sgk_internal.h"

namespace {

__device__ __forceinline__ long long binom_dev(int n, int r) {
    if (r < 0 || n < r) return 0;
    long long c = 1;
    for (int i = 1; i <= r; ++i) c = c * (n - r + i) / i;
    return c;
}

// number of tuples of length len, entries >= 0, sum <= budget
__device__ __forceinline__ long long count_dev(int len, int budget) {
    return budget < 0 ? 0 : binom_dev(budget + len, len);
}

__global__ void unrank_kernel(int d, int n, int kp1, long long ntuples, int* __restrict__ levels,
                              long long* __restrict__ sizes) {
    long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (r >= ntuples) return;
    long long rem = r;
    int budget = n;
    long long size = 1;
    for (int m = 0; m < d; ++m) {
        int v = 0;
        while (true) {
            long long c = count_dev(d - m - 1, budget - v);
            if (rem < c) break;
            rem -= c;
            ++v;
        }
        levels[r * d + m] = v;
        budget -= v;
        size *= (long long)kp1 * (v == 0 ? 1 : (1LL << (v - 1)));
    }
    sizes[r] = size;
}

// Exclusive scan of sizes into offsets[0..count], one block.
__global__ void scan_kernel(const long long* __restrict__ sizes, long long count, long long* __restrict__ offsets) {
    __shared__ long long part[1024];
    const int t = threadIdx.x;
    const long long per = (count + blockDim.x - 1) / blockDim.x;
    const long long b = t * per;
    const long long e = min(count, b + per);
    long long s = 0;
    for (long long i = b; i < e; ++i) s += sizes[i];
    part[t] = s;
    __syncthreads();
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {
        long long v = t >= off ? part[t - off] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    long long run = part[t] - s;
    for (long long i = b; i < e; ++i) {
        offsets[i] = run;
        run += sizes[i];
    }
    if (t == (int)blockDim.x - 1) offsets[count] = part[t];
}

__global__ void rank_kernel(int d, int n, long long count, const int* __restrict__ levels, long long* __restrict__ out) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= count) return;
    int budget = n;
    long long r = 0;
    for (int m = 0; m < d; ++m) {
        int l = levels[i * d + m];
        if (l < 0 || l > budget) {
            out[i] = -1;
            return;
        }
        for (int v = 0; v < l; ++v) r += count_dev(d - m - 1, budget - v);
        budget -= l;
    }
    out[i] = r;
}

}  // namespace

int64_t tuple_count(int len, int budget) {
    if (budget < 0) return 0;
    int64_t c = 1;
    for (int i = 1; i <= len; ++i) c = c * (budget + i) / i;
    return c;
}

std::vector<std::vector<int>> tuples_lex(int len, int budget) {
    std::vector<std::vector<int>> out;
    std::vector<int> cur(len, 0);
    if (len == 0) {
        out.push_back(cur);
        return out;
    }
    // odometer with the last entry fastest, skipping sums above budget
    while (true) {
        int s = 0;
        for (int v : cur) s += v;
        if (s <= budget) out.push_back(cur);
        int m = len - 1;
        while (m >= 0) {
            cur[m]++;
            int s2 = 0;
            for (int i = 0; i <= m; ++i) s2 += cur[i];
            if (s2 <= budget) break;
            cur[m] = 0;
            --m;
        }
        if (m < 0) break;
    }
    return out;
}

void build_index_on_device(sgk_index* idx) {
    sgk_ctx* ctx = idx->ctx;
    const int d = idx->d, n = idx->n, kp1 = idx->k + 1;
    const long long nt = tuple_count(d, n);
    idx->ntuples = nt;
    idx->d_levels.alloc(nt * d);
    idx->d_offsets.alloc(nt + 1);
    DevBuf<long long> sizes(nt);
    unrank_kernel<<<(unsigned)((nt + 255) / 256), 256, 0, ctx->stream>>>(d, n, kp1, nt, idx->d_levels.p, sizes.p);
    check_launch("unrank_kernel");
    scan_kernel<<<1, 1024, 0, ctx->stream>>>(sizes.p, nt, reinterpret_cast<long long*>(idx->d_offsets.p));
    check_launch("scan_kernel");
    count_launch(ctx, 2);
    idx->levels.resize(nt * d);
    idx->offsets.resize(nt + 1);
    SGK_CUDA_CHECK(cudaMemcpyAsync(idx->levels.data(), idx->d_levels.p, nt * d * sizeof(int32_t),
                                   cudaMemcpyDeviceToHost, ctx->stream));
    SGK_CUDA_CHECK(cudaMemcpyAsync(idx->offsets.data(), idx->d_offsets.p, (nt + 1) * sizeof(int64_t),
                                   cudaMemcpyDeviceToHost, ctx->stream));
    SGK_CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
    idx->dof = idx->offsets[nt];
}

void index_lookup_on_device(const sgk_index* idx, const int32_t* levels, int64_t count, int64_t* out) {
    sgk_ctx* ctx = idx->ctx;
    if (count == 0) return;
    DevBuf<int> dl(count * idx->d);
    DevBuf<long long> dout(count);
    dl.upload(levels, count * idx->d, ctx->stream);
    rank_kernel<<<(unsigned)((count + 255) / 256), 256, 0, ctx->stream>>>(idx->d, idx->n, count, dl.p, dout.p);
    check_launch("rank_kernel");
    count_launch(ctx);
    SGK_CUDA_CHECK(cudaMemcpyAsync(out, dout.p, count * sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream));
    SGK_CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
}
