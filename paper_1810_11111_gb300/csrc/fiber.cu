// Fiber engine for the change of basis along one direction of a sparse-grid
// (or partly full-grid) coefficient array.
//
// This is the unidirectional principle of Section 4 applied to the reaction
// term: the map from hierarchical coefficients to finest-cell Legendre
// coefficients, and its transpose, act on 1D fibers one direction at a time.
// For direction i, the blocks sharing the levels of the other directions form
// a group; stacked along i they hold (outer x fiber x inner) arrays whose
// fiber index is the 1D hierarchical index a_i < (k+1) 2^{N'}, N' = N -
// sum_{m != i} l_m (the "chunked" side), or a finest-cell Legendre index
// y < (k+1) 2^N (the "full" side).  Each chunk (one level) is contiguous, so
// a fiber tile is gathered with unit-stride loads along the inner extent.
//
// Work items are (group, column range) tiles sized to fit shared memory; a
// grid-stride loop over items sorted by cost keeps every SM busy.  A CTA
// stages the source fibers of its tile in shared memory and runs the
// two-scale pyramid on them.
#include <algorithm>

#include "sgk_dfloat.h"
#include "sgk_internal.h"

namespace {

__device__ __forceinline__ int level_of(int pos, int kp1) {
    int q = pos / kp1;
    return q == 0 ? 0 : 32 - __clz(q);
}

__device__ __forceinline__ long long chunk_addr(const FiberGroup& g, int o, int pos, int in, int kp1, int I) {
    int l = level_of(pos, kp1);
    int off = l ? (kp1 << (l - 1)) : 0;
    int nl = l ? (kp1 << (l - 1)) : kp1;
    return g.cbase[l] + (long long)o * nl * I + (long long)(pos - off) * I + in;
}

__device__ __forceinline__ long long full_addr(const FiberGroup& g, int o, int pos, int in, int H, int I) {
    return g.fbase + ((long long)o * H + pos) * I + in;
}

// Change of basis along one direction by the two-scale (pyramid) relations.
// FWD: hierarchical fibers (levels 0..N') -> finest-cell Legendre
// coefficients (levels refined up to Nfull with zero details above N').
// BWD: the transpose, finest Legendre moments -> hierarchical coefficients of
// levels 0..N'.
//
// Each thread owns a subtree of 2^PD finest cells of one column (PD levels
// below level t = Nfull - PD): FWD walks the t ancestors of its subtree root
// from the level-0 coefficients and expands the subtree in registers; BWD
// reduces its subtree in registers, writes the subtree's details and leaves
// the root's scaling coefficients in shared memory, where one thread per
// column finishes the t upper levels.  Shared memory holds the source tile,
// the destination tile (stored with coalesced loads/stores) and, for BWD,
// the subtree roots; two barriers per item instead of one per level.
constexpr int PD = 3;

template <typename T, int MODE, int KP1>
__global__ void __launch_bounds__(256) pyr_kernel(const FiberItem* __restrict__ items, int nitems,
                                                  const FiberGroup* __restrict__ groups, const T* __restrict__ src,
                                                  T* __restrict__ dst, const PyrFilt<T> flt, int H, int Nfull) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* tile = reinterpret_cast<T*>(smem_raw);
    __shared__ FiberGroup sg;
    T Hm[2][KP1][KP1], Gm[2][KP1][KP1];
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int r = 0; r < KP1; ++r)
#pragma unroll
            for (int s = 0; s < KP1; ++s) {
                Hm[h][r][s] = flt.H[h][r][s];
                Gm[h][r][s] = flt.G[h][r][s];
            }
    const int De = Nfull < PD ? Nfull : PD;  // levels expanded in registers
    const int t = Nfull - De;                // level of the subtree roots
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const FiberItem item = items[it];
        if (threadIdx.x < (int)(sizeof(FiberGroup) / sizeof(long long)))
            reinterpret_cast<long long*>(&sg)[threadIdx.x] =
                reinterpret_cast<const long long*>(groups + item.group)[threadIdx.x];
        __syncthreads();
        const int Np = sg.nlev - 1;  // finest hierarchical level of the fiber
        const int F = KP1 << Np;
        const int I = sg.I, nc = item.ncols, st = item.stride;
        const int src_len = MODE == FIBER_BWD ? H : F;
        const int dst_len = MODE == FIBER_FWD ? H : F;
        T* X = tile;
        T* Y = tile + (size_t)src_len * st;
        T* R = Y + (size_t)dst_len * st;  // BWD: subtree roots, (KP1 << t) rows, then a buffer of half that
        // load/store mapping: a warp per column for short inner extents
        // (lanes over rows), otherwise one column per thread with rows
        // strided; body(c, o, in, t) runs for t in [0, count) on every column
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
        const int cf = threadIdx.x % nc, rg = threadIdx.x / nc, nrg = blockDim.x / nc;
        auto for_ct = [&](int count, auto&& body) {
            if (I < 4) {
                for (int c = wid; c < nc; c += nw) {
                    const int col = item.col0 + c, o = col / I, in = col - (col / I) * I;
                    for (int q = lane; q < count; q += 32) body(c, o, in, q);
                }
            } else if (rg < nrg) {
                const int col = item.col0 + cf, o = col / I, in = col - (col / I) * I;
                for (int q = rg; q < count; q += nrg) body(cf, o, in, q);
            }
        };
        for_ct(src_len, [&](int c, int o, int in, int pos) {
            async_copy(X + pos * st + c,
                       src + (MODE == FIBER_BWD ? full_addr(sg, o, pos, in, H, I) : chunk_addr(sg, o, pos, in, KP1, I)));
        });
        async_wait_all();
        __syncthreads();
        const int units = nc << t;
        if (MODE == FIBER_FWD) {
            for (int u = threadIdx.x; u < units; u += blockDim.x) {
                const int c = u % nc, j = u / nc;
                T cell[1 << PD][KP1];
#pragma unroll
                for (int r = 0; r < KP1; ++r) cell[0][r] = X[r * st + c];
                // ancestors of the subtree root, level 1..t
                for (int n = 1; n <= t; ++n) {
                    const int an = j >> (t - n), h = an & 1, par = an >> 1;
                    T d[KP1], q[KP1];
#pragma unroll
                    for (int r = 0; r < KP1; ++r) d[r] = n <= Np ? X[((KP1 << (n - 1)) + par * KP1 + r) * st + c] : T(0);
#pragma unroll
                    for (int s2 = 0; s2 < KP1; ++s2) {
                        T acc = T(0);
#pragma unroll
                        for (int r = 0; r < KP1; ++r) {
                            // select, not index: a runtime index would put the
                            // filters in local memory
                            const T hf = h ? Hm[1][r][s2] : Hm[0][r][s2];
                            const T gf = h ? Gm[1][r][s2] : Gm[0][r][s2];
                            acc += hf * cell[0][r] + gf * d[r];
                        }
                        q[s2] = acc;
                    }
#pragma unroll
                    for (int r = 0; r < KP1; ++r) cell[0][r] = q[r];
                }
                // expand the subtree (children written over consumed parents)
#pragma unroll
                for (int l = 0; l < PD; ++l) {
                    if (l < De) {
                        const int n = t + l + 1;
#pragma unroll
                        for (int i = (1 << l) - 1; i >= 0; --i) {
                            const int par = (j << l) + i;
                            T d[KP1], p[KP1];
#pragma unroll
                            for (int r = 0; r < KP1; ++r) {
                                p[r] = cell[i][r];
                                d[r] = n <= Np ? X[((KP1 << (n - 1)) + par * KP1 + r) * st + c] : T(0);
                            }
#pragma unroll
                            for (int h = 0; h < 2; ++h)
#pragma unroll
                                for (int s2 = 0; s2 < KP1; ++s2) {
                                    T acc = T(0);
#pragma unroll
                                    for (int r = 0; r < KP1; ++r) acc += Hm[h][r][s2] * p[r] + Gm[h][r][s2] * d[r];
                                    cell[2 * i + h][s2] = acc;
                                }
                        }
                    }
                }
#pragma unroll
                for (int i = 0; i < (1 << PD); ++i)
                    if (i < (1 << De))
#pragma unroll
                        for (int s2 = 0; s2 < KP1; ++s2) Y[(((j << De) + i) * KP1 + s2) * st + c] = cell[i][s2];
            }
            __syncthreads();
            for_ct(H, [&](int c, int o, int in, int pos) { dst[full_addr(sg, o, pos, in, H, I)] = Y[pos * st + c]; });
        } else {
            for (int u = threadIdx.x; u < units; u += blockDim.x) {
                const int c = u % nc, j = u / nc;
                T cell[1 << PD][KP1];
#pragma unroll
                for (int i = 0; i < (1 << PD); ++i)
                    if (i < (1 << De))
#pragma unroll
                        for (int s2 = 0; s2 < KP1; ++s2) cell[i][s2] = X[(((j << De) + i) * KP1 + s2) * st + c];
                // reduce the subtree (parents written over consumed children)
#pragma unroll
                for (int l = PD - 1; l >= 0; --l) {
                    if (l < De) {
                        const int n = t + l + 1;  // level of the children
                        const bool keep = n <= Np;
#pragma unroll
                        for (int i = 0; i < (1 << l); ++i) {
                            T x0[KP1], x1[KP1];
#pragma unroll
                            for (int s2 = 0; s2 < KP1; ++s2) {
                                x0[s2] = cell[2 * i][s2];
                                x1[s2] = cell[2 * i + 1][s2];
                            }
                            const int par = (j << l) + i;
#pragma unroll
                            for (int r = 0; r < KP1; ++r) {
                                T sp = T(0), sd = T(0);
#pragma unroll
                                for (int s2 = 0; s2 < KP1; ++s2) {
                                    sp += Hm[0][r][s2] * x0[s2] + Hm[1][r][s2] * x1[s2];
                                    sd += Gm[0][r][s2] * x0[s2] + Gm[1][r][s2] * x1[s2];
                                }
                                cell[i][r] = sp;
                                if (keep) Y[((KP1 << (n - 1)) + par * KP1 + r) * st + c] = sd;
                            }
                        }
                    }
                }
#pragma unroll
                for (int r = 0; r < KP1; ++r) R[(j * KP1 + r) * st + c] = cell[0][r];
            }
            __syncthreads();
            // the t upper levels, one parent per thread and a barrier per
            // level, alternating between R and R2
            T* cur = R;
            T* nxt = R + (size_t)(KP1 << t) * st;
            for (int n = t; n >= 1; --n) {
                const bool keep = n <= Np;
                for (int u = threadIdx.x; u < (nc << (n - 1)); u += blockDim.x) {
                    const int c = u % nc, par = u / nc;
                    T x0[KP1], x1[KP1];
#pragma unroll
                    for (int s2 = 0; s2 < KP1; ++s2) {
                        x0[s2] = cur[((2 * par) * KP1 + s2) * st + c];
                        x1[s2] = cur[((2 * par + 1) * KP1 + s2) * st + c];
                    }
#pragma unroll
                    for (int r = 0; r < KP1; ++r) {
                        T sp = T(0), sd = T(0);
#pragma unroll
                        for (int s2 = 0; s2 < KP1; ++s2) {
                            sp += Hm[0][r][s2] * x0[s2] + Hm[1][r][s2] * x1[s2];
                            sd += Gm[0][r][s2] * x0[s2] + Gm[1][r][s2] * x1[s2];
                        }
                        nxt[(par * KP1 + r) * st + c] = sp;
                        if (keep) Y[((KP1 << (n - 1)) + par * KP1 + r) * st + c] = sd;
                    }
                }
                __syncthreads();
                T* tmp = cur;
                cur = nxt;
                nxt = tmp;
            }
            for (int u = threadIdx.x; u < nc * KP1; u += blockDim.x) {
                const int c = u % nc, r = u / nc;
                Y[r * st + c] = cur[r * st + c];
            }
            __syncthreads();
            for_ct(F, [&](int c, int o, int in, int pos) { dst[chunk_addr(sg, o, pos, in, KP1, I)] = Y[pos * st + c]; });
        }
        __syncthreads();
    }
}

}  // namespace

template <typename T>
void launch_pyr(sgk_ctx* ctx, const FiberPlan& plan, int mode, const T* src, T* dst, int H, int kp1,
                const double* two_scale) {
    if (plan.nitems == 0) return;
    PyrFilt<T> f{};
    for (int h = 0; h < 2; ++h)
        for (int r = 0; r < kp1; ++r)
            for (int s = 0; s < kp1; ++s) {
                f.H[h][r][s] = (T)two_scale[h * kp1 * kp1 + r * kp1 + s];
                f.G[h][r][s] = (T)two_scale[(2 + h) * kp1 * kp1 + r * kp1 + s];
            }
    int Nfull = 0;
    while ((kp1 << Nfull) < H) ++Nfull;
    const int grid = std::min(plan.nitems, ctx->num_sms * 8);
    const size_t smem = plan.smem_bytes;
    KTimer kt(ctx, mode);
#define SGK_PYR_CASE(M, K)                                                                                   \
    if (mode == M && kp1 == K) {                                                                             \
        allow_max_dynamic_smem(ctx->smem_optin, pyr_kernel<T, M, K>);          \
        pyr_kernel<T, M, K><<<grid, 256, smem, ctx->stream>>>(plan.items.p, plan.nitems, plan.groups.p, src, dst, \
                                                              f, H, Nfull);                                 \
    }
    SGK_PYR_CASE(FIBER_FWD, 2)
    SGK_PYR_CASE(FIBER_FWD, 3)
    SGK_PYR_CASE(FIBER_FWD, 4)
    SGK_PYR_CASE(FIBER_BWD, 2)
    SGK_PYR_CASE(FIBER_BWD, 3)
    SGK_PYR_CASE(FIBER_BWD, 4)
#undef SGK_PYR_CASE
    check_launch("pyr_kernel");
    count_launch(ctx);
}

template void launch_pyr<double>(sgk_ctx*, const FiberPlan&, int, const double*, double*, int, int, const double*);
template void launch_pyr<float>(sgk_ctx*, const FiberPlan&, int, const float*, float*, int, int, const double*);
template void launch_pyr<dfloat>(sgk_ctx*, const FiberPlan&, int, const dfloat*, dfloat*, int, int, const double*);

// Host mirror of the kernel's address arithmetic, for plan validation.
static long long chunk_addr_host(const FiberGroup& g, long long o, int pos, long long in, int kp1, int I) {
    const int q = pos / kp1;
    int l = 0;
    while ((1 << l) <= q) ++l;  // l = 0 for q = 0, else floor(log2 q) + 1
    const int off = l ? (kp1 << (l - 1)) : 0;
    const int nl = l ? (kp1 << (l - 1)) : kp1;
    return g.cbase[l] + o * nl * I + (long long)(pos - off) * I + in;
}

static void validate_item(const FiberGroup& g, const FiberItem& it, int kp1, int H, int mode, long long src_size,
                          long long dst_size) {
    const int F = kp1 << (g.nlev - 1);
    SGK_REQUIRE(g.nlev >= 1 && g.nlev <= SGK_MAX_LEVEL + 1, SGK_EINVAL, "plan: bad level count");
    SGK_REQUIRE(it.col0 >= 0 && it.ncols >= 1 && (long long)it.col0 + it.ncols <= (long long)g.O * g.I, SGK_EINVAL,
                "plan: column range outside the group");
    for (int side = 0; side < 2; ++side) {
        const bool full = (side == 0) ? mode == FIBER_BWD : mode == FIBER_FWD;
        const int len = full ? H : F;
        const long long size = side == 0 ? src_size : dst_size;
        for (int c = 0; c < it.ncols; ++c) {
            const long long col = it.col0 + c;
            const long long o = col / g.I, in = col % g.I;
            // addresses are increasing in pos within a level chunk: check the
            // first and last position of every chunk
            for (int l = 0; l < (full ? 1 : g.nlev); ++l) {
                int p0, p1;
                if (full) {
                    p0 = 0;
                    p1 = len - 1;
                } else {
                    p0 = l ? (kp1 << (l - 1)) : 0;
                    p1 = p0 + (l ? (kp1 << (l - 1)) : kp1) - 1;
                }
                for (int pos : {p0, p1}) {
                    const long long a = full ? g.fbase + (o * H + pos) * g.I + in : chunk_addr_host(g, o, pos, in, kp1, g.I);
                    SGK_REQUIRE(a >= 0 && a < size, SGK_EINVAL, "plan: address outside its buffer");
                }
            }
        }
    }
}

void finalize_plan(FiberPlan& plan, std::vector<FiberGroup>& groups, int kp1, int H, int mode, size_t elem_bytes,
                   size_t smem_budget, long long src_size, long long dst_size, cudaStream_t s) {
    std::vector<FiberItem> items;
    std::vector<long long> cost;
    // columns per item: at most what spreads the plan over about 2 x 152
    // items (a GB300's SMs), so that small transforms still fill the GPU
    long long total_cols = 0;
    for (const FiberGroup& g : groups) total_cols += (long long)g.O * g.I;
    const long long col_cap = std::max<long long>(1, (total_cols + 303) / 304);
    plan.max_src_len = 0;
    plan.max_cols = 0;
    size_t smem = 0;
    for (int gi = 0; gi < (int)groups.size(); ++gi) {
        const FiberGroup& g = groups[gi];
        const int F = kp1 << (g.nlev - 1);
        const int src_len = mode == FIBER_BWD ? H : F;
        const int dst_len = mode == FIBER_FWD ? H : F;
        long long cols = (long long)g.O * g.I;
        SGK_REQUIRE(cols < (1LL << 31), SGK_EUNSUPPORTED, "plan: too many fibers in one group");
        // the pyramid kernel stages the source and destination fibers, and
        // for BWD the subtree roots (k+1 rows per subtree of 8 finest cells)
        // twice (the upper levels alternate between two buffers)
        SGK_REQUIRE(mode == FIBER_FWD || mode == FIBER_BWD, SGK_EINVAL, "plan: mode must be FWD or BWD");
        const int tile_rows = src_len + dst_len + (mode == FIBER_BWD ? 2 * std::max(kp1, H >> 3) : 0);
        long long fit = (long long)(smem_budget / ((size_t)tile_rows * elem_bytes)) - 1;
        int maxc = (int)std::min<long long>(std::min<long long>(64, col_cap), std::max<long long>(1, fit));
        for (long long c0 = 0; c0 < cols; c0 += maxc) {
            FiberItem it;
            it.group = gi;
            it.col0 = (int)c0;
            it.ncols = (int)std::min<long long>(maxc, cols - c0);
            it.stride = it.ncols | 1;
            // an item computes whole fibers
            it.row0 = 0;
            it.nrows = dst_len;
            validate_item(g, it, kp1, H, mode, src_size, dst_size);
            items.push_back(it);
            cost.push_back((long long)src_len * it.ncols + (long long)it.nrows * it.ncols * 8);
            smem = std::max(smem, (size_t)tile_rows * it.stride * elem_bytes);
        }
        plan.max_src_len = std::max(plan.max_src_len, src_len);
    }
    // most expensive items first
    std::vector<int> order(items.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    std::vector<FiberItem> sorted(items.size());
    for (size_t i = 0; i < order.size(); ++i) sorted[i] = items[order[i]];
    plan.groups.upload(groups, s);
    plan.items.upload(sorted, s);
    plan.nitems = (int)sorted.size();
    plan.smem_bytes = smem;
    SGK_CUDA_CHECK(cudaStreamSynchronize(s));
}

// ------------------------------------------------------------- operator ---

// Rank of a tuple among lexicographic tuples of its length with sum <= n.
static long long rank_host(const std::vector<int>& l, int n) {
    int len = (int)l.size(), budget = n;
    long long r = 0;
    for (int m = 0; m < len; ++m) {
        for (int v = 0; v < l[m]; ++v) r += tuple_count(len - m - 1, budget - v);
        budget -= l[m];
    }
    return r;
}

long long tuple_rank(const std::vector<int>& l, int n) { return rank_host(l, n); }
