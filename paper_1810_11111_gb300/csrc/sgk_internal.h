// Internal declarations shared by the libsgkiif translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/sgkiif.h"

// --------------------------------------------------------------- errors ---

struct SgkError {
    int code;
    std::string msg;
};

#define SGK_CUDA_CHECK(call)                                                                   \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            throw SgkError{SGK_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)};    \
    } while (0)

#define SGK_REQUIRE(cond, code, text)                  \
    do {                                               \
        if (!(cond)) throw SgkError{(code), (text)};   \
    } while (0)

// ---------------------------------------------------- device allocations ---

// Stream for stream-ordered allocations by DevBuf on this host thread;
// nullptr (the default) selects cudaMalloc / cudaFree.  cudaFree waits for
// the whole device, which would serialise solves running concurrently on
// other streams, so a thread that owns one stream per solve sets it.
inline cudaStream_t& alloc_stream() {
    static thread_local cudaStream_t s = nullptr;
    return s;
}

// Owning device buffer; moves only.
template <typename T>
struct DevBuf {
    T* p = nullptr;
    size_t n = 0;
    cudaStream_t as = nullptr;  // stream of a stream-ordered allocation
    DevBuf() = default;
    explicit DevBuf(size_t count) { alloc(count); }
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    DevBuf(DevBuf&& o) noexcept : p(o.p), n(o.n), as(o.as) { o.p = nullptr; o.n = 0; o.as = nullptr; }
    DevBuf& operator=(DevBuf&& o) noexcept {
        if (this != &o) {
            release();
            p = o.p;
            n = o.n;
            as = o.as;
            o.p = nullptr;
            o.n = 0;
            o.as = nullptr;
        }
        return *this;
    }
    ~DevBuf() { release(); }
    void alloc(size_t count) {
        release();
        if (count == 0) return;
        cudaStream_t s = alloc_stream();
        cudaError_t e = s ? cudaMallocAsync(reinterpret_cast<void**>(&p), count * sizeof(T), s)
                          : cudaMalloc(reinterpret_cast<void**>(&p), count * sizeof(T));
        if (e != cudaSuccess) {
            p = nullptr;
            (void)cudaGetLastError();
            throw SgkError{SGK_ENOMEM, "device allocation of " + std::to_string(count * sizeof(T)) + " bytes failed"};
        }
        n = count;
        as = s;
    }
    void release() {
        if (p) {
            if (as) cudaFreeAsync(p, as);
            else cudaFree(p);
        }
        p = nullptr;
        n = 0;
        as = nullptr;
    }
    void upload(const T* host, size_t count, cudaStream_t s) {
        if (count) SGK_CUDA_CHECK(cudaMemcpyAsync(p, host, count * sizeof(T), cudaMemcpyHostToDevice, s));
    }
    void upload(const std::vector<T>& v, cudaStream_t s) {
        alloc(v.size());
        upload(v.data(), v.size(), s);
    }
};

// -------------------------------------------------------------- context ---

// Kernel classes for the optional event timing (bit i of the profile mask).
enum KernelClass {
    KC_MATVEC = 0,   // fiber engine, SIPG matvec
    KC_FWD = 1,      // fiber engine, hierarchical -> finest Legendre
    KC_BWD = 2,      // fiber engine, transpose
    KC_CELL = 3,     // cell quadrature of the reaction term / Jacobian
    KC_REDUCE = 4,   // inner products, Gram-Schmidt passes
    KC_EXPM = 5,     // exp(tau H) e_1
    KC_VECTOR = 6,   // other vector kernels
    KC_KRYLOV = 7,   // Krylov exponential: its captured graph, or the persistent Arnoldi kernel when timed alone
    KC_COUNT = 8
};

struct sgk_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int precision = SGK_FP64;
    std::string last_error;
    int64_t launches = 0;
    int num_sms = 0;
    size_t smem_optin = 0;
    bool own_stream = false;  // stream created by the library (caller passed NULL)
    bool capturing = false;   // a CUDA graph is being captured on the stream
    int persist_ctas = 0;     // CTAs of the persistent Arnoldi kernel (0 = one per SM)
    int arn_G_fixed = 0;      // lanes per output of its matvec (0 = autotuned per solver)
    double* hscal = nullptr;  // pinned host scalars (16) for step-control reads
    // event timing
    unsigned prof_mask = 0;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_pending;
    ~sgk_ctx();
};

// Raises a kernel's dynamic shared-memory limit to the most the device allows
// next to its static shared memory.  The value is the same on every call, so
// threads launching the same kernel with different sizes (a server's workers)
// cannot lower the limit under one another's launch.
template <typename K>
void allow_max_dynamic_smem(size_t smem_optin, K kern) {
    cudaFuncAttributes fa;
    SGK_CUDA_CHECK(cudaFuncGetAttributes(&fa, reinterpret_cast<const void*>(kern)));
    SGK_CUDA_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)(smem_optin - fa.sharedSizeBytes)));
}

// Asynchronous element copy global -> shared (PTX cp.async, 4 or 8 bytes):
// the copies of a thread stay in flight together until async_wait_all; the
// values never pass through registers.
template <typename T>
__device__ __forceinline__ void async_copy(T* smem_dst, const T* gmem_src) {
    static_assert(sizeof(T) == 4 || sizeof(T) == 8, "4- or 8-byte elements");
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    if constexpr (sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem_src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void async_wait_all() {
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// Every kernel launch of the library goes through this counter.
inline void count_launch(sgk_ctx* c, int n = 1) { c->launches += n; }
void check_launch(const char* what);

// Brackets the launches issued during its lifetime with CUDA events when the
// class is selected in the context's profile mask.
struct KTimer {
    sgk_ctx* ctx;
    int kc;
    cudaEvent_t a = nullptr, b = nullptr;
    KTimer(sgk_ctx* c, int k);
    ~KTimer();
};

// ------------------------------------------------------------ index set ---

struct sgk_index {
    sgk_ctx* ctx = nullptr;
    int d = 0, n = 0, k = 0;
    int64_t dof = 0;
    int64_t ntuples = 0;
    std::vector<int32_t> levels;   // ntuples x d (host copy of the device table)
    std::vector<int64_t> offsets;  // ntuples + 1
    DevBuf<int32_t> d_levels;
    DevBuf<int64_t> d_offsets;
};

// Number of tuples of length len with entries >= 0 and sum <= budget:
// C(budget + len, len).
int64_t tuple_count(int len, int budget);
// Lexicographic tuples (first entry slowest) of length len with sum <= budget.
std::vector<std::vector<int>> tuples_lex(int len, int budget);
inline int level_count(int l, int kp1) { return l == 0 ? kp1 : kp1 << (l - 1); }
inline int level_offset(int l, int kp1) { return l == 0 ? 0 : kp1 << (l - 1); }

// -------------------------------------------------- 1D tables (host C++) ---

// Sparse matrix in CSR form with sorted column indices, host and device
// (FP64 and FP32 value copies).
struct Csr {
    int rows = 0, cols = 0;
    std::vector<int> ptr, col;
    std::vector<double> val;
    DevBuf<int> d_ptr, d_col;
    DevBuf<double> d_val;
    DevBuf<float> d_valf;
    void upload(cudaStream_t s);
};

struct Tables1D {
    int N = 0, k = 0, H = 0;
    std::vector<double> alpert;  // (k+1) x 2(k+1) wavelet coefficients
    Csr T;                       // H x H: hierarchical -> finest-cell Legendre
    Csr Tt;                      // transpose of T
    // Two-scale filters, each (k+1) x (k+1) row-major: H_h[r][s] = <phi_r,
    // phi^h_s> (parent Legendre against the Legendre basis of child h) and
    // G_h[p][s] = <psi_p, phi^h_s> (wavelet against child h); stored as
    // [H_0, H_1, G_0, G_1].  A child's coefficients are
    // sum_r H_h[r][s] parent[r] + sum_p G_h[p][s] detail[p]; the transpose
    // gives the parent and detail coefficients from the two children.
    std::vector<double> two_scale;
};

// Gauss-Legendre rule on [-1, 1] with q points (Newton on P_q, long double).
void gauss_legendre(int q, std::vector<double>& x, std::vector<double>& w);
// Alpert multiwavelet coefficients (rows p = 0..k over [left Legendre 0..k,
// right Legendre 0..k]).
std::vector<double> alpert_coefficients(int k);
// Build T and its transpose for level N, degree k.
void build_transform_tables(int N, int k, Tables1D& out);
// 1D SIPG matrix in the hierarchical basis, dense row-major H x H.
std::vector<double> build_sipg_hier(const Tables1D& tab, int bc, double sigma);
// The 1D pieces of the mixed-derivative terms for a full diffusion tensor,
// dense H x H in the hierarchical basis: P[a][b] = int v_a' v_b over the
// finest cells, E[a][b] = sum over faces of [v_a] {v_b}.
void build_cross_hier(const Tables1D& tab, int bc, std::vector<double>& P, std::vector<double>& E);
// The 1D factors of the collocation matrix of the sparse-grid interpolation
// form of the reaction term (tables.cpp): A (Alpert coefficients ->
// interpolation surpluses), B (surpluses -> point values) and their
// inverses, H x H in CSR with sorted columns (host arrays only).
struct InterpFactors1D {
    Csr A, B, Binv, Ainv;
};
void build_interp_factors(int N, int k, InterpFactors1D& out);

// --------------------------------------------------------- fiber engine ---

struct FiberGroup {
    long long cbase[SGK_MAX_LEVEL + 1];  // chunked side: start of each level's chunk
    long long fbase;                     // full side: start of the block
    int nlev;                            // levels 0..nlev-1 along the fiber
    int I;                               // inner (contiguous) extent
    int O;                               // outer extent
    int pad;
};

struct FiberItem {
    int group;
    int col0;
    int ncols;
    int stride;  // smem column stride (ncols rounded to odd)
    int row0;    // output rows [row0, row0 + nrows) of the fiber
    int nrows;
};

enum FiberMode { FIBER_MATVEC = 0, FIBER_FWD = 1, FIBER_BWD = 2 };

struct FiberPlan {
    DevBuf<FiberGroup> groups;
    DevBuf<FiberItem> items;
    int nitems = 0;
    int max_src_len = 0;
    int max_cols = 0;
    size_t smem_bytes = 0;
};

// Host-side construction of a plan from groups (fills items, uploads).
// Every address a work item can touch is checked on the host against the
// source and destination sizes before the plan is uploaded.
void finalize_plan(FiberPlan& plan, std::vector<FiberGroup>& groups, int kp1, int H, int mode, size_t elem_bytes,
                   size_t smem_budget, long long src_size, long long dst_size, cudaStream_t s);

// Two-scale filters for the pyramid kernels (entries beyond k+1 unused).
template <typename T>
struct PyrFilt {
    T H[2][4][4];
    T G[2][4][4];
};

// Change of basis along one direction (plan mode FIBER_FWD or FIBER_BWD) by
// the two-scale pyramid; two_scale as in Tables1D.
template <typename T>
void launch_pyr(sgk_ctx* ctx, const FiberPlan& plan, int mode, const T* src, T* dst, int H, int kp1,
                const double* two_scale);

// ------------------------------------------------------------- operator ---

struct sgk_op {
    sgk_ctx* ctx = nullptr;
    const sgk_index* idx = nullptr;
    double kappa[SGK_MAX_DIM] = {0};
    int bc = SGK_PERIODIC;
    double sigma = 20.0;
    int H = 0;
    std::vector<double> S_dense;  // H x H host copy
    Csr S;
    // rlen[a (N+1) + L]: entries of row a with column < (k+1) 2^L (CSR rows
    // sorted by column), i.e. the row of the principal submatrix of levels
    // 0..L
    DevBuf<int> rlen;
    // gather-matvec tables: packed (level, position) of every CSR entry;
    // block offsets per (tuple, direction, level); tuple of every 256th
    // coefficient
    DevBuf<int32_t> gmv_ce;
    DevBuf<int64_t> gmv_cb;
    DevBuf<int32_t> gmv_chunk;
    DevBuf<double> gmv_cvk;  // -kappa_i S, one copy of the CSR values per direction
    DevBuf<float> gmv_cvkf;  // the same in FP32
    DevBuf<float2> gmv_cvk2;  // the same as double-float pairs (hi, lo), hi + lo = the FP64 value to 2^-48
    int64_t madds = 0;  // multiply-adds of one matvec (entries of A on the index set, per direction)
    std::vector<int> rlen_host;  // host copy of rlen
    // bound on ||A||_2 of the sparse-grid operator: sum_i |kappa_i| max(||S||_1, ||S||_inf)
    double anorm = 0.0;
    // pre-located gathers (built when the operator has at most
    // GMV_LIST_MAX entries): for output g and direction i the entries
    // gmv_eoff[g d + i] .. gmv_eoff[g d + i + 1] of gmv_ent, each {index of
    // x, index into gmv_cvk}, in row order; gmv_ecnt_host[g] = entries of g
    DevBuf<int32_t> gmv_eoff;
    DevBuf<int2> gmv_ent;
    std::vector<int32_t> gmv_ecnt_host;
    // mixed-derivative terms of a full diffusion tensor (cross.cu): the
    // direction pairs (i, j) with K_ij != 0 and K_ij; the 1D factors Q, P^T,
    // E^T, P as CSR (pointers per matrix, H + 1 each) with truncated row
    // lengths per level; per (tuple, pair) the base of its block-offset
    // table, (L + 1)^2 entries indexed by the changed levels of i and j
    int npairs = 0;
    double K[SGK_MAX_DIM * SGK_MAX_DIM] = {0};
    DevBuf<int> x_pairs, x_ptr, x_col, x_rlen;
    DevBuf<double> x_kij, x_val;
    DevBuf<float> x_valf;
    DevBuf<int64_t> x_grp, x_off;
    int64_t x_nnz = 0;
};
constexpr int64_t GMV_LIST_MAX = int64_t(1) << 24;

// Builds and checks the gather-matvec tables of an assembled operator.
void build_gmv_tables(sgk_op* op);
// Boundaries of nb contiguous slices of the coefficient vector for the
// persistent Arnoldi kernel, minimising the largest slice cost (per output
// its matvec entries, all directions, plus extra for the Gram-Schmidt
// passes, extra = 2 M), with at most cap_len outputs and cap_ent entries per
// slice.  bounds[0] = 0, bounds[nb] = dof, non-decreasing; empty when the
// caps cannot be met with nb slices.
std::vector<int64_t> arnoldi_slice_bounds(const sgk_op* op, int nb, int extra, int64_t cap_len, int64_t cap_ent);
long long tuple_rank(const std::vector<int>& l, int n);

template <typename T>
void op_matvec(const sgk_op* op, const T* x, T* y);
// Tables and application (y -= the mixed-derivative terms) of a full
// constant diffusion tensor K (d x d, row-major, symmetric).
void build_cross_tables(sgk_op* op, const double* K);
template <typename T>
void op_cross_matvec(const sgk_op* op, const T* x, T* y);

// -------------------------------------------------------------- kernels ---

// Deterministic reductions: partials per block, then one block sums them in
// a fixed order.
constexpr int RED_THREADS = 256;

#ifdef __CUDACC__
// FP64 sum over a warp (down-shuffle tree; result in lane 0).
__device__ __forceinline__ double warp_sum_f64(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// FP64 sum over the block in a fixed tree; result valid in thread 0.  Every
// thread of the block calls it (it synchronises the block).
__device__ __forceinline__ double block_sum_f64(double v, double* sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = warp_sum_f64(v);
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    v = threadIdx.x < nw ? sh[threadIdx.x] : 0.0;
    if (wid == 0) v = warp_sum_f64(v);
    __syncthreads();
    return v;
}
#endif
int reduction_blocks(const sgk_ctx* ctx, int64_t n);
