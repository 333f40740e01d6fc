// Persistent Arnoldi kernel (see arnoldi.cu): device code and launch
// templates.  Each arnoldi_d<D>.cu instantiates arn_launch_k<D> for one
// dimension, so that the variants compile in parallel.
#pragma once
#include <algorithm>

#include "sgk_gmv.h"
#include "sgk_krylov.h"

namespace sgk_arn {

constexpr int PT = 512;                        // threads per CTA, one CTA per SM
constexpr int PNW = PT / 32;                   // warps per CTA
constexpr unsigned BAR_SPIN_LIMIT = 1u << 21;  // polls (an L2 round trip each, ~0.2-0.5 us): about a second

struct ArnArgs {
    int64_t n;
    int M;
    int E;    // slice length per CTA (ceil(n / gridDim.x))
    int smem_vz;   // this CTA's slices of V and Z live in shared memory (and V also in HBM)
    int smem_loc;  // the located rows of every output of the slice live in shared memory
    int list_cap;  // > 0: the slice's pre-located gather entries (at most list_cap) live in shared memory
    const int* eoff;   // pre-located gathers (see sgk_op::gmv_eoff), or null
    const int2* ent;
    // double-float matvec (mixed precision; needs the gather lists and the
    // shared V/Z slices): operator values as (hi, lo) pairs; the gathered
    // vectors (w0, w1) and Z then hold (hi, lo) pairs instead of doubles
    const float2* cvk2;
    int df;
    const double* v;
    double* V;  // column c at V + c n
    double* w0;
    double* w1;
    double* Z;     // raw matvec outputs A v_c, column c at Z + c n (own slices only)
    double* H;     // (M + 1) x M row-major
    double* pbuf;  // gridDim.x per-CTA partials of a norm (gamma, explicit fallback)
    unsigned long long* acc;  // 3 rotating sets of FX_COLS fixed-point accumulators (FX_LIMBS words each)
    // fixed-point scales: a partial p of an inner product enters as
    // floor(p sc 2^64), the sum is read back times isc; _h for the columns of
    // V^T w (|p| <= ||A||), _n for ||w'||^2 (|p| <= ||A||^2)
    double sc_h, isc_h, sc_n, isc_n;
    unsigned* bar;  // [0] barrier arrivals (zero at launch), [1] error flag
    unsigned bar_extra;  // added to every barrier target: 0, or 1 to make the waits run out (failure test)
    KrylovScalars* ks;
    const int64_t* bounds;  // slice b = [bounds[b], bounds[b+1]) (work-balanced), or null: equal slices of E
};

constexpr int FX_COLS = SGK_MAX_KRYLOV + 2;  // columns of one accumulator set
constexpr int FX_LIMBS = 4;                   // three 56-bit limbs and a count of invalid partials
// copies of every accumulator: CTA b adds into copy b % FX_COPIES, so that
// the CTAs arriving together do not serialise on the same words
constexpr int FX_COPIES = 8;
constexpr int FX_SET = FX_COPIES * FX_COLS * FX_LIMBS;  // words of one set

// Bytes of the staged entry offsets of a slice of E outputs (D per output
// and one end), rounded up to 16.
__host__ __device__ inline size_t arn_eoff_bytes(int E, int d) { return ((sizeof(int) * ((size_t)E * d + 1)) + 15) / 16 * 16; }

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned ld_relaxed(const unsigned* p) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// All CTAs arrive; returns false if the wait ran out or another CTA failed.
// Thread 0 arrives with a release add (cumulative over the CTA's writes,
// which the CTA barrier before it orders) and polls with acquire loads,
// whose acquire the CTA barrier after it passes on to every thread; the
// error flag is looked at every 256 polls.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned target, int* s_ok) {
    __syncthreads();
    if (threadIdx.x == 0) {
        red_release_add(bar, 1u);
        int ok = 1;
        for (unsigned it = 0;; ++it) {
            if (ld_acquire(bar) >= target) break;
            if ((it & 255u) == 255u && (it >= BAR_SPIN_LIMIT || ld_relaxed(bar + 1) != 0u)) {
                ok = 0;
                break;
            }
        }
        if (!ok) atomicExch(bar + 1, 1u);
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

__device__ __forceinline__ double warp_sum(double a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    return a;
}

// out[c] = sum over CTAs b of P[c nb + b], c < ncols (the partials are
// stored column by column, so a column is one contiguous run), identical in every
// CTA; used for the norms of v and of an explicitly normalised w''.  Each thread sums a fixed subset of rows of one column (all its loads
// issued at once), the subset sums go through shared memory and one thread
// per column adds them in a fixed order: FP64 additions with every lane
// busy, no shuffle trees.  P was written by other CTAs during this launch:
// L2 loads.
__device__ __forceinline__ void colsum(const double* P, int nb, int ncols, double* out, double* tmp) {
    // RS row slots per column; ncols * RS <= max(PT, 4 ncols)
    const int RS = ncols <= PT / 32 ? 32 : (ncols <= PT / 16 ? 16 : (ncols <= PT / 8 ? 8 : 4));
    for (int base = 0; base < ncols * RS; base += PT) {
        const int t = base + threadIdx.x;
        if (t < ncols * RS) {
            const int c = t / RS, k0 = t - (t / RS) * RS;
            double v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int k = k0 + RS * q;
                v[q] = k < nb ? __ldcg(P + (int64_t)c * nb + k) : 0.0;
            }
            // the trip count depends on nb and RS only: uniform, so the
            // additions past the last row slot are not issued
            double acc = v[0];
#pragma unroll
            for (int q = 1; q < 8; ++q)
                if (RS * q < nb) acc += v[q];
            for (int k = k0 + 8 * RS; k < nb; k += RS) acc += __ldcg(P + (int64_t)c * nb + k);
            tmp[t] = acc;
        }
    }
    __syncthreads();
    if ((int)threadIdx.x < ncols) {
        const double* tc = tmp + threadIdx.x * RS;
        double a0 = 0.0, a1 = 0.0;
        for (int k = 0; k < RS; k += 2) {
            a0 += tc[k];
            a1 += tc[k + 1];
        }
        out[threadIdx.x] = a0 + a1;
    }
}

// out[c] = sum_{u < ne} Vl[c vld + u] ws[u], c < ncols (this CTA's slice,
// Vl/vld its basis columns in shared or global memory); with norm, also
// out[ncols] = sum ws[u]^2; out in shared memory, complete on return.  CH
// threads per column (a power of two, the most with nt CH <= PT, at most 32)
// sum strided elements in two chains; the CH partials of a column are added
// through shared memory in a fixed tree (quarters by four threads, then the
// four by one), so the FP64 work is spread over every warp of the CTA (FP64
// issue is slow on this part: spreading it, not shortening chains, is what
// pays).  tmp holds PT doubles, tmp2 4 (SGK_MAX_KRYLOV + 2).
__device__ __forceinline__ void slice_dots(const double* Vl, int64_t vld, int ncols, const double* ws, int ne,
                                           double* out, bool norm, double* tmp, double* tmp2) {
    const int nt = ncols + (norm ? 1 : 0);
    int CH = 32;
    while (CH > 1 && nt * CH > PT) CH >>= 1;
    const int t = threadIdx.x;
    if (t < nt * CH) {
        const int c = t / CH, k = t - (t / CH) * CH;
        const double* vc = c < ncols ? Vl + c * vld : ws;
        double a = 0.0, b = 0.0;
        int u = k;
        for (; u + CH < ne; u += 2 * CH) {
            a += vc[u] * ws[u];
            b += vc[u + CH] * ws[u + CH];
        }
        if (u < ne) a += vc[u] * ws[u];
        tmp[t] = a + b;
    }
    __syncthreads();
    const int Q = CH < 4 ? CH : 4, per = CH / Q;
    if (t < nt * Q) {
        const double* p = tmp + t * per;  // column t / Q, quarter t % Q
        double a = p[0];
        for (int i = 1; i < per; ++i) a += p[i];
        tmp2[t] = a;
    }
    __syncthreads();
    if (t < nt) {
        const double* p = tmp2 + t * Q;
        out[t] = Q == 4 ? (p[0] + p[1]) + (p[2] + p[3]) : (Q == 2 ? p[0] + p[1] : p[0]);
    }
    __syncthreads();
}

// Exact sums across CTAs.  A partial p is taken as the 128-bit integer
// P = trunc(p sc 2^64) (two's complement; sc a power of two chosen from a
// bound on |p| so that |P| < 2^110) and added to per-column accumulators of
// three 56-bit limbs with 64-bit integer atomic adds.  Integer addition is
// associative: the total is exact whatever the order of arrival, and every
// CTA reads back the same value, in every run.  A partial that is not
// finite or outside the range is counted in the fourth word and makes the
// column NaN.
constexpr unsigned long long FX_M56 = (1ull << 56) - 1;

__device__ __forceinline__ void fx_red(unsigned long long* a, double p, double sc) {
    const double q = p * sc;  // |q| < 2^46 when the bound holds
    const double aq = fabs(q);
    if (!(aq < 1125899906842624.0)) {  // 2^50; false for NaN
        atomicAdd(a + 3, 1ull);
        return;
    }
    // |P| = H 2^64 + L: the integer part, and the fraction (exact for a
    // non-negative double) scaled to 64 bits
    const double hd = floor(aq);
    unsigned long long H = __double2ull_rn(hd);
    unsigned long long L = __double2ull_rd((aq - hd) * 18446744073709551616.0);
    if (q < 0.0) {  // two's complement of the 128-bit magnitude
        L = ~L + 1ull;
        H = ~H + (L == 0ull ? 1ull : 0ull);
    }
    atomicAdd(a, L & FX_M56);
    atomicAdd(a + 1, ((L >> 56) | (H << 8)) & FX_M56);
    atomicAdd(a + 2, (unsigned long long)((long long)H >> 48));
}

// The accumulated sum of one column (its FX_COPIES copies, FX_COLS
// columns apart) times isc; L2 loads: the limbs were added by other CTAs.
__device__ __forceinline__ double fx_value(const unsigned long long* a, double isc) {
    unsigned long long s0 = 0ull, s1 = 0ull, s2 = 0ull, bad = 0ull;
#pragma unroll
    for (int k = 0; k < FX_COPIES; ++k) {
        const unsigned long long* c = a + (size_t)k * FX_COLS * FX_LIMBS;
        s0 += __ldcg(c);
        s1 += __ldcg(c + 1);
        s2 += __ldcg(c + 2);
        bad += __ldcg(c + 3);
    }
    if (bad != 0ull) return __longlong_as_double(0x7ff8000000000000ll);
    // s0 + s1 2^56 + s2 2^112 (s2 signed) as hi 2^64 + lo; the limb sums
    // stay below 2^64: at most one term below 2^56 per CTA
    unsigned long long lo = s0 + (s1 << 56);
    unsigned long long hi = (s1 >> 8) + (s2 << 48) + (lo < s0 ? 1ull : 0ull);
    const bool neg = (long long)hi < 0;
    if (neg) {  // magnitude, so that the conversion below keeps full relative precision
        lo = ~lo + 1ull;
        hi = ~hi + (lo == 0ull ? 1ull : 0ull);
    }
    const double m = __ull2double_rn(hi) * 18446744073709551616.0 + __ull2double_rn(lo);
    return (neg ? -m : m) * isc;
}

// w -= V[:, :ncols] h on this CTA's slice, one thread per element (four
// independent chains).  Writes the staged slice ws, the global w when w is
// not null (or its double-float pair to wdf when that is not null), and when
// vg is not null the next basis column w * inv to vg (global, slice offset
// included) and vs (shared, or null).
__device__ __forceinline__ void slice_update(const double* Vl, int64_t vld, int ncols, const double* h, double* w,
                                             double* ws, int64_t lo, int ne, double* vg, double* vs, double inv,
                                             float2* wdf = nullptr) {
    for (int u = threadIdx.x; u < ne; u += PT) {
        const double* vi = Vl + u;
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
        int c = 0;
        for (; c + 3 < ncols; c += 4) {
            a0 += vi[c * vld] * h[c];
            a1 += vi[(c + 1) * vld] * h[c + 1];
            a2 += vi[(c + 2) * vld] * h[c + 2];
            a3 += vi[(c + 3) * vld] * h[c + 3];
        }
        for (; c < ncols; ++c) a0 += vi[c * vld] * h[c];
        const double x = ws[u] - ((a0 + a1) + (a2 + a3));
        ws[u] = x;
        if (w) w[lo + u] = x;
        if (wdf) wdf[lo + u] = df_to_float2(df_from_double(x));
        if (vg) {
            const double y = x * inv;
            vg[u] = y;
            if (vs) vs[u] = y;
        }
    }
}

// sum of x^2 over the staged slice, written by thread 0 to *out
__device__ __forceinline__ void slice_norm2(const double* ws, int ne, double* red, double* out) {
    double a = 0.0;
    for (int u = threadIdx.x; u < ne; u += PT) a += ws[u] * ws[u];
    a = warp_sum(a);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x < 32) {
        const double t = warp_sum(threadIdx.x < PNW ? red[threadIdx.x] : 0.0);
        if (threadIdx.x == 0) *out = t;
    }
}

// The Arnoldi process of one exponential on a grid of nb CTAs of which this
// CTA is number b (slice b).  Every CTA of the grid calls it with the same
// arguments; a failed barrier or a breakdown returns from it in every CTA.
template <int D, int KP1, int G, bool DF>
__device__ __forceinline__ void arnoldi_body(const GmvArgs<double, D>& ga, const ArnArgs& a, const int nb,
                                             const int b) {
    // dynamic shared memory: [w slices: 2 E][Vs: (M+1) Es][Zs: (M+1) Es][located rows, or gather offsets
    // and entries]
    extern __shared__ __align__(16) double smem[];
    __shared__ double h1[SGK_MAX_KRYLOV + 2];
    __shared__ double h2[SGK_MAX_KRYLOV + 2];
    __shared__ double sdot[SGK_MAX_KRYLOV + 2];  // this CTA's inner products
    __shared__ double red[PNW];
    __shared__ double s_scal[4];
    // column-sum and inner-product staging: <= max(PT, 4 (SGK_MAX_KRYLOV + 2))
    __shared__ double ctmp[PT > 4 * (SGK_MAX_KRYLOV + 2) ? PT : 4 * (SGK_MAX_KRYLOV + 2)];
    __shared__ double ctmp2[4 * (SGK_MAX_KRYLOV + 2)];
    __shared__ int s_ok, s_flag;
    // double-float matvec: the correction's coefficients and the step's scale
    __shared__ float2 h2df[DF ? SGK_MAX_KRYLOV + 2 : 1];
    __shared__ float2 s_scaldf;
    const int64_t n = a.n;
    const int E = a.E;  // longest slice
    const int64_t lo = a.bounds ? a.bounds[b] : std::min<int64_t>(n, (int64_t)b * E);
    const int ne = (int)((a.bounds ? a.bounds[b + 1] : std::min<int64_t>(n, lo + E)) - lo);
    // the staged slice of w, two buffers alternating by step: the update of
    // step j (v_{j+1} from w') runs during the matvec of step j + 1
    double* const wsb0 = smem;
    double* const wsb1 = smem + E;
    // shared columns of V and Z have an odd stride: the lanes of one output
    // read different columns of Z at the same row without bank conflicts
    const int Es = E | 1;
    double* const Vs = a.smem_vz ? smem + 2 * E : nullptr;
    double* const Zs = a.smem_vz ? smem + 2 * E + (size_t)(a.M + 1) * Es : nullptr;
    unsigned char* const tail =
        reinterpret_cast<unsigned char*>(smem + 2 * E + (a.smem_vz ? 2 * (size_t)(a.M + 1) * Es : 0));
    GmvLoc<D>* const sloc = a.smem_loc ? reinterpret_cast<GmvLoc<D>*>(tail) : nullptr;
    // pre-located gathers of the slice: offsets rebased to the slice's first
    // entry, then the entries
    int* const seoff = a.list_cap > 0 ? reinterpret_cast<int*>(tail) : nullptr;
    int2* const sent = a.list_cap > 0 ? reinterpret_cast<int2*>(tail + arn_eoff_bytes(E, D)) : nullptr;
    // this slice's basis and raw-output columns: shared copies or HBM
    const double* const Vl = a.smem_vz ? Vs : a.V + lo;
    const int64_t vld = a.smem_vz ? Es : n;
    double* const Zl = a.smem_vz ? Zs : a.Z + lo;
    const int64_t zld = a.smem_vz ? Es : n;
    float2* const Zdf = reinterpret_cast<float2*>(Zl);  // Z as (hi, lo) pairs (double-float matvec)
    double* const P2 = a.pbuf;  // norms
    unsigned epoch = 0;
    auto barrier = [&]() {
        ++epoch;
        return grid_barrier(a.bar, epoch * (unsigned)nb + a.bar_extra, &s_ok);
    };
    // fixed-point reductions: phase p adds into set p % 3, read after its
    // barrier; after the barrier of phase p every CTA is done reading set
    // (p - 1) % 3, which CTA 0 then clears for phase p + 2 (its stores precede
    // its arrival at the barrier before that phase's atomics)
    unsigned fx_phase = 0;
    auto fx_set = [&](unsigned p) { return a.acc + (size_t)(p % 3u) * FX_SET; };
    // publish sdot[0..nt) (the last column with the norm scale when norm)
    auto fx_publish = [&](int nt, bool norm) {
        unsigned long long* set = fx_set(fx_phase) + (size_t)(b % FX_COPIES) * FX_COLS * FX_LIMBS;
        if ((int)threadIdx.x < nt) {
            const bool nc_col = norm && (int)threadIdx.x == nt - 1;
            fx_red(set + (size_t)threadIdx.x * FX_LIMBS, sdot[threadIdx.x], nc_col ? a.sc_n : a.sc_h);
        }
    };
    // after reading phase p: CTA 0 clears set (p + 2) % 3, next phase
    auto fx_done = [&]() {
        if (b == 0) {
            unsigned long long* old = fx_set(fx_phase + 2u);
            for (int i = threadIdx.x; i < FX_SET; i += PT) old[i] = 0ull;
        }
        ++fx_phase;
    };
    auto fx_read = [&](int nt, bool norm, double* out) {
        const unsigned long long* set = fx_set(fx_phase);
        if ((int)threadIdx.x < nt) {
            const bool nc_col = norm && (int)threadIdx.x == nt - 1;
            out[threadIdx.x] = fx_value(set + (size_t)threadIdx.x * FX_LIMBS, nc_col ? a.isc_n : a.isc_h);
        }
        fx_done();
    };
    const int r = threadIdx.x & (G - 1);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    KrylovScalars* ks = a.ks;
    if (sloc)
        for (int u = threadIdx.x; u < ne; u += PT) gmv_locate<double, D, KP1>(ga, lo + u, sloc[u]);
    if (seoff) {
        const int e0 = a.eoff[lo * D], ecount = a.eoff[(lo + ne) * D] - e0;
        if (ecount > a.list_cap) {  // the host sized the list for every slice; fail rather than overrun
            if (threadIdx.x == 0) atomicExch(a.bar + 1, 1u);
            return;
        }
        for (int i = threadIdx.x; i <= ne * D; i += PT) seoff[i] = a.eoff[lo * D + i] - e0;
        for (int i = threadIdx.x; i < ecount; i += PT) sent[i] = a.ent[e0 + i];
    }

    // the accumulator sets start cleared (before the first barrier; the
    // first atomics follow the second)
    if (b == 0)
        for (int i = threadIdx.x; i < 3 * FX_SET; i += PT) a.acc[i] = 0ull;
    // gamma = ||v||
    for (int u = threadIdx.x; u < ne; u += PT) wsb0[u] = a.v[lo + u];
    __syncthreads();
    slice_norm2(wsb0, ne, red, P2 + b);
    if (!barrier()) return;
    colsum(P2, nb, 1, s_scal, ctmp);
    __syncthreads();
    // scalar FP64 work (square roots, reciprocals, the Frobenius norm of H)
    // stays on warp 0 and is broadcast through shared memory: FP64 issue is
    // about two operations per clock per SM on this part
    if (threadIdx.x == 0) {
        const double gamma = sqrt(s_scal[0]);
        s_scal[1] = gamma > 0.0 ? 1.0 / gamma : 0.0;
        if (DF) s_scaldf = df_to_float2(df_from_double(s_scal[1]));
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
    for (int u = threadIdx.x; u < ne; u += PT) {
        const double y = wsb0[u] * scale;
        a.V[lo + u] = y;
        if (Vs) Vs[u] = y;
        // with the double-float matvec the first gathers read the pairs of
        // v / gamma from w1 (free until the second step writes it): pairs of
        // FP32 numbers have FP32's exponent range, so the pairs of an
        // unnormalised v would lose their low parts below about 1e-30 and
        // their values below about 1e-38
        if (DF) reinterpret_cast<float2*>(a.w1)[lo + u] = df_to_float2(df_from_double(y));
    }
    if (DF) {
        // one more barrier publishes the pairs; the first product is then
        // A v_0 itself (scale 1)
        if (!barrier()) return;
        scale = 1.0;
        if (threadIdx.x == 0) s_scaldf = df_to_float2(df_from_double(1.0));
        __syncthreads();
    }
    // the next matvec gathers x (written by all CTAs) and forms
    // A v_j = scale (A x - corr), corr = sum_c hp_c A v_c over the previous
    // step's columns: with the norm taken by Pythagoras, x is w' (complete at
    // the second barrier) and A v_j = (A w' - A V h2) / beta, A V being the
    // stored raw matvec outputs of the slice; after an explicit norm x is w''
    const double* x = a.v;
    const float2* xdf = reinterpret_cast<const float2*>(a.w1);
    int ncorr = 0;                 // columns of the correction (0: none)
    double fro2 = 0.0, sub = 0.0;  // kept alike by every lane of warp 0
    // the pending update of the previous step: v_{pj+1} on the slice from
    // that step's staged w (w' - V h2, or w'' after an explicit norm) times
    // pscale, into column pj + 1 of V (global and shared)
    int pj = -1, pnc = 0;
    bool pexpl = false;
    double pscale = 0.0;
    auto pending_update = [&]() {
        double* const wp = (pj & 1) ? wsb1 : wsb0;
        double* vg = a.V + (int64_t)(pj + 1) * n + lo;
        double* vs = Vs ? Vs + (int64_t)(pj + 1) * Es : nullptr;
        if (pexpl) {
            for (int u = threadIdx.x; u < ne; u += PT) {
                const double y = wp[u] * pscale;
                vg[u] = y;
                if (vs) vs[u] = y;
            }
        } else {
            slice_update(Vl, vld, pnc, h2, nullptr, wp, lo, ne, vg, vs, pscale);
        }
    };
    for (int j = 0; j < a.M; ++j) {
        double* w = (j & 1) ? a.w1 : a.w0;
        double* const ws = (j & 1) ? wsb1 : wsb0;
        const int nc = j + 1;
        // A v_j on this slice, staged in shared memory and kept in Z
        for (int base = 0; base < ne; base += PT / G) {
            const int u = base + (int)threadIdx.x / G;
            const bool live = u < ne;
            double acc;
            // the correction's columns are dealt over the virtual lanes like
            // the matrix rows (sum independent of G)
            if (DF) {
                df64 ad = gmv_accumulate_list_df<D, G>(seoff + (live ? u : 0) * D, sent, a.cvk2, xdf, r, live,
                                                       ncorr, h2df, Zdf + (live ? u : 0), zld);
                if (live && r == 0) {
                    ad = df_mul(ad, df_from_float2(s_scaldf));
                    ws[u] = df_to_double(ad);
                    Zdf[(int64_t)j * zld + u] = df_to_float2(ad);
                }
                continue;
            } else if (seoff) {
                acc = gmv_accumulate_list<D, G>(seoff + (live ? u : 0) * D, sent, ga.cvk, x, r, live, ncorr, h2,
                                                Zl + (live ? u : 0), zld);
            } else if (sloc) {
                acc = gmv_accumulate<double, D, G, 2>(ga, x, sloc[live ? u : 0], r, live, ncorr, h2,
                                                         Zl + (live ? u : 0), zld);
            } else {
                GmvLoc<D> l1;
                if (live) gmv_locate<double, D, KP1>(ga, lo + u, l1);
                acc = gmv_accumulate<double, D, G, 2>(ga, x, l1, r, live, ncorr, h2, Zl + (live ? u : 0), zld);
            }
            if (live && r == 0) {
                acc *= scale;
                ws[u] = acc;
                Zl[(int64_t)j * zld + u] = acc;
            }
        }
        if (pj >= 0) pending_update();
        __syncthreads();
        slice_dots(Vl, vld, nc, ws, ne, sdot, false, ctmp, ctmp2);
        fx_publish(nc, false);
        if (!barrier()) return;
        fx_read(nc, false, h1);
        __syncthreads();
        // w' = w - V h1, published for the next matvec
        slice_update(Vl, vld, nc, h1, DF ? nullptr : w, ws, lo, ne, nullptr, nullptr, 0.0,
                     DF ? reinterpret_cast<float2*>(w) : nullptr);
        __syncthreads();
        // second pass: V^T w' and ||w'||^2 in one reduction
        slice_dots(Vl, vld, nc, ws, ne, sdot, true, ctmp, ctmp2);
        fx_publish(nc + 1, true);
        if (!barrier()) return;
        // column j of H and the breakdown test from ||w''||^2 = b2 and
        // part = ||h1 + h2||^2: warp 0 of every CTA, every lane alike
        auto hcol = [&](double b2, double part) {
            const double f = fro2 + sub * sub + part;
            // one reciprocal square root on two lanes: 1/beta and sqrt(f)
            const double xin = lane == 0 ? b2 : f;
            const double rs = xin > 0.0 ? rsqrt(xin) : 0.0;
            const double inv = __shfl_sync(0xffffffffu, rs, 0);
            const double sf = f > 0.0 ? f * __shfl_sync(0xffffffffu, rs, 1) : 0.0;
            const double beta = b2 > 0.0 ? b2 * inv : 0.0;
            fro2 = f;
            sub = beta;
            const bool brk = !(beta > 1e-12 * sf);
            if (b == 0)
                for (int i = lane; i < nc; i += 32) a.H[(int64_t)i * a.M + j] = h1[i] + h2[i];
            if (lane == 0) {
                s_scal[1] = brk ? 0.0 : inv;
                if (DF) s_scaldf = df_to_float2(df_from_double(brk ? 0.0 : inv));
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
        };
        // ||w''||^2 = ||w'||^2 - ||h2||^2 (V orthonormal, w'' = w' - V h2);
        // when the second pass removed more than 1e-3 of ||w'||^2 (near
        // breakdown) the norm is summed explicitly instead.  With at most 32
        // columns warp 0 reads h2 itself and, in the common case, finishes
        // the column at once: one CTA barrier for the whole scalar part
        auto pyth = [&](double part, double hh, double wn2) {
            const double b2 = wn2 - hh;
            const bool flag = !(hh <= 1e-3 * wn2) || !(b2 > 0.0);
            if (lane == 0) {
                s_flag = flag;
                s_scal[0] = b2;
                s_scal[2] = part;
            }
            if (!flag) hcol(b2, part);
        };
        if (nc + 1 <= 32) {
            if (wid == 0) {
                const unsigned long long* set = fx_set(fx_phase);
                const double hv2 =
                    lane <= nc ? fx_value(set + (size_t)lane * FX_LIMBS, lane == nc ? a.isc_n : a.isc_h) : 0.0;
                if (lane <= nc) h2[lane] = hv2;
                if (DF && lane < nc) h2df[lane] = df_to_float2(df_from_double(hv2));
                __syncwarp();
                const double hv = lane < nc ? h1[lane] + hv2 : 0.0;
                const double part = warp_sum(hv * hv);
                const double hh = warp_sum(lane < nc ? hv2 * hv2 : 0.0);
                pyth(part, hh, __shfl_sync(0xffffffffu, hv2, nc));
            }
            fx_done();
        } else {
            fx_read(nc + 1, true, h2);
            __syncthreads();
            if (DF)
                for (int i = threadIdx.x; i < nc; i += PT) h2df[i] = df_to_float2(df_from_double(h2[i]));
            if (wid == 0) {
                double part = 0.0, hh = 0.0;
                for (int i = lane; i < nc; i += 32) {
                    const double hv = h1[i] + h2[i];
                    part += hv * hv;
                    hh += h2[i] * h2[i];
                }
                pyth(warp_sum(part), warp_sum(hh), h2[nc]);
            }
        }
        __syncthreads();
        const bool explicit_norm = s_flag != 0;
        if (explicit_norm) {
            // w'' in place (published), its norm through a third barrier
            slice_update(Vl, vld, nc, h2, DF ? nullptr : w, ws, lo, ne, nullptr, nullptr, 0.0,
                         DF ? reinterpret_cast<float2*>(w) : nullptr);
            __syncthreads();
            slice_norm2(ws, ne, red, P2 + b);
            if (!barrier()) return;
            colsum(P2, nb, 1, s_scal, ctmp);
            __syncthreads();
            if (wid == 0) hcol(s_scal[0], s_scal[2]);
            __syncthreads();
        }
        if (!(s_scal[1] > 0.0)) return;  // breakdown: the same decision in every CTA
        scale = s_scal[1];
        // v_{j+1} is formed during the next step's matvec (which gathers w',
        // published, and needs no column of V); the inner products after it
        // read column j + 1
        pj = j;
        pnc = nc;
        pexpl = explicit_norm;
        pscale = scale;
        ncorr = explicit_norm ? 0 : nc;
        x = w;
        xdf = reinterpret_cast<const float2*>(w);
    }
    if (pj >= 0) pending_update();  // the last column, v_M
}

template <int D, int KP1, int G, bool DF>
__global__ void __launch_bounds__(PT, 1) arnoldi_kernel(const GmvArgs<double, D> ga, const ArnArgs a) {
    arnoldi_body<D, KP1, G, DF>(ga, a, gridDim.x, blockIdx.x);
}

// Many independent Arnoldi processes in one cooperative launch.  CTA c runs
// the work items item_off[c] .. item_off[c+1]-1 in order; item (i, b) makes
// it slice b of instance i's grid of nb[i] CTAs.  The host builds the lists
// from one global order of the instances (each instance's slices take the
// same position in every list that holds them), and every CTA is resident,
// so no CTA waits on an instance that cannot start: an instance's barriers
// only involve the CTAs of its own items.
template <int D>
struct ArnMulti {
    const int* item_off;  // gridDim.x + 1
    const int2* items;    // (instance, slice)
    const GmvArgs<double, D>* ga;
    const ArnArgs* aa;
    const int* nb;
};

template <int D, int KP1, int G, bool DF>
__global__ void __launch_bounds__(PT, 1) arnoldi_multi_kernel(const ArnMulti<D> m) {
    __shared__ ArnArgs s_a;
    __shared__ GmvArgs<double, D> s_ga;
    __shared__ int s_nb;
    const int first = m.item_off[blockIdx.x], last = m.item_off[blockIdx.x + 1];
    for (int it = first; it < last; ++it) {
        const int2 w = m.items[it];
        __syncthreads();  // the previous item is done with shared memory
        {
            const int* src = reinterpret_cast<const int*>(m.aa + w.x);
            int* dst = reinterpret_cast<int*>(&s_a);
            for (int i = threadIdx.x; i < (int)(sizeof(ArnArgs) / sizeof(int)); i += PT) dst[i] = src[i];
            const int* gsrc = reinterpret_cast<const int*>(m.ga + w.x);
            int* gdst = reinterpret_cast<int*>(&s_ga);
            for (int i = threadIdx.x; i < (int)(sizeof(GmvArgs<double, D>) / sizeof(int)); i += PT) gdst[i] = gsrc[i];
            if (threadIdx.x == 0) s_nb = m.nb[w.x];
        }
        __syncthreads();
        arnoldi_body<D, KP1, G, DF>(s_ga, s_a, s_nb, w.y);
    }
}

// Launch arguments of one Arnoldi process (arnoldi_prepare).
struct ArnPrep {
    ArnArgs a;
    size_t smem = 0;
    int nb = 0, G = 0, d = 0, kp1 = 0;
};

// Device copies of the matvec arguments of a list of operators (d = D).
template <int D>
void arn_multi_upload_ga(const std::vector<const sgk_op*>& ops, DevBuf<unsigned char>& buf, cudaStream_t st) {
    std::vector<GmvArgs<double, D>> v;
    v.reserve(ops.size());
    for (const sgk_op* op : ops) v.push_back(make_gmv_args<double, D>(op));
    buf.alloc(v.size() * sizeof(GmvArgs<double, D>));
    buf.upload(reinterpret_cast<const unsigned char*>(v.data()), buf.n, st);
}

template <int D, int KP1, int G>
void arn_multi_launch(cudaStream_t st, bool df, const ArnMulti<D>& m, int grid, size_t smem, size_t smem_optin,
                      int num_sms) {
    auto kern = df ? arnoldi_multi_kernel<D, KP1, G, true> : arnoldi_multi_kernel<D, KP1, G, false>;
    allow_max_dynamic_smem(smem_optin, kern);
    int occ = 0;
    SGK_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, PT, smem));
    SGK_REQUIRE(occ >= 1 && grid <= occ * num_sms, SGK_EUNSUPPORTED, "batched Arnoldi grid does not fit");
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(PT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    SGK_CUDA_CHECK(cudaLaunchKernelEx(&cfg, kern, m));
}

// Batched launch for d = D: degree (k + 1 = kp1) and lanes per output (4 or
// 8) select the kernel; ga points at the device GmvArgs<double, D> array.
template <int D>
void arn_multi_launch_k(cudaStream_t st, int kp1, int G, bool df, const int* item_off, const int2* items,
                        const void* ga, const ArnArgs* aa, const int* nb, int grid, size_t smem, size_t smem_optin,
                        int num_sms) {
    ArnMulti<D> m;
    m.item_off = item_off;
    m.items = items;
    m.ga = static_cast<const GmvArgs<double, D>*>(ga);
    m.aa = aa;
    m.nb = nb;
#define SGK_ARN_MULTI(K, GG)                                                            \
    if (kp1 == K && G == GG) {                                                          \
        arn_multi_launch<D, K, GG>(st, df, m, grid, smem, smem_optin, num_sms);         \
        return;                                                                         \
    }
    SGK_ARN_MULTI(2, 4) SGK_ARN_MULTI(2, 8) SGK_ARN_MULTI(3, 4) SGK_ARN_MULTI(3, 8) SGK_ARN_MULTI(4, 4)
    SGK_ARN_MULTI(4, 8)
#undef SGK_ARN_MULTI
    throw SgkError{SGK_EUNSUPPORTED, "batched Arnoldi: no kernel for this degree and lane count"};
}

template <int D, int KP1, int G>
void arn_launch(sgk_ctx* ctx, const sgk_op* op, const ArnArgs& a, int nb, size_t smem) {
    auto kern = a.df ? arnoldi_kernel<D, KP1, G, true> : arnoldi_kernel<D, KP1, G, false>;
    const GmvArgs<double, D> ga = make_gmv_args<double, D>(op);
    allow_max_dynamic_smem(ctx->smem_optin, kern);
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

}  // namespace sgk_arn
