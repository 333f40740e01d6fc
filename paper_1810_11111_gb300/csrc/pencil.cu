// Fused last-direction pass of the reaction term (Section 4: reconstruction
// at the finest-mesh Gauss points and quadrature).
//
// After directions 0..d-2 have been changed to the finest-cell Legendre basis
// (fiber engine), direction d-1 still holds 1D hierarchical coefficients.
// One CTA takes a pencil: a fixed finest cell in directions 0..d-2, i.e. the
// (k+1)^{d-1} fibers of that cell's Legendre degrees, each of length
// H = (k+1) 2^N along direction d-1.  In shared memory it
//   1. changes each fiber to the finest-cell Legendre basis
//      (nodal[y] = sum_{n,p} T[y; n,p] hier[level n, cell j_n(y), p]; every
//      row of T has exactly (N+1)(k+1) entries, stored densely),
//   2. runs the cell quadrature with one thread per finest cell of the
//      pencil: Legendre -> q^d Gauss points -> f(u) or f'(u) w times the
//      weights -> Legendre moments, as nested sum-factorised loops whose
//      indices are compile-time constants (all in registers),
//   3. applies T^T (row a of T^T covers a contiguous range of y) and stores
//      the hierarchical result.
// Specialised for (d, k+1, q, species); other shapes use the unfused path.
#include <algorithm>

#include "sgk_pencil.h"

namespace {

template <int B, int E>
struct Pow {
    static constexpr int v = B * Pow<B, E - 1>::v;
};
template <int B>
struct Pow<B, 0> {
    static constexpr int v = 1;
};

template <typename T>
struct QuadTab {
    T B[8][4];  // B[g][r] = h^{-1/2} sqrt(2r+1) P_r(xi_g)
    T w[8];     // h w_g / 2
};

template <typename T, int S>
struct Rx {
    int nmono;
    int species[SGK_MAX_MONO];
    T coef[SGK_MAX_MONO];
    int exps[SGK_MAX_MONO][SGK_MAX_SPECIES];
};

template <typename T>
__device__ __forceinline__ T ipow_t(T x, int e) {
    T r = T(1);
    for (int i = 0; i < e; ++i) r *= x;
    return r;
}

// Pointwise reaction (JAC = 0) or Jacobian product (JAC = 1) for S species.
template <typename T, int S, bool JAC>
__device__ __forceinline__ void point_eval(const Rx<T, S>& rx, const T (&u)[S], const T (&w)[S], T (&out)[S]) {
#pragma unroll
    for (int s = 0; s < S; ++s) out[s] = T(0);
    for (int mo = 0; mo < rx.nmono; ++mo) {
        const int s = rx.species[mo];
        T acc = T(0);
        if (!JAC) {
            T t = rx.coef[mo];
#pragma unroll
            for (int r = 0; r < S; ++r) t *= ipow_t(u[r], rx.exps[mo][r]);
            acc = t;
        } else {
#pragma unroll
            for (int r = 0; r < S; ++r) {
                const int er = rx.exps[mo][r];
                if (er == 0) continue;
                T t = rx.coef[mo] * T(er) * w[r];
#pragma unroll
                for (int r2 = 0; r2 < S; ++r2) t *= ipow_t(u[r2], rx.exps[mo][r2] - (r2 == r ? 1 : 0));
                acc += t;
            }
        }
#pragma unroll
        for (int r = 0; r < S; ++r)
            if (r == s) out[r] += acc;
    }
}

// Recursive sum-factorised quadrature over directions DIM..D-1.
// Cin: coefficient slabs (KP1^(D-DIM) per species and set), Mout: moment
// accumulators of the same shape, wt: product of the weights of the
// directions already fixed.
template <typename T, int D, int KP1, int Q, int S, bool JAC, int DIM>
struct Quad {
    static constexpr int N = Pow<KP1, D - DIM>::v;
    static constexpr int NS = N / KP1;
    __device__ __forceinline__ static void run(const QuadTab<T>& tb, const Rx<T, S>& rx, const T (&Cu)[S][N],
                                               const T (&Cw)[S][N], T (&M)[S][N], T wt) {
#pragma unroll 1
        for (int g = 0; g < Q; ++g) {
            T su[S][NS], sw[S][NS], sm[S][NS];
#pragma unroll
            for (int s = 0; s < S; ++s)
#pragma unroll
                for (int i = 0; i < NS; ++i) {
                    T a = T(0), b = T(0);
#pragma unroll
                    for (int r = 0; r < KP1; ++r) {
                        a += tb.B[g][r] * Cu[s][r * NS + i];
                        if (JAC) b += tb.B[g][r] * Cw[s][r * NS + i];
                    }
                    su[s][i] = a;
                    sw[s][i] = b;
                    sm[s][i] = T(0);
                }
            Quad<T, D, KP1, Q, S, JAC, DIM + 1>::run(tb, rx, su, sw, sm, wt * tb.w[g]);
#pragma unroll
            for (int s = 0; s < S; ++s)
#pragma unroll
                for (int r = 0; r < KP1; ++r)
#pragma unroll
                    for (int i = 0; i < NS; ++i) M[s][r * NS + i] += tb.B[g][r] * sm[s][i];
        }
    }
};

// Last direction: the slab is a single coefficient per species.
template <typename T, int D, int KP1, int Q, int S, bool JAC>
struct Quad<T, D, KP1, Q, S, JAC, D> {
    __device__ __forceinline__ static void run(const QuadTab<T>&, const Rx<T, S>& rx, const T (&Cu)[S][1],
                                               const T (&Cw)[S][1], T (&M)[S][1], T wt) {
        T u[S], w[S], o[S];
#pragma unroll
        for (int s = 0; s < S; ++s) {
            u[s] = Cu[s][0];
            w[s] = Cw[s][0];
        }
        point_eval<T, S, JAC>(rx, u, w, o);
#pragma unroll
        for (int s = 0; s < S; ++s) M[s][0] = wt * o[s];
    }
};

template <typename T, int D, int KP1, int Q, int S, bool JAC>
__global__ void __launch_bounds__(256) pencil_kernel(const PencilArgs args, const QuadTab<T> tb, const Rx<T, S> rx) {
    constexpr int P = Pow<KP1, D - 1>::v;    // fibers per species and set
    constexpr int NC = Pow<KP1, D>::v;       // coefficients per cell
    constexpr int NSETS = JAC ? 2 * S : S;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw);
    const int H = args.H, N = args.N;
    const int W = (N + 1) * KP1;             // width of a row of T
    const T* __restrict__ Tv = reinterpret_cast<const T*>(args.Tv);
    T* hier = sm;                             // [NSETS][P][H]
    T* nod = sm + (size_t)NSETS * P * H;      // [NSETS][P][H]
    const long long npencils = args.npencils;
    for (long long pen = blockIdx.x; pen < npencils; pen += gridDim.x) {
        // fiber offsets of this pencil: o_f = sum_m (c_m (k+1) + r_m) H^{d-2-m}
        long long obase = 0;
        {
            long long rem = pen, mul = 1;
            for (int m = D - 2; m >= 0; --m) {
                const long long c = rem % args.ncell1;
                rem /= args.ncell1;
                obase += c * KP1 * mul;
                mul *= H;
            }
        }
        // 1. load the hierarchical fibers (chunks: one per level)
        for (int e = threadIdx.x; e < NSETS * P * H; e += blockDim.x) {
            const int a = e % H;
            const int f = (e / H) % P;
            const int set = e / (H * P);
            long long o = obase, mul = 1;
            int rr = f;
#pragma unroll
            for (int m = D - 2; m >= 0; --m) {
                o += (rr % KP1) * mul;
                rr /= KP1;
                mul *= H;
            }
            const int q = a / KP1;
            const int l = q == 0 ? 0 : 32 - __clz(q);
            const int off = l ? (KP1 << (l - 1)) : 0;
            const int nl = l ? (KP1 << (l - 1)) : KP1;
            const T* src = reinterpret_cast<const T*>(set < S ? args.u[set] : args.w[set - S]);
            hier[e] = src[args.cbase[l] + o * nl + (a - off)];
        }
        __syncthreads();
        // 2. to finest-cell Legendre coefficients
        for (int e = threadIdx.x; e < NSETS * P * H; e += blockDim.x) {
            const int y = e % H;
            const T* hf = hier + (e - y);
            const int c = y / KP1;
            const T* trow = Tv + (size_t)y * W;
            T acc = T(0);
#pragma unroll
            for (int p = 0; p < KP1; ++p) acc += trow[p] * hf[p];
            for (int n = 1; n <= N; ++n) {
                const int j = c >> (N - n + 1);
                const T* hp = hf + (KP1 << (n - 1)) + j * KP1;
                const T* tp = trow + n * KP1;
#pragma unroll
                for (int p = 0; p < KP1; ++p) acc += tp[p] * hp[p];
            }
            nod[e] = acc;
        }
        __syncthreads();
        // 3. cell quadrature, one thread per finest cell along the pencil
        const int ncell = H / KP1;
        for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
            T Cu[S][NC], Cw[S][NC], M[S][NC];
#pragma unroll
            for (int s = 0; s < S; ++s)
#pragma unroll
                for (int i = 0; i < NC; ++i) {
                    const int f = i / KP1, r = i % KP1;
                    Cu[s][i] = nod[((size_t)s * P + f) * H + c * KP1 + r];
                    Cw[s][i] = JAC ? nod[((size_t)(S + s) * P + f) * H + c * KP1 + r] : T(0);
                    M[s][i] = T(0);
                }
            Quad<T, D, KP1, Q, S, JAC, 0>::run(tb, rx, Cu, Cw, M, T(1));
#pragma unroll
            for (int s = 0; s < S; ++s)
#pragma unroll
                for (int i = 0; i < NC; ++i) {
                    const int f = i / KP1, r = i % KP1;
                    hier[((size_t)s * P + f) * H + c * KP1 + r] = M[s][i];
                }
        }
        __syncthreads();
        // 4. back to hierarchical coefficients (rows of T^T are contiguous
        //    ranges of y) and store
        for (int e = threadIdx.x; e < S * P * H; e += blockDim.x) {
            const int a = e % H;
            const int f = (e / H) % P;
            const int s = e / (H * P);
            const T* mf = hier + (size_t)(s * P + f) * H;
            const int q = a / KP1;
            const int l = q == 0 ? 0 : 32 - __clz(q);
            const int off = l ? (KP1 << (l - 1)) : 0;
            const int nl = l ? (KP1 << (l - 1)) : KP1;
            const int t = a - off;
            const int j = t / KP1, p = t % KP1;
            const int len = l == 0 ? H : (KP1 << (N - l + 1));
            const int y0 = l == 0 ? 0 : j * len;
            const T* tcol = Tv + l * KP1 + p;
            T acc = T(0);
            for (int y = y0; y < y0 + len; ++y) acc += tcol[(size_t)y * W] * mf[y];
            long long o = obase, mul = 1;
            int rr = f;
#pragma unroll
            for (int m = D - 2; m >= 0; --m) {
                o += (rr % KP1) * mul;
                rr /= KP1;
                mul *= H;
            }
            T* dst = reinterpret_cast<T*>(args.out[s]);
            dst[args.cbase[l] + o * nl + t] = acc;
        }
        __syncthreads();
    }
}

template <typename T, int D, int KP1, int Q, int S, bool JAC>
void launch_one(sgk_ctx* ctx, const PencilArgs& a, const QuadTab<T>& tb, const ReactionDev& rxd) {
    Rx<T, S> rx{};
    rx.nmono = rxd.nmono;
    for (int m = 0; m < rxd.nmono; ++m) {
        rx.species[m] = rxd.species[m];
        rx.coef[m] = (T)rxd.coef[m];
        for (int r = 0; r < SGK_MAX_SPECIES; ++r) rx.exps[m][r] = rxd.exps[m][r];
    }
    constexpr int P = Pow<KP1, D - 1>::v;
    constexpr int NSETS = JAC ? 2 * S : S;
    const size_t smem = (size_t)2 * NSETS * P * a.H * sizeof(T);
    SGK_REQUIRE(smem <= ctx->smem_optin, SGK_EUNSUPPORTED, "pencil exceeds shared memory");
    const int threads = std::min(256, std::max(64, a.H / KP1));
    const int grid = (int)std::min<long long>(a.npencils, (long long)ctx->num_sms * 16);
    auto kern = pencil_kernel<T, D, KP1, Q, S, JAC>;
    SGK_CUDA_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<grid, threads, smem, ctx->stream>>>(a, tb, rx);
}

template <typename T>
QuadTab<T> make_tab(const double* B, const double* w, int q, int kp1) {
    QuadTab<T> t{};
    for (int g = 0; g < q; ++g) {
        for (int r = 0; r < kp1; ++r) t.B[g][r] = (T)B[g * kp1 + r];
        t.w[g] = (T)w[g];
    }
    return t;
}

template <typename T, bool JAC>
bool dispatch(sgk_ctx* ctx, int d, int kp1, int q, int S, const PencilArgs& a, const QuadTab<T>& tb,
              const ReactionDev& rx) {
#define SGK_PENCIL(DD, KK, QQ, SS)                                 \
    if (d == DD && kp1 == KK && q == QQ && S == SS) {              \
        launch_one<T, DD, KK, QQ, SS, JAC>(ctx, a, tb, rx);        \
        return true;                                               \
    }
    SGK_PENCIL(3, 3, 5, 1)
    SGK_PENCIL(2, 3, 5, 2)
    SGK_PENCIL(2, 2, 3, 1)
    SGK_PENCIL(2, 2, 3, 2)
    SGK_PENCIL(3, 2, 3, 1)
    SGK_PENCIL(2, 3, 5, 1)
    SGK_PENCIL(4, 2, 3, 1)
#undef SGK_PENCIL
    return false;
}

}  // namespace

bool pencil_supported(int d, int kp1, int q, int S) {
    const int combos[][4] = {{3, 3, 5, 1}, {2, 3, 5, 2}, {2, 2, 3, 1}, {2, 2, 3, 2},
                             {3, 2, 3, 1}, {2, 3, 5, 1}, {4, 2, 3, 1}};
    for (auto& c : combos)
        if (c[0] == d && c[1] == kp1 && c[2] == q && c[3] == S) return true;
    return false;
}

template <typename T>
void pencil_launch(sgk_ctx* ctx, const PencilArgs& a, int d, int kp1, int q, int S, bool jac, const double* B,
                   const double* w, const ReactionDev& rx) {
    const QuadTab<T> tb = make_tab<T>(B, w, q, kp1);
    KTimer kt(ctx, KC_CELL);
    const bool ok = jac ? dispatch<T, true>(ctx, d, kp1, q, S, a, tb, rx) : dispatch<T, false>(ctx, d, kp1, q, S, a, tb, rx);
    SGK_REQUIRE(ok, SGK_EUNSUPPORTED, "no fused pencil kernel for this shape");
    check_launch("pencil_kernel");
    count_launch(ctx);
}

template void pencil_launch<double>(sgk_ctx*, const PencilArgs&, int, int, int, int, bool, const double*,
                                    const double*, const ReactionDev&);
template void pencil_launch<float>(sgk_ctx*, const PencilArgs&, int, int, int, int, bool, const double*,
                                   const double*, const ReactionDev&);
