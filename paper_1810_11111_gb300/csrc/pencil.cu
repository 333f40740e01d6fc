// Fused last-direction pass of the reaction term (Section 4: reconstruction
// at the finest-mesh Gauss points and quadrature).
//
// After directions 0..d-2 have been changed to the finest-cell Legendre basis
// (fiber engine), direction d-1 still holds 1D hierarchical coefficients.
// One CTA takes a pencil: a fixed finest cell in directions 0..d-2, i.e. the
// (k+1)^{d-1} fibers of that cell's Legendre degrees, each of length
// H = (k+1) 2^N along direction d-1.  In shared memory it
//   1. reconstructs each fiber in the finest-cell Legendre basis with the
//      two-scale relations, level by level: the children of a level-(n-1)
//      cell get H_h^T (parent coefficients) + G_h^T (level-n wavelet
//      coefficients), 2 (k+1)^2 FMAs per child cell;
//   2. runs the cell quadrature with one thread per finest cell of the
//      pencil: Legendre -> q^d Gauss points -> f(u) or f'(u) w times the
//      weights -> Legendre moments, as nested sum-factorised loops whose
//      indices are compile-time constants (registers only); f and f' are
//      dense polynomials evaluated by Horner's rule;
//   3. decomposes the moments back to hierarchical coefficients with the
//      transposed two-scale relations and stores them.
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

constexpr int PDEG = 5;  // exponents 0..4 per species

template <typename T, int KP1>
struct Filt {
    T H[2][KP1][KP1];  // H[h][r][s]
    T G[2][KP1][KP1];  // G[h][p][s]
};

template <typename T>
struct QuadTab {
    T B[8][4];  // B[g][r] = h^{-1/2} sqrt(2r+1) P_r(xi_g)
    T w[8];     // h w_g / 2
};

// f_s(u) = sum_e c[s][e] u^e (one species) or sum_{a,b} c[s][a 5 + b] u^a v^b
template <typename T, int S>
struct Poly {
    T c[S][Pow<PDEG, S>::v];
};

template <typename T, int S, bool JAC>
struct PointEval;

template <typename T, bool JAC>
struct PointEval<T, 1, JAC> {
    __device__ __forceinline__ static void run(const Poly<T, 1>& P, const T (&u)[1], const T (&w)[1], T (&o)[1]) {
        if (!JAC) {
            T f = P.c[0][PDEG - 1];
#pragma unroll
            for (int e = PDEG - 2; e >= 0; --e) f = f * u[0] + P.c[0][e];
            o[0] = f;
        } else {
            T df = T(PDEG - 1) * P.c[0][PDEG - 1];
#pragma unroll
            for (int e = PDEG - 2; e >= 1; --e) df = df * u[0] + T(e) * P.c[0][e];
            o[0] = df * w[0];
        }
    }
};

template <typename T, bool JAC>
struct PointEval<T, 2, JAC> {
    __device__ __forceinline__ static void run(const Poly<T, 2>& P, const T (&u)[2], const T (&w)[2], T (&o)[2]) {
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            // inner polynomials in v for each power of u, and their v-derivatives
            T in[PDEG], dv[PDEG];
#pragma unroll
            for (int a = 0; a < PDEG; ++a) {
                T f = P.c[s][a * PDEG + PDEG - 1];
                T g = T(PDEG - 1) * P.c[s][a * PDEG + PDEG - 1];
#pragma unroll
                for (int b = PDEG - 2; b >= 0; --b) {
                    f = f * u[1] + P.c[s][a * PDEG + b];
                    if (b >= 1) g = g * u[1] + T(b) * P.c[s][a * PDEG + b];
                }
                in[a] = f;
                dv[a] = g;
            }
            if (!JAC) {
                T f = in[PDEG - 1];
#pragma unroll
                for (int a = PDEG - 2; a >= 0; --a) f = f * u[0] + in[a];
                o[s] = f;
            } else {
                T fu = T(PDEG - 1) * in[PDEG - 1];
#pragma unroll
                for (int a = PDEG - 2; a >= 1; --a) fu = fu * u[0] + T(a) * in[a];
                T fv = dv[PDEG - 1];
#pragma unroll
                for (int a = PDEG - 2; a >= 0; --a) fv = fv * u[0] + dv[a];
                o[s] = fu * w[0] + fv * w[1];
            }
        }
    }
};

// Recursive sum-factorised quadrature over directions DIM..D-1 (see header).
template <typename T, int D, int KP1, int Q, int S, bool JAC, int DIM>
struct Quad {
    static constexpr int N = Pow<KP1, D - DIM>::v;
    static constexpr int NS = N / KP1;
    // the innermost level (whose body is the point evaluation, where most
    // of the arithmetic is) is unrolled so that its Gauss-table entries are
    // compile-time operands; the outer levels stay loops
    static constexpr int UNROLL = DIM == D - 1 ? Q : 1;
    __device__ __forceinline__ static void run(const QuadTab<T>& tb, const Poly<T, S>& P, const T (&Cu)[S][N],
                                               const T (&Cw)[S][N], T (&M)[S][N], T wt) {
#pragma unroll UNROLL
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
            Quad<T, D, KP1, Q, S, JAC, DIM + 1>::run(tb, P, su, sw, sm, wt * tb.w[g]);
#pragma unroll
            for (int s = 0; s < S; ++s)
#pragma unroll
                for (int r = 0; r < KP1; ++r)
#pragma unroll
                    for (int i = 0; i < NS; ++i) M[s][r * NS + i] += tb.B[g][r] * sm[s][i];
        }
    }
};

template <typename T, int D, int KP1, int Q, int S, bool JAC>
struct Quad<T, D, KP1, Q, S, JAC, D> {
    __device__ __forceinline__ static void run(const QuadTab<T>&, const Poly<T, S>& P, const T (&Cu)[S][1],
                                               const T (&Cw)[S][1], T (&M)[S][1], T wt) {
        T u[S], w[S], o[S];
#pragma unroll
        for (int s = 0; s < S; ++s) {
            u[s] = Cu[s][0];
            w[s] = Cw[s][0];
        }
        PointEval<T, S, JAC>::run(P, u, w, o);
#pragma unroll
        for (int s = 0; s < S; ++s) M[s][0] = wt * o[s];
    }
};

// Reconstruct P fibers (hierarchical, levels 0..N, in `src`) to the finest
// Legendre basis using scratch buffers a and b; returns the buffer holding
// the result (a, b, or src when N = 0).
template <typename T, int KP1, int P>
__device__ T* reconstruct(T* src, T* a, T* b, int H, int N, const Filt<T, KP1>& F) {
    const T* cur = src;
    T* dst = a;
    for (int n = 1; n <= N; ++n) {
        const int npar = 1 << (n - 1);
        for (int it = threadIdx.x; it < P * npar * 2; it += blockDim.x) {
            const int h = it & 1;
            const int c = (it >> 1) & (npar - 1);
            const int f = (it >> 1) >> (n - 1);
            const T* par = cur + f * H + c * KP1;
            const T* det = src + f * H + (KP1 << (n - 1)) + c * KP1;
            T pv[KP1], dv[KP1];
#pragma unroll
            for (int r = 0; r < KP1; ++r) {
                pv[r] = par[r];
                dv[r] = det[r];
            }
            T* o = dst + f * H + (2 * c + h) * KP1;
#pragma unroll
            for (int s = 0; s < KP1; ++s) {
                T acc = T(0);
#pragma unroll
                for (int r = 0; r < KP1; ++r) acc += F.H[h][r][s] * pv[r] + F.G[h][r][s] * dv[r];
                o[s] = acc;
            }
        }
        __syncthreads();
        cur = dst;
        dst = (dst == a) ? b : a;
    }
    return const_cast<T*>(cur);
}

// Decompose P fibers of finest Legendre moments (in m, destroyed) into
// hierarchical coefficients in res, using scratch a.
template <typename T, int KP1, int P>
__device__ void decompose(T* m, T* a, T* res, int H, int N, const Filt<T, KP1>& F) {
    T* cur = m;
    T* dst = a;
    for (int n = N; n >= 1; --n) {
        const int npar = 1 << (n - 1);
        for (int it = threadIdx.x; it < P * npar; it += blockDim.x) {
            const int c = it & (npar - 1);
            const int f = it >> (n - 1);
            const T* c0 = cur + f * H + 2 * c * KP1;
            T x0[KP1], x1[KP1];
#pragma unroll
            for (int s = 0; s < KP1; ++s) {
                x0[s] = c0[s];
                x1[s] = c0[KP1 + s];
            }
            T* po = dst + f * H + c * KP1;
            T* dout = res + f * H + (KP1 << (n - 1)) + c * KP1;
#pragma unroll
            for (int r = 0; r < KP1; ++r) {
                T sp = T(0), sd = T(0);
#pragma unroll
                for (int s = 0; s < KP1; ++s) {
                    sp += F.H[0][r][s] * x0[s] + F.H[1][r][s] * x1[s];
                    sd += F.G[0][r][s] * x0[s] + F.G[1][r][s] * x1[s];
                }
                po[r] = sp;
                dout[r] = sd;
            }
        }
        __syncthreads();
        T* t = cur;
        cur = dst;
        dst = t;
    }
    for (int it = threadIdx.x; it < P * KP1; it += blockDim.x) {
        const int f = it / KP1, r = it % KP1;
        res[f * H + r] = cur[f * H + r];
    }
    __syncthreads();
}

template <typename T, int D, int KP1, int Q, int S, bool JAC>
__global__ void __launch_bounds__(256) pencil_kernel(const PencilArgs args, const QuadTab<T> tb,
                                                     const Filt<T, KP1> F, const Poly<T, S> poly) {
    constexpr int P = Pow<KP1, D - 1>::v;  // fibers per species and set
    constexpr int NC = Pow<KP1, D>::v;     // coefficients per cell
    constexpr int NSETS = JAC ? 2 * S : S;
    constexpr int NBUF = NSETS + 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw);
    const int H = args.H, N = args.N;
    const int fb = P * H;  // one buffer: P fibers
    auto buf = [&](int i) { return sm + (size_t)i * fb; };
    for (long long pen = blockIdx.x; pen < args.npencils; pen += gridDim.x) {
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
        // 1. load the hierarchical fibers of every set into buffers 0..NSETS-1
        // fiber offset of fiber f: o_f = obase + sum_m r_m H^{d-2-m}
        auto fiber_offset = [&](int f) {
            long long o = obase, mul = 1;
            int rr = f;
#pragma unroll
            for (int m = D - 2; m >= 0; --m) {
                o += (rr % KP1) * mul;
                rr /= KP1;
                mul *= H;
            }
            return o;
        };
        // address of position a of fiber offset o in the level-chunked layout
        auto chunk = [&](long long o, int a) {
            const int q = a / KP1;
            const int l = q == 0 ? 0 : 32 - __clz(q);
            const int off = l ? (KP1 << (l - 1)) : 0;
            const int nl = l ? (KP1 << (l - 1)) : KP1;
            return args.cbase[l] + o * nl + (a - off);
        };
#pragma unroll 1
        for (int sf = 0; sf < NSETS * P; ++sf) {
            const int set = sf / P, f = sf - (sf / P) * P;
            const long long o = fiber_offset(f);
            const T* src = reinterpret_cast<const T*>(set < S ? args.u[set] : args.w[set - S]);
            T* dstp = sm + (size_t)sf * H;
            for (int a = threadIdx.x; a < H; a += blockDim.x) async_copy(dstp + a, src + chunk(o, a));
        }
        async_wait_all();
        __syncthreads();
        // 2. reconstruct each set; buffers rotate: a set's input buffer is
        //    free once its reconstruction is done
        int nod[NSETS];
        int freeb[2] = {NSETS, NSETS + 1};
#pragma unroll
        for (int set = 0; set < NSETS; ++set) {
            T* r = reconstruct<T, KP1, P>(buf(set), buf(freeb[0]), buf(freeb[1]), H, N, F);
            const int ri = (int)((r - sm) / fb);
            nod[set] = ri;
            if (ri == freeb[0]) freeb[0] = set;
            else if (ri == freeb[1]) freeb[1] = set;
        }
        // 3. cell quadrature, one thread per finest cell along the pencil;
        //    moments go to the input buffers of the u sets (all consumed)
        int mom[S];
#pragma unroll
        for (int s = 0; s < S; ++s) mom[s] = -1;
        {
            int used = 0;
            for (int i = 0; i < NBUF && used < S; ++i) {
                bool busy = false;
#pragma unroll
                for (int set = 0; set < NSETS; ++set) busy |= (nod[set] == i);
                if (!busy) mom[used++] = i;
            }
        }
        const int ncell = H / KP1;
        for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
            T Cu[S][NC], Cw[S][NC], M[S][NC];
#pragma unroll
            for (int s = 0; s < S; ++s)
#pragma unroll
                for (int i = 0; i < NC; ++i) {
                    const int f = i / KP1, r = i % KP1;
                    Cu[s][i] = buf(nod[s])[f * H + c * KP1 + r];
                    Cw[s][i] = JAC ? buf(nod[S + s])[f * H + c * KP1 + r] : T(0);
                    M[s][i] = T(0);
                }
            Quad<T, D, KP1, Q, S, JAC, 0>::run(tb, poly, Cu, Cw, M, T(1));
#pragma unroll
            for (int s = 0; s < S; ++s)
#pragma unroll
                for (int i = 0; i < NC; ++i) {
                    const int f = i / KP1, r = i % KP1;
                    buf(mom[s])[f * H + c * KP1 + r] = M[s][i];
                }
        }
        __syncthreads();
        // 4. decompose each species' moments (nodal buffers are free now)
#pragma unroll
        for (int s = 0; s < S; ++s) {
            int sc = -1, rs = -1;
            for (int i = 0; i < NBUF; ++i) {
                bool busy = false;
#pragma unroll
                for (int t = 0; t < S; ++t) busy |= (mom[t] == i);
                if (busy) continue;
                if (sc < 0) sc = i;
                else if (rs < 0) rs = i;
            }
            decompose<T, KP1, P>(buf(mom[s]), buf(sc), buf(rs), H, N, F);
            // 5. store
            T* dst = reinterpret_cast<T*>(args.out[s]);
            const T* res = buf(rs);
#pragma unroll 1
            for (int f = 0; f < P; ++f) {
                const long long o = fiber_offset(f);
                const T* rp = res + (size_t)f * H;
                for (int a = threadIdx.x; a < H; a += blockDim.x) dst[chunk(o, a)] = rp[a];
            }
            __syncthreads();
        }
    }
}

template <typename T, int D, int KP1, int Q, int S, bool JAC>
void launch_one(sgk_ctx* ctx, const PencilArgs& a, const QuadTab<T>& tb, const double* two_scale,
                const ReactionDev& rxd) {
    Filt<T, KP1> F{};
    for (int h = 0; h < 2; ++h)
        for (int r = 0; r < KP1; ++r)
            for (int s = 0; s < KP1; ++s) {
                F.H[h][r][s] = (T)two_scale[h * KP1 * KP1 + r * KP1 + s];
                F.G[h][r][s] = (T)two_scale[(2 + h) * KP1 * KP1 + r * KP1 + s];
            }
    Poly<T, S> poly{};
    for (int m = 0; m < rxd.nmono; ++m) {
        int idx = 0;
        for (int r = 0; r < S; ++r) idx = idx * PDEG + rxd.exps[m][r];
        poly.c[rxd.species[m]][idx] += (T)rxd.coef[m];
    }
    constexpr int P = Pow<KP1, D - 1>::v;
    constexpr int NBUF = (JAC ? 2 * S : S) + 2;
    const size_t smem = (size_t)NBUF * P * a.H * sizeof(T);
    SGK_REQUIRE(smem <= ctx->smem_optin, SGK_EUNSUPPORTED, "pencil exceeds shared memory");
    const int threads = std::min(256, std::max(64, a.H / KP1));
    const int grid = (int)std::min<long long>(a.npencils, (long long)ctx->num_sms * 16);
    auto kern = pencil_kernel<T, D, KP1, Q, S, JAC>;
    allow_max_dynamic_smem(ctx->smem_optin, kern);
    kern<<<grid, threads, smem, ctx->stream>>>(a, tb, F, poly);
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

#define SGK_PENCIL_SHAPES(X) \
    X(3, 3, 5, 1)            \
    X(2, 3, 5, 2)            \
    X(2, 2, 3, 1)            \
    X(2, 2, 3, 2)            \
    X(3, 2, 3, 1)            \
    X(2, 3, 5, 1)            \
    X(4, 2, 3, 1)

template <typename T, bool JAC>
bool dispatch(sgk_ctx* ctx, int d, int kp1, int q, int S, const PencilArgs& a, const QuadTab<T>& tb,
              const double* two_scale, const ReactionDev& rx) {
#define SGK_PENCIL(DD, KK, QQ, SS)                                     \
    if (d == DD && kp1 == KK && q == QQ && S == SS) {                  \
        launch_one<T, DD, KK, QQ, SS, JAC>(ctx, a, tb, two_scale, rx); \
        return true;                                                   \
    }
    SGK_PENCIL_SHAPES(SGK_PENCIL)
#undef SGK_PENCIL
    return false;
}

}  // namespace

bool pencil_supported(int d, int kp1, int q, int S, const ReactionDev& rx) {
    for (int m = 0; m < rx.nmono; ++m)
        for (int r = 0; r < S; ++r)
            if (rx.exps[m][r] >= PDEG) return false;
#define SGK_PENCIL_OK(DD, KK, QQ, SS) \
    if (d == DD && kp1 == KK && q == QQ && S == SS) return true;
    SGK_PENCIL_SHAPES(SGK_PENCIL_OK)
#undef SGK_PENCIL_OK
    return false;
}

template <typename T>
void pencil_launch(sgk_ctx* ctx, const PencilArgs& a, int d, int kp1, int q, int S, bool jac, const double* B,
                   const double* w, const double* two_scale, const ReactionDev& rx) {
    const QuadTab<T> tb = make_tab<T>(B, w, q, kp1);
    KTimer kt(ctx, KC_CELL);
    const bool ok = jac ? dispatch<T, true>(ctx, d, kp1, q, S, a, tb, two_scale, rx)
                        : dispatch<T, false>(ctx, d, kp1, q, S, a, tb, two_scale, rx);
    SGK_REQUIRE(ok, SGK_EUNSUPPORTED, "no fused pencil kernel for this shape");
    check_launch("pencil_kernel");
    count_launch(ctx);
}

template void pencil_launch<double>(sgk_ctx*, const PencilArgs&, int, int, int, int, bool, const double*,
                                    const double*, const double*, const ReactionDev&);
template void pencil_launch<float>(sgk_ctx*, const PencilArgs&, int, int, int, int, bool, const double*,
                                   const double*, const double*, const ReactionDev&);
