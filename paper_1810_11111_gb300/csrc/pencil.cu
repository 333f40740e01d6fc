// Fused last-direction pass of the reaction term (Section 4: reconstruction
// at the finest-mesh Gauss points and quadrature).
//
// After directions 0..d-2 have been changed to the finest-cell Legendre basis
// (fiber engine), direction d-1 still holds 1D hierarchical coefficients.
// One CTA takes a pencil: a fixed finest cell in directions 0..d-2, i.e. the
// (k+1)^{d-1} fibers of that cell's Legendre degrees, each of length
// H = (k+1) 2^N along direction d-1.  In shared memory it
//   1. reconstructs each fiber in the finest-cell Legendre basis with the
//      two-scale relations (the children of a level-(n-1) cell get
//      H_h^T (parent coefficients) + G_h^T (level-n wavelet coefficients),
//      2 (k+1)^2 FMAs per child cell), one thread per subtree of up to 8
//      finest cells expanded in registers: one barrier per set;
//   2. runs the cell quadrature with one thread per finest cell of the
//      pencil: Legendre -> q^d Gauss points -> f(u) or f'(u) w times the
//      weights -> Legendre moments, as nested sum-factorised loops whose
//      indices are compile-time constants; f and f' are dense polynomials
//      evaluated by Horner's rule;
//   3. decomposes the moments back to hierarchical coefficients with the
//      transposed two-scale relations (subtrees of up to 3 levels reduced in
//      registers, one barrier per 3 levels) and stores them.
// Specialised for (d, k+1, q, species); other shapes use the unfused path.
#include <algorithm>
#include <type_traits>

#include "sgk_dfloat.h"
#include "sgk_pencil.h"

namespace {

template <typename T>
__device__ __forceinline__ void volatile_write(T* p, const T& v) {
    *reinterpret_cast<volatile T*>(p) = v;
}
template <>
__device__ __forceinline__ void volatile_write<dfloat>(dfloat* p, const dfloat& v) {
    volatile float* f = reinterpret_cast<volatile float*>(p);
    f[0] = v.hi;
    f[1] = v.lo;
}

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

template <typename T>
__device__ __forceinline__ bool is_zero(const T& v) {
    return v == T(0);
}
template <>
__device__ __forceinline__ bool is_zero<dfloat>(const dfloat& v) {
    return v.hi == 0.0f && v.lo == 0.0f;
}

// Horner's rule that skips the zero coefficients (the reactions are sparse
// polynomials, e.g. -c u^3): the tests are on kernel parameters, uniform
// over the grid, and adding an exact zero is exact, so the value is bitwise
// that of the dense rule
template <typename T>
__device__ __forceinline__ T horner_sparse(const T (&c)[PDEG], const T& u) {
    T f = T(0);
    bool started = false;
#pragma unroll
    for (int e = PDEG - 1; e >= 0; --e) {
        if (started) f = f * u;
        if (!is_zero(c[e])) {
            f = started ? f + c[e] : c[e];
            started = true;
        }
    }
    return f;
}

template <typename T, bool JAC>
struct PointEval<T, 1, JAC> {
    __device__ __forceinline__ static void run(const Poly<T, 1>& P, const T (&u)[1], const T (&w)[1], T (&o)[1]) {
        if (!JAC) {
            o[0] = horner_sparse<T>(P.c[0], u[0]);
        } else {
            // f'(u) = sum_{e >= 1} e c_e u^{e-1}
            T dc[PDEG];
#pragma unroll
            for (int e = 0; e + 1 < PDEG; ++e) dc[e] = T(e + 1) * P.c[0][e + 1];
            dc[PDEG - 1] = T(0);
            o[0] = horner_sparse<T>(dc, u[0]) * w[0];
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
    // compile-time operands; the outer levels stay loops.  In double-float
    // the unrolled code outgrows the instruction cache (fetch stalls led the
    // profile), so that level stays a loop too: measured 0.66 against
    // 0.76 ms per F pass at level 6 together with the register cap below
    static constexpr int UNROLL = (DIM == D - 1 && !std::is_same<T, dfloat>::value) ? Q : 1;
    // The Gauss points are symmetric about the cell centre and P_r(-x) =
    // (-1)^r P_r(x), so the table rows of points g and Q-1-g differ only in
    // the sign of the odd degrees (and the weights agree): the values at
    // both points come from the even and odd partial sums, E + O and E - O,
    // and their moments from the sum and difference of the two points' inner
    // results.  That halves the multiply-adds of both transforms on the inner
    // levels, whose partial sums are short enough (NS <= k+1) to keep the
    // second point's inputs live while the first point recurses; the middle
    // point of an odd rule (x = 0) has only even degrees.  Used for FP32
    // (the Jacobian passes: 0.177 against 0.182 ms at level 6); the
    // double-float pass, bound by issue latency rather than arithmetic,
    // measured 1-3% slower with it
    static constexpr bool SYM = NS <= KP1 && std::is_same<T, float>::value;
    __device__ __forceinline__ static void run(const QuadTab<T>& tb, const Poly<T, S>& P, const T (&Cu)[S][N],
                                               const T (&Cw)[S][N], T (&M)[S][N], T wt) {
        if constexpr (SYM)
            run_sym(tb, P, Cu, Cw, M, wt);
        else
            run_plain(tb, P, Cu, Cw, M, wt);
    }
    __device__ __forceinline__ static void run_sym(const QuadTab<T>& tb, const Poly<T, S>& P, const T (&Cu)[S][N],
                                                   const T (&Cw)[S][N], T (&M)[S][N], T wt) {
        constexpr int PAIRS = Q / 2;
#pragma unroll(UNROLL > 1 ? PAIRS : 1)
        for (int g = 0; g < PAIRS; ++g) {
            T ua[S][NS], ub[S][NS], wa[S][NS], wb[S][NS], ma[S][NS], mb[S][NS];
#pragma unroll
            for (int s = 0; s < S; ++s)
#pragma unroll
                for (int i = 0; i < NS; ++i) {
                    T e = T(0), o = T(0), ew = T(0), ow = T(0);
#pragma unroll
                    for (int r = 0; r < KP1; ++r) {
                        if (r & 1) {
                            o += tb.B[g][r] * Cu[s][r * NS + i];
                            if (JAC) ow += tb.B[g][r] * Cw[s][r * NS + i];
                        } else {
                            e += tb.B[g][r] * Cu[s][r * NS + i];
                            if (JAC) ew += tb.B[g][r] * Cw[s][r * NS + i];
                        }
                    }
                    ua[s][i] = e + o;
                    ub[s][i] = e - o;
                    wa[s][i] = ew + ow;
                    wb[s][i] = ew - ow;
                    ma[s][i] = T(0);
                    mb[s][i] = T(0);
                }
            const T wg = wt * tb.w[g];
            Quad<T, D, KP1, Q, S, JAC, DIM + 1>::run(tb, P, ua, wa, ma, wg);
            Quad<T, D, KP1, Q, S, JAC, DIM + 1>::run(tb, P, ub, wb, mb, wg);
#pragma unroll
            for (int s = 0; s < S; ++s)
#pragma unroll
                for (int i = 0; i < NS; ++i) {
                    const T sp = ma[s][i] + mb[s][i], sd = ma[s][i] - mb[s][i];
#pragma unroll
                    for (int r = 0; r < KP1; ++r) M[s][r * NS + i] += tb.B[g][r] * ((r & 1) ? sd : sp);
                }
        }
        if constexpr (Q & 1) {
            constexpr int g = Q / 2;
            T u[S][NS], w[S][NS], m[S][NS];
#pragma unroll
            for (int s = 0; s < S; ++s)
#pragma unroll
                for (int i = 0; i < NS; ++i) {
                    T e = T(0), ew = T(0);
#pragma unroll
                    for (int r = 0; r < KP1; r += 2) {
                        e += tb.B[g][r] * Cu[s][r * NS + i];
                        if (JAC) ew += tb.B[g][r] * Cw[s][r * NS + i];
                    }
                    u[s][i] = e;
                    w[s][i] = ew;
                    m[s][i] = T(0);
                }
            Quad<T, D, KP1, Q, S, JAC, DIM + 1>::run(tb, P, u, w, m, wt * tb.w[g]);
#pragma unroll
            for (int s = 0; s < S; ++s)
#pragma unroll
                for (int r = 0; r < KP1; r += 2)
#pragma unroll
                    for (int i = 0; i < NS; ++i) M[s][r * NS + i] += tb.B[g][r] * m[s][i];
        }
    }
    __device__ __forceinline__ static void run_plain(const QuadTab<T>& tb, const Poly<T, S>& P, const T (&Cu)[S][N],
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

// Outermost quadrature level with the cell's coefficients read from shared
// memory (coefficient e = f (k+1) + r of the cell at pu[r PS + f]: fiber f,
// position r along the pencil) instead of registers, which keeps only the
// moments and the inner levels' partial sums live.
template <typename T, int D, int KP1, int Q, int S, bool JAC, int PS>
struct QuadTop {
    static constexpr int NC = Pow<KP1, D>::v;
    static constexpr int NS = NC / KP1;
    // volatile: re-read at every Gauss point (hoisting the loads out of the
    // loop would hold all of them in registers again)
    __device__ __forceinline__ static T at(const T* p, int e) {
        return volatile_read(p + (e % KP1) * PS + e / KP1);
    }
    __device__ __forceinline__ static void run(const QuadTab<T>& tb, const Poly<T, S>& P, const T* const (&pu)[S],
                                               const T* const (&pw)[S], T (&M)[S][NC]) {
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
                        a += tb.B[g][r] * at(pu[s], r * NS + i);
                        if (JAC) b += tb.B[g][r] * at(pw[s], r * NS + i);
                    }
                    su[s][i] = a;
                    sw[s][i] = b;
                    sm[s][i] = T(0);
                }
            Quad<T, D, KP1, Q, S, JAC, 1>::run(tb, P, su, sw, sm, tb.w[g]);
#pragma unroll
            for (int s = 0; s < S; ++s)
#pragma unroll
                for (int r = 0; r < KP1; ++r)
#pragma unroll
                    for (int i = 0; i < NS; ++i) M[s][r * NS + i] += tb.B[g][r] * sm[s][i];
        }
    }
    // The same with the moments of one species accumulated in shared memory
    // (moment e of the cell at ms[e * mstride]) instead of registers: the
    // NC accumulators then hold no registers across the inner levels, which
    // is what makes the double-float pass spill at its register cap
    __device__ __forceinline__ static void run_shared(const QuadTab<T>& tb, const Poly<T, S>& P,
                                                      const T* const (&pu)[S], const T* const (&pw)[S], T* ms,
                                                      int mstride) {
        static_assert(S == 1, "shared moments: one species");
#pragma unroll
        for (int e = 0; e < NC; ++e) volatile_write(ms + e * mstride, T(0));
#pragma unroll 1
        for (int g = 0; g < Q; ++g) {
            T su[S][NS], sw[S][NS], sm[S][NS];
#pragma unroll
            for (int i = 0; i < NS; ++i) {
                T a = T(0), b = T(0);
#pragma unroll
                for (int r = 0; r < KP1; ++r) {
                    a += tb.B[g][r] * at(pu[0], r * NS + i);
                    if (JAC) b += tb.B[g][r] * at(pw[0], r * NS + i);
                }
                su[0][i] = a;
                sw[0][i] = b;
                sm[0][i] = T(0);
            }
            Quad<T, D, KP1, Q, S, JAC, 1>::run(tb, P, su, sw, sm, tb.w[g]);
#pragma unroll
            for (int r = 0; r < KP1; ++r)
#pragma unroll
                for (int i = 0; i < NS; ++i) {
                    T* p = ms + (r * NS + i) * mstride;
                    volatile_write(p, volatile_read(p) + tb.B[g][r] * sm[0][i]);
                }
        }
    }
};

// Two-scale pyramids on register subtrees.  In shared memory a buffer holds
// the P fibers of one set interleaved, position pos of fiber f at
// pos PS + f (PS = P rounded up to odd: threads on consecutive fibers, or
// on consecutive cells of one fiber, hit distinct banks).
constexpr int PD = 3;  // levels of a subtree expanded or reduced in registers

// Forward (hierarchical levels 0..N in X -> finest-cell Legendre
// coefficients in Y) for the subtree of 2^De finest cells under node j of
// level t = N - De of fiber f: walks the t ancestors of that node from the
// level-0 coefficients, then expands the subtree, children over consumed
// parents.
template <typename T, int KP1, int PS>
__device__ __forceinline__ void fwd_subtree(const T* X, T* Y, int f, int j, int t, int De, const Filt<T, KP1>& F) {
    T cell[1 << PD][KP1];
#pragma unroll
    for (int r = 0; r < KP1; ++r) cell[0][r] = X[r * PS + f];
    for (int n = 1; n <= t; ++n) {
        const int an = j >> (t - n), h = an & 1, par = an >> 1;
        T d[KP1], q[KP1];
#pragma unroll
        for (int r = 0; r < KP1; ++r) d[r] = X[((KP1 << (n - 1)) + par * KP1 + r) * PS + f];
#pragma unroll
        for (int s2 = 0; s2 < KP1; ++s2) {
            T acc = T(0);
#pragma unroll
            for (int r = 0; r < KP1; ++r) {
                // select, not index: a runtime index would put the filters
                // in local memory
                const T hf = h ? F.H[1][r][s2] : F.H[0][r][s2];
                const T gf = h ? F.G[1][r][s2] : F.G[0][r][s2];
                acc += hf * cell[0][r] + gf * d[r];
            }
            q[s2] = acc;
        }
#pragma unroll
        for (int r = 0; r < KP1; ++r) cell[0][r] = q[r];
    }
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
                    d[r] = X[((KP1 << (n - 1)) + par * KP1 + r) * PS + f];
                }
#pragma unroll
                for (int h = 0; h < 2; ++h)
#pragma unroll
                    for (int s2 = 0; s2 < KP1; ++s2) {
                        T acc = T(0);
#pragma unroll
                        for (int r = 0; r < KP1; ++r) acc += F.H[h][r][s2] * p[r] + F.G[h][r][s2] * d[r];
                        cell[2 * i + h][s2] = acc;
                    }
            }
        }
    }
#pragma unroll
    for (int i = 0; i < (1 << PD); ++i)
        if (i < (1 << De))
#pragma unroll
            for (int s2 = 0; s2 < KP1; ++s2) Y[(((j << De) + i) * KP1 + s2) * PS + f] = cell[i][s2];
}

// Transposed step for subtree j of fiber f: its 2^De nodes of level Lhi,
// node m stored at position m stride of Mb (stride = (k+1) 2^{N - Lhi};
// the finest cells are contiguous), reduced over De levels; the details of
// levels Lhi - De + 1 .. Lhi go to Y (hierarchical layout) and the root
// (level Lhi - De) in place over the first node, or to Y when it is level 0.
template <typename T, int KP1, int PS>
__device__ __forceinline__ void bwd_subtree(T* Mb, T* Y, int f, int j, int Lhi, int De, int stride,
                                            const Filt<T, KP1>& F) {
    T cell[1 << PD][KP1];
#pragma unroll
    for (int i = 0; i < (1 << PD); ++i)
        if (i < (1 << De))
#pragma unroll
            for (int s2 = 0; s2 < KP1; ++s2) cell[i][s2] = Mb[(((j << De) + i) * stride + s2) * PS + f];
#pragma unroll
    for (int l = PD - 1; l >= 0; --l) {
        if (l < De) {
            const int n = Lhi - De + l + 1;  // level of the children
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
                        sp += F.H[0][r][s2] * x0[s2] + F.H[1][r][s2] * x1[s2];
                        sd += F.G[0][r][s2] * x0[s2] + F.G[1][r][s2] * x1[s2];
                    }
                    cell[i][r] = sp;
                    Y[((KP1 << (n - 1)) + par * KP1 + r) * PS + f] = sd;
                }
            }
        }
    }
    const bool top = Lhi == De;
#pragma unroll
    for (int r = 0; r < KP1; ++r) {
        if (top) Y[r * PS + f] = cell[0][r];
        else Mb[((j << De) * stride + r) * PS + f] = cell[0][r];
    }
}

// Register limit per element type: 128 for FP32 (eight 64-thread CTAs per
// SM, no spills; a 96-register cap with spills measured slower), the
// architectural 255 for FP64 (its cell loops need them), and 128 for
// double-float (eight CTAs per SM, as many as shared memory allows; a few
// spills, but 128, 144, 168, 192 and 216 measured 0.66, 0.68, 0.68, 0.72
// and 0.73 ms per F pass at level 6).
template <typename T, int D, int KP1, int Q, int S, bool JAC>
__global__ void __maxnreg__((sizeof(T) == 4 || std::is_same<T, dfloat>::value) ? 128 : 255)
    pencil_kernel(const PencilArgs args, const QuadTab<T> tb, const Filt<T, KP1> F, const Poly<T, S> poly) {
    constexpr int P = Pow<KP1, D - 1>::v;  // fibers per species and set
    constexpr int PS = P | 1;              // odd fiber stride in shared memory
    constexpr int NC = Pow<KP1, D>::v;     // coefficients per cell
    constexpr int NSETS = JAC ? 2 * S : S;
    // double-float, one species: the moments live in shared memory (the
    // pass then does not spill at its register cap: 0.651 against 0.661 ms
    // per F evaluation at level 6, bitwise the same sums)
    constexpr bool SHARED_MOMENTS = std::is_same<T, dfloat>::value && S == 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ long long s_of[P];
    T* sm = reinterpret_cast<T*>(smem_raw);
    const int H = args.H, N = args.N;
    const int bs = H * PS;  // one buffer: the P fibers of one set
    auto buf = [&](int i) { return sm + (size_t)i * bs; };
    const int De = N < PD ? N : PD;  // levels of a forward subtree
    const int t = N - De;            // level of the forward subtree roots
    for (long long pen = blockIdx.x; pen < args.npencils; pen += gridDim.x) {
        // source offset of every fiber: o_f = obase + sum_m r_m H^{d-2-m}
        if ((int)threadIdx.x < P) {
            long long o = 0, rem = pen, mul = 1;
            for (int m = D - 2; m >= 0; --m) {
                const long long c = rem % args.ncell1;
                rem /= args.ncell1;
                o += c * KP1 * mul;
                mul *= H;
            }
            int rr = threadIdx.x;
            mul = 1;
            for (int m = D - 2; m >= 0; --m) {
                o += (rr % KP1) * mul;
                rr /= KP1;
                mul *= H;
            }
            s_of[threadIdx.x] = o;
        }
        __syncthreads();
        // 1. load every set's hierarchical fibers into buffers 0..NSETS-1.
        //    Position a of fiber offset o lives in the level-l chunk at
        //    cbase[l] + o nl + (a - off); l, nl and a - off depend on a only
        for (int a = threadIdx.x; a < H; a += blockDim.x) {
            const int q = a / KP1;
            const int l = q == 0 ? 0 : 32 - __clz(q);
            const int off = l ? (KP1 << (l - 1)) : 0;
            const long long nl = l ? (KP1 << (l - 1)) : KP1;
            const long long base = args.cbase[l] + (a - off);
#pragma unroll
            for (int set = 0; set < NSETS; ++set) {
                const T* src = reinterpret_cast<const T*>(set < S ? args.u[set] : args.w[set - S]) + base;
                T* dst = buf(set) + a * PS;
#pragma unroll
                for (int f = 0; f < P; ++f) async_copy(dst + f, src + s_of[f] * nl);
            }
        }
        async_wait_all();
        __syncthreads();
        // 2. forward pyramids, one set after the other: set 0 into the spare
        //    buffer NSETS, set k >= 1 into buffer k-1 (freed by set k-1)
        const int units = P << t;
#pragma unroll 1
        for (int set = 0; set < NSETS; ++set) {
            const T* X = buf(set);
            T* Y = buf(set == 0 ? NSETS : set - 1);
            for (int u = threadIdx.x; u < units; u += blockDim.x)
                fwd_subtree<T, KP1, PS>(X, Y, u % P, u / P, t, De, F);
            __syncthreads();
        }
        // nodal buffer of set k: NSETS for k = 0, k - 1 otherwise; buffer
        // NSETS - 1 is free
        // 3. cell quadrature, one thread per finest cell along the pencil;
        //    the moments of species s overwrite its nodal u values (each
        //    thread reads and writes only its own cell)
        const int ncell = H / KP1;
        for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
            const T* pu[S];
            const T* pw[S];
#pragma unroll
            for (int s = 0; s < S; ++s) {
                pu[s] = buf(s == 0 ? NSETS : s - 1) + c * KP1 * PS;
                pw[s] = JAC ? buf(S + s - 1) + c * KP1 * PS : pu[s];
            }
            if constexpr (SHARED_MOMENTS) {
                // moments in the free buffer NSETS - 1 (KP1 PS >= NC rows of
                // ncell), moment e of cell c at e ncell + c
                T* ms = buf(NSETS - 1) + c;
                QuadTop<T, D, KP1, Q, S, JAC, PS>::run_shared(tb, poly, pu, pw, ms, ncell);
                T* mo = const_cast<T*>(pu[0]);
#pragma unroll
                for (int i = 0; i < NC; ++i) mo[(i % KP1) * PS + i / KP1] = volatile_read(ms + i * ncell);
            } else {
                T M[S][NC];
#pragma unroll
                for (int s = 0; s < S; ++s)
#pragma unroll
                    for (int i = 0; i < NC; ++i) M[s][i] = T(0);
                QuadTop<T, D, KP1, Q, S, JAC, PS>::run(tb, poly, pu, pw, M);
#pragma unroll
                for (int s = 0; s < S; ++s) {
                    T* mo = const_cast<T*>(pu[s]);
#pragma unroll
                    for (int i = 0; i < NC; ++i) mo[(i % KP1) * PS + i / KP1] = M[s][i];
                }
            }
        }
        __syncthreads();
        // 4. per species: backward pyramid (stages of up to PD levels, roots
        //    kept in place between them) into the free buffer, then store
        T* Y = buf(NSETS - 1);
#pragma unroll 1
        for (int s = 0; s < S; ++s) {
            T* Mb = buf(s == 0 ? NSETS : s - 1);
            for (int Lhi = N; Lhi > 0;) {
                const int de = Lhi < PD ? Lhi : PD;
                const int nu = P << (Lhi - de), stride = KP1 << (N - Lhi);
                for (int u = threadIdx.x; u < nu; u += blockDim.x)
                    bwd_subtree<T, KP1, PS>(Mb, Y, u % P, u / P, Lhi, de, stride, F);
                __syncthreads();
                Lhi -= de;
            }
            if (N == 0) {  // one cell: the moments are the coefficients
                for (int u = threadIdx.x; u < KP1 * PS; u += blockDim.x) Y[u] = Mb[u];
                __syncthreads();
            }
            T* dst = reinterpret_cast<T*>(args.out[s]);
            for (int a = threadIdx.x; a < H; a += blockDim.x) {
                const int q = a / KP1;
                const int l = q == 0 ? 0 : 32 - __clz(q);
                const int off = l ? (KP1 << (l - 1)) : 0;
                const long long nl = l ? (KP1 << (l - 1)) : KP1;
                T* d0 = dst + args.cbase[l] + (a - off);
                const T* y = Y + a * PS;
#pragma unroll
                for (int f = 0; f < P; ++f) d0[s_of[f] * nl] = y[f];
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
    double pc[S][Pow<PDEG, S>::v] = {};
    for (int m = 0; m < rxd.nmono; ++m) {
        int idx = 0;
        for (int r = 0; r < S; ++r) idx = idx * PDEG + rxd.exps[m][r];
        pc[rxd.species[m]][idx] += rxd.coef[m];
    }
    Poly<T, S> poly{};
    for (int sp = 0; sp < S; ++sp)
        for (int i = 0; i < Pow<PDEG, S>::v; ++i) poly.c[sp][i] = (T)pc[sp][i];
    constexpr int P = Pow<KP1, D - 1>::v;
    constexpr int NBUF = (JAC ? 2 * S : S) + 1;
    const size_t smem = (size_t)NBUF * (P | 1) * a.H * sizeof(T);
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
    bool ok = false;
    if constexpr (std::is_same<T, dfloat>::value) {
        // double-float serves the F passes only (Jacobian products stay FP32)
        SGK_REQUIRE(!jac, SGK_EUNSUPPORTED, "no double-float Jacobian pencil");
        ok = dispatch<T, false>(ctx, d, kp1, q, S, a, tb, two_scale, rx);
    } else {
        ok = jac ? dispatch<T, true>(ctx, d, kp1, q, S, a, tb, two_scale, rx)
                 : dispatch<T, false>(ctx, d, kp1, q, S, a, tb, two_scale, rx);
    }
    SGK_REQUIRE(ok, SGK_EUNSUPPORTED, "no fused pencil kernel for this shape");
    check_launch("pencil_kernel");
    count_launch(ctx);
}

template void pencil_launch<double>(sgk_ctx*, const PencilArgs&, int, int, int, int, bool, const double*,
                                    const double*, const double*, const ReactionDev&);
template void pencil_launch<float>(sgk_ctx*, const PencilArgs&, int, int, int, int, bool, const double*,
                                   const double*, const double*, const ReactionDev&);
template void pencil_launch<dfloat>(sgk_ctx*, const PencilArgs&, int, int, int, int, bool, const double*,
                                    const double*, const double*, const ReactionDev&);
