// Sparse-grid interpolation form of the reaction term, on the device.
//
// Not the paper's F: the paper projects f(u_h) at the Gauss points of the
// finest full grid (Section 4); its first stated future direction (Section 5)
// is an evaluation that uses the structure of the basis instead.  This form
// takes F_I(U) = the Alpert coefficients of the sparse-grid interpolant of
// f(u_h) on nested collocation points (one point per coefficient; the 1D
// factors and their definitions are in tables.cpp):
//
//   u at the points = C U,  C = (B along every direction)(A along every direction),
//   F_I(U)         = C^{-1} f(C U),  C^{-1} = (A^{-1} ...)(B^{-1} ...).
//
// Each 1D factor maps every level to the same or coarser levels only (A,
// A^{-1}) or to the same or finer ones only (B, B^{-1}), so on the sparse
// index set (closed under lowering a level) its application along one
// direction is exact fiber by fiber with each fiber truncated to its own
// highest level -- the unidirectional principle of Section 4.  sgt_kernel
// applies one factor along one direction as a gather: every output
// coefficient walks its truncated CSR row, like one direction of the
// diffusion matvec, with the same block-offset tables.  Work per F: 4d
// passes of at most a few tens of multiply-adds per coefficient, no finest
// full grid.
//
// In point values the implicit stage U - c (F_I(U) + S) = W decouples into
// one small equation per collocation point, u - c f(u) = (C (W + c S))_p,
// solved by Newton's method at each point (interp_newton_kernel); then
// U = C^{-1} u and F_I(U) = C^{-1} f(u) in one pass over both vector sets.
// The transforms and the point kernels run in FP64 in both precision modes.
#include <algorithm>
#include <cmath>

#include "sgk_solver.h"

namespace {

struct SgtArgs {
    int64_t n;
    int N;
    const int64_t* __restrict__ offsets;
    const int32_t* __restrict__ levels;
    const int32_t* __restrict__ chunk;
    const int64_t* __restrict__ cb;
    const int32_t* __restrict__ rp;
    const int32_t* __restrict__ rlen;
    const int32_t* __restrict__ ce;
    const double* __restrict__ val;
};

// y = (I x .. x T x .. x I) x along direction dir on the sparse set, for
// nvec vectors stacked with stride ld; output vector v goes to y + v ld for
// v < nsplit and to y2 + (v - nsplit) ld otherwise.  G consecutive lanes
// share one output (G divides 32): lane r takes the row entries r, r + G, ...
// in two chains, four loads issued before their multiply-adds, and the G
// partial sums are added by XOR shuffles in a fixed order.  G > 1 shortens
// the longest rows' dependent chains (the level-0 rows of A and A^{-1} walk
// the whole fiber), which bound a launch on small index sets; G = 1 keeps
// the per-output decoding cheapest where the FP64 pipe is the bound.
template <int D, int KP1, int G>
__global__ void __launch_bounds__(256) sgt_kernel(SgtArgs a, int dir, int nvec, int64_t ld,
                                                  const double* __restrict__ x, double* __restrict__ y,
                                                  double* __restrict__ y2, int nsplit) {
    // 32-bit index arithmetic: the index set has at most 2^30 coefficients
    // (checked when the tables are built)
    const int g = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G);
    const int r = (int)(threadIdx.x & (G - 1));
    const bool live = g < a.n;
    if (G == 1 && !live) return;
    int q0 = 0, qe = 0;
    const int64_t* __restrict__ base = a.cb;
    int oI = 0, in = 0, I = 1;
    if (live) {
        int lo = a.chunk[g >> 8], hi = a.chunk[(g >> 8) + 1];
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (a.offsets[mid] <= g) lo = mid;
            else hi = mid - 1;
        }
        const int t = lo;
        int e = g - (int)a.offsets[t];
        int lv[D], sh[D], cnt[D], c[D];
        int sum = 0;
#pragma unroll
        for (int m = 0; m < D; ++m) {
            lv[m] = a.levels[t * D + m];
            sum += lv[m];
            sh[m] = lv[m] > 0 ? lv[m] - 1 : 0;
            cnt[m] = KP1 << sh[m];
        }
#pragma unroll
        for (int m = D - 1; m >= 0; --m) {
            const int q = (e >> sh[m]) / KP1;
            c[m] = e - q * cnt[m];
            e = q;
        }
        int o = 0, cd = 0, ldir = 0;
#pragma unroll
        for (int m = 0; m < D; ++m) {
            if (m < dir) o = o * cnt[m] + c[m];
            if (m == dir) {
                cd = c[m];
                ldir = lv[m];
            }
        }
#pragma unroll
        for (int m = D - 1; m >= 0; --m)
            if (m > dir) {
                in += c[m] * I;
                I *= cnt[m];
            }
        const int nl = a.N + 1;
        const int np = a.N - (sum - ldir);
        const int ai = (ldir ? (KP1 << (ldir - 1)) : 0) + cd;
        q0 = a.rp[ai];
        qe = q0 + a.rlen[ai * nl + np];
        base = a.cb + ((int64_t)t * D + dir) * nl;
        oI = o * I * KP1;
    }
    // index of the source coefficient of a packed (level, position) entry
    auto src = [&](int pk) {
        const int lb = pk >> 16;
        return (int)base[lb] + (lb ? (oI << (lb - 1)) : oI) + (pk & 0xffff) * I + in;
    };
    for (int v = 0; v < nvec; ++v) {
        const double* __restrict__ xv = x + v * ld;
        double s0 = 0.0, s1 = 0.0;
        int q = q0 + r;
        for (; q + 3 * G < qe; q += 4 * G) {
            const double x0 = xv[src(a.ce[q])], x1 = xv[src(a.ce[q + G])];
            const double x2 = xv[src(a.ce[q + 2 * G])], x3 = xv[src(a.ce[q + 3 * G])];
            s0 += a.val[q] * x0;
            s1 += a.val[q + G] * x1;
            s0 += a.val[q + 2 * G] * x2;
            s1 += a.val[q + 3 * G] * x3;
        }
        if (q + G < qe) {
            const double x0 = xv[src(a.ce[q])], x1 = xv[src(a.ce[q + G])];
            s0 += a.val[q] * x0;
            s1 += a.val[q + G] * x1;
            q += 2 * G;
        }
        if (q < qe) s0 += a.val[q] * xv[src(a.ce[q])];
        double t = s0 + s1;
#pragma unroll
        for (int o = 1; o < G; o <<= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (live && r == 0) {
            double* out = v < nsplit ? y + v * ld : y2 + (v - nsplit) * ld;
            out[g] = t;
        }
    }
}

// f_s(u) = sum over the species' monomials of coef prod_r u_r^e
__device__ __forceinline__ double ipow(double u, int e) {
    double r = 1.0;
    for (int i = 0; i < e; ++i) r *= u;
    return r;
}

__device__ __forceinline__ void react(const ReactionDev& rx, const double* u, double* f, double* J) {
    const int S = rx.nspecies;
    for (int s = 0; s < S; ++s) {
        f[s] = 0.0;
        if (J)
            for (int r = 0; r < S; ++r) J[s * SGK_MAX_SPECIES + r] = 0.0;
    }
    for (int m = 0; m < rx.nmono; ++m) {
        const int s = rx.species[m];
        double v = rx.coef[m];
        for (int r = 0; r < S; ++r) v *= ipow(u[r], rx.exps[m][r]);
        f[s] += v;
        if (J)
            for (int r = 0; r < S; ++r) {
                const int er = rx.exps[m][r];
                if (er == 0) continue;
                double dv = rx.coef[m] * er;
                for (int r2 = 0; r2 < S; ++r2) dv *= ipow(u[r2], r2 == r ? er - 1 : rx.exps[m][r2]);
                J[s * SGK_MAX_SPECIES + r] += dv;
            }
    }
}

// out = f(u) at every point (species stacked with stride n)
__global__ void interp_f_kernel(ReactionDev rx, const double* __restrict__ u, double* __restrict__ out, int64_t n) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    double uu[SGK_MAX_SPECIES], f[SGK_MAX_SPECIES];
    for (int s = 0; s < rx.nspecies; ++s) uu[s] = u[s * n + g];
    react(rx, uu, f, nullptr);
    for (int s = 0; s < rx.nspecies; ++s) out[s * n + g] = f[s];
}

// out = f'(u) w at every point
__global__ void interp_jac_kernel(ReactionDev rx, const double* __restrict__ u, const double* __restrict__ w,
                                  double* __restrict__ out, int64_t n) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    double uu[SGK_MAX_SPECIES], f[SGK_MAX_SPECIES], J[SGK_MAX_SPECIES * SGK_MAX_SPECIES];
    const int S = rx.nspecies;
    for (int s = 0; s < S; ++s) uu[s] = u[s * n + g];
    react(rx, uu, f, J);
    for (int s = 0; s < S; ++s) {
        double acc = 0.0;
        for (int r = 0; r < S; ++r) acc += J[s * SGK_MAX_SPECIES + r] * w[r * n + g];
        out[s * n + g] = acc;
    }
}

__global__ void interp_outcome_reset_kernel(int* status, int* iters) {
    *status = SGK_OK;
    *iters = 0;
}

// Per point: u - c f(u) = w by Newton's method from u = w, the S x S
// Jacobian I - c f'(u) solved by Gaussian elimination with partial
// pivoting.  A point has converged when a correction is at most 1e-14 of
// max(|u|, |w|) (sup norms over the species); one more correction follows
// (quadratic convergence takes it to rounding).  Writes u and f(u) into
// uf[0 .. S n) and uf[S n .. 2 S n).  A point that does not converge within
// max_iter corrections, or meets a singular or non-finite Jacobian, sets
// *status = SGK_ENEWTON; *iters receives the most corrections any point took.
__global__ void interp_newton_kernel(ReactionDev rx, double c, const double* __restrict__ w, double* __restrict__ uf,
                                     int64_t n, int max_iter, int* status, int* iters) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    const int S = rx.nspecies;
    double u[SGK_MAX_SPECIES], ww[SGK_MAX_SPECIES], f[SGK_MAX_SPECIES], J[SGK_MAX_SPECIES * SGK_MAX_SPECIES];
    double wmax = 0.0;
    for (int s = 0; s < S; ++s) {
        ww[s] = w[s * n + g];
        u[s] = ww[s];
        wmax = fmax(wmax, fabs(ww[s]));
    }
    int it = 0, extra = 0;
    bool ok = rx.nmono == 0;
    while (!ok && it < max_iter) {
        react(rx, u, f, J);
        double A[SGK_MAX_SPECIES][SGK_MAX_SPECIES + 1];
        for (int s = 0; s < S; ++s) {
            for (int r = 0; r < S; ++r) A[s][r] = (s == r ? 1.0 : 0.0) - c * J[s * SGK_MAX_SPECIES + r];
            A[s][S] = -(u[s] - c * f[s] - ww[s]);
        }
        bool singular = false;
        for (int col = 0; col < S; ++col) {
            int piv = col;
            for (int r = col + 1; r < S; ++r)
                if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
            if (!(fabs(A[piv][col]) > 0.0)) {
                singular = true;
                break;
            }
            if (piv != col)
                for (int r = 0; r <= S; ++r) {
                    const double tmp = A[col][r];
                    A[col][r] = A[piv][r];
                    A[piv][r] = tmp;
                }
            for (int r = col + 1; r < S; ++r) {
                const double m = A[r][col] / A[col][col];
                for (int q = col; q <= S; ++q) A[r][q] -= m * A[col][q];
            }
        }
        if (singular) break;
        double dmax = 0.0, umax = 0.0;
        for (int s = S - 1; s >= 0; --s) {
            double v = A[s][S];
            for (int r = s + 1; r < S; ++r) v -= A[s][r] * A[r][S];
            A[s][S] = v / A[s][s];
        }
        for (int s = 0; s < S; ++s) {
            u[s] += A[s][S];
            dmax = fmax(dmax, fabs(A[s][S]));
            umax = fmax(umax, fabs(u[s]));
        }
        ++it;
        if (!isfinite(dmax) || !isfinite(umax)) break;
        if (extra) {
            ok = true;
        } else if (dmax <= 1e-14 * fmax(umax, wmax)) {
            extra = 1;
            if (dmax == 0.0) ok = true;
        }
    }
    if (!ok) *status = SGK_ENEWTON;
    atomicMax(iters, it);
    react(rx, u, f, nullptr);
    for (int s = 0; s < S; ++s) {
        uf[s * n + g] = u[s];
        uf[(S + s) * n + g] = f[s];
    }
}

// largest index set whose transform passes use eight lanes per output
constexpr int64_t SGT_WIDE_MAX_N = int64_t(1) << 18;

SgtArgs sgt_args(const sgk_solver* s, int which) {
    const sgk_op* op = s->ops[0];
    const sgk_index* idx = s->idx;
    const InterpFactorDev& F = s->IP.f[which];
    SgtArgs a;
    a.n = idx->dof;
    a.N = idx->n;
    a.offsets = idx->d_offsets.p;
    a.levels = idx->d_levels.p;
    a.chunk = op->gmv_chunk.p;
    a.cb = op->gmv_cb.p;
    a.rp = F.rp.p;
    a.rlen = F.rlen.p;
    a.ce = F.ce.p;
    a.val = F.val.p;
    return a;
}

template <int D>
void launch_sgt_d(const sgk_solver* s, int which, int dir, int nvec, const double* x, double* y, double* y2,
                  int nsplit) {
    const SgtArgs a = sgt_args(s, which);
    cudaStream_t st = s->ctx->stream;
    // eight lanes per output on small index sets (latency-bound launches),
    // one on large ones (FP64-pipe-bound)
    const bool wide = a.n <= SGT_WIDE_MAX_N;
    const unsigned blocks = (unsigned)((a.n * (wide ? 8 : 1) + 255) / 256);
#define SGK_SGT(KP, GG) sgt_kernel<D, KP, GG><<<blocks, 256, 0, st>>>(a, dir, nvec, a.n, x, y, y2, nsplit)
    switch (s->idx->k + 1) {
        case 2: if (wide) SGK_SGT(2, 8); else SGK_SGT(2, 1); break;
        case 3: if (wide) SGK_SGT(3, 8); else SGK_SGT(3, 1); break;
        case 4: if (wide) SGK_SGT(4, 8); else SGK_SGT(4, 1); break;
        default: throw SgkError{SGK_EUNSUPPORTED, "interp: degree must be 1..3"};
    }
#undef SGK_SGT
}

void launch_sgt(sgk_solver* s, int which, int dir, int nvec, const double* x, double* y, double* y2, int nsplit) {
    switch (s->idx->d) {
        case 1: launch_sgt_d<1>(s, which, dir, nvec, x, y, y2, nsplit); break;
        case 2: launch_sgt_d<2>(s, which, dir, nvec, x, y, y2, nsplit); break;
        case 3: launch_sgt_d<3>(s, which, dir, nvec, x, y, y2, nsplit); break;
        case 4: launch_sgt_d<4>(s, which, dir, nvec, x, y, y2, nsplit); break;
        case 5: launch_sgt_d<5>(s, which, dir, nvec, x, y, y2, nsplit); break;
        case 6: launch_sgt_d<6>(s, which, dir, nvec, x, y, y2, nsplit); break;
        default: throw SgkError{SGK_EUNSUPPORTED, "interp: d must be 1..6"};
    }
    check_launch("sgt_kernel");
    count_launch(s->ctx);
}

// The 2d passes of C (first = A, second = B) or C^{-1} (first = B^{-1},
// second = A^{-1}) on nvec stacked vectors: x -> y (vectors v >= nsplit to
// y2), through the two scratch buffers.
void chain(sgk_solver* s, int first, int second, int nvec, const double* x, double* y, double* y2, int nsplit) {
    const int d = s->idx->d, npass = 2 * d;
    double* buf[2] = {s->IP.t0.p, s->IP.t1.p};
    const double* src = x;
    for (int ps = 0; ps < npass; ++ps) {
        const bool last = ps == npass - 1;
        double* dst = last ? y : buf[ps & 1];
        launch_sgt(s, ps < d ? first : second, ps % d, nvec, src, dst, last ? y2 : nullptr, last ? nsplit : nvec);
        src = dst;
    }
}

unsigned point_blocks(int64_t n) { return (unsigned)((n + 255) / 256); }

}  // namespace

enum { IF_A = 0, IF_B = 1, IF_BINV = 2, IF_AINV = 3 };

void interp_to_points(sgk_solver* s, const double* U, double* P, int nvec) {
    KTimer kt(s->ctx, KC_FWD);
    chain(s, IF_A, IF_B, nvec, U, P, nullptr, nvec);
}

void interp_from_points(sgk_solver* s, const double* P, double* U, int nvec, double* U2, int nsplit) {
    KTimer kt(s->ctx, KC_BWD);
    chain(s, IF_BINV, IF_AINV, nvec, P, U, U2, U2 ? nsplit : nvec);
}

void interp_evalF(sgk_solver* s, const double* U, double* F) {
    const int S = s->nspecies;
    const int64_t n = s->n;
    interp_to_points(s, U, s->IP.p0.p, S);
    {
        KTimer kt(s->ctx, KC_CELL);
        interp_f_kernel<<<point_blocks(n), 256, 0, s->ctx->stream>>>(s->rx, s->IP.p0.p, s->IP.p1.p, n);
        check_launch("interp_f_kernel");
        count_launch(s->ctx);
    }
    interp_from_points(s, s->IP.p1.p, F, S, nullptr, S);
}

void interp_evalJ(sgk_solver* s, const double* U, const double* w, double* jw) {
    const int S = s->nspecies;
    const int64_t n = s->n;
    interp_to_points(s, U, s->IP.p0.p, S);
    interp_to_points(s, w, s->IP.p1.p, S);
    {
        KTimer kt(s->ctx, KC_CELL);
        interp_jac_kernel<<<point_blocks(n), 256, 0, s->ctx->stream>>>(s->rx, s->IP.p0.p, s->IP.p1.p,
                                                                       s->IP.p1.p + (int64_t)S * n, n);
        check_launch("interp_jac_kernel");
        count_launch(s->ctx);
    }
    interp_from_points(s, s->IP.p1.p + (int64_t)S * n, jw, S, nullptr, S);
}

void interp_implicit(sgk_solver* s, const double* Wp, double c, double* U, double* Fr, int* status, int* iters) {
    const int S = s->nspecies;
    const int64_t n = s->n;
    interp_to_points(s, Wp, s->IP.p0.p, S);
    {
        KTimer kt(s->ctx, KC_CELL);
        interp_outcome_reset_kernel<<<1, 1, 0, s->ctx->stream>>>(status, iters);
        check_launch("interp_outcome_reset");
        count_launch(s->ctx);
        interp_newton_kernel<<<point_blocks(n), 256, 0, s->ctx->stream>>>(s->rx, c, s->IP.p0.p, s->IP.p1.p, n,
                                                                          s->opts.max_iter, status, iters);
        check_launch("interp_newton_kernel");
        count_launch(s->ctx);
    }
    interp_from_points(s, s->IP.p1.p, U, 2 * S, Fr, S);
}

// Host tables of the four factors (packed columns, truncated row lengths),
// every address checked against the 1D space, and the work buffers.
void interp_build(sgk_solver* s) {
    const sgk_index* idx = s->idx;
    const int N = idx->n, kp1 = idx->k + 1, nl = N + 1, H = kp1 << N;
    SGK_REQUIRE(idx->dof <= (int64_t(1) << 30), SGK_EUNSUPPORTED,
                "interpolation form: at most 2^30 coefficients per species");
    InterpFactors1D F;
    build_interp_factors(N, idx->k, F);
    const Csr* mats[4] = {&F.A, &F.B, &F.Binv, &F.Ainv};
    cudaStream_t st = s->ctx->stream;
    for (int w = 0; w < 4; ++w) {
        const Csr& M = *mats[w];
        SGK_REQUIRE(M.rows == H && (int)M.ptr.size() == H + 1, SGK_EINVAL, "interp: factor size mismatch");
        std::vector<int32_t> ce(M.col.size());
        std::vector<int32_t> rl((size_t)H * nl, 0);
        for (int a = 0; a < H; ++a)
            for (int q = M.ptr[a]; q < M.ptr[a + 1]; ++q) {
                const int b = M.col[q];
                SGK_REQUIRE(b >= 0 && b < H, SGK_EINVAL, "interp: column outside the 1D space");
                SGK_REQUIRE(q == M.ptr[a] || M.col[q - 1] < b, SGK_EINVAL, "interp: unsorted row");
                int lb = 0;
                while (b >= level_offset(lb, kp1) + level_count(lb, kp1)) ++lb;
                ce[q] = (lb << 16) | (b - level_offset(lb, kp1));
                for (int L = lb; L < nl; ++L) rl[(size_t)a * nl + L] += 1;
            }
        InterpFactorDev& D = s->IP.f[w];
        D.rp.upload(M.ptr, st);
        D.rlen.upload(rl, st);
        D.ce.upload(ce, st);
        D.val.upload(M.val, st);
        SGK_CUDA_CHECK(cudaStreamSynchronize(st));  // the host vectors go out of scope
    }
    const size_t NS = (size_t)s->nspecies * idx->dof;
    s->IP.t0.alloc(2 * NS);
    s->IP.t1.alloc(2 * NS);
    s->IP.p0.alloc(2 * NS);
    s->IP.p1.alloc(2 * NS);
    s->IP.outcome.alloc(2);
    SGK_CUDA_CHECK(cudaMemsetAsync(s->IP.outcome.p, 0, 2 * sizeof(int), st));
    s->IP.on = true;
}

