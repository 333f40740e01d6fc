// IIF time stepping with a Newton implicit stage: IIF2 (eq. krylov5) and the
// r-th order schemes of eqs. krylov3, krylov4 (IIF3 is eq. krylov6).
//
//   v_s   = U_s^n + dt/2 F_s(U^n)                    (predictor)
//   W_s   = gamma V_M exp(dt H_M) e_1 ~ exp(dt A_s) v_s  (per species)
//   solve G(U) = U - dt/2 F(U) - W = 0 by Newton from U = W:
//         (I - dt/2 J_F(U)) delta = -G(U), U += delta,
//   inner solver: CG for one species (symmetric), restarted GMRES for systems;
//   outer stop ||G||_2 <= tol max(||W||_2, ||G(W)||_2) (relative to the
//   stage's scale); on failure the step is undone.
// For order r the predictor weight dt/2 becomes alpha_0 dt, each older
// F(U^{n-i}) adds alpha_{-i} dt exp((i+1) dt A_s) F_s(U^{n-i}) to W_s, and
// the Newton weight is alpha_1 dt.  F(U, t) includes the source terms at the
// time of its argument.
//
// All vectors live on the device; the host only reads back the scalars that
// decide loop exits (none at all in the device-driven step).  In SGK_MIXED
// mode the Jacobian products J_F(U) w of the inner solve run in FP32 (on an
// FP32 copy of the transformed U), and so does the first residual of a step,
// which only seeds the first correction and never accepts; every other F
// that fixes the answer -- the predictor's F(U^n) and each Newton residual's
// F(U) -- runs in double-float arithmetic (about 1e-14 relative, FP64 where
// the fused pencil kernel does not serve the shape), so Newton's fixed point
// is that of the FP64 path and the outer stop is the same ||G||_2 <= tol
// max(||W||_2, ||G(W)||_2) in both modes (an inexact Jacobian only changes
// the convergence rate).  With the interpolation form of F (interp.cu) the
// implicit stage is solved pointwise at the collocation points instead, in
// FP64 in both modes.  The Krylov exponential keeps its
// double-float matvec and FP64 reductions, and the inner products, norms and
// state stay FP64.  The Newton and CG vector steps are fused with their
// inner products and control decisions.
#include <cmath>
#include <cstring>
#include <type_traits>

#include "sgk_dfloat.h"
#include "sgk_krylov.h"
#include "sgk_pencil.h"
#include "sgk_quad.h"
#include "sgk_solver.h"

namespace {

struct StepCtl {
    double stop, last_g, cg_stop, wnorm, tol;
    int it, status, cg_iters;
    int fvalid;  // Fv holds F(U) for the current U (Newton accepted at its last residual evaluation)
    int pred_skipped;  // this step took F(U^n) from Fv
    int pad;
    long long newton_iters, inner_iters;
};

// The step's control logic (that of the host loop), on one device thread.
__device__ __forceinline__ void newton_init(StepCtl* c, double wnorm, double tol) {
    c->wnorm = wnorm;
    c->tol = tol;
    c->stop = 0.0;  // set at the first residual evaluation
    c->last_g = 0.0;
    c->it = 0;
    c->status = SGK_ENEWTON;
    c->cg_iters = 0;
    c->fvalid = 0;  // U becomes W; the predictor has used the previous F
    c->newton_iters = 0;
    c->inner_iters = 0;
}

// returns 1 to take another Newton correction
// first_low: this evaluation's F ran in FP32 (the first residual of a mixed
// step, which only seeds the first correction): it never accepts
__device__ __forceinline__ unsigned newton_decide(StepCtl* c, double g, int max_iter, int first_low) {
    c->last_g = g;
    // the stop is relative to the stage's scale, max(||W||, ||G(W)||), fixed
    // at the first evaluation (U = W)
    if (c->it == 0) c->stop = c->tol * fmax(c->wnorm, g);
    unsigned go = 0;
    if (!isfinite(g)) c->status = SGK_ENEWTON;
    else if (first_low && c->it == 0) go = 1;
    else if (g <= c->stop) c->status = SGK_OK;
    else if (c->it >= max_iter) c->status = SGK_ENEWTON;
    else go = 1;
    // accepted at this evaluation: F(U) of the new state is in Fv
    c->fvalid = c->status == SGK_OK ? 1 : 0;
    return go;
}

__device__ __forceinline__ unsigned cg_begin(StepCtl* c, double r, double inner_tol, int inner_max) {
    c->cg_stop = inner_tol * inner_tol * r;
    c->cg_iters = 0;
    return (inner_max > 0 && r > c->cg_stop) ? 1u : 0u;
}

__device__ __forceinline__ unsigned cg_continue(StepCtl* c, double r, int inner_max) {
    c->cg_iters += 1;
    return (c->cg_iters < inner_max && r > c->cg_stop) ? 1u : 0u;
}

__device__ __forceinline__ void newton_advance(StepCtl* c) {
    c->inner_iters += c->cg_iters;
    c->newton_iters += 1;
    c->it += 1;
}

// Deterministic FP64 sum completed by the last block to arrive: every block
// stores its partial, counts itself in, and the block that arrives last sums
// the partials in index order with the tree of the two-kernel reduction
// (reduce_final), so the value is bitwise that of vk_dot on the same grid;
// it resets the counter and calls fin(total) on thread 0.
template <typename Fin>
__device__ __forceinline__ void finish_sum(double acc, double* partials, unsigned* counter, Fin&& fin) {
    __shared__ double sh[32];
    __shared__ int s_last;
    acc = block_sum_f64(acc, sh);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = acc;
        __threadfence();
        s_last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double t = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) t += __ldcg(partials + i);
    t = block_sum_f64(t, sh);
    if (threadIdx.x == 0) {
        *counter = 0u;
        fin(t);
    }
}

// Condition of the predictor's F evaluation: run it unless Fv already holds
// F(U) (the previous step ended with an accepted residual evaluation at U,
// which is the same computation).
__global__ void predictor_if_kernel(StepCtl* c, cudaGraphConditionalHandle h) {
    c->pred_skipped = c->fvalid;
    cudaGraphSetConditional(h, c->fvalid ? 0u : 1u);
}

// U[i] = src[i]; any bitwise change of U clears the cached-F flag
__global__ void set_state_kernel(double* __restrict__ U, const double* __restrict__ src, long long n, StepCtl* c) {
    bool changed = false;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double v = src[i];
        changed |= __double_as_longlong(v) != __double_as_longlong(U[i]);
        U[i] = v;
    }
    if (__syncthreads_or(changed) && threadIdx.x == 0) atomicExch(&c->fvalid, 0);
}

// t^n of the state, read by the source kernels of the step's graphs
__global__ void set_time_kernel(double* tdev, double t) { *tdev = t; }

// F[i] += sum_m e^{lam_m (t^n + toff)} S[m n + i] (the source terms of one
// species; toff = 0 for F(U^n), dt for the Newton stage F(U^{n+1}))
__global__ void source_add_kernel(double* __restrict__ F, const double* __restrict__ S, const double* __restrict__ lam,
                                  int nterms, const double* __restrict__ tdev, double toff, long long n) {
    const double t = *tdev + toff;
    double c[SGK_MAX_SOURCE_TERMS];
#pragma unroll
    for (int m = 0; m < SGK_MAX_SOURCE_TERMS; ++m) c[m] = m < nterms ? exp(lam[m] * t) : 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double acc = F[i];
#pragma unroll
        for (int m = 0; m < SGK_MAX_SOURCE_TERMS; ++m)
            if (m < nterms) acc += c[m] * S[m * n + i];
        F[i] = acc;
    }
}

// The last block to arrive runs fin() on thread 0 (no sum).
template <typename Fin>
__device__ __forceinline__ void finish_last(unsigned* counter, Fin&& fin) {
    __shared__ int s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        __threadfence();
        *counter = 0u;
        fin();
    }
}

#define SGK_GRID_STRIDE(i, n) \
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (n); i += (long long)gridDim.x * blockDim.x)

// The Newton / CG vector steps fused with their inner products and, in the
// device-driven step (ctl not null), with the control decisions.  Each runs
// on the grid of vk_dot (reduction_blocks x RED_THREADS), so its elementwise
// results and sums are bitwise those of the separate kernels.

// out = ||W|| and the Newton set-up
__global__ void norm_init_kernel(const double* __restrict__ W, long long n, double* partials, unsigned* cnt,
                                 double* out, StepCtl* ctl, double tol) {
    double acc = 0.0;
    SGK_GRID_STRIDE(i, n) acc += W[i] * W[i];
    finish_sum(acc, partials, cnt, [&](double t) {
        const double wn = sqrt(t);
        *out = wn;
        if (ctl) newton_init(ctl, wn, tol);
    });
}

// G = U - c F - W, out = ||G|| and the Newton decision
__global__ void residual_norm_kernel(const double* __restrict__ U, const double* __restrict__ F,
                                     const double* __restrict__ W, double c, double* __restrict__ G, long long n,
                                     double* partials, unsigned* cnt, double* out, StepCtl* ctl,
                                     cudaGraphConditionalHandle h, int max_iter, int first_low) {
    double acc = 0.0;
    SGK_GRID_STRIDE(i, n) {
        const double g = U[i] - c * F[i] - W[i];
        G[i] = g;
        acc += g * g;
    }
    finish_sum(acc, partials, cnt, [&](double t) {
        const double g = sqrt(t);
        *out = g;
        if (ctl) cudaGraphSetConditional(h, newton_decide(ctl, g, max_iter, first_low));
    });
}

// CG start: x = 0, r = p = -G, rr = r.r and the first CG decision
__global__ void cg_start_kernel(const double* __restrict__ G, double* __restrict__ x, double* __restrict__ r,
                                double* __restrict__ p, long long n, double* partials, unsigned* cnt, double* rr,
                                StepCtl* ctl, double inner_tol, int inner_max, cudaGraphConditionalHandle h) {
    double acc = 0.0;
    SGK_GRID_STRIDE(i, n) {
        const double g = G[i];
        const double v = -1.0 * g + 0.0 * g;  // the axpby(-1, G, 0, G) of the unfused form
        x[i] = 0.0;
        r[i] = v;
        p[i] = v;
        acc += v * v;
    }
    finish_sum(acc, partials, cnt, [&](double t) {
        *rr = t;
        if (ctl) cudaGraphSetConditional(h, cg_begin(ctl, t, inner_tol, inner_max));
    });
}

// q = p - c Jp and pq = p.q
template <typename T>
__global__ void jac_finish_dot_kernel(const double* __restrict__ p, const T* __restrict__ Jp, double c,
                                      double* __restrict__ q, long long n, double* partials, unsigned* cnt,
                                      double* pq) {
    double acc = 0.0;
    SGK_GRID_STRIDE(i, n) {
        const double v = p[i] - c * (double)Jp[i];
        q[i] = v;
        acc += p[i] * v;
    }
    finish_sum(acc, partials, cnt, [&](double t) { *pq = t; });
}

// alpha = rr / pq; x += alpha p; r -= alpha q; rr_new = r.r
__global__ void cg_update_dot_kernel(double* __restrict__ x, double* __restrict__ r, const double* __restrict__ p,
                                     const double* __restrict__ q, const double* rr, const double* pq, long long n,
                                     double* partials, unsigned* cnt, double* rr_new) {
    const double alpha = *rr / *pq;
    double acc = 0.0;
    SGK_GRID_STRIDE(i, n) {
        x[i] += alpha * p[i];
        const double v = r[i] - alpha * q[i];
        r[i] = v;
        acc += v * v;
    }
    finish_sum(acc, partials, cnt, [&](double t) { *rr_new = t; });
}

// p = r + (rr_new / rr) p; then rr = rr_new (after every block has read rr)
// and the next CG decision
__global__ void cg_direction_kernel(double* __restrict__ p, const double* __restrict__ r, const double* rr_new,
                                    double* rr, long long n, unsigned* cnt, StepCtl* ctl, int inner_max,
                                    cudaGraphConditionalHandle h) {
    const double beta = *rr_new / *rr;
    SGK_GRID_STRIDE(i, n) p[i] = r[i] + beta * p[i];
    finish_last(cnt, [&]() {
        const double v = *rr_new;
        *rr = v;
        if (ctl) cudaGraphSetConditional(h, cg_continue(ctl, v, inner_max));
    });
}

// U += x and the Newton advance
__global__ void newton_step_kernel(double* __restrict__ U, const double* __restrict__ x, long long n, unsigned* cnt,
                                   StepCtl* ctl) {
    SGK_GRID_STRIDE(i, n) U[i] = 1.0 * U[i] + 1.0 * x[i];
    finish_last(cnt, [&]() {
        if (ctl) newton_advance(ctl);
    });
}

#undef SGK_GRID_STRIDE

// fused-kernel counters of a solver (each zero between launches)
enum { FC_NORM, FC_RESID, FC_CGSTART, FC_JAC, FC_CGUPD, FC_CGDIR, FC_STEP, FC_COUNT };

// Launch a fused kernel on the grid of vk_dot (so sums match it bitwise).
template <typename K, typename... Args>
void launch_fused(sgk_solver* s, long long N, const char* what, K kern, Args... args) {
    KTimer kt(s->ctx, KC_VECTOR);
    kern<<<reduction_blocks(s->ctx, N), RED_THREADS, 0, s->ctx->stream>>>(args...);
    check_launch(what);
    count_launch(s->ctx);
}

double read_scalar(sgk_solver* s, const double* dptr) {
    SGK_CUDA_CHECK(cudaMemcpyAsync(s->ctx->hscal, dptr, sizeof(double), cudaMemcpyDeviceToHost, s->ctx->stream));
    SGK_CUDA_CHECK(cudaStreamSynchronize(s->ctx->stream));
    return s->ctx->hscal[0];
}

// Runs body() through a cached CUDA graph: captured on first use (kernel
// timers off, launches counted once), then replayed with one launch.
template <class Body>
void run_graph(sgk_solver* s, GraphCache& g, int kc, Body&& body) {
    sgk_ctx* ctx = s->ctx;
    if (!s->use_graphs || ctx->prof_mask) {  // kernel timing needs individual launches
        body();
        return;
    }
    if (!g.exec) {
        const int64_t before = ctx->launches;
        cudaGraph_t graph = nullptr;
        ctx->capturing = true;
        SGK_CUDA_CHECK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
        try {
            body();
        } catch (...) {
            cudaStreamEndCapture(ctx->stream, &graph);
            if (graph) cudaGraphDestroy(graph);
            ctx->capturing = false;
            throw;
        }
        const cudaError_t e = cudaStreamEndCapture(ctx->stream, &graph);
        ctx->capturing = false;
        SGK_CUDA_CHECK(e);
        const cudaError_t ei = cudaGraphInstantiate(&g.exec, graph, 0);
        cudaGraphDestroy(graph);
        SGK_CUDA_CHECK(ei);
        g.nlaunch = ctx->launches - before;
        ctx->launches = before;
    }
    KTimer kt(ctx, kc);
    SGK_CUDA_CHECK(cudaGraphLaunch(g.exec, ctx->stream));
    count_launch(ctx, (int)g.nlaunch);
}

template <typename T>
T* qbuf(sgk_solver* s) {
    return sizeof(T) == 8 ? reinterpret_cast<T*>(s->q64.p) : reinterpret_cast<T*>(s->q32.p);
}

// quad buffer carving: [unod S][wnod S][tmp][spin S][spout S]
template <typename T>
struct QuadPtrs {
    T* unod[SGK_MAX_SPECIES];
    T* wnod[SGK_MAX_SPECIES];
    T* tmp;
    T* spin[SGK_MAX_SPECIES];
    T* spout[SGK_MAX_SPECIES];
};

template <typename T>
QuadPtrs<T> qptrs(sgk_solver* s) {
    QuadPtrs<T> p{};
    T* b = qbuf<T>(s);
    const long long F = s->Q.full_size, n = s->n;
    for (int i = 0; i < s->nspecies; ++i) p.unod[i] = b + i * F;
    for (int i = 0; i < s->nspecies; ++i) p.wnod[i] = b + (s->nspecies + i) * F;
    p.tmp = b + 2LL * s->nspecies * F;
    T* sp = b + (2LL * s->nspecies + 1) * F;
    for (int i = 0; i < s->nspecies; ++i) p.spin[i] = sp + i * n;
    for (int i = 0; i < s->nspecies; ++i) p.spout[i] = sp + (s->nspecies + i) * n;
    return p;
}

// Directions changed by the fiber engine: all d (unfused) or 0..d-2 (the
// last one is fused with the cell quadrature in the pencil kernel).
int fiber_dims(const sgk_solver* s) { return s->Q.fused ? s->Q.d - 1 : s->Q.d; }

template <typename T>
void forward_species(sgk_solver* s, const T* src, T* dst, T* tmp) {
    const int nd = fiber_dims(s);
    if (nd == 0) {
        SGK_CUDA_CHECK(cudaMemcpyAsync(dst, src, s->n * sizeof(T), cudaMemcpyDeviceToDevice, s->ctx->stream));
        return;
    }
    quad_forward<T>(s->ctx, s->Q, src, dst, tmp, nd);
}

template <typename T>
void backward_species(sgk_solver* s, T* mom, T* tmp, T* out) {
    const int nd = fiber_dims(s);
    if (nd == 0) {
        SGK_CUDA_CHECK(cudaMemcpyAsync(out, mom, s->n * sizeof(T), cudaMemcpyDeviceToDevice, s->ctx->stream));
        return;
    }
    quad_backward<T>(s->ctx, s->Q, mom, tmp, out, nd);
}

template <typename T>
void cell_pass(sgk_solver* s, bool jac, T* const* u, T* const* w, T* const* out) {
    const Quad& Q = s->Q;
    if (!Q.fused) {
        if constexpr (std::is_same<T, dfloat>::value) SGK_REQUIRE(false, SGK_EUNSUPPORTED, "double-float cell pass");
        else quad_cells<T>(s->ctx, Q, s->rx, jac, u, w, out);
        return;
    }
    PencilArgs a{};
    a.H = Q.H;
    a.N = Q.N;
    a.ncell1 = 1 << Q.N;
    a.npencils = 1;
    for (int m = 0; m < Q.d - 1; ++m) a.npencils *= a.ncell1;
    for (int l = 0; l <= Q.N; ++l) a.cbase[l] = Q.layout_offsets[Q.d - 1][l];
    for (int sp = 0; sp < s->nspecies; ++sp) {
        a.u[sp] = u[sp];
        a.w[sp] = jac ? w[sp] : nullptr;
        a.out[sp] = out[sp];
    }
    pencil_launch<T>(s->ctx, a, Q.d, Q.kp1, Q.q, s->nspecies, jac, Q.B_host.data(), Q.w_host.data(),
                     Q.tab.two_scale.data(), s->rx);
}

// F(U) for species-stacked FP64 U into FP64 F; caches the transformed U in
// unod for the Jacobian products that follow.
template <typename T>
void evalF_T(sgk_solver* s, const double* U, double* F) {
    QuadPtrs<T> p = qptrs<T>(s);
    const long long n = s->n;
    for (int sp = 0; sp < s->nspecies; ++sp) {
        const T* src;
        if (sizeof(T) == 8) src = reinterpret_cast<const T*>(U + sp * n);
        else {
            vk_convert(s->ctx, U + sp * n, reinterpret_cast<float*>(p.spin[sp]), n);
            src = p.spin[sp];
        }
        forward_species<T>(s, src, p.unod[sp], p.tmp);
    }
    cell_pass<T>(s, false, p.unod, nullptr, p.wnod);
    for (int sp = 0; sp < s->nspecies; ++sp) {
        if (sizeof(T) == 8) {
            backward_species<T>(s, p.wnod[sp], p.tmp, reinterpret_cast<T*>(F + sp * n));
        } else {
            backward_species<T>(s, p.wnod[sp], p.tmp, p.spout[sp]);
            vk_convert(s->ctx, reinterpret_cast<const float*>(p.spout[sp]), F + sp * n, n);
        }
    }
    s->unod_valid = true;
}

// J_F(U) w for the U cached in unod; output in T.
template <typename T>
void evalJ_T(sgk_solver* s, const double* w, T* out) {
    QuadPtrs<T> p = qptrs<T>(s);
    const long long n = s->n;
    for (int sp = 0; sp < s->nspecies; ++sp) {
        const T* src;
        if (sizeof(T) == 8) src = reinterpret_cast<const T*>(w + sp * n);
        else {
            vk_convert(s->ctx, w + sp * n, reinterpret_cast<float*>(p.spin[sp]), n);
            src = p.spin[sp];
        }
        forward_species<T>(s, src, p.wnod[sp], p.tmp);
    }
    cell_pass<T>(s, true, p.unod, p.wnod, p.wnod);
    for (int sp = 0; sp < s->nspecies; ++sp) backward_species<T>(s, p.wnod[sp], p.tmp, out + sp * n);
}

// F(U) in double-float arithmetic (the fused pencil path): U split into
// FP32 pairs, the FP64 work buffers and plans reused for the pairs, the
// result summed back to FP64; caches the transformed U (pairs) in unod.
void evalF_df(sgk_solver* s, const double* U, double* F) {
    QuadPtrs<dfloat> p = qptrs<dfloat>(s);
    const long long n = s->n;
    for (int sp = 0; sp < s->nspecies; ++sp) {
        vk_convert(s->ctx, U + sp * n, p.spin[sp], n);
        forward_species<dfloat>(s, p.spin[sp], p.unod[sp], p.tmp);
    }
    cell_pass<dfloat>(s, false, p.unod, nullptr, p.wnod);
    for (int sp = 0; sp < s->nspecies; ++sp) {
        backward_species<dfloat>(s, p.wnod[sp], p.tmp, p.spout[sp]);
        vk_convert(s->ctx, p.spout[sp], F + sp * n, n);
    }
    s->unod_valid = true;
}

// The reaction passes of every F that fixes the answer: FP64, or in mixed
// mode double-float where the fused pencil kernel serves the shape.
bool df_reaction(const sgk_solver* s) { return s->prec == SGK_MIXED && s->Q.fused; }

// F(U, t^n + toff): the reaction passes (about 1e-14 relative accuracy in
// both precision modes), then the source terms in FP64
//
// In mixed mode the FP32 Jacobian passes that follow read an FP32 copy of
// the transformed U, made here.  lo: a mixed-mode F that only seeds a
// Newton correction and never decides acceptance runs in FP32 (and leaves
// its FP32 transform for the Jacobian passes directly).
// F += sum_m e^{lambda_m (t^n + toff)} S_m per species (FP64)
void add_sources(sgk_solver* s, double* F, double toff) {
    if (!s->has_src) return;
    const long long n = s->n;
    for (int sp = 0; sp < s->nspecies; ++sp) {
        if (!s->nsrc[sp]) continue;
        KTimer kt(s->ctx, KC_VECTOR);
        source_add_kernel<<<(int)std::min<long long>((n + 255) / 256, 4LL * s->ctx->num_sms), 256, 0,
                            s->ctx->stream>>>(F + sp * n, s->src_S[sp].p, s->src_lam.p + sp * SGK_MAX_SOURCE_TERMS,
                                              s->nsrc[sp], s->tdev.p, toff, n);
        check_launch("source_add");
        count_launch(s->ctx);
    }
}

void evalF(sgk_solver* s, const double* U, double* F, double toff, bool lo = false) {
    if (s->IP.on) {
        // the interpolation form (FP64 in both modes; no Jacobian cache)
        interp_evalF(s, U, F);
        add_sources(s, F, toff);
        return;
    }
    if (lo && s->prec == SGK_MIXED) {
        evalF_T<float>(s, U, F);
    } else if (df_reaction(s)) {
        evalF_df(s, U, F);
    } else {
        evalF_T<double>(s, U, F);
    }
    if (s->prec == SGK_MIXED && !lo) {
        const long long m = (long long)s->nspecies * s->Q.full_size;
        if (df_reaction(s)) vk_convert(s->ctx, reinterpret_cast<const dfloat*>(s->q64.p), s->q32.p, m);
        else vk_convert(s->ctx, s->q64.p, s->q32.p, m);
    }
    add_sources(s, F, toff);
}

// writes t^n to the device before a step (or a stand-alone F) reads it
void write_time(sgk_solver* s) {
    if (!s->has_src) return;
    set_time_kernel<<<1, 1, 0, s->ctx->stream>>>(s->tdev.p, s->t);
    check_launch("set_time");
    count_launch(s->ctx);
}

// destroys every cached graph (they are captured again on next use)
void drop_graphs(sgk_solver* s) {
    for (GraphCache* g :
         {&s->g_step, &s->g_pre, &s->g_post, &s->g_pred, &s->g_pred_f, &s->g_resid, &s->g_resid0, &s->g_cg}) {
        if (g->exec) cudaGraphExecDestroy(g->exec);
        *g = GraphCache{};
    }
    for (int sp = 0; sp < SGK_MAX_SPECIES; ++sp) {
        if (s->g_krylov[sp].exec) cudaGraphExecDestroy(s->g_krylov[sp].exec);
        s->g_krylov[sp] = GraphCache{};
        for (GraphCache& g : s->g_krylovh[sp]) {
            if (g.exec) cudaGraphExecDestroy(g.exec);
            g = GraphCache{};
        }
    }
}

// q = p - dt/2 J_F(U) p (stacked FP64); with pq also pq = p.q
void apply_newton_matrix(sgk_solver* s, const double* pv, double* q, double* pq = nullptr) {
    const long long N = s->n * s->nspecies;
    const double c = s->newton_c;
    double* const part = s->partials.p;
    unsigned* const cnt = s->fcnt.p + FC_JAC;
    if (s->prec == SGK_FP64) {
        evalJ_T<double>(s, pv, s->jw64.p);
        if (pq) launch_fused(s, N, "jac_finish_dot", jac_finish_dot_kernel<double>, pv, (const double*)s->jw64.p, c, q,
                             N, part, cnt, pq);
        else vk_jac_finish<double>(s->ctx, pv, s->jw64.p, c, q, N);
    } else {
        evalJ_T<float>(s, pv, s->jw32.p);
        if (pq) launch_fused(s, N, "jac_finish_dot", jac_finish_dot_kernel<float>, pv, (const float*)s->jw32.p, c, q,
                             N, part, cnt, pq);
        else vk_jac_finish<float>(s->ctx, pv, s->jw32.p, c, q, N);
    }
}

template <typename T>
KrylovWork<T> krylov_work(sgk_solver* s, int species) {
    KrylovWork<T> kw;
    kw.V = sizeof(T) == 8 ? reinterpret_cast<T*>(s->V64.p) : reinterpret_cast<T*>(s->V32.p);
    kw.w = sizeof(T) == 8 ? reinterpret_cast<T*>(s->w64.p) : reinterpret_cast<T*>(s->w32.p);
    kw.H = s->Hm.p;
    kw.h1 = s->h1.p;
    kw.h2 = s->h2.p;
    kw.y = s->ky.p;
    kw.scal = s->scal.p;
    kw.partials = s->partials.p;
    kw.expm_ws = s->expm_ws.p;
    kw.ks = s->ks.p + species;
    kw.counter = s->counters.p;
    return kw;
}

void cg_solve(sgk_solver* s, const double* G, double* x, int& iters) {
    const long long N = s->n * s->nspecies;
    double* r = s->cg_r.p;
    double* pv = s->cg_p.p;
    double* q = s->cg_q.p;
    double* const rr = s->scal.p + 2;
    double* const rr_new = s->scal.p + 3;
    double* const pq = s->scal.p + 4;
    launch_fused(s, N, "cg_start", cg_start_kernel, G, x, r, pv, N, s->partials.p, s->fcnt.p + FC_CGSTART, rr,
                 (StepCtl*)nullptr, 0.0, 0, cudaGraphConditionalHandle{});
    double rr_h = read_scalar(s, rr);
    const double stop = s->opts.inner_tol * s->opts.inner_tol * rr_h;
    iters = 0;
    while (iters < s->opts.inner_max && rr_h > stop) {
        run_graph(s, s->g_cg, KC_VECTOR, [&]() {
            apply_newton_matrix(s, pv, q, pq);
            launch_fused(s, N, "cg_update", cg_update_dot_kernel, x, r, (const double*)pv, (const double*)q,
                         (const double*)rr, (const double*)pq, N, s->partials.p, s->fcnt.p + FC_CGUPD, rr_new);
            launch_fused(s, N, "cg_direction", cg_direction_kernel, pv, (const double*)r, (const double*)rr_new, rr,
                         N, s->fcnt.p + FC_CGDIR, (StepCtl*)nullptr, 0, cudaGraphConditionalHandle{});
        });
        rr_h = read_scalar(s, rr);
        ++iters;
    }
}

void gmres_solve_host(sgk_solver* s, const double* G, double* x, int& iters) {
    sgk_ctx* ctx = s->ctx;
    const long long N = s->n * s->nspecies;
    const int restart = s->opts.gmres_restart;
    double* b = s->cg_p.p;
    double* r = s->cg_r.p;
    double* w = s->cg_q.p;
    double* V = s->gm_V.p;
    double* beta = s->scal.p + 2;
    double* hn2 = s->scal.p + 3;
    double* rep = s->gm_report.p;
    vk_axpby(ctx, -1.0, G, 0.0, G, b, N);
    SGK_CUDA_CHECK(cudaMemsetAsync(x, 0, N * sizeof(double), ctx->stream));
    vk_dot(ctx, b, b, N, s->partials.p, beta, 1, nullptr);
    const double bnorm = read_scalar(s, beta);
    iters = 0;
    if (bnorm == 0.0) return;
    const double tol = s->opts.inner_tol * bnorm;
    while (iters < s->opts.inner_max) {
        if (iters == 0) {
            SGK_CUDA_CHECK(cudaMemcpyAsync(r, b, N * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
        } else {
            apply_newton_matrix(s, x, w);
            vk_axpby(ctx, 1.0, b, -1.0, w, r, N);
        }
        vk_dot(ctx, r, r, N, s->partials.p, beta, 1, nullptr);
        const double beta_h = read_scalar(s, beta);
        if (beta_h <= tol) break;
        const int m = std::min(restart, s->opts.inner_max - iters);
        gmres_init(ctx, s->gm_g.p, restart + 1, beta, s->scal.p + 5);
        vk_scale_from(ctx, r, V, N, s->scal.p + 5, nullptr);
        int used = 0;
        double last_g = beta_h;
        for (int j = 0; j < m; ++j) {
            apply_newton_matrix(s, V + (long long)j * N, w);
            vk_mdot<double>(ctx, V, N, j + 1, w, N, s->partials.p, s->h1.p, nullptr);
            vk_gs_update<double>(ctx, V, N, j + 1, s->h1.p, w, N, nullptr);
            vk_mdot<double>(ctx, V, N, j + 1, w, N, s->partials.p, s->h2.p, nullptr);
            vk_gs_update<double>(ctx, V, N, j + 1, s->h2.p, w, N, nullptr);
            vk_dot(ctx, w, w, N, s->partials.p, hn2, 0, nullptr);
            gmres_givens(ctx, j, restart, s->gm_H.p, s->gm_cs.p, s->gm_sn.p, s->gm_g.p, s->h1.p, s->h2.p, hn2, rep);
            SGK_CUDA_CHECK(cudaMemcpyAsync(s->ctx->hscal, rep, 4 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
            SGK_CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
            used = j + 1;
            ++iters;
            last_g = s->ctx->hscal[0];
            if (s->ctx->hscal[0] <= tol || s->ctx->hscal[1] <= 1e-12 * s->ctx->hscal[2]) break;
            vk_scale_from(ctx, w, V + (long long)(j + 1) * N, N, rep + 3, nullptr);
        }
        gmres_solve(ctx, used, restart, s->gm_H.p, s->gm_g.p, s->gm_y.p);
        vk_basis_accumulate(ctx, V, N, used, s->gm_y.p, x, N);
        if (last_g <= tol) break;
    }
}

// The implicit stage U - c F_I(U, t^{n+1}) = W of the interpolation form:
// Wp = W + c S(t^{n+1}), the pointwise solve at the collocation points, U and
// Fv = F_I(U) + S(t^{n+1}) (the next predictor's F); outcome to status, iters.
void interp_stage(sgk_solver* s, int* status, int* iters) {
    const long long N = s->n * s->nspecies;
    const double c = s->newton_c;
    const double* Wp = s->W.p;
    if (s->has_src) {
        SGK_CUDA_CHECK(cudaMemsetAsync(s->G.p, 0, N * sizeof(double), s->ctx->stream));
        add_sources(s, s->G.p, s->dt);
        vk_axpby(s->ctx, 1.0, s->W.p, c, s->G.p, s->G.p, N);
        Wp = s->G.p;
    }
    interp_implicit(s, Wp, c, s->U.p, s->Fv.p, status, iters);
    add_sources(s, s->Fv.p, s->dt);
}

// StepCtl after the interpolation stage of a step graph: the pointwise
// solve's outcome (status, most corrections in it) becomes the step's
__global__ void interp_ctl_finish_kernel(StepCtl* c) {
    c->newton_iters = c->it;
    c->inner_iters = 0;
    c->last_g = 0.0;
    c->fvalid = c->status == SGK_OK ? 1 : 0;
}

int newton(sgk_solver* s) {
    sgk_ctx* ctx = s->ctx;
    if (s->IP.on) {
        int* o = s->IP.outcome.p;
        interp_stage(s, o, o + 1);
        int h[2] = {0, 0};
        SGK_CUDA_CHECK(cudaMemcpyAsync(h, o, 2 * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
        SGK_CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
        s->stats.newton_iters += h[1];
        s->stats.last_newton_residual = 0.0;
        return h[0] == SGK_OK ? SGK_OK : SGK_ENEWTON;
    }
    const long long N = s->n * s->nspecies;
    const double dt2 = s->newton_c;
    SGK_CUDA_CHECK(cudaMemcpyAsync(s->U.p, s->W.p, N * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
    launch_fused(s, N, "norm", norm_init_kernel, (const double*)s->W.p, N, s->partials.p, s->fcnt.p + FC_NORM,
                 s->scal.p + 6, (StepCtl*)nullptr, 0.0);
    const double wnorm = read_scalar(s, s->scal.p + 6);
    double stop = 0.0;  // relative to max(||W||, ||G(W)||), set at the first evaluation
    // mixed mode: the first residual (at W) runs in FP32 and only seeds the
    // first correction; every residual that can accept runs accurately
    const bool first_low = s->prec == SGK_MIXED;
    for (int it = 0; it <= s->opts.max_iter; ++it) {
        const bool lo = first_low && it == 0;
        run_graph(s, lo ? s->g_resid0 : s->g_resid, KC_VECTOR, [&]() {
            evalF(s, s->U.p, s->Fv.p, s->dt, lo);
            launch_fused(s, N, "residual", residual_norm_kernel, (const double*)s->U.p, (const double*)s->Fv.p,
                         (const double*)s->W.p, dt2, s->G.p, N, s->partials.p, s->fcnt.p + FC_RESID, s->scal.p + 7,
                         (StepCtl*)nullptr, cudaGraphConditionalHandle{}, 0, 0);
        });
        const double g = read_scalar(s, s->scal.p + 7);
        s->stats.last_newton_residual = g;
        if (!std::isfinite(g)) break;
        if (it == 0) stop = s->opts.tol * std::max(wnorm, g);
        if (!lo && g <= stop) return SGK_OK;
        if (it == s->opts.max_iter) break;
        int inner = 0;
        if (s->nspecies == 1) cg_solve(s, s->G.p, s->cg_x.p, inner);
        else gmres_solve_host(s, s->G.p, s->cg_x.p, inner);
        s->stats.inner_iters += inner;
        s->stats.newton_iters += 1;
        launch_fused(s, N, "newton_step", newton_step_kernel, s->U.p, (const double*)s->cg_x.p, N,
                     s->fcnt.p + FC_STEP, (StepCtl*)nullptr);
    }
    return SGK_ENEWTON;
}

}  // namespace

// ------------------------------------------------------------ interface ---

void solver_eval_reaction(sgk_solver* s, const double* U, double* F) {
    SGK_REQUIRE(s->has_rx, SGK_EINVAL, "solver has no reaction term");
    write_time(s);
    evalF(s, U, F, 0.0);
}

void solver_jacobian_apply(sgk_solver* s, const double* U, const double* w, double* jw) {
    SGK_REQUIRE(s->has_rx, SGK_EINVAL, "solver has no reaction term");
    if (s->IP.on) {
        interp_evalJ(s, U, w, jw);
        return;
    }
    const long long n = s->n;
    if (s->prec == SGK_FP64) {
        QuadPtrs<double> p = qptrs<double>(s);
        for (int sp = 0; sp < s->nspecies; ++sp) forward_species<double>(s, U + sp * n, p.unod[sp], p.tmp);
        evalJ_T<double>(s, w, jw);
    } else {
        QuadPtrs<float> p = qptrs<float>(s);
        for (int sp = 0; sp < s->nspecies; ++sp) {
            vk_convert(s->ctx, U + sp * n, p.spin[sp], n);
            forward_species<float>(s, p.spin[sp], p.unod[sp], p.tmp);
        }
        evalJ_T<float>(s, w, s->jw32.p);
        vk_convert(s->ctx, s->jw32.p, jw, n * s->nspecies);
    }
    s->unod_valid = false;
}

// W = exp(tau A_s) v by the Krylov projection (tau < 0: tau = dt)
namespace {

// One Krylov projection W = gamma V_M exp(tau H_M) e_1 (eq. krylov8) of v.
void krylov_projection(sgk_solver* s, int species, const double* v, double* W, double tau) {
    const sgk_op* op = s->ops[species];
    const long long n = s->n;
    // the matvec inside Arnoldi is FP64 or double-float (mixed mode, in the
    // persistent kernel): an FP32 matvec costs a few 1e-6 of relative
    // accuracy per exponential on these stiff operators
    if (s->persistent) {
        PersistentWork pw;
        pw.w_alt = s->w64b.p;
        pw.Z = s->zbuf.p;
        pw.pbuf = s->pbuf.p;
        pw.bar = s->pbar.p + 2 * species;
        pw.G = s->arn_G;
        pw.bounds = s->abounds.p;
        pw.E = s->aE;
        pw.list_ent = s->alist;
        krylov_expv_persistent(s->ctx, op, pw, krylov_work<double>(s, species), v, W, n, s->M, tau);
    } else {
        auto mv = [op](const double* x, double* y) { op_matvec<double>(op, x, y); };
        krylov_expv_dev<double>(s->ctx, krylov_work<double>(s, species), mv, v, W, n, s->M, tau);
    }
}

// KrylovScalars::err_max = 0 for every species (the start of a step)
__global__ void krylov_est_clear_kernel(KrylovScalars* ks, int nspecies) {
    if (threadIdx.x < nspecies) ks[threadIdx.x].err_max = 0.0;
}

}  // namespace

void krylov_est_clear(sgk_solver* s) {
    krylov_est_clear_kernel<<<1, 32, 0, s->ctx->stream>>>(s->ks.p, s->nspecies);
    check_launch("krylov_est_clear");
    count_launch(s->ctx);
}

// exp(tau A) v: the paper's single projection, or with ksub > 1 the
// semigroup product exp(tau A) = exp((tau / ksub) A)^ksub taken as ksub
// successive projections, the last of which writes W
void solver_krylov_expv(sgk_solver* s, int species, const double* v, double* W, double tau) {
    if (tau < 0.0) tau = s->dt;
    const int ns = s->ksub;
    const double* src = v;
    for (int i = 0; i < ns; ++i) {
        double* dst = ((ns - 1 - i) & 1) ? s->ktmp.p : W;
        krylov_projection(s, species, src, dst, tau / ns);
        src = dst;
    }
    if (!s->use_graphs || !s->ctx->capturing) s->stats.krylov_calls += 1;
}

void solver_set_krylov_substeps(sgk_solver* s, int ksub) {
    if (ksub > 1 && s->ktmp.n < (size_t)s->n) s->ktmp.alloc(s->n);
    s->stats.krylov_substeps = ksub;
    if (ksub != s->ksub) {
        s->ksub = ksub;
        drop_graphs(s);
    }
}

// exp(dt H) e_1 and W = gamma V y of species 0 after its Arnoldi process
// ran outside the solver (batched launch)
void solver_krylov_finish(sgk_solver* s, int species, double* W) {
    krylov_finish(s->ctx, krylov_work<double>(s, species), W, s->n, s->M, s->dt);
    if (!s->use_graphs || !s->ctx->capturing) s->stats.krylov_calls += 1;
}

// ------------------------------------------------ device-driven step ---
//
// With graphs on and one species (CG) or no reaction, a whole IIF2 step is
// one CUDA graph: the Newton iteration and the CG iteration are conditional
// while-nodes whose conditions are set by one-thread control kernels from the
// residual norms, so a step needs one host synchronisation (to read the
// outcome) instead of one per Newton and CG iteration.  The control logic is
// that of the host loop: stop at ||G|| <= tol max(||W||, ||G(W)||), at most
// max_iter corrections, CG to a relative residual inner_tol.

namespace {

// Adds a while-node at the capture position of ctx->stream: pre(h) is
// captured first (it sets the first condition), then the node, whose body
// body(h) is captured on aux (ctx->stream points there meanwhile).
template <typename Pre, typename Body>
void capture_cond(sgk_ctx* ctx, cudaStream_t aux, cudaGraphConditionalNodeType type, Pre&& pre, Body&& body) {
    cudaStream_t st = ctx->stream;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    SGK_CUDA_CHECK(cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, nullptr, &nd));
    SGK_REQUIRE(cs == cudaStreamCaptureStatusActive, SGK_ECUDA, "step graph: stream is not capturing");
    cudaGraphConditionalHandle h;
    SGK_CUDA_CHECK(cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault));
    pre(h);
    SGK_CUDA_CHECK(cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, nullptr, &nd));
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = type;
    p.conditional.size = 1;
    cudaGraphNode_t node = nullptr;
    SGK_CUDA_CHECK(cudaGraphAddNode(&node, g, deps, nullptr, nd, &p));
    SGK_CUDA_CHECK(cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    cudaGraph_t bodyg = p.conditional.phGraph_out[0];
    SGK_CUDA_CHECK(cudaStreamBeginCaptureToGraph(aux, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    ctx->stream = aux;
    try {
        body(h);
    } catch (...) {
        ctx->stream = st;
        cudaGraph_t tmp = nullptr;
        cudaStreamEndCapture(aux, &tmp);
        throw;
    }
    ctx->stream = st;
    cudaGraph_t out = nullptr;
    SGK_CUDA_CHECK(cudaStreamEndCapture(aux, &out));
}

template <typename Pre, typename Body>
void capture_while(sgk_ctx* ctx, cudaStream_t aux, Pre&& pre, Body&& body) {
    capture_cond(ctx, aux, cudaGraphCondTypeWhile, pre, body);
}

bool step_graph_eligible(const sgk_solver* s) {
    return s->use_graphs && s->scheme == SGK_IIF2 && (!s->has_rx || s->nspecies == 1 || s->IP.on);
}

// part: STEP_WHOLE (one graph per step), or the two halves of a step whose
// Arnoldi process runs elsewhere (a batched launch): STEP_PRE (state copy,
// predictor, v) and STEP_POST (exp(dt H) e_1, the combination, the Newton
// solve); one species only for the halves.
enum { STEP_WHOLE = 0, STEP_PRE = 1, STEP_POST = 2 };

void build_step_graph(sgk_solver* s, int part = STEP_WHOLE) {
    sgk_ctx* ctx = s->ctx;
    const long long n = s->n, N = n * s->nspecies;
    const double dt2 = 0.5 * s->dt;
    StepCtl* ctl = reinterpret_cast<StepCtl*>(s->ctl.p);
    for (int i = 0; i < 2; ++i)
        if (!s->aux[i]) SGK_CUDA_CHECK(cudaStreamCreateWithFlags(&s->aux[i], cudaStreamNonBlocking));
    const int64_t before = ctx->launches;
    cudaGraph_t graph = nullptr;
    ctx->capturing = true;
    SGK_CUDA_CHECK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    try {
      if (part != STEP_POST) {
        SGK_CUDA_CHECK(cudaMemcpyAsync(s->Uprev.p, s->U.p, N * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
        krylov_est_clear(s);
        if (s->has_rx) {
            // F(U^n) for the predictor, unless the last step left it in Fv
            capture_cond(
                ctx, s->aux[0], cudaGraphCondTypeIf,
                [&](cudaGraphConditionalHandle h) {
                    predictor_if_kernel<<<1, 1, 0, ctx->stream>>>(ctl, h);
                    check_launch("predictor_if");
                    count_launch(ctx);
                },
                [&](cudaGraphConditionalHandle) {
                    const int64_t m0 = ctx->launches;
                    evalF(s, s->U.p, s->Fv.p, 0.0);
                    s->n_predf = ctx->launches - m0;
                });
            vk_axpby(ctx, 1.0, s->U.p, dt2, s->Fv.p, s->vv.p, N);
        } else {
            SGK_CUDA_CHECK(
                cudaMemcpyAsync(s->vv.p, s->U.p, N * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
        }
      }
      if (part == STEP_PRE) {
        s->n_pre = ctx->launches - before;
      } else {
        if (part == STEP_WHOLE)
            for (int sp = 0; sp < s->nspecies; ++sp) solver_krylov_expv(s, sp, s->vv.p + sp * n, s->W.p + sp * n);
        else
            solver_krylov_finish(s, 0, s->W.p);
        SGK_CUDA_CHECK(cudaMemcpyAsync(s->U.p, s->W.p, N * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
        if (s->has_rx && s->IP.on) {
            // the interpolation form: the implicit stage is straight-line
            interp_stage(s, &ctl->status, &ctl->it);
            interp_ctl_finish_kernel<<<1, 1, 0, ctx->stream>>>(ctl);
            check_launch("interp_ctl_finish");
            count_launch(ctx);
            s->n_prefix = ctx->launches - before;
        } else if (s->has_rx) {
            double* const rr = s->scal.p + 2;
            double* const rr_new = s->scal.p + 3;
            double* const pq = s->scal.p + 4;
            launch_fused(s, N, "norm", norm_init_kernel, (const double*)s->W.p, N, s->partials.p,
                         s->fcnt.p + FC_NORM, s->scal.p + 6, ctl, s->opts.tol);
            // mixed mode: the first residual (at W) in FP32, never accepting
            const int first_low = s->prec == SGK_MIXED ? 1 : 0;
            auto resid = [&](cudaGraphConditionalHandle h, bool lo) {
                evalF(s, s->U.p, s->Fv.p, s->dt, lo);
                launch_fused(s, N, "residual", residual_norm_kernel, (const double*)s->U.p, (const double*)s->Fv.p,
                             (const double*)s->W.p, dt2, s->G.p, N, s->partials.p, s->fcnt.p + FC_RESID,
                             s->scal.p + 7, ctl, h, s->opts.max_iter, lo ? first_low : 0);
            };
            int64_t mark = 0;
            capture_while(
                ctx, s->aux[0],
                [&](cudaGraphConditionalHandle h) { resid(h, first_low != 0); },
                [&](cudaGraphConditionalHandle hn) {
                    s->n_prefix = ctx->launches - before;
                    mark = ctx->launches;
                    double* x = s->cg_x.p;
                    double* r = s->cg_r.p;
                    double* pv = s->cg_p.p;
                    double* q = s->cg_q.p;
                    capture_while(
                        ctx, s->aux[1],
                        [&](cudaGraphConditionalHandle hc) {
                            launch_fused(s, N, "cg_start", cg_start_kernel, (const double*)s->G.p, x, r, pv, N,
                                         s->partials.p, s->fcnt.p + FC_CGSTART, rr, ctl, s->opts.inner_tol,
                                         s->opts.inner_max, hc);
                            s->n_cgpre = ctx->launches - mark;
                        },
                        [&](cudaGraphConditionalHandle hc) {
                            mark = ctx->launches;
                            apply_newton_matrix(s, pv, q, pq);
                            launch_fused(s, N, "cg_update", cg_update_dot_kernel, x, r, (const double*)pv,
                                         (const double*)q, (const double*)rr, (const double*)pq, N, s->partials.p,
                                         s->fcnt.p + FC_CGUPD, rr_new);
                            launch_fused(s, N, "cg_direction", cg_direction_kernel, pv, (const double*)r,
                                         (const double*)rr_new, rr, N, s->fcnt.p + FC_CGDIR, ctl,
                                         s->opts.inner_max, hc);
                            s->n_cgbody = ctx->launches - mark;
                        });
                    mark = ctx->launches;
                    launch_fused(s, N, "newton_step", newton_step_kernel, s->U.p, (const double*)x, N,
                                 s->fcnt.p + FC_STEP, ctl);
                    s->n_adv = ctx->launches - mark;
                    mark = ctx->launches;
                    resid(hn, false);
                    s->n_resid = ctx->launches - mark;
                });
        } else {
            s->n_prefix = ctx->launches - before;
        }
      }
    } catch (...) {
        cudaStreamEndCapture(ctx->stream, &graph);
        if (graph) cudaGraphDestroy(graph);
        ctx->capturing = false;
        ctx->launches = before;
        throw;
    }
    const cudaError_t e = cudaStreamEndCapture(ctx->stream, &graph);
    ctx->capturing = false;
    ctx->launches = before;
    SGK_CUDA_CHECK(e);
    GraphCache& g = part == STEP_WHOLE ? s->g_step : (part == STEP_PRE ? s->g_pre : s->g_post);
    const cudaError_t ei = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    SGK_CUDA_CHECK(ei);
}

// Pinned host record of one device-driven step: StepCtl, the Krylov
// scalars and the barrier flags of every species.
struct StepRecord {
    StepCtl c;
    KrylovScalars ks[SGK_MAX_SPECIES];
    unsigned flags[2 * SGK_MAX_SPECIES];
};

}  // namespace

// Copies of a launched step's outcome to its host record.
static void step_record(sgk_solver* s, int slot);

// Queues one device-driven step (graph launch and the copies of its
// outcome) without waiting.
void solver_step_launch(sgk_solver* s, int slot) {
    sgk_ctx* ctx = s->ctx;
    if (!s->g_step.exec) build_step_graph(s);
    write_time(s);
    {
        KTimer kt(ctx, KC_KRYLOV);
        SGK_CUDA_CHECK(cudaGraphLaunch(s->g_step.exec, ctx->stream));
    }
    s->split_last = false;
    step_record(s, slot);
}

bool solver_split_eligible(const sgk_solver* s) {
    return solver_device_steps(s) && s->nspecies == 1 && s->persistent && s->ksub == 1;
}

ArnJob solver_arnoldi_job(sgk_solver* s) {
    ArnJob j;
    j.ctx = s->ctx;
    j.op = s->ops[0];
    j.pw.w_alt = s->w64b.p;
    j.pw.Z = s->zbuf.p;
    j.pw.pbuf = s->pbuf.p;
    j.pw.bar = s->pbar.p;
    j.pw.G = s->arn_G;
    j.pw.bounds = s->abounds.p;
    j.pw.E = s->aE;
    j.pw.list_ent = s->alist;
    j.kw = krylov_work<double>(s, 0);
    j.v = s->vv.p;
    j.n = s->n;
    j.M = s->M;
    return j;
}

void solver_step_launch_pre(sgk_solver* s) {
    if (!s->g_pre.exec) build_step_graph(s, STEP_PRE);
    write_time(s);
    SGK_CUDA_CHECK(cudaGraphLaunch(s->g_pre.exec, s->ctx->stream));
}

void solver_step_launch_post(sgk_solver* s, int slot) {
    if (!s->g_post.exec) build_step_graph(s, STEP_POST);
    SGK_CUDA_CHECK(cudaGraphLaunch(s->g_post.exec, s->ctx->stream));
    s->split_last = true;
    step_record(s, slot);
}

static void step_record(sgk_solver* s, int slot) {
    sgk_ctx* ctx = s->ctx;
    StepRecord* h = static_cast<StepRecord*>(s->hrec) + slot;
    if (s->has_rx)
        SGK_CUDA_CHECK(cudaMemcpyAsync(&h->c, s->ctl.p, sizeof(StepCtl), cudaMemcpyDeviceToHost, ctx->stream));
    SGK_CUDA_CHECK(cudaMemcpyAsync(h->ks, s->ks.p, s->nspecies * sizeof(KrylovScalars), cudaMemcpyDeviceToHost,
                                   ctx->stream));
    if (s->persistent)
        SGK_CUDA_CHECK(cudaMemcpyAsync(h->flags, s->pbar.p, 2 * s->nspecies * sizeof(unsigned),
                                       cudaMemcpyDeviceToHost, ctx->stream));
}

// Completes a launched step once its stream has drained (the caller
// synchronised it): statistics, and on failure the rollback of the state.
int solver_step_finish(sgk_solver* s, int slot, const double* restore) {
    sgk_ctx* ctx = s->ctx;
    const long long N = s->n * s->nspecies;
    StepRecord* h = static_cast<StepRecord*>(s->hrec) + slot;
    StepCtl c{};
    if (s->has_rx) c = h->c;
    int rc = s->has_rx ? c.status : SGK_OK;
    count_launch(ctx, (int)((s->split_last ? s->n_pre : 0) + s->n_prefix -
                            (s->has_rx && c.pred_skipped ? s->n_predf : 0) +
                            c.newton_iters * (s->n_cgpre + s->n_adv + s->n_resid) + c.inner_iters * s->n_cgbody));
    s->stats.newton_iters += c.newton_iters;
    s->stats.inner_iters += c.inner_iters;
    if (s->has_rx) s->stats.last_newton_residual = c.last_g;
    s->stats.krylov_calls += s->nspecies;
    s->stats.last_krylov_err_est = 0.0;
    for (int sp = 0; sp < s->nspecies; ++sp) {
        s->stats.krylov_breakdowns += h->ks[sp].breakdown;
        s->stats.last_m_eff = h->ks[sp].m_eff;
        s->stats.last_krylov_err_est = std::max(s->stats.last_krylov_err_est, h->ks[sp].err_max);
    }
    s->stats.max_krylov_err_est = std::max(s->stats.max_krylov_err_est, s->stats.last_krylov_err_est);
    bool timed_out = false;
    if (s->persistent)
        for (int sp = 0; sp < s->nspecies; ++sp) timed_out = timed_out || h->flags[2 * sp + 1] != 0u;
    if (timed_out) {
        SGK_CUDA_CHECK(cudaMemsetAsync(s->pbar.p, 0, 2 * s->nspecies * sizeof(unsigned), ctx->stream));
        rc = SGK_ETIMEOUT;
    }
    if (rc != SGK_OK) {
        SGK_CUDA_CHECK(cudaMemcpyAsync(s->U.p, restore ? restore : s->Uprev.p, N * sizeof(double),
                                       cudaMemcpyDeviceToDevice, ctx->stream));
        solver_state_changed(s);
        SGK_CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
    } else {
        s->stats.steps += 1;
        s->t += s->dt;
        s->fv_valid = s->has_rx;
    }
    return rc;
}

int solver_step_async(sgk_solver* s, int nsteps) {
    if (!solver_device_steps(s)) return solver_step(s, nsteps);
    if (s->async_rc != SGK_OK) return SGK_OK;  // a queued step failed: nothing more runs until it is reported
    sgk_ctx* ctx = s->ctx;
    const long long N = s->n * s->nspecies;
    if (!s->ring.p) {
        // up to 32 queued steps, and at most 256 MB of saved states
        const long long cap = (256LL << 20) / (N * (long long)sizeof(double));
        s->ring_slots = (int)std::max(1LL, std::min<long long>(SGK_ASYNC_SLOTS, cap));
        s->ring.alloc((size_t)s->ring_slots * N);
    }
    for (int k = 0; k < nsteps; ++k) {
        if (s->nqueued == s->ring_slots) {
            solver_drain(s);
            if (s->async_rc != SGK_OK) break;
        }
        const int slot = s->nqueued;
        SGK_CUDA_CHECK(cudaMemcpyAsync(s->ring.p + slot * N, s->U.p, N * sizeof(double), cudaMemcpyDeviceToDevice,
                                       ctx->stream));
        solver_step_launch(s, slot);
        ++s->nqueued;
    }
    return SGK_OK;
}

void solver_drain(sgk_solver* s) {
    if (s->nqueued == 0) return;
    const long long N = s->n * s->nspecies;
    const int q = s->nqueued;
    s->nqueued = 0;
    SGK_CUDA_CHECK(cudaStreamSynchronize(s->ctx->stream));
    for (int slot = 0; slot < q; ++slot) {
        const int rc = solver_step_finish(s, slot, s->ring.p + slot * N);
        if (rc != SGK_OK) {
            // the state is that before the failing step; the steps queued
            // after it are discarded, and so are any barrier flags they left
            if (s->persistent)
                SGK_CUDA_CHECK(cudaMemsetAsync(s->pbar.p, 0, 2 * s->nspecies * sizeof(unsigned), s->ctx->stream));
            SGK_CUDA_CHECK(cudaStreamSynchronize(s->ctx->stream));
            if (s->async_rc == SGK_OK) s->async_rc = rc;
            break;
        }
    }
}

bool solver_device_steps(const sgk_solver* s) { return step_graph_eligible(s) && !s->ctx->prof_mask; }

void solver_set_state(sgk_solver* s, int species, const double* src_dev) {
    const long long n = s->n;
    s->nhist = 0;  // a new state has no F(U^{n-1}): IIFr restarts with an IIF2 step
    if (s->has_rx && s->ctl.p) {
        // the device keeps the cached F(U) when the new state equals the old
        set_state_kernel<<<reduction_blocks(s->ctx, n), RED_THREADS, 0, s->ctx->stream>>>(
            s->U.p + species * n, src_dev, n, reinterpret_cast<StepCtl*>(s->ctl.p));
        check_launch("set_state");
        count_launch(s->ctx);
        s->fv_valid = false;  // host-driven steps do not read the device flag
    } else {
        SGK_CUDA_CHECK(cudaMemcpyAsync(s->U.p + species * n, src_dev, n * sizeof(double), cudaMemcpyDeviceToDevice,
                                       s->ctx->stream));
        solver_state_changed(s);
    }
}

void solver_set_source(sgk_solver* s, int species, int nterms, const double* lambda, const double* coeffs_dev) {
    const long long n = s->n;
    if (nterms > 0) {
        if (!s->src_S[species].p) s->src_S[species].alloc((size_t)SGK_MAX_SOURCE_TERMS * n);
        if (!s->src_lam.p) s->src_lam.alloc(SGK_MAX_SPECIES * SGK_MAX_SOURCE_TERMS);
        if (!s->tdev.p) s->tdev.alloc(1);
        SGK_CUDA_CHECK(cudaMemcpyAsync(s->src_S[species].p, coeffs_dev, nterms * n * sizeof(double),
                                       cudaMemcpyDeviceToDevice, s->ctx->stream));
        SGK_CUDA_CHECK(cudaMemcpyAsync(s->src_lam.p + species * SGK_MAX_SOURCE_TERMS, lambda, nterms * sizeof(double),
                                       cudaMemcpyHostToDevice, s->ctx->stream));
        SGK_CUDA_CHECK(cudaStreamSynchronize(s->ctx->stream));  // lambda is pageable host memory
    }
    s->nsrc[species] = nterms;
    s->has_src = false;
    for (int sp = 0; sp < s->nspecies; ++sp) s->has_src = s->has_src || s->nsrc[sp] > 0;
    // the graphs hold the source launches with their term counts, and F changed
    drop_graphs(s);
    s->nhist = 0;
    solver_state_changed(s);
}

void solver_set_time(sgk_solver* s, double t) {
    if (t == s->t) return;  // the cached F values stay valid
    s->t = t;
    s->nhist = 0;
    solver_state_changed(s);
}

void solver_state_changed(sgk_solver* s) {
    s->fv_valid = false;
    if (s->ctl.p)
        SGK_CUDA_CHECK(
            cudaMemsetAsync(&reinterpret_cast<StepCtl*>(s->ctl.p)->fvalid, 0, sizeof(int), s->ctx->stream));
}

namespace {

}  // namespace

// The accuracy guard of synchronous steps: true when the projections just
// taken missed the tolerance and the sub-projections can still be doubled
// (doubles them)
static bool krylov_refine(sgk_solver* s) {
    if (!(s->ktol > 0.0) || !(s->stats.last_krylov_err_est > s->ktol) || s->ksub >= s->kmax) return false;
    solver_set_krylov_substeps(s, std::min(2 * s->ksub, s->kmax));
    s->stats.krylov_refinements += 1;
    return true;
}

bool solver_step_retake(sgk_solver* s) {
    if (!krylov_refine(s)) return false;
    // back to the step's starting state (a device-driven IIF2 step keeps no
    // history beyond U and t)
    SGK_CUDA_CHECK(cudaMemcpyAsync(s->U.p, s->Uprev.p, s->n * s->nspecies * sizeof(double), cudaMemcpyDeviceToDevice,
                                   s->ctx->stream));
    solver_state_changed(s);
    s->t -= s->dt;
    s->stats.steps -= 1;
    return true;
}

int solver_step(sgk_solver* s, int nsteps) {
    sgk_ctx* ctx = s->ctx;
    if (solver_device_steps(s)) {
        for (int step = 0; step < nsteps; ++step) {
            do {
                solver_step_launch(s);
                SGK_CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
                const int rc = solver_step_finish(s);
                if (rc != SGK_OK) return rc;
            } while (solver_step_retake(s));
        }
        return SGK_OK;
    }
    const long long n = s->n, N = n * s->nspecies;
    // restores the solver's graph setting when a step ends, however it ends
    struct GraphsSetting {
        sgk_solver* s;
        bool v;
        ~GraphsSetting() { s->use_graphs = v; }
    };
    for (int step = 0; step < nsteps; ++step) {
        SGK_CUDA_CHECK(cudaMemcpyAsync(s->Uprev.p, s->U.p, N * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
        write_time(s);
        // IIFr (eqs. krylov3, krylov4) at the highest order r the history
        // allows: W = exp(dt A)(U^n + alpha_0 dt F(U^n)) + sum_{i=1}^{r-2}
        // alpha_{-i} dt exp((i+1) dt A) F(U^{n-i}), Newton weight alpha_1 dt
        // (IIF2: dt/2 and dt/2; IIF3: 2/3, -1/12 and 5/12).  The graph caches
        // hold the weights of the full order, so start-up steps run without
        // them.
        const int r_full = s->has_rx ? s->scheme : SGK_IIF2;
        const int r = std::min(r_full, 2 + s->nhist);
        double alpha[SGK_IIF_MAX_ORDER];
        iif_alpha(r, alpha);
        const double cpred = alpha[1] * s->dt;
        s->newton_c = alpha[0] * s->dt;
        GraphsSetting keep{s, s->use_graphs};
        if (r < r_full) s->use_graphs = false;
        // F(U^n) for the predictor, unless the last step left it in Fv; the
        // device-side flag of the step graph is stale after a host-driven step
        const bool have_f = s->fv_valid;
        run_graph(s, have_f ? s->g_pred_f : s->g_pred, KC_VECTOR, [&]() {
            if (s->has_rx) {
                if (!have_f) evalF(s, s->U.p, s->Fv.p, 0.0);
                vk_axpby(ctx, 1.0, s->U.p, cpred, s->Fv.p, s->vv.p, N);
            } else {
                SGK_CUDA_CHECK(cudaMemcpyAsync(s->vv.p, s->U.p, N * sizeof(double), cudaMemcpyDeviceToDevice,
                                               ctx->stream));
            }
        });
        // the step's exponentials; with the accuracy guard on, taken again
        // with twice the sub-projections while their estimate misses the
        // tolerance (nothing of the state has changed yet)
        for (;;) {
            krylov_est_clear(s);
            for (int sp = 0; sp < s->nspecies; ++sp) {
                run_graph(s, s->g_krylov[sp], KC_KRYLOV,
                          [&]() { solver_krylov_expv(s, sp, s->vv.p + sp * n, s->W.p + sp * n); });
                s->stats.krylov_calls += s->use_graphs ? 1 : 0;
            }
            for (int i = 1; i <= r - 2; ++i)
                for (int sp = 0; sp < s->nspecies; ++sp) {
                    run_graph(s, s->g_krylovh[sp][i - 1], KC_KRYLOV, [&]() {
                        solver_krylov_expv(s, sp, s->Fhist.p + (i - 1) * N + sp * n, s->W2.p + sp * n,
                                           (i + 1) * s->dt);
                        vk_axpby(ctx, 1.0, s->W.p + sp * n, alpha[i + 1] * s->dt, s->W2.p + sp * n,
                                 s->W.p + sp * n, n);
                    });
                    s->stats.krylov_calls += s->use_graphs ? 1 : 0;
                }
            if (!(s->ktol > 0.0)) break;
            KrylovScalars kq[SGK_MAX_SPECIES];
            SGK_CUDA_CHECK(cudaMemcpyAsync(kq, s->ks.p, s->nspecies * sizeof(KrylovScalars), cudaMemcpyDeviceToHost,
                                           ctx->stream));
            SGK_CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
            s->stats.last_krylov_err_est = 0.0;
            for (int sp = 0; sp < s->nspecies; ++sp)
                s->stats.last_krylov_err_est = std::max(s->stats.last_krylov_err_est, kq[sp].err_max);
            if (!krylov_refine(s)) break;
        }
        // F(U^n) becomes F(U^{n-1}) of the next step if this one succeeds
        if (r_full > 2)
            SGK_CUDA_CHECK(
                cudaMemcpyAsync(s->Fstage.p, s->Fv.p, N * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
        int rc = SGK_OK;
        if (!s->has_rx) {
            SGK_CUDA_CHECK(cudaMemcpyAsync(s->U.p, s->W.p, N * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
        } else {
            rc = newton(s);
        }
        KrylovScalars ks[SGK_MAX_SPECIES];
        unsigned flags[2 * SGK_MAX_SPECIES] = {0};
        SGK_CUDA_CHECK(cudaMemcpyAsync(ks, s->ks.p, s->nspecies * sizeof(KrylovScalars), cudaMemcpyDeviceToHost,
                                       ctx->stream));
        if (s->persistent)
            SGK_CUDA_CHECK(cudaMemcpyAsync(flags, s->pbar.p, 2 * s->nspecies * sizeof(unsigned),
                                           cudaMemcpyDeviceToHost, ctx->stream));
        SGK_CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
        // a grid barrier of the persistent Arnoldi kernel ran out of time:
        // clear the sticky flags and report it
        bool timed_out = false;
        for (int sp = 0; sp < s->nspecies; ++sp) timed_out = timed_out || flags[2 * sp + 1] != 0u;
        if (timed_out) {
            SGK_CUDA_CHECK(cudaMemsetAsync(s->pbar.p, 0, 2 * s->nspecies * sizeof(unsigned), ctx->stream));
            rc = SGK_ETIMEOUT;
        }
        s->stats.last_krylov_err_est = 0.0;
        for (int sp = 0; sp < s->nspecies; ++sp) {
            s->stats.krylov_breakdowns += ks[sp].breakdown;
            s->stats.last_m_eff = ks[sp].m_eff;
            s->stats.last_krylov_err_est = std::max(s->stats.last_krylov_err_est, ks[sp].err_max);
        }
        s->stats.max_krylov_err_est = std::max(s->stats.max_krylov_err_est, s->stats.last_krylov_err_est);
        if (rc != SGK_OK) {
            SGK_CUDA_CHECK(cudaMemcpyAsync(s->U.p, s->Uprev.p, N * sizeof(double), cudaMemcpyDeviceToDevice,
                                           ctx->stream));
            solver_state_changed(s);
            SGK_CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
            return rc;
        }
        s->stats.steps += 1;
        s->t += s->dt;
        if (r_full > 2) {
            // shift the history by one step: F(U^{n-i}) -> slot i, F(U^n) -> slot 0
            for (int k = std::min(s->nhist, r_full - 3); k >= 1; --k)
                SGK_CUDA_CHECK(cudaMemcpyAsync(s->Fhist.p + k * N, s->Fhist.p + (k - 1) * N, N * sizeof(double),
                                               cudaMemcpyDeviceToDevice, ctx->stream));
            SGK_CUDA_CHECK(
                cudaMemcpyAsync(s->Fhist.p, s->Fstage.p, N * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
            s->nhist = std::min(s->nhist + 1, r_full - 2);
        }
        // newton() returns OK right after the residual evaluation at the final
        // U; the step graph's flag says the same
        if (s->has_rx) {
            static const int one = 1;
            SGK_CUDA_CHECK(cudaMemcpyAsync(&reinterpret_cast<StepCtl*>(s->ctl.p)->fvalid, &one, sizeof(int),
                                           cudaMemcpyHostToDevice, ctx->stream));
            s->fv_valid = true;
        }
    }
    return SGK_OK;
}

void iif_alpha(int r, double* alpha) {
    // In the scaled time s = tau / dt the basis polynomial of node -i (i =
    // -1..r-2) is prod_{k != i} (s + k) / (k - i); its coefficients are built
    // factor by factor (ascending powers) and integrated over [0, 1].
    for (int a = 0; a < r; ++a) {
        const int i = a - 1;
        double c[SGK_IIF_MAX_ORDER + 1] = {1.0};
        int deg = 0;
        for (int k = -1; k <= r - 2; ++k) {
            if (k == i) continue;
            for (int p = deg + 1; p >= 0; --p) c[p] = ((p > 0 ? c[p - 1] : 0.0) + k * c[p]) / (k - i);
            ++deg;
        }
        double integral = 0.0;
        for (int p = deg; p >= 0; --p) integral += c[p] / (p + 1);
        alpha[a] = integral;
    }
}

void solver_alloc(sgk_solver* s) {
    const long long n = s->n, S = s->nspecies, N = n * S;
    const int M = s->M;
    s->stats.krylov_substeps = s->ksub;
    s->U.alloc(N);
    s->Uprev.alloc(N);
    s->W.alloc(N);
    s->vv.alloc(N);
    if (s->scheme > SGK_IIF2) {
        s->Fhist.alloc((size_t)(s->scheme - 2) * N);
        s->Fstage.alloc(N);
        s->W2.alloc(N);
    }
    SGK_CUDA_CHECK(cudaMemsetAsync(s->U.p, 0, N * sizeof(double), s->ctx->stream));
    // the fused Gram-Schmidt kernels read whole 128-element slices (past n in
    // the last one, multiplied by zero): pad the basis and keep it finite
    s->V64.alloc((M + 1) * n + 128);
    SGK_CUDA_CHECK(cudaMemsetAsync(s->V64.p, 0, s->V64.n * sizeof(double), s->ctx->stream));
    s->w64.alloc(n);
    s->Hm.alloc((M + 1) * M);
    s->h1.alloc(std::max(M, s->opts.gmres_restart) + 1);
    s->h2.alloc(std::max(M, s->opts.gmres_restart) + 1);
    s->ky.alloc(M + 1);
    s->scal.alloc(16);
    const size_t nblk = std::max<size_t>(reduction_blocks(s->ctx, N), (size_t)((n + 127) / 128));
    s->partials.alloc(nblk * (std::max(M, s->opts.gmres_restart) + 1) + 16);
    s->expm_ws.alloc(8 * (size_t)M * M);
    s->ks.alloc(S);
    s->counters.alloc(4);
    s->fcnt.alloc(FC_COUNT);
    SGK_CUDA_CHECK(cudaMemsetAsync(s->fcnt.p, 0, FC_COUNT * sizeof(unsigned), s->ctx->stream));
    s->ctl.alloc(sizeof(StepCtl));
    SGK_CUDA_CHECK(cudaMallocHost(&s->hrec, SGK_ASYNC_SLOTS * sizeof(StepRecord)));
    SGK_CUDA_CHECK(cudaMemsetAsync(s->ctl.p, 0, sizeof(StepCtl), s->ctx->stream));
    // the persistent kernel's gather holds the diagonal terms only: an
    // operator with mixed-derivative terms takes the launch-sequence path
    bool cross = false;
    for (int sp = 0; sp < S; ++sp) cross = cross || s->ops[sp]->npairs > 0;
    s->persistent = std::getenv("SGK_NO_PERSISTENT") == nullptr && !cross && n <= arnoldi_persistent_max_n(s->ctx);
    if (s->persistent) {
        s->w64b.alloc(n);
        s->zbuf.alloc((size_t)(M + 1) * n);
        s->pbuf.alloc(arnoldi_persistent_pbuf_size(s->ctx, M));
        s->pbar.alloc(2 * S);
        SGK_CUDA_CHECK(cudaMemsetAsync(s->pbar.p, 0, 2 * S * sizeof(unsigned), s->ctx->stream));
        // slices of about equal work (the species share one index set)
        int64_t E = 0, lent = 0;
        const std::vector<int64_t> bnd = arnoldi_balanced_bounds(s->ctx, s->ops[0], M, &E, &lent);
        if (!bnd.empty() && E >= 1 && E <= 12 * 1024) {  // else equal slices
            s->aE = E;
            s->alist = lent;
            s->abounds.upload(bnd, s->ctx->stream);
        }
        // tune the matvec's lanes per output on this operator and size (the
        // runs use the Krylov workspace and W, which hold nothing yet)
        PersistentWork pw;
        pw.w_alt = s->w64b.p;
        pw.Z = s->zbuf.p;
        pw.pbuf = s->pbuf.p;
        pw.bar = s->pbar.p;
        pw.bounds = s->abounds.p;
        pw.E = s->aE;
        pw.list_ent = s->alist;
        s->arn_G = s->ctx->arn_G_fixed > 0
                       ? s->ctx->arn_G_fixed
                       : arnoldi_autotune(s->ctx, s->ops[0], pw, krylov_work<double>(s, 0), s->W.p, n, M);
        SGK_CUDA_CHECK(cudaMemsetAsync(s->pbar.p, 0, 2 * S * sizeof(unsigned), s->ctx->stream));
    }
    SGK_CUDA_CHECK(cudaMemsetAsync(s->counters.p, 0, 4 * sizeof(unsigned), s->ctx->stream));
    SGK_CUDA_CHECK(cudaMemsetAsync(s->Hm.p, 0, (M + 1) * M * sizeof(double), s->ctx->stream));
    if (s->has_rx && s->rform == SGK_REACTION_INTERP) {
        // the interpolation form needs no finest-grid buffers and no inner solver
        s->Fv.alloc(N);
        s->G.alloc(N);
        interp_build(s);
    } else if (s->has_rx) {
        s->Fv.alloc(N);
        s->G.alloc(N);
        s->cg_x.alloc(N);
        s->cg_r.alloc(N);
        s->cg_p.alloc(N);
        s->cg_q.alloc(N);
        const long long qsize = (2 * S + 1) * s->Q.full_size + 2 * S * n;
        // FP64 buffers for F (both modes) and, in mixed mode, FP32 buffers
        // for the Jacobian products
        s->q64.alloc(qsize);
        if (s->prec == SGK_FP64) {
            s->jw64.alloc(N);
        } else {
            s->q32.alloc(qsize);
            s->jw32.alloc(N);
        }
        if (S > 1) {
            const int R = s->opts.gmres_restart;
            s->gm_V.alloc((R + 1) * N);
            s->gm_H.alloc((R + 1) * R);
            s->gm_cs.alloc(R);
            s->gm_sn.alloc(R);
            s->gm_g.alloc(R + 1);
            s->gm_y.alloc(R);
            s->gm_report.alloc(4);
        }
    }
}

sgk_solver::~sgk_solver() {
    if (hrec) cudaFreeHost(hrec);
    for (cudaStream_t& a : aux)
        if (a) cudaStreamDestroy(a);
    for (GraphCache* g : {&g_step, &g_pre, &g_post, &g_pred, &g_pred_f, &g_resid, &g_resid0, &g_cg})
        if (g->exec) cudaGraphExecDestroy(g->exec);
    for (auto& gs : g_krylovh)
        for (auto& g : gs)
            if (g.exec) cudaGraphExecDestroy(g.exec);
    for (auto& g : g_krylov)
        if (g.exec) cudaGraphExecDestroy(g.exec);
}
