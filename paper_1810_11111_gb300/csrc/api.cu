// C ABI of libsgkiif (declared and documented in include/sgkiif.h).  Every
// entry point catches errors and turns them into a status code; the message
// is kept on the context.
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <memory>

#include "sgk_pencil.h"
#include "sgk_solver.h"

void check_launch(const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) throw SgkError{SGK_ECUDA, std::string(what) + ": " + cudaGetErrorString(e)};
}

static cudaEvent_t take_event(sgk_ctx* c) {
    if (!c->ev_pool.empty()) {
        cudaEvent_t e = c->ev_pool.back();
        c->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    SGK_CUDA_CHECK(cudaEventCreate(&e));
    return e;
}

KTimer::KTimer(sgk_ctx* c, int k) : ctx(c), kc(k) {
    if (!ctx->capturing && (ctx->prof_mask & (1u << kc))) {
        a = take_event(ctx);
        b = take_event(ctx);
        cudaEventRecord(a, ctx->stream);
    }
}

KTimer::~KTimer() {
    if (a) {
        cudaEventRecord(b, ctx->stream);
        ctx->ev_pending.push_back({kc, {a, b}});
    }
}

sgk_ctx::~sgk_ctx() {
    for (auto& p : ev_pending) {
        cudaEventDestroy(p.second.first);
        cudaEventDestroy(p.second.second);
    }
    for (auto e : ev_pool) cudaEventDestroy(e);
    if (hscal) cudaFreeHost(hscal);
    if (own_stream && stream) cudaStreamDestroy(stream);
}

void build_index_on_device(sgk_index* idx);
void index_lookup_on_device(const sgk_index* idx, const int32_t* levels, int64_t count, int64_t* out);
int64_t level_dof(int d, int N, int k);

// empty kernel whose attributes tell which device image of the library loaded
__global__ void binary_probe_kernel() {}


namespace {

template <typename F>
int guarded(sgk_ctx* ctx, F&& f) {
    try {
        int rc = f();
        if (ctx && rc == SGK_OK) ctx->last_error.clear();
        return rc;
    } catch (const SgkError& e) {
        if (ctx) ctx->last_error = e.msg;
        return e.code;
    } catch (const std::bad_alloc&) {
        if (ctx) ctx->last_error = "host allocation failed";
        return SGK_ENOMEM;
    } catch (const std::exception& e) {
        if (ctx) ctx->last_error = e.what();
        return SGK_EINVAL;
    }
}

void set_device(sgk_ctx* ctx) { SGK_CUDA_CHECK(cudaSetDevice(ctx->device)); }

}  // namespace

extern "C" {

int sgk_ctx_create(sgk_ctx** out, int device, void* cuda_stream, int precision) {
    if (!out) return SGK_EINVAL;
    *out = nullptr;
    if (precision != SGK_FP64 && precision != SGK_MIXED) return SGK_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        (void)cudaGetLastError();
        return SGK_ECUDA;
    }
    auto* c = new (std::nothrow) sgk_ctx();
    if (!c) return SGK_ENOMEM;
    c->device = device;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    c->precision = precision;
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        (void)cudaGetLastError();
        delete c;
        return SGK_ECUDA;
    }
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    c->smem_optin = (size_t)optin;
    if (cudaMallocHost(reinterpret_cast<void**>(&c->hscal), 16 * sizeof(double)) != cudaSuccess) {
        (void)cudaGetLastError();
        c->hscal = nullptr;
        delete c;
        return SGK_ENOMEM;
    }
    if (!c->stream) {
        // a blocking stream: ordered with the legacy default stream, and
        // capturable into CUDA graphs (the legacy stream itself is not)
        if (cudaStreamCreate(&c->stream) != cudaSuccess) {
            (void)cudaGetLastError();
            delete c;
            return SGK_ECUDA;
        }
        c->own_stream = true;
    }
    *out = c;
    return SGK_OK;
}

int sgk_ctx_destroy(sgk_ctx* ctx) {
    delete ctx;
    return SGK_OK;
}

const char* sgk_last_error(const sgk_ctx* ctx) { return ctx ? ctx->last_error.c_str() : "null context"; }

int64_t sgk_ctx_launch_count(const sgk_ctx* ctx) { return ctx ? ctx->launches : -1; }

int sgk_binary_arch(int* arch) {
    if (!arch) return SGK_EINVAL;
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, reinterpret_cast<const void*>(binary_probe_kernel)) != cudaSuccess) {
        (void)cudaGetLastError();
        return SGK_ECUDA;
    }
    *arch = fa.binaryVersion;
    return SGK_OK;
}

int sgk_ctx_profile(sgk_ctx* ctx, unsigned mask) {
    if (!ctx) return SGK_EINVAL;
    ctx->prof_mask = mask & ((1u << KC_COUNT) - 1);
    return SGK_OK;
}

int sgk_ctx_profile_read(sgk_ctx* ctx, double* ms, int64_t* launches) {
    if (!ctx || !ms || !launches) return SGK_EINVAL;
    return guarded(ctx, [&]() {
        set_device(ctx);
        SGK_CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
        for (int i = 0; i < KC_COUNT; ++i) {
            ms[i] = 0.0;
            launches[i] = 0;
        }
        for (auto& p : ctx->ev_pending) {
            float t = 0.f;
            SGK_CUDA_CHECK(cudaEventElapsedTime(&t, p.second.first, p.second.second));
            ms[p.first] += t;
            launches[p.first] += 1;
            ctx->ev_pool.push_back(p.second.first);
            ctx->ev_pool.push_back(p.second.second);
        }
        ctx->ev_pending.clear();
        return SGK_OK;
    });
}

int sgk_index_build(sgk_ctx* ctx, int d, int n, int k, sgk_index** out) {
    if (!ctx || !out) return SGK_EINVAL;
    *out = nullptr;
    return guarded(ctx, [&]() {
        SGK_REQUIRE(d >= 1 && d <= SGK_MAX_DIM, SGK_EINVAL, "d must be in [1, 6]");
        SGK_REQUIRE(n >= 0 && n <= SGK_MAX_LEVEL, SGK_EINVAL, "n must be in [0, 12]");
        SGK_REQUIRE(k >= 1 && k <= 3, SGK_EINVAL, "k must be in [1, 3]");
        set_device(ctx);
        std::unique_ptr<sgk_index> idx(new sgk_index());
        idx->ctx = ctx;
        idx->d = d;
        idx->n = n;
        idx->k = k;
        build_index_on_device(idx.get());
        *out = idx.release();
        return SGK_OK;
    });
}

int sgk_index_destroy(sgk_index* idx) {
    delete idx;
    return SGK_OK;
}

int64_t sgk_index_dof(const sgk_index* idx) { return idx ? idx->dof : -1; }

int64_t sgk_dof(int d, int n, int k) {
    if (d < 1 || d > SGK_MAX_DIM || n < 0 || n > SGK_MAX_LEVEL || k < 1 || k > 3) return -1;
    return level_dof(d, n, k);
}
int64_t sgk_index_ntuples(const sgk_index* idx) { return idx ? idx->ntuples : -1; }

int sgk_index_export(const sgk_index* idx, int32_t* levels, int64_t* offsets, int64_t cap) {
    if (!idx || !levels || !offsets) return SGK_EINVAL;
    return guarded(idx->ctx, [&]() {
        SGK_REQUIRE(cap >= idx->ntuples, SGK_EINVAL, "buffer too small for the tuple table");
        set_device(idx->ctx);
        // fresh copy from the device table (the host copy was taken from it too)
        SGK_CUDA_CHECK(cudaMemcpyAsync(levels, idx->d_levels.p, idx->ntuples * idx->d * sizeof(int32_t),
                                       cudaMemcpyDeviceToHost, idx->ctx->stream));
        SGK_CUDA_CHECK(cudaMemcpyAsync(offsets, idx->d_offsets.p, (idx->ntuples + 1) * sizeof(int64_t),
                                       cudaMemcpyDeviceToHost, idx->ctx->stream));
        SGK_CUDA_CHECK(cudaStreamSynchronize(idx->ctx->stream));
        return SGK_OK;
    });
}

int sgk_index_lookup(const sgk_index* idx, const int32_t* levels, int64_t count, int64_t* block_ids) {
    if (!idx || (count > 0 && (!levels || !block_ids)) || count < 0) return SGK_EINVAL;
    return guarded(idx->ctx, [&]() {
        set_device(idx->ctx);
        index_lookup_on_device(idx, levels, count, block_ids);
        return SGK_OK;
    });
}

namespace {
int operator_assemble(sgk_ctx* ctx, const sgk_index* idx, const double* kappa, const double* Kfull, int bc,
                      double sigma, sgk_op** out) {
    return guarded(ctx, [&]() {
        SGK_REQUIRE(bc == SGK_PERIODIC || bc == SGK_DIRICHLET0, SGK_EINVAL, "bc must be periodic or Dirichlet");
        SGK_REQUIRE(sigma > 0 && std::isfinite(sigma), SGK_EINVAL, "sigma must be positive");
        for (int i = 0; i < idx->d; ++i)
            SGK_REQUIRE(kappa[i] > 0 && std::isfinite(kappa[i]), SGK_EINVAL, "kappa must be positive");
        const int H = (idx->k + 1) << idx->n;
        SGK_REQUIRE(H <= 8192, SGK_EUNSUPPORTED, "1D space too large ((k+1) 2^n > 8192)");
        set_device(ctx);
        std::unique_ptr<sgk_op> op(new sgk_op());
        op->ctx = ctx;
        op->idx = idx;
        op->bc = bc;
        op->sigma = sigma;
        op->H = H;
        for (int i = 0; i < idx->d; ++i) op->kappa[i] = kappa[i];
        Tables1D tab;
        build_transform_tables(idx->n, idx->k, tab);
        op->S_dense = build_sipg_hier(tab, bc, sigma);
        Csr& S = op->S;
        S.rows = S.cols = H;
        S.ptr.assign(H + 1, 0);
        for (int a = 0; a < H; ++a) {
            for (int b = 0; b < H; ++b) {
                const double v = op->S_dense[(size_t)a * H + b];
                if (v != 0.0) {
                    S.col.push_back(b);
                    S.val.push_back(v);
                }
            }
            S.ptr[a + 1] = (int)S.col.size();
        }
        S.upload(ctx->stream);
        {
            const int nl = idx->n + 1;
            std::vector<int> rl((size_t)H * nl);
            for (int a = 0; a < H; ++a)
                for (int L = 0; L < nl; ++L) {
                    const int lim = (idx->k + 1) << L;
                    int c = 0;
                    for (int e = S.ptr[a]; e < S.ptr[a + 1] && S.col[e] < lim; ++e) ++c;
                    rl[(size_t)a * nl + L] = c;
                }
            op->rlen.upload(rl, ctx->stream);
            SGK_CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
        }
        build_gmv_tables(op.get());
        if (Kfull) {
            for (int e = 0; e < idx->d * idx->d; ++e) op->K[e] = Kfull[e];
            build_cross_tables(op.get(), Kfull);
        }
        *out = op.release();
        return SGK_OK;
    });
}
}  // namespace

int sgk_operator_assemble(sgk_ctx* ctx, const sgk_index* idx, const double* kappa, int bc, double sigma,
                          sgk_op** out) {
    if (!ctx || !idx || !kappa || !out) return SGK_EINVAL;
    *out = nullptr;
    return operator_assemble(ctx, idx, kappa, nullptr, bc, sigma, out);
}

int sgk_operator_assemble_full(sgk_ctx* ctx, const sgk_index* idx, const double* K, int bc, double sigma,
                               sgk_op** out) {
    if (!ctx || !idx || !K || !out) return SGK_EINVAL;
    *out = nullptr;
    const int d = idx->d;
    // symmetric positive definite: Cholesky on the host
    double L[SGK_MAX_DIM * SGK_MAX_DIM] = {0};
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j)
            if (!std::isfinite(K[i * d + j]) || K[i * d + j] != K[j * d + i]) {
                ctx->last_error = "K must be finite and symmetric";
                return SGK_EINVAL;
            }
    for (int j = 0; j < d; ++j) {
        double s = K[j * d + j];
        for (int m = 0; m < j; ++m) s -= L[j * d + m] * L[j * d + m];
        if (!(s > 0.0)) {
            ctx->last_error = "K must be positive definite";
            return SGK_EINVAL;
        }
        L[j * d + j] = std::sqrt(s);
        for (int i = j + 1; i < d; ++i) {
            double t = K[i * d + j];
            for (int m = 0; m < j; ++m) t -= L[i * d + m] * L[j * d + m];
            L[i * d + j] = t / L[j * d + j];
        }
    }
    double kd[SGK_MAX_DIM];
    for (int i = 0; i < d; ++i) kd[i] = K[i * d + i];
    return operator_assemble(ctx, idx, kd, K, bc, sigma, out);
}

int64_t sgk_operator_madds(const sgk_op* op) { return op ? op->madds : -1; }

int sgk_operator_destroy(sgk_op* op) {
    delete op;
    return SGK_OK;
}

int sgk_operator_export_1d(const sgk_op* op, double* out, int64_t cap) {
    if (!op || !out) return SGK_EINVAL;
    return guarded(op->ctx, [&]() {
        SGK_REQUIRE(cap >= (int64_t)op->H * op->H, SGK_EINVAL, "buffer too small");
        // reconstruct from the uploaded CSR so that the export shows what the kernels use
        std::vector<int> ptr(op->H + 1), col(op->S.col.size());
        std::vector<double> val(op->S.val.size());
        set_device(op->ctx);
        SGK_CUDA_CHECK(cudaMemcpyAsync(ptr.data(), op->S.d_ptr.p, ptr.size() * sizeof(int), cudaMemcpyDeviceToHost,
                                       op->ctx->stream));
        SGK_CUDA_CHECK(cudaMemcpyAsync(col.data(), op->S.d_col.p, col.size() * sizeof(int), cudaMemcpyDeviceToHost,
                                       op->ctx->stream));
        SGK_CUDA_CHECK(cudaMemcpyAsync(val.data(), op->S.d_val.p, val.size() * sizeof(double),
                                       cudaMemcpyDeviceToHost, op->ctx->stream));
        SGK_CUDA_CHECK(cudaStreamSynchronize(op->ctx->stream));
        std::memset(out, 0, sizeof(double) * op->H * op->H);
        for (int a = 0; a < op->H; ++a)
            for (int e = ptr[a]; e < ptr[a + 1]; ++e) out[(size_t)a * op->H + col[e]] = val[e];
        return SGK_OK;
    });
}

int sgk_cross_blocks_1d(int n, int k, int bc, double* P, double* E, int64_t cap) {
    if (!P || !E || n < 0 || n > 10 || k < 1 || k > 3 || (bc != SGK_PERIODIC && bc != SGK_DIRICHLET0))
        return SGK_EINVAL;
    const int64_t H = (int64_t)(k + 1) << n;
    if (cap < H * H) return SGK_EINVAL;
    try {
        Tables1D tab;
        build_transform_tables(n, k, tab);
        std::vector<double> p, e;
        build_cross_hier(tab, bc, p, e);
        std::memcpy(P, p.data(), sizeof(double) * H * H);
        std::memcpy(E, e.data(), sizeof(double) * H * H);
    } catch (...) {
        return SGK_ENOMEM;
    }
    return SGK_OK;
}

int sgk_interp_factors_1d(int n, int k, int which, double* out, int64_t cap) {
    if (!out || n < 0 || n > 10 || k < 1 || k > 3 || which < 0 || which > 3) return SGK_EINVAL;
    const int64_t H = (int64_t)(k + 1) << n;
    if (cap < H * H) return SGK_EINVAL;
    try {
        InterpFactors1D F;
        build_interp_factors(n, k, F);
        const Csr* M[4] = {&F.A, &F.B, &F.Binv, &F.Ainv};
        std::memset(out, 0, sizeof(double) * H * H);
        for (int a = 0; a < H; ++a)
            for (int e = M[which]->ptr[a]; e < M[which]->ptr[a + 1]; ++e) out[a * H + M[which]->col[e]] = M[which]->val[e];
    } catch (const SgkError& e) {
        return e.code;
    } catch (...) {
        return SGK_ENOMEM;
    }
    return SGK_OK;
}

int sgk_matvec(const sgk_op* op, const void* x_dev, void* y_dev, int precision) {
    if (!op || !x_dev || !y_dev || x_dev == y_dev) return SGK_EINVAL;
    return guarded(op->ctx, [&]() {
        set_device(op->ctx);
        if (precision == SGK_FP64)
            op_matvec<double>(op, static_cast<const double*>(x_dev), static_cast<double*>(y_dev));
        else if (precision == SGK_MIXED)
            op_matvec<float>(op, static_cast<const float*>(x_dev), static_cast<float*>(y_dev));
        else
            throw SgkError{SGK_EINVAL, "precision must be SGK_FP64 or SGK_MIXED"};
        return SGK_OK;
    });
}

int sgk_project_separable(sgk_ctx* ctx, const sgk_index* idx, int nterms, const double* amp, const int* wavenum,
                          const int* kind, double const_term, double* coeffs_dev) {
    if (!ctx || !idx || !coeffs_dev || nterms < 0 || (nterms > 0 && (!amp || !wavenum || !kind))) return SGK_EINVAL;
    return guarded(ctx, [&]() {
        for (int t = 0; t < nterms * idx->d; ++t) {
            SGK_REQUIRE(kind[t] == 0 || kind[t] == 1, SGK_EINVAL, "kind must be 0 (sin) or 1 (cos)");
        }
        set_device(ctx);
        Tables1D tab;
        build_transform_tables(idx->n, idx->k, tab);
        tab.Tt.upload(ctx->stream);
        project_separable_dev(ctx, idx, tab, nterms, amp, wavenum, kind, const_term, coeffs_dev);
        return SGK_OK;
    });
}

int sgk_dirichlet_load(sgk_ctx* ctx, const sgk_index* idx, const double* kappa, double sigma, int nterms,
                       const double* amp, const int* wavenum, const int* kind, double const_term, double* b_dev) {
    if (!ctx || !idx || !kappa || !b_dev || nterms < 0 || (nterms > 0 && (!amp || !wavenum || !kind))) return SGK_EINVAL;
    return guarded(ctx, [&]() {
        SGK_REQUIRE(sigma > 0.0, SGK_EINVAL, "sigma must be positive");
        for (int i = 0; i < idx->d; ++i) SGK_REQUIRE(kappa[i] > 0.0, SGK_EINVAL, "kappa must be positive");
        for (int t = 0; t < nterms * idx->d; ++t)
            SGK_REQUIRE(kind[t] == 0 || kind[t] == 1, SGK_EINVAL, "kind must be 0 (sin) or 1 (cos)");
        set_device(ctx);
        Tables1D tab;
        build_transform_tables(idx->n, idx->k, tab);
        tab.Tt.upload(ctx->stream);
        dirichlet_load_dev(ctx, idx, tab, kappa, sigma, nterms, amp, wavenum, kind, const_term, b_dev);
        return SGK_OK;
    });
}

int sgk_solver_create(sgk_ctx* ctx, int nspecies, const sgk_op* const* ops, const sgk_reaction* f, int scheme,
                      int krylov_m, double dt, const sgk_newton_opts* opts, sgk_solver** out) {
    return sgk_solver_create_form(ctx, nspecies, ops, f, scheme, krylov_m, dt, opts, SGK_REACTION_QUADRATURE, out);
}

int sgk_solver_create_form(sgk_ctx* ctx, int nspecies, const sgk_op* const* ops, const sgk_reaction* f, int scheme,
                           int krylov_m, double dt, const sgk_newton_opts* opts, int reaction_form,
                           sgk_solver** out) {
    if (!ctx || !ops || !out) return SGK_EINVAL;
    *out = nullptr;
    if (reaction_form != SGK_REACTION_QUADRATURE && reaction_form != SGK_REACTION_INTERP) return SGK_EINVAL;
    return guarded(ctx, [&]() {
        SGK_REQUIRE(nspecies >= 1 && nspecies <= SGK_MAX_SPECIES, SGK_EINVAL, "nspecies must be in [1, 4]");
        SGK_REQUIRE(scheme >= SGK_IIF2 && scheme <= SGK_IIF_MAX_ORDER, SGK_EUNSUPPORTED,
                    "scheme must be an IIF order in [2, 6]");
        SGK_REQUIRE(krylov_m >= 1 && krylov_m <= SGK_MAX_KRYLOV, SGK_EINVAL, "krylov_m must be in [1, 128]");
        SGK_REQUIRE(dt > 0 && std::isfinite(dt), SGK_EINVAL, "dt must be positive");
        const sgk_index* idx = nullptr;
        for (int s = 0; s < nspecies; ++s) {
            SGK_REQUIRE(ops[s] != nullptr, SGK_EINVAL, "null operator");
            SGK_REQUIRE(ops[s]->ctx == ctx, SGK_EINVAL, "operator from another context");
            if (!idx) idx = ops[s]->idx;
            SGK_REQUIRE(ops[s]->idx == idx, SGK_EINVAL, "operators on different index sets");
        }
        set_device(ctx);
        std::unique_ptr<sgk_solver> s(new sgk_solver());
        static std::atomic<uint64_t> next_uid{1};
        s->uid = next_uid.fetch_add(1);
        s->ctx = ctx;
        s->idx = idx;
        s->nspecies = nspecies;
        for (int i = 0; i < nspecies; ++i) s->ops[i] = ops[i];
        s->M = krylov_m;
        s->dt = dt;
        s->scheme = scheme;
        s->newton_c = 0.5 * dt;
        s->prec = ctx->precision;
        s->n = idx->dof;
        s->rx.nspecies = nspecies;
        s->rx.nmono = 0;
        if (f && f->nmono > 0) {
            SGK_REQUIRE(f->nspecies == nspecies, SGK_EINVAL, "reaction species count mismatch");
            SGK_REQUIRE(f->nmono <= SGK_MAX_MONO, SGK_EUNSUPPORTED, "at most 16 monomials");
            SGK_REQUIRE(f->species && f->coef && f->exps, SGK_EINVAL, "null reaction arrays");
            s->rx.nmono = f->nmono;
            for (int m = 0; m < f->nmono; ++m) {
                SGK_REQUIRE(f->species[m] >= 0 && f->species[m] < nspecies, SGK_EINVAL, "bad monomial species");
                s->rx.species[m] = f->species[m];
                s->rx.coef[m] = f->coef[m];
                for (int r = 0; r < nspecies; ++r) {
                    const int e = f->exps[m * nspecies + r];
                    SGK_REQUIRE(e >= 0 && e <= 4, SGK_EINVAL, "exponents must be in [0, 4]");
                    s->rx.exps[m][r] = e;
                }
            }
        }
        s->has_rx = s->rx.nmono > 0;
        s->use_graphs = std::getenv("SGK_NO_GRAPHS") == nullptr;
        const bool fp64 = s->prec == SGK_FP64;
        // the oracle's outer tolerance in both modes (F is FP64-accurate in
        // both); the mixed inner solve, whose Jacobian products are FP32,
        // stops at 1e-6: a tighter solve of an FP32 operator buys nothing
        s->opts.tol = 1e-12;
        s->opts.max_iter = 50;
        s->opts.inner_tol = fp64 ? 1e-13 : 1e-6;
        s->opts.inner_max = 500;
        s->opts.gmres_restart = 50;
        if (opts) {
            if (opts->tol > 0) s->opts.tol = opts->tol;
            if (opts->max_iter > 0) s->opts.max_iter = opts->max_iter;
            if (opts->inner_tol > 0) s->opts.inner_tol = opts->inner_tol;
            if (opts->inner_max > 0) s->opts.inner_max = opts->inner_max;
            if (opts->gmres_restart > 0) s->opts.gmres_restart = std::min(opts->gmres_restart, SGK_MAX_KRYLOV);
        }
        s->rform = reaction_form;
        if (s->has_rx && reaction_form != SGK_REACTION_INTERP) {
            const int p = reaction_degree(s->rx);
            const int k = idx->k;
            const int q = std::max(1, (p * k + k + 1 + 1) / 2);
            SGK_REQUIRE(q <= 8, SGK_EUNSUPPORTED, "reaction degree too high for the quadrature tables");
            quad_build(s->Q, idx, q, nspecies, true);
            s->Q.fused = pencil_supported(idx->d, idx->k + 1, q, nspecies, s->rx) && std::getenv("SGK_NO_FUSED") == nullptr;
            const size_t elem = fp64 ? 8 : 4;
            const double need = (double)((2 * nspecies + 1) * s->Q.full_size) * elem;
            size_t free_b = 0, total_b = 0;
            SGK_CUDA_CHECK(cudaMemGetInfo(&free_b, &total_b));
            SGK_REQUIRE(need < 0.9 * (double)free_b, SGK_ENOMEM, "finest full grid does not fit in device memory");
        }
        solver_alloc(s.get());
        SGK_CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
        *out = s.release();
        return SGK_OK;
    });
}

int sgk_solver_destroy(sgk_solver* s) {
    if (s) {
        cudaSetDevice(s->ctx->device);
        cudaStreamSynchronize(s->ctx->stream);
    }
    delete s;
    return SGK_OK;
}

int sgk_solver_set_state(sgk_solver* s, int species, const double* coeffs, int on_device) {
    if (!s || !coeffs) return SGK_EINVAL;
    return guarded(s->ctx, [&]() {
        SGK_REQUIRE(species >= 0 && species < s->nspecies, SGK_EINVAL, "bad species");
        set_device(s->ctx);
        solver_drain(s);
        const double* src = coeffs;
        if (!on_device) {  // staged in the predictor's buffer (free between steps)
            SGK_CUDA_CHECK(cudaMemcpyAsync(s->vv.p + species * s->n, coeffs, s->n * sizeof(double),
                                           cudaMemcpyHostToDevice, s->ctx->stream));
            src = s->vv.p + species * s->n;
        }
        solver_set_state(s, species, src);
        if (!on_device) SGK_CUDA_CHECK(cudaStreamSynchronize(s->ctx->stream));
        return SGK_OK;
    });
}

int sgk_solver_step(sgk_solver* s, int nsteps) {
    if (!s || nsteps < 0) return SGK_EINVAL;
    return guarded(s->ctx, [&]() {
        set_device(s->ctx);
        solver_drain(s);
        int rc = s->async_rc;  // a queued step failed: report it before stepping on
        s->async_rc = SGK_OK;
        if (rc == SGK_OK) rc = solver_step(s, nsteps);
        if (rc == SGK_ENEWTON) s->ctx->last_error = "Newton did not converge; state rolled back";
        SGK_CUDA_CHECK(cudaStreamSynchronize(s->ctx->stream));
        if (rc != SGK_OK) throw SgkError{rc, s->ctx->last_error};
        return SGK_OK;
    });
}

int sgk_solver_get_state(const sgk_solver* s, int species, double* out, int64_t cap, int on_device) {
    if (!s || !out) return SGK_EINVAL;
    return guarded(s->ctx, [&]() {
        SGK_REQUIRE(species >= 0 && species < s->nspecies, SGK_EINVAL, "bad species");
        SGK_REQUIRE(cap >= s->n, SGK_EINVAL, "buffer too small");
        set_device(s->ctx);
        solver_drain(const_cast<sgk_solver*>(s));
        SGK_CUDA_CHECK(cudaMemcpyAsync(out, s->U.p + species * s->n, s->n * sizeof(double),
                                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                       s->ctx->stream));
        if (!on_device) SGK_CUDA_CHECK(cudaStreamSynchronize(s->ctx->stream));
        return SGK_OK;
    });
}

int sgk_solver_stats(const sgk_solver* s, sgk_stats* out) {
    if (!s || !out) return SGK_EINVAL;
    return guarded(s->ctx, [&]() {
        set_device(s->ctx);
        solver_drain(const_cast<sgk_solver*>(s));
        *out = s->stats;
        out->krylov_substeps = s->ksub;
        return SGK_OK;
    });
}

int sgk_solver_step_async(sgk_solver* s, int nsteps) {
    if (!s || nsteps < 0) return SGK_EINVAL;
    return guarded(s->ctx, [&]() {
        set_device(s->ctx);
        const int rc = solver_step_async(s, nsteps);  // the synchronous fallback reports at once
        if (rc == SGK_ENEWTON) s->ctx->last_error = "Newton did not converge; state rolled back";
        if (rc != SGK_OK) throw SgkError{rc, s->ctx->last_error};
        return SGK_OK;
    });
}

int sgk_solver_wait(sgk_solver* s) {
    if (!s) return SGK_EINVAL;
    return guarded(s->ctx, [&]() {
        set_device(s->ctx);
        solver_drain(s);
        const int rc = s->async_rc;
        s->async_rc = SGK_OK;
        if (rc != SGK_OK)
            throw SgkError{rc, rc == SGK_ENEWTON ? "Newton did not converge; state rolled back"
                                                 : "a queued step failed; state rolled back"};
        return SGK_OK;
    });
}

int sgk_iif_alpha(int r, double* alpha) {
    if (r < 2 || r > SGK_IIF_MAX_ORDER || !alpha) return SGK_EINVAL;
    iif_alpha(r, alpha);
    return SGK_OK;
}

int sgk_solver_set_source(sgk_solver* s, int species, int nterms, const double* lambda, const double* coeffs_dev) {
    if (!s) return SGK_EINVAL;
    return guarded(s->ctx, [&]() {
        SGK_REQUIRE(species >= 0 && species < s->nspecies, SGK_EINVAL, "bad species");
        SGK_REQUIRE(nterms >= 0 && nterms <= SGK_MAX_SOURCE_TERMS, SGK_EINVAL, "nterms must be in [0, 8]");
        SGK_REQUIRE(nterms == 0 || (lambda && coeffs_dev), SGK_EINVAL, "null source arrays");
        for (int m = 0; m < nterms; ++m) SGK_REQUIRE(std::isfinite(lambda[m]), SGK_EINVAL, "non-finite lambda");
        SGK_REQUIRE(nterms == 0 || s->has_rx, SGK_EUNSUPPORTED, "a source term needs a reaction term");
        set_device(s->ctx);
        solver_drain(s);
        solver_set_source(s, species, nterms, lambda, coeffs_dev);
        SGK_CUDA_CHECK(cudaStreamSynchronize(s->ctx->stream));
        return SGK_OK;
    });
}

int sgk_solver_set_time(sgk_solver* s, double t) {
    if (!s) return SGK_EINVAL;
    return guarded(s->ctx, [&]() {
        SGK_REQUIRE(std::isfinite(t), SGK_EINVAL, "non-finite time");
        set_device(s->ctx);
        solver_drain(s);
        solver_set_time(s, t);
        return SGK_OK;
    });
}

int sgk_solver_set_krylov_substeps(sgk_solver* s, int substeps) {
    if (!s) return SGK_EINVAL;
    return guarded(s->ctx, [&]() {
        SGK_REQUIRE(substeps >= 1 && substeps <= SGK_MAX_KRYLOV_SUBSTEPS, SGK_EINVAL,
                    "krylov substeps must be 1..SGK_MAX_KRYLOV_SUBSTEPS");
        set_device(s->ctx);
        solver_drain(s);
        solver_set_krylov_substeps(s, substeps);
        return SGK_OK;
    });
}

int sgk_solver_set_krylov_tolerance(sgk_solver* s, double tol, int max_substeps) {
    if (!s) return SGK_EINVAL;
    return guarded(s->ctx, [&]() {
        SGK_REQUIRE(std::isfinite(tol) && tol >= 0.0, SGK_EINVAL, "krylov tolerance must be finite and >= 0");
        SGK_REQUIRE(max_substeps >= 1 && max_substeps <= SGK_MAX_KRYLOV_SUBSTEPS, SGK_EINVAL,
                    "max substeps must be 1..SGK_MAX_KRYLOV_SUBSTEPS");
        set_device(s->ctx);
        solver_drain(s);
        s->ktol = tol;
        s->kmax = max_substeps;
        return SGK_OK;
    });
}

int sgk_solver_get_time(const sgk_solver* s, double* t) {
    if (!s || !t) return SGK_EINVAL;
    return guarded(s->ctx, [&]() {
        set_device(s->ctx);
        solver_drain(const_cast<sgk_solver*>(s));  // queued steps advance the time when they finish
        *t = s->t;
        return SGK_OK;
    });
}

int sgk_reaction_eval(sgk_solver* s, const double* u_dev, double* f_dev) {
    if (!s || !u_dev || !f_dev) return SGK_EINVAL;
    return guarded(s->ctx, [&]() {
        set_device(s->ctx);
        solver_drain(s);
        solver_eval_reaction(s, u_dev, f_dev);
        return SGK_OK;
    });
}

int sgk_jacobian_apply(sgk_solver* s, const double* u_dev, const double* w_dev, double* jw_dev) {
    if (!s || !u_dev || !w_dev || !jw_dev) return SGK_EINVAL;
    return guarded(s->ctx, [&]() {
        set_device(s->ctx);
        solver_drain(s);
        solver_jacobian_apply(s, u_dev, w_dev, jw_dev);
        return SGK_OK;
    });
}

int sgk_krylov_expv(sgk_solver* s, int species, const double* v_dev, double* w_dev, int* m_eff) {
    if (!s || !v_dev || !w_dev) return SGK_EINVAL;
    return guarded(s->ctx, [&]() {
        SGK_REQUIRE(species >= 0 && species < s->nspecies, SGK_EINVAL, "bad species");
        set_device(s->ctx);
        solver_drain(s);
        solver_krylov_expv(s, species, v_dev, w_dev);
        KrylovScalars ks{};
        unsigned flags[2] = {0u, 0u};
        SGK_CUDA_CHECK(cudaMemcpyAsync(&ks, s->ks.p + species, sizeof(ks), cudaMemcpyDeviceToHost, s->ctx->stream));
        if (s->persistent)
            SGK_CUDA_CHECK(cudaMemcpyAsync(flags, s->pbar.p + 2 * species, sizeof(flags), cudaMemcpyDeviceToHost,
                                           s->ctx->stream));
        SGK_CUDA_CHECK(cudaStreamSynchronize(s->ctx->stream));
        if (m_eff) *m_eff = ks.m_eff;
        if (flags[1] != 0u) {  // a grid barrier of the persistent kernel ran out of time
            SGK_CUDA_CHECK(cudaMemsetAsync(s->pbar.p + 2 * species, 0, 2 * sizeof(unsigned), s->ctx->stream));
            SGK_CUDA_CHECK(cudaStreamSynchronize(s->ctx->stream));
            throw SgkError{SGK_ETIMEOUT, "persistent Arnoldi: a grid barrier wait ran out"};
        }
        return SGK_OK;
    });
}

int sgk_krylov_export(const sgk_solver* s, double* H, double* V, int64_t cap_V) {
    if (!s) return SGK_EINVAL;
    return guarded(s->ctx, [&]() {
        set_device(s->ctx);
        solver_drain(const_cast<sgk_solver*>(s));
        const long long n = s->n;
        const int M = s->M;
        if (H)
            SGK_CUDA_CHECK(cudaMemcpyAsync(H, s->Hm.p, (size_t)(M + 1) * M * sizeof(double), cudaMemcpyDeviceToHost,
                                           s->ctx->stream));
        if (V) {
            SGK_REQUIRE(cap_V >= (M + 1) * n, SGK_EINVAL, "buffer too small for the basis");
            SGK_CUDA_CHECK(cudaMemcpyAsync(V, s->V64.p, (size_t)(M + 1) * n * sizeof(double), cudaMemcpyDeviceToHost,
                                           s->ctx->stream));
        }
        SGK_CUDA_CHECK(cudaStreamSynchronize(s->ctx->stream));
        return SGK_OK;
    });
}

int sgk_expm_e1(sgk_ctx* ctx, int m, const double* X, double tau, double* y) {
    if (!ctx || !X || !y || m < 1 || m > SGK_MAX_KRYLOV) return SGK_EINVAL;
    return guarded(ctx, [&]() {
        set_device(ctx);
        DevBuf<double> dX((size_t)m * m), ws(8 * (size_t)m * m), dy(m);
        dX.upload(X, (size_t)m * m, ctx->stream);
        expm_e1(ctx, dX.p, m, nullptr, m, tau, ws.p, dy.p);
        SGK_CUDA_CHECK(cudaMemcpyAsync(y, dy.p, m * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        SGK_CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
        return SGK_OK;
    });
}

}  // extern "C"
