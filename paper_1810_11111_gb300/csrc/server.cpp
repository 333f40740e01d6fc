// Request loop around the IIF2 solver: continuous batching of whole solves
// on one GPU (the service around the method; the paper has no counterpart).
//
// Submitted requests wait in a FIFO.  The dispatcher admits a request when a
// worker is idle and the request's estimated device memory fits in the budget
// left by the running ones; a request that does not fit is overtaken by later
// ones that do, until it has waited longer than the aging limit, after which
// nothing behind it is admitted until it runs.  Each worker thread owns a
// CUDA stream and one library context per precision on it, builds the index
// set, operators and solver of its request, takes the steps, copies the
// state to the host and frees everything, so admitted requests overlap on
// the GPU through their streams and keep their Krylov bases and state on the
// device for their whole run.  The persistent Arnoldi kernel of each worker
// gets an equal share of the SMs, so that the cooperative grids of all
// workers fit on the device together.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "sgk_batchcore.h"
#include "sgk_internal.h"
#include "sgk_quad.h"

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

struct InitCopy {
    std::vector<double> coeffs;
    std::vector<double> amp;
    std::vector<int> wavenum, kind;
    double const_term = 0.0;
};

struct Req {
    int64_t ticket = 0;
    int d = 0, n = 0, k = 0, S = 1, bc = SGK_PERIODIC, M = 0, nsteps = 0, prec = SGK_FP64;
    double dt = 0.0;
    double ktol = 0.0;  // Krylov accuracy guard (0: off) and its limit
    int kmax = 1;
    int form = SGK_REACTION_QUADRATURE;  // form of the reaction term
    std::vector<double> kappa;  // S x d
    int nmono = 0;
    std::vector<int> rx_species, rx_exps;
    std::vector<double> rx_coef;
    InitCopy init[SGK_MAX_SPECIES];
    int64_t est = 0;
    Clock::time_point t_submit, t_admit, t_done;
    bool done = false;
    sgk_result_info info{};
    std::vector<double> result;
};


}  // namespace

// sum over level tuples |l|_1 <= N of prod_m (k+1) 2^{max(l_m - 1, 0)}
int64_t level_dof(int d, int N, int k) {
    std::vector<int64_t> cnt(N + 1, 0);  // cnt[s]: dof of tuples with sum s, built dimension by dimension
    cnt[0] = 1;
    for (int m = 0; m < d; ++m) {
        std::vector<int64_t> nxt(N + 1, 0);
        for (int s = 0; s <= N; ++s)
            if (cnt[s])
                for (int l = 0; s + l <= N; ++l) nxt[s + l] += cnt[s] * level_count(l, k + 1);
        cnt.swap(nxt);
    }
    int64_t t = 0;
    for (int64_t c : cnt) t += c;
    return t;
}

extern "C" double sgk_estimate_work(int d, int n, int k, int nspecies, int krylov_m, int has_reaction) {
    if (d < 1 || d > SGK_MAX_DIM || n < 0 || n > SGK_MAX_LEVEL || k < 1 || k > 3 || nspecies < 1 ||
        nspecies > SGK_MAX_SPECIES || krylov_m < 1 || krylov_m > SGK_MAX_KRYLOV)
        return -1.0;
    const double dof = (double)level_dof(d, n, k), M = krylov_m, kp1 = k + 1;
    // a row of the 1D matrix along one direction visits about 13 entries
    // (measured on the index sets of this library's workloads)
    double w = M * (2.0 * 13.0 * d * dof) + 4.0 * M * M * dof;
    if (has_reaction == 2) {
        // the interpolation form: per step about three applications of the
        // collocation transforms (2d passes each of 1D rows of about (k+1)(n+2)
        // entries) and the pointwise solve
        w += 3.0 * 2.0 * (2.0 * d) * kp1 * (n + 2.0) * dof + 40.0 * dof;
    } else if (has_reaction) {
        const double cells = std::pow(2.0, (double)n * d);
        const int q = 2 * k + 1;  // Gauss points of a cubic reaction, ceil((3k + k + 1) / 2)
        double per_cell = 0.0;  // sum-factorised stages, forward and back
        for (int m = 0; m < d; ++m) per_cell += 2.0 * std::pow((double)q, m + 1) * std::pow(kp1, d - m);
        w += 3.0 * 2.0 * cells * per_cell;
    }
    return w * nspecies;
}

extern "C" int sgk_partition(int count, const double* cost, int nparts, int* part_of) {
    if (count < 0 || nparts < 1 || (count > 0 && (!cost || !part_of))) return SGK_EINVAL;
    std::vector<int> order(count);
    for (int i = 0; i < count; ++i) {
        if (!(cost[i] >= 0.0) || !std::isfinite(cost[i])) return SGK_EINVAL;
        order[i] = i;
    }
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    std::vector<double> load(nparts, 0.0);
    for (int i : order) {
        int best = 0;
        for (int p = 1; p < nparts; ++p)
            if (load[p] < load[best]) best = p;
        part_of[i] = best;
        load[best] += cost[i];
    }
    return SGK_OK;
}

struct sgk_server {
    int device = 0;
    int nworkers = 0;
    int64_t budget = 0;
    double aging_ms = 2000.0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Req>> queue;
    std::unordered_map<int64_t, std::shared_ptr<Req>> tickets;
    std::vector<std::shared_ptr<Req>> slot;  // request assigned to each worker
    std::vector<std::thread> threads;
    bool stopping = false;
    int64_t next_ticket = 1;
    int64_t reserved = 0, peak_reserved = 0;
    int64_t submitted = 0, completed = 0, failed = 0, rejected = 0;
    int running = 0, max_concurrent = 0;
    // the engine: single-species requests (d 2..4) stepped together, one
    // batch step of all of them per tick (batch_core_tick), joining and
    // leaving at tick boundaries
    bool engine_on = true;
    int eng_max = 64;                           // most requests in the engine at once
    std::deque<std::shared_ptr<Req>> eng_new;   // admitted, not yet set up
    int eng_count = 0;                          // admitted to the engine and not finished
    std::condition_variable cv_eng;
    std::thread eng_thread;

    static bool engine_eligible(const Req& r) { return r.S == 1 && r.d >= 2 && r.d <= 4; }

    // under mu: admit queued requests in arrival order, each to the engine
    // (when eligible and it has room) or to an idle worker, while its
    // memory estimate fits what the running requests leave of the budget;
    // a request that does not fit is overtaken by later ones until it has
    // waited past the aging limit, after which it blocks everything behind it
    void admit_locked() {
        const auto now = Clock::now();
        for (auto it = queue.begin(); it != queue.end();) {
            const std::shared_ptr<Req> r = *it;
            const bool fits = reserved + r->est <= budget;
            const bool eng = engine_on && engine_eligible(*r);
            int w = -1;
            if (!eng)
                for (int i = 0; i < nworkers && w < 0; ++i)
                    if (!slot[i]) w = i;
            const bool room = eng ? eng_count < eng_max : w >= 0;
            if (fits && room) {
                it = queue.erase(it);
                r->t_admit = now;
                reserved += r->est;
                peak_reserved = std::max(peak_reserved, reserved);
                ++running;
                max_concurrent = std::max(max_concurrent, running);
                if (eng) {
                    eng_new.push_back(r);
                    ++eng_count;
                } else {
                    slot[w] = r;
                }
                continue;
            }
            if (!fits && ms_between(r->t_submit, now) > aging_ms) break;
            ++it;
        }
        cv_work.notify_all();
        cv_eng.notify_all();
    }

    // under mu: a request's outcome, its memory back to the budget, the
    // next admissions
    void finish_locked(const std::shared_ptr<Req>& r, int rc, const std::string& err, int worker) {
        r->info.status = rc;
        r->info.worker = worker;
        std::snprintf(r->info.error, sizeof(r->info.error), "%s", err.c_str());
        r->t_done = Clock::now();
        r->info.queue_ms = ms_between(r->t_submit, r->t_admit);
        r->info.run_ms = ms_between(r->t_admit, r->t_done);
        r->info.latency_ms = ms_between(r->t_submit, r->t_done);
        r->done = true;
        reserved -= r->est;
        --running;
        ++completed;
        if (rc != SGK_OK) ++failed;
        admit_locked();
    }

    void worker(int w);
    void engine();
};

namespace {

int run_request(sgk_ctx* ctx, Req& r, std::string& err) {
    sgk_index* idx = nullptr;
    sgk_op* ops[SGK_MAX_SPECIES] = {nullptr};
    sgk_solver* sol = nullptr;
    DevBuf<double> u0;
    // the first failing call's status and text (later calls reset the text)
    auto chk = [&](int code) {
        if (code != SGK_OK && err.empty()) err = ctx->last_error.empty() ? "status " + std::to_string(code)
                                                                         : ctx->last_error;
        return code;
    };
    int rc = chk(sgk_index_build(ctx, r.d, r.n, r.k, &idx));
    if (rc == SGK_OK) {
        for (int s = 0; s < r.S && rc == SGK_OK; ++s)
            rc = chk(sgk_operator_assemble(ctx, idx, &r.kappa[(size_t)s * r.d], r.bc, 20.0, &ops[s]));
    }
    if (rc == SGK_OK) {
        sgk_reaction f{};
        f.nspecies = r.S;
        f.nmono = r.nmono;
        f.species = r.rx_species.data();
        f.coef = r.rx_coef.data();
        f.exps = r.rx_exps.data();
        rc = chk(sgk_solver_create_form(ctx, r.S, ops, &f, SGK_IIF2, r.M, r.dt, nullptr, r.form, &sol));
        if (rc == SGK_OK && r.ktol > 0.0) rc = chk(sgk_solver_set_krylov_tolerance(sol, r.ktol, r.kmax));
    }
    const int64_t dof = idx ? idx->dof : 0;
    if (rc == SGK_OK) {
        try {
            u0.alloc(dof);
        } catch (const SgkError& e) {
            rc = e.code;
            err = e.msg;
        }
    }
    for (int s = 0; s < r.S && rc == SGK_OK; ++s) {
        const InitCopy& in = r.init[s];
        if (!in.coeffs.empty()) {
            rc = (int64_t)in.coeffs.size() == dof ? chk(sgk_solver_set_state(sol, s, in.coeffs.data(), 0))
                                                  : chk(SGK_EINVAL);
        } else {
            rc = chk(sgk_project_separable(ctx, idx, (int)in.amp.size(), in.amp.data(), in.wavenum.data(),
                                           in.kind.data(), in.const_term, u0.p));
            if (rc == SGK_OK) rc = chk(sgk_solver_set_state(sol, s, u0.p, 1));
        }
    }
    if (rc == SGK_OK) rc = chk(sgk_solver_step(sol, r.nsteps));
    if (sol) {
        sgk_stats st{};
        sgk_solver_stats(sol, &st);
        r.info.steps = st.steps;
        r.info.newton_iters = st.newton_iters;
        r.info.krylov_err_est = st.max_krylov_err_est;
        r.info.inner_iters = st.inner_iters;
        if (rc == SGK_OK) {
            r.result.resize((size_t)r.S * dof);
            for (int s = 0; s < r.S && rc == SGK_OK; ++s)
                rc = chk(sgk_solver_get_state(sol, s, r.result.data() + (size_t)s * dof, dof, 0));
        }
    }
    r.info.dof = dof;
    sgk_solver_destroy(sol);
    for (int s = 0; s < r.S; ++s) sgk_operator_destroy(ops[s]);
    sgk_index_destroy(idx);
    return rc;
}

}  // namespace

void sgk_server::worker(int w) {
    cudaSetDevice(device);
    cudaStream_t stream = nullptr;
    sgk_ctx* ctx[2] = {nullptr, nullptr};
    bool ok = cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) == cudaSuccess;
    // this thread's device buffers are stream-ordered on its own stream, so
    // that freeing one request's memory does not wait for the other workers
    if (ok) alloc_stream() = stream;
    ok = ok && sgk_ctx_create(&ctx[0], device, stream, SGK_FP64) == SGK_OK;
    ok = ok && sgk_ctx_create(&ctx[1], device, stream, SGK_MIXED) == SGK_OK;
    if (ok)
        for (sgk_ctx* c : ctx) c->persist_ctas = std::max(1, c->num_sms / nworkers);
    for (;;) {
        std::shared_ptr<Req> r;
        {
            std::unique_lock<std::mutex> lk(mu);
            cv_work.wait(lk, [&] { return slot[w] != nullptr || (stopping && queue.empty()); });
            if (!slot[w]) break;
            r = slot[w];
        }
        int rc = SGK_ECUDA;
        std::string err = ok ? "" : "worker could not create its stream or contexts";
        if (ok) {
            sgk_ctx* c = ctx[r->prec == SGK_MIXED ? 1 : 0];
            c->last_error.clear();
            try {
                rc = run_request(c, *r, err);
            } catch (const std::exception& e) {
                rc = SGK_ECUDA;
                err = e.what();
            } catch (...) {
                rc = SGK_ECUDA;
                err = "unknown exception";
            }
        }
        {
            std::lock_guard<std::mutex> lk(mu);
            slot[w] = nullptr;
            finish_locked(r, rc, err, w);
        }
        cv_done.notify_all();
    }
    for (sgk_ctx* c : ctx) sgk_ctx_destroy(c);
    if (stream) cudaStreamDestroy(stream);
}

namespace {

// A request in the engine: its own context (on one of the engine's
// streams), index set, operator and solver, and the steps taken so far.
struct Live {
    std::shared_ptr<Req> r;
    sgk_ctx* ctx = nullptr;
    sgk_index* idx = nullptr;
    sgk_op* op = nullptr;
    sgk_solver* sol = nullptr;
    int64_t done = 0;
    ~Live() {
        sgk_solver_destroy(sol);
        sgk_operator_destroy(op);
        sgk_index_destroy(idx);
        sgk_ctx_destroy(ctx);
    }
};

// Sets a request up on stream st; SGK_OK or the failing call's status.
int engine_setup(int device, cudaStream_t st, Live& L, std::string& err, int num_sms) {
    Req& r = *L.r;
    int rc = sgk_ctx_create(&L.ctx, device, st, r.prec);
    if (rc != SGK_OK) {
        err = "engine context";
        return rc;
    }
    auto chk = [&](int code) {
        if (code != SGK_OK && err.empty())
            err = L.ctx->last_error.empty() ? "status " + std::to_string(code) : L.ctx->last_error;
        return code;
    };
    const int64_t dof = level_dof(r.d, r.n, r.k);
    // the Arnoldi grid sized to the DOF (slices of at most 384 coefficients)
    // and the batched kernels' lane count, so that no tuning runs stall the
    // engine's other requests
    L.ctx->persist_ctas = (int)std::max<int64_t>(1, std::min<int64_t>(num_sms, (dof + 383) / 384));
    L.ctx->arn_G_fixed = 8;
    rc = chk(sgk_index_build(L.ctx, r.d, r.n, r.k, &L.idx));
    if (rc == SGK_OK) rc = chk(sgk_operator_assemble(L.ctx, L.idx, r.kappa.data(), r.bc, 20.0, &L.op));
    if (rc == SGK_OK) {
        sgk_reaction f{};
        f.nspecies = 1;
        f.nmono = r.nmono;
        f.species = r.rx_species.data();
        f.coef = r.rx_coef.data();
        f.exps = r.rx_exps.data();
        rc = chk(sgk_solver_create_form(L.ctx, 1, &L.op, &f, SGK_IIF2, r.M, r.dt, nullptr, r.form, &L.sol));
        if (rc == SGK_OK && r.ktol > 0.0) rc = chk(sgk_solver_set_krylov_tolerance(L.sol, r.ktol, r.kmax));
    }
    if (rc != SGK_OK) return rc;
    const InitCopy& in = r.init[0];
    if (!in.coeffs.empty()) {
        rc = (int64_t)in.coeffs.size() == dof ? chk(sgk_solver_set_state(L.sol, 0, in.coeffs.data(), 0))
                                              : chk(SGK_EINVAL);
    } else {
        try {
            DevBuf<double> u0(dof);
            rc = chk(sgk_project_separable(L.ctx, L.idx, (int)in.amp.size(), in.amp.data(), in.wavenum.data(),
                                           in.kind.data(), in.const_term, u0.p));
            if (rc == SGK_OK) rc = chk(sgk_solver_set_state(L.sol, 0, u0.p, 1));
            SGK_CUDA_CHECK(cudaStreamSynchronize(st));
        } catch (const SgkError& e) {
            rc = e.code;
            err = e.msg;
        }
    }
    return rc;
}

}  // namespace

void sgk_server::engine() {
    cudaSetDevice(device);
    BatchCore core;
    const bool ok = core.init(device, 8) == SGK_OK;
    std::vector<std::unique_ptr<Live>> live;
    int next_stream = 0;
    auto retire = [&](std::unique_ptr<Live>& L, int rc, const std::string& err) {
        if (rc == SGK_OK && L->sol) {
            Req& r = *L->r;
            const int64_t dof = L->idx->dof;
            sgk_stats st{};
            sgk_solver_stats(L->sol, &st);
            r.info.steps = st.steps;
            r.info.newton_iters = st.newton_iters;
            r.info.krylov_err_est = st.max_krylov_err_est;
            r.info.inner_iters = st.inner_iters;
            r.info.dof = dof;
            r.result.resize((size_t)dof);
            rc = sgk_solver_get_state(L->sol, 0, r.result.data(), dof, 0);
        }
        std::shared_ptr<Req> r = L->r;
        L.reset();  // device memory back before the budget is
        {
            std::lock_guard<std::mutex> lk(mu);
            --eng_count;
            finish_locked(r, rc, err, -1);
        }
        cv_done.notify_all();
    };
    for (;;) {
        std::deque<std::shared_ptr<Req>> fresh;
        {
            std::unique_lock<std::mutex> lk(mu);
            cv_eng.wait(lk, [&] { return !eng_new.empty() || !live.empty() || (stopping && queue.empty()); });
            if (eng_new.empty() && live.empty()) break;
            fresh.swap(eng_new);
        }
        // join: set the new requests up between ticks
        for (auto& r : fresh) {
            std::unique_ptr<Live> L(new Live());
            L->r = r;
            std::string err;
            int rc = SGK_ECUDA;
            if (ok) {
                cudaStream_t st = core.streams[next_stream++ % core.streams.size()];
                alloc_stream() = st;  // the request's buffers stream-ordered on its stream
                try {
                    rc = engine_setup(device, st, *L, err, core.num_sms);
                } catch (const std::exception& e) {
                    rc = SGK_ECUDA;
                    err = e.what();
                }
                alloc_stream() = nullptr;
            } else {
                err = "engine could not create its streams";
            }
            if (rc != SGK_OK || r->nsteps == 0) {
                if (L->ctx) alloc_stream() = L->ctx->stream;
                retire(L, rc, err);
                alloc_stream() = nullptr;
            } else {
                live.push_back(std::move(L));
            }
        }
        if (live.empty()) continue;
        // one step of every live request
        std::vector<sgk_solver*> sols;
        for (auto& L : live) sols.push_back(L->sol);
        std::vector<int> status;
        std::string tick_err;
        // the batched plan's buffers (rebuilt when the set changes) stream-
        // ordered on the batch stream, so that freeing them does not wait
        // for the workers' streams
        alloc_stream() = core.bstream;
        try {
            batch_core_tick(core, sols, status);
            alloc_stream() = nullptr;
        } catch (const SgkError& e) {
            alloc_stream() = nullptr;
            status.assign(sols.size(), e.code);
            tick_err = e.msg;
        } catch (const std::exception& e) {
            alloc_stream() = nullptr;
            status.assign(sols.size(), SGK_ECUDA);
            tick_err = e.what();
        }
        // leave: finished or failed requests
        for (size_t i = 0; i < live.size(); ++i) {
            std::unique_ptr<Live>& L = live[i];
            if (status[i] == BATCH_STEP_RETAKE) continue;  // the step is taken again next tick
            if (status[i] == SGK_OK) ++L->done;
            if (status[i] != SGK_OK || L->done >= L->r->nsteps) {
                std::string err = tick_err;
                if (status[i] != SGK_OK && err.empty())
                    err = L->ctx->last_error.empty() ? "step status " + std::to_string(status[i])
                                                     : L->ctx->last_error;
                alloc_stream() = L->ctx->stream;
                retire(L, status[i], err);
                alloc_stream() = nullptr;
            }
        }
        live.erase(std::remove_if(live.begin(), live.end(), [](const std::unique_ptr<Live>& L) { return !L; }),
                   live.end());
    }
}

// ------------------------------------------------------------------ C ABI ---

extern "C" {

int64_t sgk_estimate_bytes(int d, int n, int k, int nspecies, int krylov_m, int precision, int has_reaction) {
    if (d < 1 || d > SGK_MAX_DIM || n < 0 || n > SGK_MAX_LEVEL || k < 1 || k > 3 || nspecies < 1 ||
        nspecies > SGK_MAX_SPECIES || krylov_m < 1 || krylov_m > SGK_MAX_KRYLOV ||
        (precision != SGK_FP64 && precision != SGK_MIXED))
        return -1;
    const double dof = (double)level_dof(d, n, k);
    const double S = nspecies, N = dof * S, M = krylov_m;
    const double H = (double)((k + 1) << n);
    const double ntup = (double)tuple_count(d, n);
    double b = 0.0;
    // index set; per species an operator: CSR of the 1D matrix (rows of at
    // most min(H, 64 (k+1)) entries), truncated row lengths, gather tables
    b += ntup * (4.0 * d + 8.0);
    b += S * (H * std::min(H, 64.0 * (k + 1)) * 20.0 + H * (n + 1) * 4.0 + ntup * d * (n + 1) * 8.0 + dof / 32.0);
    // solver: state and Krylov workspace (FP64 basis, two work vectors,
    // partial sums of the Gram-Schmidt reductions)
    b += 8.0 * (4.0 * N + 2.0 * (M + 1.0) * dof + 128.0 + 3.0 * dof);
    b += 8.0 * (std::max(N / 128.0 + 1.0, 160.0) * (std::max(M, 50.0) + 1.0) + 8.0 * M * M + 3.0 * 160.0 * (M + 1.0));
    if (has_reaction == 2) {
        // the interpolation form: F and the stage buffer, the scratch and
        // point-value buffers of the transforms (2 S dof each), and the four
        // 1D factors (rows of at most (n+1)(k+1) entries on average)
        b += 8.0 * (2.0 * N + 8.0 * N) + 4.0 * (H * (n + 1.0) * (k + 1.0) * 16.0 + H * (n + 2.0) * 4.0);
    } else if (has_reaction) {
        const double elem = precision == SGK_FP64 ? 8.0 : 4.0;
        const double full = std::pow(H, d);
        b += 8.0 * 6.0 * N + elem * ((2.0 * S + 1.0) * full + 2.0 * S * dof + N);
        // mixed: the FP32 buffers of the Jacobian products above, the FP64
        // ones of F and FP32 copies of the sparse vectors
        if (precision == SGK_MIXED) b += 8.0 * ((2.0 * S + 1.0) * full + 2.0 * S * dof) + 4.0 * 3.0 * N;
        if (nspecies > 1) b += 8.0 * 51.0 * N;            // GMRES(50) basis
        // change-of-basis tables and work plans
        b += 2.0 * H * (n + 1) * (k + 1) * 12.0 + 64.0 * 1024.0 * d;
    }
    b = b * 1.05 + 16.0 * 1024 * 1024;  // allocator granularity and small buffers
    return b > 9.0e18 ? -1 : (int64_t)b;
}

int sgk_server_create(int device, int nworkers, int64_t mem_budget_bytes, double aging_ms, sgk_server** out) {
    if (!out || nworkers < 1 || nworkers > 64 || mem_budget_bytes < 0) return SGK_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        (void)cudaGetLastError();
        return SGK_ECUDA;
    }
    size_t free_b = 0, total_b = 0;
    if (cudaSetDevice(device) != cudaSuccess || cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        (void)cudaGetLastError();
        return SGK_ECUDA;
    }
    std::unique_ptr<sgk_server> srv(new (std::nothrow) sgk_server());
    if (!srv) return SGK_ENOMEM;
    srv->device = device;
    srv->nworkers = nworkers;
    srv->budget = mem_budget_bytes > 0 ? std::min<int64_t>(mem_budget_bytes, (int64_t)free_b)
                                       : (int64_t)(0.8 * (double)free_b);
    srv->aging_ms = aging_ms > 0 ? aging_ms : 2000.0;
    srv->slot.assign(nworkers, nullptr);
    try {
        for (int w = 0; w < nworkers; ++w) srv->threads.emplace_back([s = srv.get(), w] { s->worker(w); });
        srv->eng_thread = std::thread([s = srv.get()] { s->engine(); });
    } catch (...) {
        {
            std::lock_guard<std::mutex> lk(srv->mu);
            srv->stopping = true;
        }
        srv->cv_work.notify_all();
        srv->cv_eng.notify_all();
        for (auto& t : srv->threads) t.join();
        if (srv->eng_thread.joinable()) srv->eng_thread.join();
        return SGK_ENOMEM;
    }
    *out = srv.release();
    return SGK_OK;
}

int sgk_server_submit(sgk_server* srv, const sgk_request* q, int64_t* ticket) {
    if (!srv || !q || !ticket) return SGK_EINVAL;
    *ticket = 0;
    const int S = q->nspecies;
    if (S < 1 || S > SGK_MAX_SPECIES || q->d < 1 || q->d > SGK_MAX_DIM || q->n < 0 || q->n > SGK_MAX_LEVEL ||
        q->k < 1 || q->k > 3 || q->krylov_m < 1 || q->krylov_m > SGK_MAX_KRYLOV || !(q->dt > 0) || q->nsteps < 0 ||
        !q->kappa || (q->precision != SGK_FP64 && q->precision != SGK_MIXED) ||
        (q->bc != SGK_PERIODIC && q->bc != SGK_DIRICHLET0) || !std::isfinite(q->krylov_tol) ||
        q->krylov_tol < 0.0 ||
        (q->krylov_tol > 0.0 && (q->krylov_max_substeps < 1 || q->krylov_max_substeps > SGK_MAX_KRYLOV_SUBSTEPS)) ||
        (q->reaction_form != SGK_REACTION_QUADRATURE && q->reaction_form != SGK_REACTION_INTERP))
        return SGK_EINVAL;
    if (q->reaction.nmono < 0 || q->reaction.nmono > SGK_MAX_MONO ||
        (q->reaction.nmono > 0 &&
         (q->reaction.nspecies != S || !q->reaction.species || !q->reaction.coef || !q->reaction.exps)))
        return SGK_EINVAL;
    auto r = std::make_shared<Req>();
    r->d = q->d;
    r->n = q->n;
    r->k = q->k;
    r->S = S;
    r->bc = q->bc;
    r->M = q->krylov_m;
    r->dt = q->dt;
    r->nsteps = q->nsteps;
    r->prec = q->precision;
    r->ktol = q->krylov_tol;
    r->kmax = q->krylov_tol > 0.0 ? q->krylov_max_substeps : 1;
    r->form = q->reaction_form;
    r->kappa.assign(q->kappa, q->kappa + (size_t)S * q->d);
    r->nmono = q->reaction.nmono;
    if (r->nmono > 0) {
        r->rx_species.assign(q->reaction.species, q->reaction.species + r->nmono);
        r->rx_coef.assign(q->reaction.coef, q->reaction.coef + r->nmono);
        r->rx_exps.assign(q->reaction.exps, q->reaction.exps + (size_t)r->nmono * S);
    }
    const int64_t dof = level_dof(q->d, q->n, q->k);
    for (int s = 0; s < S; ++s) {
        const sgk_init& in = q->init[s];
        InitCopy& c = r->init[s];
        if (in.coeffs) {
            c.coeffs.assign(in.coeffs, in.coeffs + dof);
        } else {
            if (in.nterms < 0 || (in.nterms > 0 && (!in.amp || !in.wavenum || !in.kind))) return SGK_EINVAL;
            c.amp.assign(in.amp, in.amp + in.nterms);
            c.wavenum.assign(in.wavenum, in.wavenum + (size_t)in.nterms * q->d);
            c.kind.assign(in.kind, in.kind + (size_t)in.nterms * q->d);
            c.const_term = in.const_term;
        }
    }
    r->est = sgk_estimate_bytes(q->d, q->n, q->k, S, q->krylov_m, q->precision,
                                r->nmono > 0 ? (r->form == SGK_REACTION_INTERP ? 2 : 1) : 0);
    std::lock_guard<std::mutex> lk(srv->mu);
    if (srv->stopping) return SGK_EINVAL;
    if (r->est < 0 || r->est > srv->budget) {
        ++srv->rejected;
        return SGK_ENOMEM;
    }
    r->ticket = srv->next_ticket++;
    r->t_submit = Clock::now();
    r->info.nspecies = S;
    r->info.est_bytes = r->est;
    srv->tickets[r->ticket] = r;
    srv->queue.push_back(r);
    ++srv->submitted;
    *ticket = r->ticket;
    srv->admit_locked();
    return SGK_OK;
}

int sgk_server_poll(sgk_server* srv, int64_t ticket) {
    if (!srv) return -1;
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->tickets.find(ticket);
    if (it == srv->tickets.end()) return -1;
    return it->second->done ? 1 : 0;
}

int sgk_server_wait(sgk_server* srv, int64_t ticket, double timeout_ms, sgk_result_info* info, double* out,
                    int64_t cap) {
    if (!srv) return SGK_EINVAL;
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->tickets.find(ticket);
    if (it == srv->tickets.end()) return SGK_EINVAL;
    std::shared_ptr<Req> r = it->second;
    auto ready = [&] { return r->done; };
    if (timeout_ms < 0) {
        srv->cv_done.wait(lk, ready);
    } else if (!srv->cv_done.wait_for(lk, std::chrono::duration<double, std::milli>(timeout_ms), ready)) {
        return SGK_ETIMEOUT;
    }
    if (out && cap < (int64_t)r->result.size()) return SGK_EINVAL;
    if (info) *info = r->info;
    if (out && !r->result.empty()) std::memcpy(out, r->result.data(), r->result.size() * sizeof(double));
    srv->tickets.erase(it);
    return SGK_OK;
}

int sgk_server_get_stats(sgk_server* srv, sgk_server_stats* out) {
    if (!srv || !out) return SGK_EINVAL;
    std::lock_guard<std::mutex> lk(srv->mu);
    out->submitted = srv->submitted;
    out->completed = srv->completed;
    out->failed = srv->failed;
    out->rejected = srv->rejected;
    out->queued = (int64_t)srv->queue.size();
    out->running = srv->running;
    out->budget_bytes = srv->budget;
    out->reserved_bytes = srv->reserved;
    out->peak_reserved_bytes = srv->peak_reserved;
    out->max_concurrent = srv->max_concurrent;
    return SGK_OK;
}

int sgk_server_destroy(sgk_server* srv) {
    if (!srv) return SGK_OK;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stopping = true;
    }
    srv->cv_work.notify_all();
    srv->cv_eng.notify_all();
    for (auto& t : srv->threads) t.join();
    if (srv->eng_thread.joinable()) srv->eng_thread.join();
    delete srv;
    return SGK_OK;
}

int sgk_server_set_engine(sgk_server* srv, int on, int max_requests) {
    if (!srv || max_requests < 0) return SGK_EINVAL;
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->engine_on = on != 0;
    if (max_requests > 0) srv->eng_max = max_requests;
    return SGK_OK;
}

}  // extern "C"
