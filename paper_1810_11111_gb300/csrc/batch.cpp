// Batched stepping of many independent IIF2 problems on one device (the
// service around the method; the paper has no counterpart).
//
// Every instance has its own context (so that its persistent Arnoldi grid
// can be sized to its DOF), index set, operators and solver; the contexts
// share the batch's streams round-robin.  A batch step runs, for the
// instances whose step can be split (one species, persistent Arnoldi):
//   1. per instance, on its stream, the first half of its device-driven step
//      (state copy, predictor, v = U + dt/2 F(U)) as one CUDA graph;
//   2. on the batch stream, after all of those, the Arnoldi processes of
//      every instance in one persistent cooperative launch per kernel class
//      (arnoldi_batch_*: a device work list of (instance, slice) items per
//      CTA, so one grid barrier schedule serves all instances of a class);
//   3. per instance, on its stream, the second half (exp(dt H) e_1, the
//      combination, the Newton solve) as one CUDA graph.
// Other device-driven instances take whole-step graphs on their streams;
// the rest (systems, host-driven) step one by one.  The host waits once per
// stream and batch step.
#include <algorithm>
#include <memory>
#include <vector>

#include <cuda_runtime.h>

#include "sgk_internal.h"
#include "sgk_quad.h"
#include "sgk_krylov.h"
#include "sgk_solver.h"

namespace {

struct Instance {
    sgk_ctx* ctx = nullptr;
    sgk_index* idx = nullptr;
    sgk_op* ops[SGK_MAX_SPECIES] = {nullptr};
    sgk_solver* sol = nullptr;
    int S = 1;
    int status = SGK_OK;
    int stream = 0;
    ~Instance() {
        sgk_solver_destroy(sol);
        for (sgk_op* o : ops) sgk_operator_destroy(o);
        sgk_index_destroy(idx);
        sgk_ctx_destroy(ctx);
    }
};

}  // namespace

struct sgk_batch {
    int device = 0;
    int slice_len = 384;
    bool fused = true;  // batched Arnoldi launches (else whole-step graphs per instance)
    std::vector<cudaStream_t> streams;
    cudaStream_t bstream = nullptr;  // the batched Arnoldi launches
    std::vector<cudaEvent_t> ev;     // one per stream, joins them into bstream
    cudaEvent_t evb = nullptr;       // forks bstream back to the streams
    int num_sms = 0;
    size_t smem_optin = 0;
    std::vector<std::unique_ptr<Instance>> inst;
    ArnBatchPlan* plan = nullptr;
    std::vector<Instance*> plan_set;  // instances of the plan, in job order
    int64_t batched_launches = 0;
    ~sgk_batch() {
        arnoldi_batch_free(plan);
        inst.clear();
        for (cudaStream_t s : streams)
            if (s) cudaStreamDestroy(s);
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
        if (evb) cudaEventDestroy(evb);
        if (bstream) cudaStreamDestroy(bstream);
    }
};

extern "C" {

int sgk_batch_create(int device, int nstreams, int slice_len, sgk_batch** out) {
    if (!out || nstreams < 1 || nstreams > 256 || slice_len < 0) return SGK_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev || cudaSetDevice(device) != cudaSuccess) {
        (void)cudaGetLastError();
        return SGK_ECUDA;
    }
    std::unique_ptr<sgk_batch> b(new (std::nothrow) sgk_batch());
    if (!b) return SGK_ENOMEM;
    b->device = device;
    if (slice_len > 0) b->slice_len = slice_len;
    for (int i = 0; i < nstreams; ++i) {
        cudaStream_t s = nullptr;
        cudaEvent_t e = nullptr;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            (void)cudaGetLastError();
            return SGK_ECUDA;
        }
        b->streams.push_back(s);
        b->ev.push_back(e);
    }
    int optin = 0;
    if (cudaStreamCreateWithFlags(&b->bstream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->evb, cudaEventDisableTiming) != cudaSuccess ||
        cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess) {
        (void)cudaGetLastError();
        return SGK_ECUDA;
    }
    b->smem_optin = (size_t)optin;
    *out = b.release();
    return SGK_OK;
}

int sgk_batch_add(sgk_batch* b, const sgk_request* q, int* index) {
    if (!b || !q || !index || !q->kappa) return SGK_EINVAL;
    const int S = q->nspecies;
    if (S < 1 || S > SGK_MAX_SPECIES) return SGK_EINVAL;
    cudaSetDevice(b->device);
    std::unique_ptr<Instance> in(new (std::nothrow) Instance());
    if (!in) return SGK_ENOMEM;
    in->S = S;
    in->stream = (int)(b->inst.size() % b->streams.size());
    int rc = sgk_ctx_create(&in->ctx, b->device, b->streams[in->stream], q->precision);
    if (rc != SGK_OK) return rc;
    rc = sgk_index_build(in->ctx, q->d, q->n, q->k, &in->idx);
    if (rc != SGK_OK) return rc;
    const int64_t dof = in->idx->dof;
    // persistent Arnoldi grid: slices of at most slice_len coefficients
    in->ctx->persist_ctas =
        (int)std::max<int64_t>(1, std::min<int64_t>(in->ctx->num_sms, (dof + b->slice_len - 1) / b->slice_len));
    for (int s = 0; s < S && rc == SGK_OK; ++s)
        rc = sgk_operator_assemble(in->ctx, in->idx, q->kappa + (size_t)s * q->d, q->bc, 20.0, &in->ops[s]);
    if (rc != SGK_OK) return rc;
    rc = sgk_solver_create(in->ctx, S, in->ops, &q->reaction, SGK_IIF2, q->krylov_m, q->dt, nullptr, &in->sol);
    if (rc != SGK_OK) return rc;
    try {
        DevBuf<double> u0(dof);
        for (int s = 0; s < S && rc == SGK_OK; ++s) {
            const sgk_init& ii = q->init[s];
            if (ii.coeffs) {
                rc = sgk_solver_set_state(in->sol, s, ii.coeffs, 0);
            } else {
                rc = sgk_project_separable(in->ctx, in->idx, ii.nterms, ii.amp, ii.wavenum, ii.kind, ii.const_term,
                                           u0.p);
                if (rc == SGK_OK) rc = sgk_solver_set_state(in->sol, s, u0.p, 1);
            }
        }
        SGK_CUDA_CHECK(cudaStreamSynchronize(in->ctx->stream));
    } catch (const SgkError& e) {
        return e.code;
    }
    if (rc != SGK_OK) return rc;
    *index = (int)b->inst.size();
    b->inst.push_back(std::move(in));
    return SGK_OK;
}

int sgk_batch_set_fused(sgk_batch* b, int on) {
    if (!b) return SGK_EINVAL;
    b->fused = on != 0;
    return SGK_OK;
}

int64_t sgk_batch_launches(const sgk_batch* b) { return b ? b->batched_launches : -1; }

int sgk_batch_step(sgk_batch* b, int nsteps, int* status) {
    if (!b || nsteps < 0) return SGK_EINVAL;
    cudaSetDevice(b->device);
    int first = SGK_OK;
    try {
        for (int step = 0; step < nsteps; ++step) {
            // the split instances share the batched Arnoldi launches; the
            // plan is rebuilt when that set changes (an instance failed)
            std::vector<Instance*> split, queued;
            if (b->fused)
                for (auto& in : b->inst)
                    if (in->status == SGK_OK && solver_split_eligible(in->sol) &&
                        arnoldi_batch_supports(solver_arnoldi_job(in->sol)))
                        split.push_back(in.get());
            if (split != b->plan_set) {
                arnoldi_batch_free(b->plan);
                b->plan = nullptr;
                b->plan_set.clear();
                if (!split.empty()) {
                    std::vector<ArnJob> jobs;
                    for (Instance* in : split) jobs.push_back(solver_arnoldi_job(in->sol));
                    b->plan = arnoldi_batch_plan(jobs, b->num_sms, b->smem_optin, b->bstream);
                    b->plan_set = split;
                }
            }
            if (!split.empty()) {
                for (Instance* in : split) solver_step_launch_pre(in->sol);
                for (size_t i = 0; i < b->streams.size(); ++i) {
                    SGK_CUDA_CHECK(cudaEventRecord(b->ev[i], b->streams[i]));
                    SGK_CUDA_CHECK(cudaStreamWaitEvent(b->bstream, b->ev[i], 0));
                }
                b->batched_launches += arnoldi_batch_launch(b->plan, b->bstream);
                SGK_CUDA_CHECK(cudaEventRecord(b->evb, b->bstream));
                for (cudaStream_t s : b->streams) SGK_CUDA_CHECK(cudaStreamWaitEvent(s, b->evb, 0));
                for (Instance* in : split) {
                    solver_step_launch_post(in->sol);
                    queued.push_back(in);
                }
            }
            // the other device-driven steps, whole
            for (auto& in : b->inst) {
                if (in->status != SGK_OK || std::find(split.begin(), split.end(), in.get()) != split.end()) continue;
                if (solver_device_steps(in->sol)) {
                    solver_step_launch(in->sol);
                    queued.push_back(in.get());
                }
            }
            for (cudaStream_t s : b->streams) SGK_CUDA_CHECK(cudaStreamSynchronize(s));
            for (Instance* in : queued) in->status = solver_step_finish(in->sol);
            for (auto& in : b->inst)
                if (in->status == SGK_OK && !solver_device_steps(in->sol)) in->status = sgk_solver_step(in->sol, 1);
        }
    } catch (const SgkError& e) {
        return e.code;
    }
    for (size_t i = 0; i < b->inst.size(); ++i) {
        if (status) status[i] = b->inst[i]->status;
        if (first == SGK_OK && b->inst[i]->status != SGK_OK) first = b->inst[i]->status;
    }
    return first;
}

int64_t sgk_batch_dof(const sgk_batch* b, int index) {
    if (!b || index < 0 || index >= (int)b->inst.size()) return -1;
    return b->inst[index]->idx->dof;
}

int sgk_batch_count(const sgk_batch* b) { return b ? (int)b->inst.size() : -1; }

int sgk_batch_get_state(const sgk_batch* b, int index, int species, double* out, int64_t cap) {
    if (!b || index < 0 || index >= (int)b->inst.size() || !out) return SGK_EINVAL;
    const Instance& in = *b->inst[index];
    if (species < 0 || species >= in.S) return SGK_EINVAL;
    return sgk_solver_get_state(in.sol, species, out, cap, 0);
}

int sgk_batch_destroy(sgk_batch* b) {
    delete b;
    return SGK_OK;
}

}  // extern "C"
