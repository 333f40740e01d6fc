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
#include "sgk_batchcore.h"
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

BatchCore::~BatchCore() {
    arnoldi_batch_free(plan);
    for (cudaStream_t st : streams)
        if (st) cudaStreamDestroy(st);
    for (cudaEvent_t e : ev)
        if (e) cudaEventDestroy(e);
    if (evb) cudaEventDestroy(evb);
    if (bstream) cudaStreamDestroy(bstream);
}

int BatchCore::init(int dev, int nstreams) {
    device = dev;
    for (int i = 0; i < nstreams; ++i) {
        cudaStream_t st = nullptr;
        cudaEvent_t e = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            (void)cudaGetLastError();
            if (st) cudaStreamDestroy(st);
            return SGK_ECUDA;
        }
        streams.push_back(st);
        ev.push_back(e);
    }
    int optin = 0;
    if (cudaStreamCreateWithFlags(&bstream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&evb, cudaEventDisableTiming) != cudaSuccess ||
        cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return SGK_ECUDA;
    }
    smem_optin = (size_t)optin;
    return SGK_OK;
}

void batch_core_tick(BatchCore& core, const std::vector<sgk_solver*>& sols, std::vector<int>& status) {
    status.assign(sols.size(), SGK_OK);
    // the split solvers share the batched Arnoldi launches; the plan is
    // rebuilt when that set changes
    std::vector<sgk_solver*> split;
    std::vector<uint64_t> split_uid;
    std::vector<int> split_idx, queued;
    if (core.fused)
        for (size_t i = 0; i < sols.size(); ++i)
            if (solver_split_eligible(sols[i]) && arnoldi_batch_supports(solver_arnoldi_job(sols[i]))) {
                split.push_back(sols[i]);
                split_uid.push_back(sols[i]->uid);
                split_idx.push_back((int)i);
            }
    if (split_uid != core.plan_set) {
        arnoldi_batch_free(core.plan);
        core.plan = nullptr;
        core.plan_set.clear();
        if (!split.empty()) {
            std::vector<ArnJob> jobs;
            for (sgk_solver* s : split) jobs.push_back(solver_arnoldi_job(s));
            core.plan = arnoldi_batch_plan(jobs, core.num_sms, core.smem_optin, core.bstream);
            core.plan_set = split_uid;
        }
    }
    if (!split.empty()) {
        for (sgk_solver* s : split) solver_step_launch_pre(s);
        for (size_t i = 0; i < core.streams.size(); ++i) {
            SGK_CUDA_CHECK(cudaEventRecord(core.ev[i], core.streams[i]));
            SGK_CUDA_CHECK(cudaStreamWaitEvent(core.bstream, core.ev[i], 0));
        }
        core.launches += arnoldi_batch_launch(core.plan, core.bstream);
        SGK_CUDA_CHECK(cudaEventRecord(core.evb, core.bstream));
        for (cudaStream_t st : core.streams) SGK_CUDA_CHECK(cudaStreamWaitEvent(st, core.evb, 0));
        for (size_t k = 0; k < split.size(); ++k) {
            solver_step_launch_post(split[k]);
            queued.push_back(split_idx[k]);
        }
    }
    // the other device-driven steps, whole
    for (size_t i = 0; i < sols.size(); ++i) {
        if (std::find(split_idx.begin(), split_idx.end(), (int)i) != split_idx.end()) continue;
        if (solver_device_steps(sols[i])) {
            solver_step_launch(sols[i]);
            queued.push_back((int)i);
        }
    }
    for (cudaStream_t st : core.streams) SGK_CUDA_CHECK(cudaStreamSynchronize(st));
    for (int i : queued) {
        status[i] = solver_step_finish(sols[i]);
        if (status[i] == SGK_OK && solver_step_retake(sols[i])) status[i] = BATCH_STEP_RETAKE;
    }
    for (size_t i = 0; i < sols.size(); ++i)
        if (!solver_device_steps(sols[i])) status[i] = sgk_solver_step(sols[i], 1);
}

struct sgk_batch {
    int device = 0;
    int slice_len = 384;
    BatchCore core;
    std::vector<std::unique_ptr<Instance>> inst;
    ~sgk_batch() { inst.clear(); }
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
    const int rc = b->core.init(device, nstreams);
    if (rc != SGK_OK) return rc;
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
    in->stream = (int)(b->inst.size() % b->core.streams.size());
    int rc = sgk_ctx_create(&in->ctx, b->device, b->core.streams[in->stream], q->precision);
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
    rc = sgk_solver_create_form(in->ctx, S, in->ops, &q->reaction, SGK_IIF2, q->krylov_m, q->dt, nullptr,
                                q->reaction_form, &in->sol);
    if (rc != SGK_OK) return rc;
    if (q->krylov_tol != 0.0) {
        rc = sgk_solver_set_krylov_tolerance(in->sol, q->krylov_tol, q->krylov_max_substeps);
        if (rc != SGK_OK) return rc;
    }
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
    b->core.fused = on != 0;
    return SGK_OK;
}

int64_t sgk_batch_launches(const sgk_batch* b) { return b ? b->core.launches : -1; }

int sgk_batch_step(sgk_batch* b, int nsteps, int* status) {
    if (!b || nsteps < 0) return SGK_EINVAL;
    cudaSetDevice(b->device);
    int first = SGK_OK;
    try {
        // steps left per instance: a step the accuracy guard rolled back is
        // taken again in the next tick
        std::vector<int> left(b->inst.size(), nsteps);
        for (;;) {
            std::vector<sgk_solver*> sols;
            std::vector<size_t> act;
            for (size_t i = 0; i < b->inst.size(); ++i)
                if (b->inst[i]->status == SGK_OK && left[i] > 0) {
                    sols.push_back(b->inst[i]->sol);
                    act.push_back(i);
                }
            if (sols.empty()) break;
            std::vector<int> st;
            batch_core_tick(b->core, sols, st);
            for (size_t k = 0; k < act.size(); ++k) {
                if (st[k] == BATCH_STEP_RETAKE) continue;
                b->inst[act[k]]->status = st[k];
                left[act[k]] -= 1;
            }
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

int sgk_batch_stats(const sgk_batch* b, int index, sgk_stats* out) {
    if (!b || !out || index < 0 || index >= (int)b->inst.size()) return SGK_EINVAL;
    return sgk_solver_stats(b->inst[index]->sol, out);
}

int sgk_batch_destroy(sgk_batch* b) {
    delete b;
    return SGK_OK;
}

}  // extern "C"
