// Stepping many independent solvers together: the streams, events and
// batched Arnoldi plan shared by sgk_batch (batch.cpp) and the request
// server's engine (server.cpp).
#pragma once

#include <vector>

#include "sgk_krylov.h"
#include "sgk_solver.h"

struct BatchCore {
    int device = 0;
    int num_sms = 0;
    size_t smem_optin = 0;
    bool fused = true;  // batched Arnoldi launches (else whole-step graphs per solver)
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> ev;     // one per stream, joins them into bstream
    cudaStream_t bstream = nullptr;  // the batched Arnoldi launches
    cudaEvent_t evb = nullptr;       // forks bstream back to the streams
    ArnBatchPlan* plan = nullptr;
    // serial numbers (sgk_solver::uid) of the plan's solvers, in job order:
    // the plan holds their device pointers, so it is rebuilt whenever this
    // set changes -- compared by serial number, never by address
    std::vector<uint64_t> plan_set;
    int64_t launches = 0;               // kernels of the batched Arnoldi path
    BatchCore() = default;
    BatchCore(const BatchCore&) = delete;
    BatchCore& operator=(const BatchCore&) = delete;
    ~BatchCore();
    // streams and events on device; SGK_OK or SGK_ECUDA
    int init(int device, int nstreams);
};

// Status of a solver's step in a tick whose Krylov accuracy guard asked for
// more sub-projections: the step was rolled back (state, time and step
// count as before it) and is to be taken again in the next tick
constexpr int BATCH_STEP_RETAKE = -1;

// One step of every solver in sols, each on its context's stream (one of
// core.streams): the split ones (solver_split_eligible, batched-Arnoldi
// class) share the batched Arnoldi launches between their pre- and
// post-Krylov graphs; other device-driven ones take whole-step graphs; the
// host-driven ones step alone after the others.  status[i] receives the
// status of solver i's step (a failed step is rolled back by the solver;
// BATCH_STEP_RETAKE: rolled back by the accuracy guard).
// The host waits for every stream once.  Throws SgkError on CUDA errors.
void batch_core_tick(BatchCore& core, const std::vector<sgk_solver*>& sols, std::vector<int>& status);
