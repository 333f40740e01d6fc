// IIF solver object: shared declarations.
#pragma once

#include "sgk_krylov.h"
#include "sgk_quad.h"

// most device-driven steps queued without waiting
constexpr int SGK_ASYNC_SLOTS = 32;

// An instantiated CUDA graph of a fixed launch sequence and the number of
// kernels it holds.
struct GraphCache {
    cudaGraphExec_t exec = nullptr;
    int64_t nlaunch = 0;
};

// Device tables of one 1D factor of the interpolation form of the reaction
// term (interp.cu): CSR row pointers, truncated row lengths per level,
// packed (level << 16 | position) columns, values.
struct InterpFactorDev {
    DevBuf<int32_t> rp, rlen, ce;
    DevBuf<double> val;
};

// The sparse-grid interpolation form of F (SGK_REACTION_INTERP): the factors
// A, B, B^{-1}, A^{-1}; two scratch buffers of the direction passes and two
// of point values (2 S n each); the pointwise Newton outcome (status, most
// corrections).
struct InterpPlan {
    bool on = false;
    InterpFactorDev f[4];
    DevBuf<double> t0, t1, p0, p1;
    DevBuf<int> outcome;
};

struct sgk_solver {
    // serial number, never reused in the process (a destroyed solver's
    // address can be handed to a new one; plans that hold device pointers
    // of their solvers are keyed by this)
    uint64_t uid = 0;
    sgk_ctx* ctx = nullptr;
    const sgk_index* idx = nullptr;
    int nspecies = 1;
    const sgk_op* ops[SGK_MAX_SPECIES] = {nullptr};
    ReactionDev rx;
    bool has_rx = false;
    int M = 0;
    double dt = 0.0;
    int scheme = SGK_IIF2;
    double newton_c = 0.0;  // c of the implicit stage U - c F(U) = W (alpha_1 dt: dt/2 IIF2, 5/12 dt IIF3)
    // IIFr, r > 2: F(U^{n-1}), ..., F(U^{n-r+2}) of the last steps (nhist of
    // them valid, N values each), the staged F(U^n) of the running step, and
    // exp((i+1) dt A) F(U^{n-i})
    DevBuf<double> Fhist, Fstage, W2;
    int nhist = 0;
    // source terms: F_s(U, t) += sum_m e^{lambda_m t} S_{s,m}; t^n of the
    // state on the host and, written before each step, on the device
    double t = 0.0;
    bool has_src = false;
    int nsrc[SGK_MAX_SPECIES] = {0};
    DevBuf<double> src_S[SGK_MAX_SPECIES];  // SGK_MAX_SOURCE_TERMS * n each, allocated on first use
    DevBuf<double> src_lam;                 // SGK_MAX_SPECIES * SGK_MAX_SOURCE_TERMS
    DevBuf<double> tdev;                    // t^n
    sgk_newton_opts opts{};
    int prec = SGK_FP64;
    long long n = 0;  // dof per species
    Quad Q;
    // SGK_REACTION_QUADRATURE (the paper's finest-grid F, Q above) or
    // SGK_REACTION_INTERP (IP below)
    int rform = SGK_REACTION_QUADRATURE;
    InterpPlan IP;
    bool unod_valid = false;
    // state and Newton vectors (species-stacked FP64)
    DevBuf<double> U, Uprev, W, vv, Fv, G, cg_x, cg_r, cg_p, cg_q;
    // Krylov workspace
    DevBuf<double> V64, w64;
    DevBuf<float> V32, w32;
    DevBuf<double> Hm, h1, h2, ky, scal, partials, expm_ws;
    DevBuf<KrylovScalars> ks;
    // exp(tau A) v as ksub successive projections of tau / ksub (1: the
    // paper's single projection); ktmp is their intermediate vector
    int ksub = 1;
    DevBuf<double> ktmp;
    // accuracy guard of synchronous steps: while the step's estimate is
    // above ktol (> 0), its exponentials are taken again with twice the
    // sub-projections, up to kmax
    double ktol = 0.0;
    int kmax = 1;
    DevBuf<unsigned> counters;
    DevBuf<unsigned> fcnt;  // arrival counters of the fused Newton / CG kernels (zero between launches)
    // persistent Arnoldi: second work vector, partial sums, per species a
    // barrier counter and an error flag
    bool persistent = false;
    int arn_G = 0;  // autotuned lanes per output of the persistent matvec
    DevBuf<double> w64b, zbuf, pbuf;
    DevBuf<unsigned> pbar;
    DevBuf<int64_t> abounds;  // work-balanced slices of the persistent kernel
    int64_t aE = 0;           // longest of them
    int64_t alist = 0;        // most pre-located gather entries of one of them
    // reaction passes: [unod S][wnod S][tmp][spin S][spout S], T = double or float
    DevBuf<double> q64, jw64;
    DevBuf<float> q32, jw32;
    // GMRES (systems)
    DevBuf<double> gm_V, gm_H, gm_cs, gm_sn, gm_g, gm_y, gm_report;
    bool use_graphs = true;
    GraphCache g_krylov[SGK_MAX_SPECIES], g_pred, g_pred_f, g_resid, g_resid0, g_cg;
    GraphCache g_krylovh[SGK_MAX_SPECIES][SGK_IIF_MAX_ORDER - 2];  // the history projections of IIFr
    // Fv holds F(U) for the current U (a host-driven or device-driven step
    // ended with an accepted residual evaluation there); cleared whenever U
    // changes otherwise
    bool fv_valid = false;
    int64_t n_predf = 0;        // launches of the predictor's F in the step graph
    // device-driven step: the whole IIF2 step (predictor, Krylov, Newton with
    // CG) as one graph whose loops are conditional while-nodes
    GraphCache g_step;
    // the same step in two graphs around an Arnoldi process run elsewhere
    // (batched launch); n_pre kernels in the first
    GraphCache g_pre, g_post;
    int64_t n_pre = 0;
    bool split_last = false;  // the last launched step used the two graphs
    cudaStream_t aux[2] = {nullptr, nullptr};  // capture streams of the loop bodies
    DevBuf<unsigned char> ctl;                 // StepCtl on the device
    // kernels per segment of the step graph (for the launch count)
    int64_t n_prefix = 0, n_resid = 0, n_cgpre = 0, n_cgbody = 0, n_adv = 0;
    // pinned host records of launched device-driven steps: slot 0 for a
    // synchronous step, slots 0..nqueued-1 for queued ones
    void* hrec = nullptr;
    int nqueued = 0;      // steps queued by solver_step_async, not yet finished
    int ring_slots = 0;   // capacity of the queue
    DevBuf<double> ring;  // the state before each queued step (ring_slots x N), for the rollback
    int async_rc = 0;     // first failure among finished queued steps, reported by sgk_solver_wait
    sgk_stats stats{};
    ~sgk_solver();
};

void solver_alloc(sgk_solver* s);
// Interpolation form of the reaction term (interp.cu).  interp_build makes
// the factor tables and buffers; interp_evalF: F = C^{-1} f(C U) (no
// sources); interp_evalJ: jw = C^{-1} (f'(C U) (C w)); interp_implicit: from
// Wp = W + c S, solves u - c f(u) = C Wp at every collocation point and
// writes U = C^{-1} u and Fr = C^{-1} f(u), the outcome (SGK_OK or
// SGK_ENEWTON, most Newton corrections of a point) to *status and *iters on
// the device.  All vectors species-stacked on the device.
void interp_build(sgk_solver* s);
void interp_evalF(sgk_solver* s, const double* U, double* F);
void interp_evalJ(sgk_solver* s, const double* U, const double* w, double* jw);
void interp_implicit(sgk_solver* s, const double* Wp, double c, double* U, double* Fr, int* status, int* iters);
void interp_to_points(sgk_solver* s, const double* U, double* P, int nvec);
void interp_from_points(sgk_solver* s, const double* P, double* U, int nvec, double* U2, int nsplit);
// alpha_1, alpha_0, alpha_{-1}, ..., alpha_{-(r-2)} of eq. krylov4
void iif_alpha(int r, double* alpha);
// Device-driven steps (one graph per step) are used when graphs are on, no
// kernel timing is active and the implicit solve is CG (one species) or
// absent.  solver_step_launch queues one such step on the solver's stream;
// after that stream has been synchronised, solver_step_finish reads its
// outcome (rolling the state back on failure) and returns the status.
bool solver_device_steps(const sgk_solver* s);
// U was written from outside a step (or rolled back): the cached F(U) no
// longer applies
void solver_state_changed(sgk_solver* s);
// U_species = src (device, n values); keeps the cached F(U) on the device when
// nothing changed
void solver_set_state(sgk_solver* s, int species, const double* src_dev);
// slot: the host record that receives the step's outcome; restore: the state
// to roll back to on failure (null: the step graph's own copy)
void solver_step_launch(sgk_solver* s, int slot = 0);
int solver_step_finish(sgk_solver* s, int slot = 0, const double* restore = nullptr);
// After a successful device-driven step finished by solver_step_finish: if
// the Krylov accuracy guard wants more sub-projections (and doubles them),
// the step is rolled back (state, time, step count) and true is returned.
bool solver_step_retake(sgk_solver* s);
// The same device-driven step with its Arnoldi process run by the caller
// (one species, persistent Arnoldi): solver_step_launch_pre queues the state
// copy, the predictor and v = U + dt/2 F(U); the caller then runs the
// Arnoldi process of solver_arnoldi_job(s) (after pre, on any stream
// ordered with it); solver_step_launch_post queues exp(dt H) e_1, the
// combination and the Newton solve and the outcome copies;
// solver_step_finish completes it as for solver_step_launch.
bool solver_split_eligible(const sgk_solver* s);
ArnJob solver_arnoldi_job(sgk_solver* s);
void solver_step_launch_pre(sgk_solver* s);
void solver_step_launch_post(sgk_solver* s, int slot = 0);
void solver_krylov_finish(sgk_solver* s, int species, double* W);
// Queue nsteps device-driven steps without waiting (synchronous steps when
// the solver is not device-driven); solver_drain finishes the queued ones in
// order and keeps the first failure for sgk_solver_wait.
int solver_step_async(sgk_solver* s, int nsteps);
void solver_drain(sgk_solver* s);
int solver_step(sgk_solver* s, int nsteps);
void solver_eval_reaction(sgk_solver* s, const double* U, double* F);
void solver_jacobian_apply(sgk_solver* s, const double* U, const double* w, double* jw);
void solver_krylov_expv(sgk_solver* s, int species, const double* v, double* W, double tau = -1.0);
// exp(tau A) v as ksub >= 1 successive projections of tau / ksub from the
// next step on (drops the cached graphs when it changes)
void solver_set_krylov_substeps(sgk_solver* s, int ksub);
// replaces the source terms of one species (coeffs_dev: nterms * n device values)
void solver_set_source(sgk_solver* s, int species, int nterms, const double* lambda, const double* coeffs_dev);
void solver_set_time(sgk_solver* s, double t);
