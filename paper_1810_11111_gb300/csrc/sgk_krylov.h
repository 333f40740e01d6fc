// Krylov exponential and vector kernels: shared declarations.
#pragma once

struct dfloat;
#include <vector>

#include <functional>

#include "sgk_internal.h"

struct KrylovScalars {
    double gamma;
    double inv_gamma;
    double inv_beta;
    double fro2;
    int stop;       // set by breakdown (or gamma == 0): later steps return at once
    int m_eff;      // Krylov dimension reached
    int breakdown;  // 1 if truncated by happy breakdown
    int pad;
    // a-posteriori estimate of the projection's error relative to the
    // result: h_{m+1,m} |e_m^T exp(tau H_m) e_1| / ||exp(tau H_m) e_1||
    // (0 after a happy breakdown, where the projection is exact)
    double err_est;
    // the largest err_est since the solver last cleared it: a step clears
    // it at its start, so it holds the largest over the step's projections
    // (every exponential and every sub-projection of one)
    double err_max;
};

struct PadeCoef {
    double c[14];
};

// Device workspace of one Krylov exponential; V holds M+1 columns of n.
template <typename T>
struct KrylovWork {
    T* V = nullptr;
    T* w = nullptr;
    double* H = nullptr;      // (M+1) x M row-major
    double* h1 = nullptr;     // M+1
    double* h2 = nullptr;     // M+1
    double* y = nullptr;      // M
    double* scal = nullptr;   // [0] gamma^2, [1] ||w||^2
    double* partials = nullptr;
    double* expm_ws = nullptr;  // 8 M^2
    KrylovScalars* ks = nullptr;
    unsigned* counter = nullptr;  // last-block counter of the fused reductions (zero between kernels)
};

// Extra device workspace of the persistent Arnoldi kernel (arnoldi.cu).
struct PersistentWork {
    double* w_alt = nullptr;  // second work vector (n)
    double* Z = nullptr;      // raw matvec outputs, (M + 1) n
    double* pbuf = nullptr;   // arnoldi_persistent_pbuf_size doubles
    unsigned* bar = nullptr;  // [0] barrier arrivals, [1] error flag (sticky until the host clears it)
    int G = 0;                // lanes per output in the matvec (0: default)
    const int64_t* bounds = nullptr;  // work-balanced slices (device, grid + 1 entries), or null
    int64_t E = 0;                    // longest slice when bounds is set
    int64_t list_ent = 0;             // most pre-located gather entries of a slice when bounds is set
};

// CTAs of the persistent kernel on this context.
int arnoldi_persistent_ctas(const sgk_ctx* ctx);
// Largest n (and the partial-sum buffer size) the persistent kernel takes on
// this context's device.
int64_t arnoldi_persistent_max_n(const sgk_ctx* ctx);
size_t arnoldi_persistent_pbuf_size(const sgk_ctx* ctx, int M);
// Work-balanced slices for the persistent kernel (arnoldi_slice_bounds with
// the caps that keep the slice's pre-located gathers and Krylov columns in
// shared memory); empty when no such partition exists.  E and list_ent
// receive the longest slice and its most gather entries.
std::vector<int64_t> arnoldi_balanced_bounds(const sgk_ctx* ctx, const sgk_op* op, int M, int64_t* E,
                                             int64_t* list_ent);
// gamma, V (M + 1 columns), H and m_eff of the Krylov space of v, in one
// cooperative launch.
void arnoldi_persistent(sgk_ctx* ctx, const sgk_op* op, const PersistentWork& pw, const KrylovWork<double>& kw,
                        const double* v, int64_t n, int M);
// Times the candidate lane counts of the matvec on this operator and size
// (scratch: n doubles of device memory) and returns the fastest; the runs
// overwrite the Krylov workspace.  Not while a graph is being captured.
int arnoldi_autotune(sgk_ctx* ctx, const sgk_op* op, PersistentWork pw, const KrylovWork<double>& kw, double* scratch,
                     int64_t n, int M);
// One Arnoldi process of a batch of independent instances (its context,
// operator, workspaces and input vector).
struct ArnJob {
    sgk_ctx* ctx = nullptr;
    const sgk_op* op = nullptr;
    PersistentWork pw;
    KrylovWork<double> kw;
    const double* v = nullptr;
    int64_t n = 0;
    int M = 0;
};
struct ArnBatchPlan;
// Whether an instance can join a batched launch (d 2..4, degree 1..3, a
// persistent-size vector).
bool arnoldi_batch_supports(const ArnJob& j);
// Schedules the jobs' Arnoldi processes into one cooperative launch per
// kernel class and uploads the work lists; the plan holds device memory
// until arnoldi_batch_free.
ArnBatchPlan* arnoldi_batch_plan(const std::vector<ArnJob>& jobs, int num_sms, size_t smem_optin, cudaStream_t st);
// Queues the plan's launches on st (the barrier counters reset first);
// returns the number of kernels launched.
int arnoldi_batch_launch(const ArnBatchPlan* plan, cudaStream_t st);
int arnoldi_batch_classes(const ArnBatchPlan* plan);
void arnoldi_batch_free(ArnBatchPlan* plan);
// expm and the combination W = gamma V y after an Arnoldi process (the rest
// of krylov_expv_persistent)
void krylov_finish(sgk_ctx* ctx, const KrylovWork<double>& kw, double* W, long long n, int M, double dt);

// exp(dt A) v by the persistent Arnoldi kernel, expm and the combination
void krylov_expv_persistent(sgk_ctx* ctx, const sgk_op* op, const PersistentWork& pw, const KrylovWork<double>& kw,
                            const double* v, double* W, long long n, int M, double dt);

PadeCoef pade13_coefficients();
void vk_dot(sgk_ctx* ctx, const double* a, const double* b, long long n, double* partials, double* out, int mode,
            const int* stop);
template <typename T>
void vk_mdot(sgk_ctx* ctx, const T* V, long long ldv, int ncols, const T* w, long long n, double* partials,
             double* out, const int* stop);
template <typename T>
void vk_gs_update(sgk_ctx* ctx, const T* V, long long ldv, int ncols, const double* h, T* w, long long n,
                  const int* stop);
void vk_convert(sgk_ctx* ctx, const double* x, float* y, long long n);
void vk_convert(sgk_ctx* ctx, const float* x, double* y, long long n);
void vk_convert(sgk_ctx* ctx, const double* x, dfloat* y, long long n);
void vk_convert(sgk_ctx* ctx, const dfloat* x, double* y, long long n);
void vk_convert(sgk_ctx* ctx, const dfloat* x, float* y, long long n);
void vk_axpby(sgk_ctx* ctx, double a, const double* x, double b, const double* y, double* z, long long n);
void vk_residual(sgk_ctx* ctx, const double* U, const double* F, const double* W, double c, double* G, long long n);
template <typename T>
void vk_jac_finish(sgk_ctx* ctx, const double* p, const T* Jp, double c, double* q, long long n);
void vk_cg_update(sgk_ctx* ctx, double* x, double* r, const double* p, const double* q, const double* rr,
                  const double* pq, long long n);
void vk_cg_direction(sgk_ctx* ctx, double* p, const double* r, const double* rr_new, const double* rr_old,
                     long long n);
void vk_copy_scalar(sgk_ctx* ctx, double* dst, const double* src);
void vk_basis_accumulate(sgk_ctx* ctx, const double* V, long long ldv, int m, const double* y, double* x,
                         long long n);
void vk_scale_from(sgk_ctx* ctx, const double* x, double* y, long long n, const double* s, const int* stop);
void gmres_givens(sgk_ctx* ctx, int j, int ld, double* Hg, double* cs, double* sn, double* g, const double* h1,
                  const double* h2, const double* hn2, double* report);
void gmres_solve(sgk_ctx* ctx, int m, int ld, const double* Hg, const double* g, double* y);
void gmres_init(sgk_ctx* ctx, double* g, int len, const double* beta, double* inv_beta);
void expm_e1(sgk_ctx* ctx, const double* H, int M, const int* m_dev, int m_fixed, double tau, double* ws, double* y);
template <typename T>
void krylov_expv_dev(sgk_ctx* ctx, const KrylovWork<T>& kw, const std::function<void(const T*, T*)>& matvec,
                     const double* v, double* W, long long n, int M, double dt);
