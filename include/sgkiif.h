/*
 * sgkiif.h -- C ABI of libsgkiif, a CUDA (sm_103a) implementation of the
 * sparse-grid Krylov implicit-integration-factor DG method for
 * reaction-diffusion equations u_t = div(k grad u) + f(u) on [0,1]^d
 * (Liu, Cheng, Chen, Zhang, arXiv:1810.11111).
 *
 * Conventions shared by every call
 * --------------------------------
 * Status: every call that can fail returns an int status (SGK_OK = 0).  No
 *   C++ exception crosses this boundary.  The text of the last error of a
 *   context is returned by sgk_last_error().
 * Memory: the library owns every device buffer behind an opaque handle.  The
 *   caller owns every host buffer and every device buffer it passes in
 *   ("_dev" pointers are device pointers on the context's device, allocated
 *   by the caller, e.g. through PyTorch).  Handles are destroyed by the
 *   caller, children (solver, operator, index) before the context.
 * Streams: all device work of a context is issued on the stream given to
 *   sgk_ctx_create (0 = legacy default stream).  Calls returning host data
 *   synchronise that stream; the others are asynchronous unless noted.
 * Threads: a context and its children must be used by one host thread at a
 *   time.
 * Coefficient layout (sparse-grid vectors): the sparse-grid space is the sum
 *   of W_l over level tuples |l|_1 <= n (Section 2.1, eq. sp13).  Tuples are
 *   in lexicographic order with l_1 varying slowest; each tuple owns one
 *   contiguous block, row-major over the local 1D indices
 *   t_m = j_m (k+1) + p_m (dimension d fastest), where j_m is the support
 *   cell and p_m the degree of the 1D function on level l_m (eq. sp9, sp14).
 *   1D functions: level 0 = sqrt(2p+1) P_p(2x-1); level n >= 1 =
 *   2^{n/2} f_p(2^n x - (2j+1)) with Alpert's multiwavelets f_p fixed by
 *   vanishing moments (f_p orthogonal to x^i, i <= p+k) and the sign rule
 *   "first right-half Legendre coefficient of magnitude > 1e-8, scanned from
 *   degree k down, is positive".
 * Species-stacked vectors hold species s at offset s * dof.
 */
#ifndef SGKIIF_H
#define SGKIIF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define SGK_OK 0
#define SGK_EINVAL 1        /* bad argument (null, out of range, mismatch) */
#define SGK_ENOMEM 2        /* device or host allocation failed */
#define SGK_EUNSUPPORTED 3  /* valid request outside what is implemented */
#define SGK_ENEWTON 4       /* Newton did not converge; state rolled back */
#define SGK_ETIMEOUT 5      /* a bounded device wait ran out */
#define SGK_ECUDA 6         /* a CUDA runtime call failed */

/* precision modes */
#define SGK_FP64 0   /* all arithmetic in FP64 */
#define SGK_MIXED 1  /* solvers: the Jacobian products J_F(U) w of the
                        Newton inner solve, and the first residual of a step
                        (which seeds the first correction and never accepts),
                        in FP32; the Krylov matvec and every other F(U) (the
                        predictor's and each accepting Newton residual's) in
                        double-float arithmetic (pairs of FP32 numbers, about
                        48 significand bits; F in FP64 where the fused
                        reaction kernel does not serve the shape); the
                        Gram-Schmidt inner products and norms, exp(tau H), the
                        state and the Newton residual vector in FP64.  The
                        interpolation form of F (SGK_REACTION_INTERP) runs in
                        FP64 in both modes.  sgk_matvec with SGK_MIXED is
                        plain FP32. */

/* boundary conditions (Section 2.1, eq. sp3) */
#define SGK_PERIODIC 0
#define SGK_DIRICHLET0 1   /* homogeneous Dirichlet */

/* time schemes (Section 3) */
#define SGK_IIF2 2         /* eq. krylov5 */
#define SGK_IIF3 3         /* eq. krylov6 */
#define SGK_IIF_MAX_ORDER 6 /* schemes 2..6: the r-th order IIF of eqs. krylov3, krylov4 */

#define SGK_MAX_DIM 6
#define SGK_MAX_LEVEL 12
#define SGK_MAX_SPECIES 4
#define SGK_MAX_SOURCE_TERMS 8
#define SGK_MAX_KRYLOV 128

typedef struct sgk_ctx sgk_ctx;
typedef struct sgk_index sgk_index;
typedef struct sgk_op sgk_op;
typedef struct sgk_solver sgk_solver;

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device`, issuing work on `cuda_stream`
 * (a cudaStream_t; NULL makes the library create its own blocking stream,
 * which stays ordered with the legacy default stream).  Repeated sequences
 * (Krylov exponential, CG iteration, residual) are captured into CUDA graphs
 * on this stream, so it must not be the legacy default stream itself.  precision is SGK_FP64 or
 * SGK_MIXED and selects the arithmetic of solvers created on this context.
 * Errors: SGK_EINVAL (null out, bad precision), SGK_ECUDA (no such device). */
int sgk_ctx_create(sgk_ctx** out, int device, void* cuda_stream, int precision);
int sgk_ctx_destroy(sgk_ctx* ctx);
/* Text of the last error on this context ("" if none).  Owned by ctx. */
const char* sgk_last_error(const sgk_ctx* ctx);
/* Number of kernel launches this context has issued since creation. */
int64_t sgk_ctx_launch_count(const sgk_ctx* ctx);
/* Target architecture of the library's device code as the runtime sees it
 * (cudaFuncGetAttributes binaryVersion of one of its kernels, major * 10 +
 * minor: 103 for sm_103a) in *arch.  No counterpart in the paper; a check
 * that the loaded binary is the one built for this GPU.  Errors: SGK_EINVAL
 * (null arch), SGK_ECUDA (no device, or no image of the kernels loads on
 * it). */
int sgk_binary_arch(int* arch);
/* Measured arithmetic peak of one pipe (no counterpart in the paper; the
 * denominator of the ALU-bound rooflines).  Runs a kernel of independent
 * fused multiply-add chains (8 per thread, 8 CTAs of 256 threads per SM, on a
 * private stream of `device`, about 20 ms per launch, 3 untimed and 5 timed
 * launches) and writes the best timed rate in flop/s (2 per FMA) to
 * *flops_per_s.  kind: SGK_PEAK_FP32_FMA or SGK_PEAK_FP64_FMA.  Allocates
 * and frees a small device buffer; synchronises with its own events only.
 * Errors: SGK_EINVAL (null out, unknown kind, no such device), SGK_ECUDA. */
#define SGK_PEAK_FP32_FMA 0
#define SGK_PEAK_FP64_FMA 1
int sgk_alu_peak(int device, int kind, double* flops_per_s);
/* Kernel timing for benchmarks (no counterpart in the paper).  While bit i of
 * mask is set, every launch of kernel class i is bracketed by two CUDA events
 * on the context's stream.  Classes: 0 SIPG matvec, 1 change of basis to the
 * finest grid, 2 its transpose, 3 cell quadrature of the reaction term,
 * 4 inner products and Gram-Schmidt passes, 5 exp(tau H) e_1, 6 other vector
 * kernels, 7 a whole Krylov exponential replayed as one CUDA graph.  While
 * timing is enabled, sequences that are normally replayed as CUDA graphs run
 * as individual launches so that each kernel can be timed.  mask = 0
 * disables timing. */
int sgk_ctx_profile(sgk_ctx* ctx, unsigned mask);
/* Sum of event-timed milliseconds and launch counts per class (arrays of 8)
 * since the previous read; synchronises the stream and resets the sums. */
int sgk_ctx_profile_read(sgk_ctx* ctx, double* ms, int64_t* launches);

/* -------------------------------------------------------------- index set */

/* Build the sparse-grid index set {(l, j, p) : |l|_1 <= n} of degree-k
 * multiwavelets in d dimensions (Section 2.1, eqs. sp10-sp14) on the device:
 * enumerates the level tuples in the layout order above, their block sizes
 * (k+1)^d prod_m max(1, 2^{l_m-1}) and block offsets, and the level hash
 * (tuple -> block id).  d in [1, 6], n in [0, 12], k in [1, 3], else
 * SGK_EINVAL. */
int sgk_index_build(sgk_ctx* ctx, int d, int n, int k, sgk_index** out);
int sgk_index_destroy(sgk_index* idx);
/* Number of coefficients per species, (k+1)^d sum_l prod_m max(1,2^{l_m-1}). */
int64_t sgk_index_dof(const sgk_index* idx);
/* Number of level tuples, C(n+d, d). */
int64_t sgk_index_ntuples(const sgk_index* idx);
/* The same count as sgk_index_dof without building anything (host only, no
 * device needed): (k+1)^d sum_{|l|_1 <= n} prod_m max(1, 2^{l_m-1}), the
 * dimension of the space of eq. sp14.  -1 for d, n or k out of range. */
int64_t sgk_dof(int d, int n, int k);
/* Copy the tuple table to host: levels[ntuples*d] (row per tuple) and
 * offsets[ntuples+1] (block starts, offsets[ntuples] = dof).  cap is the
 * number of tuples the buffers hold; SGK_EINVAL if cap < ntuples.
 * Synchronises. */
int sgk_index_export(const sgk_index* idx, int32_t* levels, int64_t* offsets, int64_t cap);
/* Level hash: block id of each of `count` level tuples levels[count*d]
 * (host arrays), -1 for tuples outside the set.  Runs on the device.
 * Synchronises. */
int sgk_index_lookup(const sgk_index* idx, const int32_t* levels, int64_t count, int64_t* block_ids);

/* --------------------------------------------------------------- operator */

/* Assemble the SIPG diffusion operator A = -B for k(x) = diag(kappa) with
 * penalty sigma / h_n on every finest-mesh face (Section 2.1, bilinear form
 * B; the paper takes sigma = 20).  The 1D matrix S (one per bc) is built
 * once on the host in the hierarchical basis; A = -sum_i kappa_i S along
 * direction i restricted to the index set (unidirectional principle,
 * Section 4).  kappa: host array of d positive values.  bc: SGK_PERIODIC or
 * SGK_DIRICHLET0.  Errors: SGK_EINVAL.  For a tensor with off-diagonal
 * entries see sgk_operator_assemble_full. */
int sgk_operator_assemble(sgk_ctx* ctx, const sgk_index* idx, const double* kappa, int bc, double sigma,
                          sgk_op** out);
/* The same operator for a full constant symmetric positive definite
 * diffusion tensor K (Section 2.1: the PDE's k(x) constant with off-diagonal
 * entries; the bilinear form B with k grad u . grad v and the face terms of
 * eq. sp3).  K: host array d x d, row-major, symmetric, positive definite
 * (checked by a Cholesky factorisation), else SGK_EINVAL.  The diagonal
 * enters as for sgk_operator_assemble; every pair i < j with K_ij != 0 adds
 * -K_ij B_ij, B_ij = P x P^T + P^T x P - E x P^T - P^T x E - E^T x P -
 * P x E^T in 1D factors along i and j (P: test-function derivative against
 * trial value over the finest cells; E: test jump against trial average over
 * the faces), restricted to the index set.  sgk_matvec applies it in two
 * launches (the diagonal gather, then the mixed terms); solvers on such an
 * operator run the Arnoldi process as a sequence of launches instead of the
 * persistent kernel. */
int sgk_operator_assemble_full(sgk_ctx* ctx, const sgk_index* idx, const double* K, int bc, double sigma,
                               sgk_op** out);
/* Multiply-adds of one sgk_matvec: the entries of the 1D matrix rows each
 * output coefficient visits, summed over directions (the algorithmic work of
 * the unidirectional matvec of Section 4); -1 for a null handle. */
int64_t sgk_operator_madds(const sgk_op* op);
int sgk_operator_destroy(sgk_op* op);
/* Copy the 1D hierarchical matrix S (size H x H, H = (k+1) 2^n, row-major,
 * zeros included) to host `out` (cap >= H*H doubles).  Synchronises. */
int sgk_operator_export_1d(const sgk_op* op, double* out, int64_t cap);
/* y = A x on the device (eq. krylov1's A applied to a coefficient vector).
 * x_dev, y_dev: caller-owned device arrays of dof elements, FP64 when
 * precision == SGK_FP64 and FP32 when precision == SGK_MIXED; they must not
 * overlap.  Asynchronous. */
int sgk_matvec(const sgk_op* op, const void* x_dev, void* y_dev, int precision);

/* The 1D pieces of the mixed-derivative terms of the SIPG form of Section 2
 * for a full constant SPD diffusion tensor K (off-diagonal K_ij), in the
 * hierarchical basis of level n, degree k (H = (k+1) 2^n):
 *   P[a*H + b] = sum over finest cells of int v_a' v_b dx,
 *   E[a*H + b] = sum over faces of [v_a] {v_b} (jump of v_a, left trace minus
 *                right trace, one-sided times the outward normal on
 *                zero-Dirichlet boundary faces; average of the traces of v_b,
 *                one-sided on boundary faces).
 * Per pair i < j the operator adds -K_ij times
 *   P x P^T + P^T x P - E x P^T - P^T x E - E^T x P - P x E^T
 * (factors along directions i and j).  Host-only (the matvec with these
 * terms is sgk_operator_assemble_full's); P and E are host arrays of
 * cap >= H*H doubles.  n <= 10.  Errors: SGK_EINVAL (arguments), SGK_ENOMEM. */
int sgk_cross_blocks_1d(int n, int k, int bc, double* P, double* E, int64_t cap);

/* The 1D factors of the collocation matrix of the sparse-grid interpolation
 * form of the reaction term (SGK_REACTION_INTERP, see sgk_solver_create_form;
 * not the paper's F) at level n, degree k (H = (k+1) 2^n), as a dense
 * row-major H x H host array (cap >= H*H doubles):
 *   which = 0: A      Alpert coefficients -> interpolation surpluses,
 *           1: B      surpluses -> values at the collocation points,
 *           2: B^{-1} values -> surpluses,
 *           3: A^{-1} surpluses -> Alpert coefficients.
 * Host-only, n <= 10.  Errors: SGK_EINVAL (arguments), SGK_ENOMEM. */
int sgk_interp_factors_1d(int n, int k, int which, double* out, int64_t cap);

/* ------------------------------------------------------------- projection */

/* L2 projection (Theorem 2.4: u_h(0) = P u_0) of
 *   u_0(x) = const_term + sum_t amp[t] prod_m g_{t,m}(2 pi wavenum[t*d+m] x_m)
 * with g = sin for kind 0 and cos for kind 1, into coeffs_dev (device, FP64,
 * dof elements).  amp, wavenum, kind are host arrays of nterms (times d)
 * entries.  1D integrals use 12-point Gauss quadrature per finest cell.
 * Asynchronous. */
int sgk_project_separable(sgk_ctx* ctx, const sgk_index* idx, int nterms, const double* amp, const int* wavenum,
                          const int* kind, double const_term, double* coeffs_dev);
/* Load vector of non-zero Dirichlet data (Section 2.1: the boundary term of
 * L(v) for u = g on dOmega): b_a = -int_{dOmega} (k grad v_a . n - sigma/h
 * v_a) g ds, h the finest mesh size, k = diag(kappa), for g the restriction
 * to the boundary of const_term + sum_t amp[t] prod_m g_{t,m}(2 pi
 * wavenum[t*d+m] x_m), g = sin (kind 0) or cos (kind 1) -- the family of
 * sgk_project_separable.  The paper prints the penalty part with a plus
 * sign; the sign taken here is the one under which smooth solutions satisfy
 * the scheme (exact for polynomial data of degree <= k).  With the
 * zero-Dirichlet operator (SGK_DIRICHLET0, same kappa and sigma) the
 * semi-discrete system is dU/dt = A U + F(U) + b; data e^{lambda t} g(x)
 * enter a solver as the source term (lambda, b) (sgk_solver_set_source).
 * kappa: host array of d positive values; b_dev: caller-owned device array
 * of dof doubles.  Synchronises.  Errors: SGK_EINVAL. */
int sgk_dirichlet_load(sgk_ctx* ctx, const sgk_index* idx, const double* kappa, double sigma, int nterms,
                       const double* amp, const int* wavenum, const int* kind, double const_term, double* b_dev);

/* ---------------------------------------------------------------- solver */

/* Polynomial reaction term: f_s(u) = sum over monomials m with species[m] == s
 * of coef[m] prod_r u_r^{exps[m*nspecies + r]}.  Host arrays. */
typedef struct sgk_reaction {
    int nspecies;            /* 1 .. SGK_MAX_SPECIES */
    int nmono;               /* number of monomials (0 = no reaction) */
    const int* species;      /* [nmono] species whose f the monomial adds to */
    const double* coef;      /* [nmono] */
    const int* exps;         /* [nmono * nspecies] exponents, each 0..4 */
} sgk_reaction;

/* Newton / inner-solver options; zero fields take the defaults shown. */
typedef struct sgk_newton_opts {
    double tol;        /* outer stop ||G||_2 <= tol max(||W||_2, ||G(W)||_2), relative to
                          the stage's scale (W the exponential term, G(W) the first
                          residual); 1e-12 */
    int max_iter;      /* outer cap; 50 */
    double inner_tol;  /* CG/GMRES relative residual; 1e-13 (FP64), 1e-6 (mixed) */
    int inner_max;     /* inner iteration cap; 500 */
    int gmres_restart; /* GMRES restart length (systems); 50 */
} sgk_newton_opts;

/* Create an IIF solver for nspecies species on one index set.  scheme is
 * the order r of the IIF scheme (eqs. krylov3, krylov4), 2 <= r <=
 * SGK_IIF_MAX_ORDER: SGK_IIF2 (eq. krylov5), SGK_IIF3 (eq. krylov6), ...
 * The exp(dt A) terms of U^n and F(U^n) are one Krylov projection of
 * U^n + alpha_0 dt F(U^n); every older F(U^{n-i}) is a projection over
 * (i+1) dt; the Newton weight is alpha_1 dt.  A step uses the highest order
 * its history of F values allows: the first step after creation,
 * sgk_solver_set_state, sgk_solver_set_time or sgk_solver_set_source is an
 * IIF2 step, the next an IIF3 step, and so on up to r (with this start-up
 * the global order is min(r, 3)).  ops[s] is the diffusion operator of
 * species s (all on the same index set).  krylov_m in [1, 128], dt > 0.  The
 * reaction term uses finest-mesh Gauss quadrature with q = ceil((p k + k + 1)/2)
 * points per direction for total polynomial degree p, i.e. the exact L2
 * projection of f(u_h).  The finest full grid must fit in device memory
 * ((k+1) 2^n)^d nodal values per species); else SGK_ENOMEM.
 * opts may be NULL.  Errors: SGK_EINVAL, SGK_ENOMEM, SGK_EUNSUPPORTED (scheme
 * out of range). */
int sgk_solver_create(sgk_ctx* ctx, int nspecies, const sgk_op* const* ops, const sgk_reaction* f, int scheme,
                      int krylov_m, double dt, const sgk_newton_opts* opts, sgk_solver** out);

/* Forms of the reaction term F(U) */
#define SGK_REACTION_QUADRATURE 0 /* the paper's: the L2 projection of f(u_h) by
                                     Gauss quadrature on the finest full grid
                                     (Section 4), as sgk_solver_create */
#define SGK_REACTION_INTERP 1     /* a deviation from the paper, for its first
                                     stated future direction (Section 5: an
                                     evaluation of the reaction integral that
                                     uses the structure of the basis): the
                                     Alpert coefficients of the sparse-grid
                                     interpolant of f(u_h) on nested
                                     collocation points, one per coefficient */

/* sgk_solver_create with a choice of the reaction form.  With
 * SGK_REACTION_INTERP, F_I(U) = C^{-1} f(C U), C the collocation matrix of
 * the sparse set (u_h at the points), applied as 2d passes of 1D factors
 * along the directions (sgk_interp_factors_1d); equal to the quadrature form
 * for linear f, within an interpolation error of it otherwise.  It needs no
 * finest full grid, so every shape whose sparse-grid vectors fit in device
 * memory is accepted.  The implicit stage U - c F_I(U) = W becomes one
 * equation per collocation point, u - c f(u) = (C W)_p, solved by Newton's
 * method at each point to rounding (at most opts->max_iter corrections,
 * else SGK_ENEWTON and the step is rolled back); sgk_stats counts the most
 * corrections any point took per step, and no inner iterations.  The
 * transforms and the point solve run in FP64 in both precision modes; IIF2
 * steps with any species count run as one CUDA graph.  Errors as
 * sgk_solver_create, and SGK_EINVAL for an unknown form. */
int sgk_solver_create_form(sgk_ctx* ctx, int nspecies, const sgk_op* const* ops, const sgk_reaction* f, int scheme,
                           int krylov_m, double dt, const sgk_newton_opts* opts, int reaction_form,
                           sgk_solver** out);
int sgk_solver_destroy(sgk_solver* s);
/* The weights of the r-th order IIF scheme (eq. krylov4) into alpha[0..r-1]:
 * alpha_1, alpha_0, alpha_{-1}, ..., alpha_{-(r-2)} (the integrals over one
 * step of the Lagrange basis polynomials on the nodes t^{n+1}, t^n, ...,
 * t^{n+2-r}).  Host-only; 2 <= r <= SGK_IIF_MAX_ORDER, else SGK_EINVAL. */
int sgk_iif_alpha(int r, double* alpha);
/* Set the coefficients of one species (FP64, dof elements) from host memory
 * (on_device = 0) or from a device array (on_device = 1). */
int sgk_solver_set_state(sgk_solver* s, int species, const double* coeffs, int on_device);
/* Take nsteps steps of the solver's scheme.  Arnoldi breakdown truncates the Krylov basis and
 * is not an error.  On Newton failure the state is rolled back to the start
 * of the failing step and SGK_ENEWTON is returned.  Synchronises. */
int sgk_solver_step(sgk_solver* s, int nsteps);
/* Queue nsteps steps without waiting for them, for callers that keep the GPU
 * busy while the host prepares more work.  Applies when the step is one
 * device-driven graph (IIF2 with one species or no reaction, graphs on, no
 * kernel timing); otherwise the steps run synchronously, as in
 * sgk_solver_step, and a failure is returned at once.  Up to 32 steps are
 * queued (fewer when 32 saved states would exceed 256 MB); beyond that the
 * call waits for the queued ones.  Each queued step saves the state it starts
 * from, so a failing step is rolled back as in sgk_solver_step and the steps
 * queued after it are discarded.  The outcome is reported by
 * sgk_solver_wait; every other call on the solver first finishes the queued
 * steps (sgk_solver_step also reports a pending failure). */
int sgk_solver_step_async(sgk_solver* s, int nsteps);
/* Wait for the queued steps.  Returns SGK_OK, or the status of the first
 * failing one (SGK_ENEWTON, SGK_ETIMEOUT), with the state rolled back to
 * the start of that step. */
int sgk_solver_wait(sgk_solver* s);
/* Copy one species' coefficients (FP64) to host (on_device = 0) or to a
 * device array (on_device = 1); cap >= dof.  Host copies synchronise. */
int sgk_solver_get_state(const sgk_solver* s, int species, double* out, int64_t cap, int on_device);

/* Source term of species s for u_t = div(k grad u) + f(u) + s(x, t)
 * (Examples 2 and 3, Section 4), given as nterms terms e^{lambda_m t} g_m(x):
 * the scheme's F becomes F(U, t) = P f(u_h) + sum_m e^{lambda_m t} S_m with
 * S_m = P g_m, the caller's projected coefficient vectors (for separable g_m
 * from sgk_project_separable).  Every F is taken at the time of its argument:
 * F(U^n) at t^n, the Newton stage F(U^{n+1}) at t^n + dt, and IIF3's
 * F(U^{n-1}) at t^n - dt.
 * lambda: host array of nterms finite values.  coeffs_dev: device array of
 * nterms * dof FP64 values, term m at offset m * dof; the solver copies it
 * (the caller keeps ownership).  nterms = 0 removes the species' source;
 * nterms <= SGK_MAX_SOURCE_TERMS.  The source is added in FP64 in both
 * precision modes.  A source needs a reaction term (a monomial with
 * coefficient 0 is one): SGK_EUNSUPPORTED otherwise.  Errors: SGK_EINVAL (bad
 * species or nterms, null pointers, non-finite lambda).  Synchronises. */
int sgk_solver_set_source(sgk_solver* s, int species, int nterms, const double* lambda, const double* coeffs_dev);
/* The time t^n of the current state: 0 at creation, dt more after every
 * accepted step (a failed step leaves it).  Setting it drops the cached
 * F(U^n) and IIF3's F(U^{n-1}) (the next IIF3 step is an IIF2 step) unless t
 * equals the current time. */
int sgk_solver_set_time(sgk_solver* s, double t);
int sgk_solver_get_time(const sgk_solver* s, double* t);
/* Sub-projections of the exponential (an extension: the paper takes one
 * projection of dimension M per exponential, eq. krylov8).  With substeps =
 * s > 1 every exp(tau A) v of the following steps (also sgk_krylov_expv) is
 * the semigroup product exp((tau/s) A)^s v taken as s successive
 * projections of dimension M, each of a time span tau/s.  Its error falls
 * steeply with the span when tau rho(A) is large; the cost is s Arnoldi
 * processes.  Use it where the a-posteriori estimate (sgk_stats) is above
 * the accuracy wanted.  1 <= substeps <= SGK_MAX_KRYLOV_SUBSTEPS; 1 restores
 * the paper's method.  A solver with substeps > 1 steps with its own
 * Arnoldi launches inside sgk_batch (not the batched ones).  Drains queued
 * steps; allocates one more vector of dof doubles on first use.  Errors:
 * SGK_EINVAL (null, substeps out of range), SGK_ENOMEM. */
#define SGK_MAX_KRYLOV_SUBSTEPS 64
int sgk_solver_set_krylov_substeps(sgk_solver* s, int substeps);
/* Accuracy guard on the Krylov projections (an extension, as above).  With
 * tol > 0, every synchronous sgk_solver_step compares the a-posteriori
 * estimate of its projections (sgk_stats) with tol and, while it is larger
 * and the sub-projections number less than max_substeps, doubles them (as
 * sgk_solver_set_krylov_substeps, kept for the following steps) and takes
 * the step's exponentials again: IIF2 steps run as one graph restart from
 * their starting state, the host-driven steps (systems, IIF3 and higher)
 * redo their exponentials before the Newton stage.  The count of doublings
 * is sgk_stats.krylov_refinements.  Batches and the server apply it to the
 * instances and requests that set sgk_request.krylov_tol: a rolled-back step
 * is taken again in the next batch step, which then still gives every
 * instance its nsteps steps.  Queued steps (sgk_solver_step_async) report
 * the estimate without acting on it.  tol = 0 turns the guard off (the
 * default).  Drains queued steps.  Errors:
 * SGK_EINVAL (null, tol negative or not finite, max_substeps outside
 * 1..SGK_MAX_KRYLOV_SUBSTEPS). */
int sgk_solver_set_krylov_tolerance(sgk_solver* s, double tol, int max_substeps);

typedef struct sgk_stats {
    int64_t steps;           /* steps taken since creation */
    int64_t newton_iters;    /* total Newton corrections */
    int64_t inner_iters;     /* total CG/GMRES iterations */
    int64_t krylov_calls;    /* Krylov exponentials evaluated */
    int64_t krylov_breakdowns; /* of which truncated by happy breakdown */
    int last_m_eff;          /* Krylov dimension of the last exponential */
    double last_newton_residual;
    /* A-posteriori estimate of the Krylov projection's error in the last
     * step (largest over species, over the step's exponentials and over
     * their sub-projections), relative to the projected result:
     * h_{m+1,m} |e_m^T exp(dt H_m) e_1| / ||exp(dt H_m) e_1|| (the
     * residual-type estimate of Saad 1992; 0 after a happy breakdown).  The
     * paper takes a fixed M with no error control (Section 3); this reports
     * how far that M is from converged without changing the method. */
    double last_krylov_err_est;
    double max_krylov_err_est;  /* the largest of those over all steps taken */
    int krylov_substeps;        /* sub-projections per exponential now (1: the paper's method) */
    int64_t krylov_refinements; /* times the accuracy guard doubled them */
} sgk_stats;
int sgk_solver_stats(const sgk_solver* s, sgk_stats* out);

/* Component entry points of the step, for testing and benchmarking.  All
 * vectors are caller-owned device arrays, FP64, species-stacked.  They use
 * the solver's precision mode internally and are asynchronous. */
/* F(U) = (int f(u_h) v_a dx)_a, finest-grid Gauss quadrature (Section 4),
 * plus the source terms at the solver's time t^n when set; FP64 in both
 * precision modes. */
int sgk_reaction_eval(sgk_solver* s, const double* u_dev, double* f_dev);
/* J_F(U) w = (int f'(u_h) w_h v_a dx)_a with the same quadrature (FP32
 * passes in SGK_MIXED). */
int sgk_jacobian_apply(sgk_solver* s, const double* u_dev, const double* w_dev, double* jw_dev);
/* w = gamma V_M exp(dt H_M) e_1 ~ exp(dt A_s) v for species s (eqs.
 * krylov7-krylov8, Arnoldi with classical Gram-Schmidt applied twice).
 * m_eff (host, may be NULL) receives the Krylov dimension used.  With
 * sub-projections (sgk_solver_set_krylov_substeps) w is their product and
 * m_eff, like sgk_krylov_export, describes the last of them.
 * Synchronises.  SGK_ETIMEOUT: a grid barrier of the persistent Arnoldi
 * kernel ran out of time (w is then undefined; the solver stays usable).
 * Setting the environment variable SGK_TEST_BARRIER_STALL makes those
 * barriers wait for one CTA more than the grid has, so that the bounded
 * waits run out (failure test). */
int sgk_krylov_expv(sgk_solver* s, int species, const double* v_dev, double* w_dev, int* m_eff);
/* Copy the Hessenberg matrix ((M+1) x M, row-major) and the Krylov basis
 * (M+1 columns of dof, column-major, FP64) of the last sgk_krylov_expv call
 * to host.  Either pointer may be NULL.  Synchronises. */
int sgk_krylov_export(const sgk_solver* s, double* H, double* V, int64_t cap_V);
/* y = exp(tau X) e_1 for the m x m row-major matrix X (host), by Pade(13)
 * scaling and squaring on the device (Section 3; Higham 2005).  m in
 * [1, 128].  y: host array of m doubles.  Synchronises. */
int sgk_expm_e1(sgk_ctx* ctx, int m, const double* X, double tau, double* y);

/* Largest m accepted by sgk_expm_e1_noalloc. */
#define SGK_EXPM_NOALLOC_MAX_M 64
/* The same y = exp(tau X) e_1 as sgk_expm_e1, for callers that must not
 * allocate device memory while they run: code that is being recorded into a
 * CUDA graph (where cudaMalloc/cudaFree are not recorded and cudaFree
 * synchronises the device), latency-critical loops, and processes whose
 * device memory is owned by another allocator (e.g. a framework's caching
 * allocator).  The paper has no counterpart; this is a service entry point.
 * X_dev (m x m, row-major) and y_dev (m doubles) are caller-owned device
 * arrays on the current device; the work is queued on cuda_stream (NULL =
 * legacy default stream) and the call returns without synchronising.
 * Scratch: for m <= 56 the work matrices live in the shared memory of one
 * eight-CTA thread-block cluster (up to 196 KB per CTA) and calls are
 * independent of each other.  For 56 < m <= 64 they live in a fixed
 * 8 * 64 * 64 doubles (256 KB) array compiled into the library, held by
 * every GPU that loads it until the process exits; m above
 * SGK_EXPM_NOALLOC_MAX_M is rejected with SGK_EINVAL.  The first call on a
 * device does a one-time set-up there: it looks up that array's device
 * address (cudaGetSymbolAddress) and raises the cluster kernel's
 * shared-memory limit (cudaFuncSetAttribute), so make one call on each
 * device before any stream capture.  The set-up is kept per device and made
 * again if the device's context changes (after cudaDeviceReset), so that an
 * address from a destroyed context is never used.  Calls with m > 56 share
 * the one array: those that may overlap on the GPU (different streams, or
 * different host threads) race and must be serialised by the caller.  No
 * context, no allocation, no host copy.  Errors: SGK_EINVAL (bad m or null
 * pointer), SGK_ECUDA (no current device, or the set-up or launch failed). */
int sgk_expm_e1_noalloc(int m, const double* X_dev, double tau, double* y_dev, void* cuda_stream);

/* -------------------------------------------------------------- serving */

/* A request loop that runs whole IIF2 solves (the problem of Section 2 with
 * the scheme of eq. krylov5, one per request) as they arrive.  The paper has
 * no counterpart; this is the service around the method.
 *
 * Continuous batching: a server owns an engine thread (see
 * sgk_server_set_engine) and nworkers worker threads, each with its own CUDA
 * stream on one device.  A submitted request waits in a queue until the
 * engine has room (single-species requests) or a worker is idle (the others),
 * and its estimated device memory (sgk_estimate_bytes) fits in what the
 * admitted requests leave of the budget; requests are admitted in arrival
 * order, except that a request that does not fit yet lets later ones that do
 * fit go first unless it has waited longer than the aging limit.  Admitted
 * requests run concurrently: the engine's requests step together in batched
 * launches, the workers' kernels overlap with them on the GPU; each keeps
 * its Krylov basis and state on the device until it finishes, and its memory
 * returns to the budget when it does.  Results do not depend on what else
 * runs: a request gives the same coefficients alone and in a mix on a server
 * with the same worker count and engine setting. */
typedef struct sgk_server sgk_server;

/* Initial data of one species: coefficients (host, dof doubles) if coeffs is
 * not NULL, else the L2 projection of const_term + sum_t amp[t] prod_m
 * g_{t,m}(2 pi wavenum[t*d+m] x_m) as for sgk_project_separable. */
typedef struct sgk_init {
    const double* coeffs;
    int nterms;
    const double* amp;
    const int* wavenum;
    const int* kind;
    double const_term;
} sgk_init;

typedef struct sgk_request {
    int d, n, k;             /* sparse grid V_N^k in d dimensions (as sgk_index_build) */
    int nspecies;            /* 1 .. SGK_MAX_SPECIES */
    int bc;                  /* SGK_PERIODIC | SGK_DIRICHLET0 */
    const double* kappa;     /* [nspecies * d] diagonal diffusion per species */
    sgk_reaction reaction;   /* as for sgk_solver_create (nspecies must match) */
    int krylov_m;            /* 1 .. SGK_MAX_KRYLOV */
    double dt;               /* > 0 */
    int nsteps;              /* >= 0 IIF2 steps */
    int precision;           /* SGK_FP64 | SGK_MIXED */
    sgk_init init[SGK_MAX_SPECIES];
    double krylov_tol;       /* > 0: the Krylov accuracy guard (sgk_solver_set_krylov_tolerance); 0: off */
    int krylov_max_substeps; /* its limit, 1 .. SGK_MAX_KRYLOV_SUBSTEPS (ignored when krylov_tol = 0) */
    int reaction_form;       /* SGK_REACTION_QUADRATURE (0, the paper's) | SGK_REACTION_INTERP */
} sgk_request;

typedef struct sgk_result_info {
    int status;              /* SGK_OK or the solve's error code */
    int nspecies;
    int64_t dof;             /* per species */
    int64_t steps;           /* steps taken */
    int64_t est_bytes;       /* device memory reserved at admission */
    double queue_ms;         /* submit -> admission */
    double run_ms;           /* admission -> result on the host */
    double latency_ms;       /* submit -> result on the host */
    int worker;              /* worker that ran it */
    int64_t newton_iters, inner_iters;
    char error[160];         /* error text when status != SGK_OK, else empty */
    double krylov_err_est;   /* largest a-posteriori Krylov error estimate over its steps (sgk_stats) */
} sgk_result_info;

typedef struct sgk_server_stats {
    int64_t submitted, completed, failed, rejected;
    int64_t queued, running;
    int64_t budget_bytes, reserved_bytes, peak_reserved_bytes;
    int max_concurrent;      /* most requests running at once so far */
} sgk_server_stats;

/* Device memory a request will hold while it runs (index, operators, solver
 * workspace including the finest-grid reaction buffers), in bytes; -1 for an
 * invalid shape.  Host only. */
int64_t sgk_estimate_bytes(int d, int n, int k, int nspecies, int krylov_m, int precision, int has_reaction);

/* Estimated arithmetic of one IIF2 step of a problem, for sharding
 * independent instances across GPUs (no counterpart in the paper): per
 * species the Arnoldi process (M matvecs of 2 (entries per row) DOF operations and
 * the two Gram-Schmidt passes, 4 M^2 DOF) and, with a reaction, about three
 * finest-grid passes (predictor, residual and one Jacobian product: the
 * sum-factorised quadrature of (2^n)^d cells).  Relative units: only ratios
 * between instances matter.  -1 for an invalid shape.  Host only. */
double sgk_estimate_work(int d, int n, int k, int nspecies, int krylov_m, int has_reaction);
/* Split `count` independent work items of estimated cost cost[i] >= 0 over
 * nparts parts (ranks) so that the largest part sum is small: the items in
 * order of decreasing cost (ties by index), each to the part with the
 * smallest sum so far (ties by part index) -- the longest-processing-time
 * rule, at most 4/3 of the optimum.  part_of[count] receives each item's
 * part; deterministic, so every rank computes the same split without
 * communicating.  Errors: SGK_EINVAL (null arrays, count < 0, nparts < 1, a
 * negative or non-finite cost).  Host only. */
int sgk_partition(int count, const double* cost, int nparts, int* part_of);

/* Start a server on device with nworkers (1 .. 64) workers and a device
 * memory budget of mem_budget_bytes (0 = 80% of the memory free at start).
 * aging_ms: how long a request that does not fit may be overtaken (<= 0:
 * 2000 ms).  Errors: SGK_EINVAL, SGK_ECUDA, SGK_ENOMEM. */
int sgk_server_create(int device, int nworkers, int64_t mem_budget_bytes, double aging_ms, sgk_server** out);
/* The server's engine (on by default): single-species requests with d in
 * 2..4 are not given to a worker but join a running batch, stepped one IIF2
 * step per tick for all of its requests together (iteration-level
 * continuous batching): per request a pre-Krylov CUDA graph, then one
 * persistent cooperative Arnoldi launch per kernel class for all of them
 * (as sgk_batch), then per request a post-Krylov graph with the Newton
 * solve.  Requests join between ticks once admitted (same memory rule) and
 * leave after their last step; their result info reports worker -1.
 * Systems (host-driven GMRES) stay with the workers.  on = 0 sends every
 * request to the workers; max_requests > 0 caps the requests in the engine
 * at once (default 64).  Takes effect for requests admitted after the call.
 * Errors: SGK_EINVAL. */
int sgk_server_set_engine(sgk_server* srv, int on, int max_requests);
/* Queue a request; every host array it points to is copied before the call
 * returns.  *ticket identifies it.  Errors: SGK_EINVAL (bad request),
 * SGK_ENOMEM (its estimate exceeds the whole budget: rejected). */
int sgk_server_submit(sgk_server* srv, const sgk_request* req, int64_t* ticket);
/* 1 if the request has finished, 0 if not, negative for an unknown ticket. */
int sgk_server_poll(sgk_server* srv, int64_t ticket);
/* Wait up to timeout_ms (< 0: no limit) for a request; on completion fill
 * info (may be NULL) and copy its final coefficients (species-stacked,
 * nspecies * dof doubles) to out (may be NULL; cap in doubles), then forget
 * the ticket.  Returns SGK_OK once finished (the solve's own status is in
 * info->status), SGK_ETIMEOUT if still running, SGK_EINVAL for an unknown
 * ticket or a too-small buffer. */
int sgk_server_wait(sgk_server* srv, int64_t ticket, double timeout_ms, sgk_result_info* info, double* out,
                    int64_t cap);
int sgk_server_get_stats(sgk_server* srv, sgk_server_stats* out);
/* Finish every queued and running request, then stop the workers. */
int sgk_server_destroy(sgk_server* srv);

/* ------------------------------------------------------------- batching */

/* Many independent IIF2 problems of uneven size stepped together on one
 * device (the paper's method applied to each, eqs. krylov5-krylov8 per
 * instance; no counterpart in the paper).  Each instance owns its index set,
 * operators and solver on its own library context; instances are spread
 * round-robin over the batch's nstreams streams.  A batch step runs the
 * Arnoldi processes (eqs. krylov7, krylov8) of all single-species instances
 * with d in 2..4 in one persistent cooperative launch per kernel class
 * (d, degree, lanes per output, arithmetic): each CTA walks a device work
 * list of (instance, slice) items, built once by list scheduling, so that
 * instances of uneven size share the SMs within one grid.  Around it, per
 * instance on its stream, one CUDA graph before (predictor) and one after
 * (exp(tau H) e_1, combination, and the Newton/CG loops as conditional
 * graph nodes).  Other instances take one whole-step graph each.  The host
 * waits for all streams once per batch step.  The Arnoldi grid of an
 * instance is sized to its DOF (slices of at most slice_len coefficients
 * per CTA, 0 = 384); the lanes per output of its matvec are autotuned when
 * the instance is added.  Results do not depend on the stream count, on
 * the batched launch or on the other instances. */
typedef struct sgk_batch sgk_batch;

/* Errors: SGK_EINVAL, SGK_ECUDA (no such device or stream creation failed). */
int sgk_batch_create(int device, int nstreams, int slice_len, sgk_batch** out);
/* Add an instance described by req (its nsteps is ignored; its krylov_tol
 * and krylov_max_substeps set the instance's accuracy guard); host arrays
 * are read during the call.  *index receives the instance number (0, 1,
 * ...).  Errors: as sgk_index_build / sgk_operator_assemble /
 * sgk_solver_create / sgk_solver_set_krylov_tolerance. */
int sgk_batch_add(sgk_batch* b, const sgk_request* req, int* index);
/* Take nsteps steps of every active instance.  status (may be NULL) receives
 * per instance the status of its last step; an instance whose step fails is
 * rolled back to the start of that step and takes no further steps.  A step
 * that an instance's accuracy guard rolls back is taken again in a later
 * batch step of the same call.  Returns SGK_OK if every instance succeeded,
 * else the first failing status. */
int sgk_batch_step(sgk_batch* b, int nsteps, int* status);
int64_t sgk_batch_dof(const sgk_batch* b, int index);
int sgk_batch_count(const sgk_batch* b);
/* Copy one species' coefficients of an instance to host memory (cap >= dof). */
int sgk_batch_get_state(const sgk_batch* b, int index, int species, double* out, int64_t cap);
/* Statistics of one instance's solver (as sgk_solver_stats). */
int sgk_batch_stats(const sgk_batch* b, int index, sgk_stats* out);
int sgk_batch_destroy(sgk_batch* b);
/* on = 0: run every instance's Arnoldi process inside its own whole-step
 * graph instead of the batched launches (for comparison); default 1. */
int sgk_batch_set_fused(sgk_batch* b, int on);
/* Kernels launched by the batched Arnoldi path so far (barrier reset and one
 * per class and batch step); -1 for a null handle. */
int64_t sgk_batch_launches(const sgk_batch* b);

#ifdef __cplusplus
}
#endif
#endif /* SGKIIF_H */
