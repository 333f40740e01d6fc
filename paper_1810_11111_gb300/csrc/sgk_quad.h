// Finest-grid quadrature of the reaction term: shared declarations.
#pragma once

#include "sgk_internal.h"

#define SGK_MAX_MONO 16

// Polynomial reaction, device copy passed by value to kernels.
struct ReactionDev {
    int nspecies = 1;
    int nmono = 0;
    int species[SGK_MAX_MONO] = {0};
    double coef[SGK_MAX_MONO] = {0};
    int exps[SGK_MAX_MONO][SGK_MAX_SPECIES] = {{0}};
};

struct Quad {
    const sgk_index* idx = nullptr;
    int d = 0, N = 0, kp1 = 0, q = 0, H = 0, nspecies = 1, maxstage = 0;
    Tables1D tab;
    std::vector<std::vector<long long>> layout_offsets;  // R_i block offsets, i = 0..d
    std::vector<long long> layout_size;                  // R_i total sizes
    long long full_size = 0;                             // H^d
    FiberPlan fwd[SGK_MAX_DIM][2], bwd[SGK_MAX_DIM][2];  // [direction][fp64, fp32]
    DevBuf<double> B64, w64;
    DevBuf<float> B32, w32;
    std::vector<double> B_host, w_host;  // q x (k+1) and q
    bool fused = false;                  // last direction runs in the pencil kernel
};

int reaction_degree(const ReactionDev& rx);
long long tuple_rank(const std::vector<int>& l, int n);
void quad_build(Quad& Q, const sgk_index* idx, int q, int nspecies, bool need_jacobian);
// Change of basis along directions 0..ndims-1 (ndims = d: to the full finest
// grid) and its transpose.
template <typename T>
void quad_forward(sgk_ctx* ctx, const Quad& Q, const T* in, T* final_nodal, T* tmp, int ndims);
template <typename T>
void quad_backward(sgk_ctx* ctx, const Quad& Q, T* moments, T* tmp, T* out, int ndims);
template <typename T>
void quad_cells(sgk_ctx* ctx, const Quad& Q, const ReactionDev& rx, bool jac, const T* const* u, const T* const* w,
                T* const* out);
void project_separable_dev(sgk_ctx* ctx, const sgk_index* idx, const Tables1D& tab, int nterms, const double* amp,
                           const int* wavenum, const int* kind, double c0, double* U);
// Load of non-zero Dirichlet data g (the restriction to the boundary of
// c0 + sum_t amp_t prod_m g_{t,m}(2 pi w x_m), as for the projection) on the
// device: b_a = -int_{dOmega} (k grad v_a . n - sigma/h v_a) g ds.
void dirichlet_load_dev(sgk_ctx* ctx, const sgk_index* idx, const Tables1D& tab, const double* kappa, double sigma,
                        int nterms, const double* amp, const int* wavenum, const int* kind, double c0, double* b);
