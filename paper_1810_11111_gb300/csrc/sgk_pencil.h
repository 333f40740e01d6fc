// Fused last-direction reaction pass: shared declarations.
#pragma once

#include "sgk_quad.h"

struct PencilArgs {
    int H, N, ncell1, pad;
    long long npencils;
    long long cbase[SGK_MAX_LEVEL + 1];  // level chunks of the last direction
    const void* u[SGK_MAX_SPECIES];      // R_{d-1} of U per species
    const void* w[SGK_MAX_SPECIES];      // R_{d-1} of w per species (Jacobian)
    void* out[SGK_MAX_SPECIES];          // G_{d-1} per species
    const void* Tv;                      // rows of T, (N+1)(k+1) entries each
};

bool pencil_supported(int d, int kp1, int q, int S);
template <typename T>
void pencil_launch(sgk_ctx* ctx, const PencilArgs& a, int d, int kp1, int q, int S, bool jac, const double* B,
                   const double* w, const ReactionDev& rx);
