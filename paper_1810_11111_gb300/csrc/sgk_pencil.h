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
};

bool pencil_supported(int d, int kp1, int q, int S, const ReactionDev& rx);
// two_scale: [H_0, H_1, G_0, G_1], each (k+1) x (k+1) (Tables1D::two_scale)
template <typename T>
void pencil_launch(sgk_ctx* ctx, const PencilArgs& a, int d, int kp1, int q, int S, bool jac, const double* B,
                   const double* w, const double* two_scale, const ReactionDev& rx);
