// Persistent Arnoldi kernel instantiated for d = 4 (see arnoldi.cu).
#include "sgk_arnoldi.cuh"

template void sgk_arn::arn_launch_k<4>(sgk_ctx*, const sgk_op*, const sgk_arn::ArnArgs&, int, size_t, int);
