// Persistent Arnoldi kernel instantiated for d = 4 (see arnoldi.cu).
#include "sgk_arnoldi.cuh"

template void sgk_arn::arn_launch_k<4>(sgk_ctx*, const sgk_op*, const sgk_arn::ArnArgs&, int, size_t, int);
template void sgk_arn::arn_multi_launch_k<4>(cudaStream_t, int, int, bool, const int*, const int2*, const void*,
                                              const sgk_arn::ArnArgs*, const int*, int, size_t, size_t, int);
template void sgk_arn::arn_multi_upload_ga<4>(const std::vector<const sgk_op*>&, DevBuf<unsigned char>&, cudaStream_t);
