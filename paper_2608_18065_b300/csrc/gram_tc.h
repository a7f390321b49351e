// gram_tc.h -- T = A A^T for FP32 A with split BF16x3 tcgen05 products.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace nqs {
// Whether the tensor-core Gram is compiled in and usable on this device.
bool gram_tc_available();
// Kernels one call of gram_tc_bf16x3 launches.
int gram_tc_launches();
// Bytes of scratch the split (hi/lo BF16 copies of A) needs.
size_t gram_tc_split_bytes(int64_t R, int64_t np);
// T[R x R] (FP64, both triangles) = A A^T, A row-major [R x np] FP32.
cudaError_t gram_tc_bf16x3(const float *A, int64_t R, int64_t np, double *T, void *scratch,
                           cudaStream_t st);
}  // namespace nqs
