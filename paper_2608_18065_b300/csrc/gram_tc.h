// gram_tc.h -- T = A A^T for FP32 A with split BF16x3 tcgen05 products, and
// the centring / O'x stages that share its split (hi, lo) planes.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace nqs {
// Whether the tensor-core Gram is usable on this device (sm_103 and a
// tensor-map encoder from the driver).
bool gram_tc_available();
// Kernels one call of gram_tc_bf16x3 launches.
int gram_tc_launches();
// Bytes of scratch: the hi/lo planes [2][R][Kpad] bf16 and the K-slice partials.
size_t gram_tc_split_bytes(int64_t R, int64_t np);
// T[R x R] (FP64, both triangles) = A A^T, A row-major [R x np] FP32, from
// the four BF16 products of the split with compensated FP32 chunk sums.  *err
// (device int) receives NQS_ERR_TIMEOUT if a bounded device wait ran out.
cudaError_t gram_tc_bf16x3(const float *A, int64_t R, int64_t np, double *T, void *scratch,
                           int *err, cudaStream_t st);
// Step path: centre O (FP32, rows = Re block then Im block of ns samples) with
// the column means as FP32 pairs (hi, lo), scale by 1/sqrt(ns), split into
// the scratch planes ...
cudaError_t center_split(const float *O, int64_t ns, int64_t np, int64_t R, const float2 *mean,
                         void *scratch, cudaStream_t st);
// ... T from those planes (splits: K-slices per output tile, 0 = built-in
// plan, capped at gram_tc_max_splits) ...
cudaError_t gram_from_center_split(const void *scratch, int64_t R, int64_t np, double *T, int *err,
                                   cudaStream_t st, int splits = 0);
// Largest K-split the scratch of gram_tc_split_bytes(R, np) holds, and the
// built-in plan's choice.
int gram_tc_max_splits(int64_t R, int64_t np);
int gram_tc_default_splits(int64_t R, int64_t np);
// T in FP64 from the same planes (exact products, FP64 sums), only when
// *gate (device) is non-zero: the fallback when T + lambda I from the
// tensor cores is not positive definite at the requested lambda.
cudaError_t gram_split_f64(const void *scratch, int64_t R, int64_t np, double *T,
                           const int32_t *gate, cudaStream_t st);
// ... and partial sums of O'x from the same planes.
cudaError_t gemv_split(const void *scratch, int64_t R, int64_t np, const double *x, int rows_per,
                       double *part, cudaStream_t st);
}  // namespace nqs
