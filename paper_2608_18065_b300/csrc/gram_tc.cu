// gram_tc.cu -- placeholder until the tcgen05 kernel is in.
#include "gram_tc.h"

namespace nqs {
bool gram_tc_available() { return false; }
int gram_tc_launches() { return 0; }
size_t gram_tc_split_bytes(int64_t, int64_t) { return 0; }
cudaError_t gram_tc_bf16x3(const float *, int64_t, int64_t, double *, void *, cudaStream_t) {
  return cudaErrorNotSupported;
}
}  // namespace nqs
