// recur_f32.cu -- float instantiation of the recurrence launchers.
#include "recur_impl.cuh"

namespace nqs {
template cudaError_t run_forward<float>(const RecDesc &, int, FwdArgs<float>, int, cudaStream_t);
template cudaError_t run_bwd<float>(const RecDesc &, BwdArgs<float>, cudaStream_t);
template cudaError_t run_grad<float>(const RecDesc &, GradArgs<float, float>, cudaStream_t);
template int eloc_max_grid<float>(const RecDesc &);
}  // namespace nqs
