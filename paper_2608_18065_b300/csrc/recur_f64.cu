// recur_f64.cu -- double instantiation of the recurrence launchers.
#include "recur_impl.cuh"

namespace nqs {
template cudaError_t run_forward<double>(const RecDesc &, int, FwdArgs<double>, int, cudaStream_t);
template cudaError_t run_bwd<double>(const RecDesc &, BwdArgs<double>, cudaStream_t);
template cudaError_t run_grad<double>(const RecDesc &, GradArgs<double, double>, cudaStream_t);
template int eloc_max_grid<double>(const RecDesc &);
}  // namespace nqs
