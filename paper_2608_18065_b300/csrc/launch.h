// launch.h -- internal host interface between the C-ABI layer and the
// templated recurrence kernels (one instantiation unit per precision).
#pragma once
#include <cuda_runtime.h>

#include "jacobian.cuh"

namespace nqs {

struct RecDesc {
  int dim, dh, N, Lx, cplx, marshall, zmask;
  int sm_count;
};

// Rows per CTA of each recurrence kernel.
template <typename T> struct Rows {
  static constexpr int SAMPLE_RT = 1, SAMPLE_RG = 8;
  static constexpr int ELOC_RT = sizeof(T) == 4 ? 4 : 2, ELOC_RG = 16;
  static constexpr int ELOC_RT_2D = sizeof(T) == 4 ? 4 : 1;
  static constexpr int BWD_RT = 1, BWD_RG = 8;
};

// Rows per thread of the local-energy sweep: fewer at hidden size 256 in 2D
// FP32, where four state buffers of 64 rows would exceed shared memory, and
// one at 200, where each thread holds 25 units.
template <typename T> constexpr int eloc_rt(int dim, int dh) {
  return dh == 200 ? 1  // 25 units per thread
         : dim == 2 ? (sizeof(T) == 4 && dh >= 256 ? 2 : Rows<T>::ELOC_RT_2D) : Rows<T>::ELOC_RT;
}

inline int eloc_rows(const RecDesc &d, bool f32) {
  return (f32 ? eloc_rt<float>(d.dim, d.dh) : eloc_rt<double>(d.dim, d.dh)) * 16;
}

// mode: MODE_SAMPLE / MODE_GIVEN / MODE_ELOC.  For MODE_ELOC, a.ntiles must
// be set; *grid_out receives the persistent grid used (for colbuf sizing,
// pass max_grid as the cap).
template <typename T>
cudaError_t run_forward(const RecDesc &d, int mode, FwdArgs<T> a, int max_grid, cudaStream_t st);
template <typename T> cudaError_t run_bwd(const RecDesc &d, BwdArgs<T> a, cudaStream_t st);
template <typename T> cudaError_t run_grad(const RecDesc &d, GradArgs<T, T> a, cudaStream_t st);
// Upper bound of the persistent ELOC grid (colbuf sizing).
template <typename T> int eloc_max_grid(const RecDesc &d);
bool dh_supported(int dh);

}  // namespace nqs
