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

inline int eloc_rows(const RecDesc &d, bool f32) {
  if (f32) return (d.dim == 2 ? Rows<float>::ELOC_RT_2D : Rows<float>::ELOC_RT) * 16;
  return (d.dim == 2 ? Rows<double>::ELOC_RT_2D : Rows<double>::ELOC_RT) * 16;
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
