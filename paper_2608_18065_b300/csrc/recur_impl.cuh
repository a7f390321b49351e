// recur_impl.cuh -- host launchers of the templated recurrence kernels,
// dispatching the runtime hidden size and lattice dimension onto the
// compile-time instantiations.
#pragma once
#include "launch.h"

namespace nqs {

#define NQS_DISPATCH_DH(dh, ...)                          \
  switch (dh) {                                           \
    case 8: { constexpr int DH = 8; __VA_ARGS__; } break;    \
    case 16: { constexpr int DH = 16; __VA_ARGS__; } break;  \
    case 32: { constexpr int DH = 32; __VA_ARGS__; } break;  \
    case 64: { constexpr int DH = 64; __VA_ARGS__; } break;  \
    case 96: { constexpr int DH = 96; __VA_ARGS__; } break;  \
    case 128: { constexpr int DH = 128; __VA_ARGS__; } break;  \
    case 200: { constexpr int DH = 200; __VA_ARGS__; } break;  \
    case 256: { constexpr int DH = 256; __VA_ARGS__; } break;  \
    default: return cudaErrorInvalidValue;                \
  }

// Unit groups of the sampling / given-configuration sweeps: the FP32 d_h = 64
// sweep runs two hidden units per thread (eight warps per CTA) instead of
// four, the others the default tile.
template <typename T, int DH> constexpr int sample_groups() {
  return (sizeof(T) == 4 && DH == 64) ? 32 : 0;
}

// Shared memory above this leaves the large weight blocks in global memory.
constexpr size_t SMEM_STAGE_LIMIT = 200 * 1024;

template <typename T, int DH, int DIM, int RT, int RG, int MODE, int UGX = 0>
static cudaError_t fwd_one(const RecDesc &d, FwdArgs<T> a, int max_grid, cudaStream_t st) {
  constexpr int R = RT * RG;
  constexpr int UG = UGX ? UGX : Tile<DH>::UG;
  auto kern = k_forward<T, DH, DIM, RT, RG, MODE, true, UGX>;
  size_t smem = fwd_smem_bytes<T, DH, DIM, R>(d.N, true);
  if constexpr (DH >= 96) {
    if (smem > SMEM_STAGE_LIMIT) {
      smem = fwd_smem_bytes<T, DH, DIM, R>(d.N, false);
      kern = k_forward<T, DH, DIM, RT, RG, MODE, false, UGX>;
    }
  }
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (MODE != MODE_ELOC) a.ntiles = (int)((a.nrows + R - 1) / R);
  int grid = a.ntiles;
  if (MODE == MODE_ELOC) grid = grid < max_grid ? grid : max_grid;
  if (grid <= 0) return cudaSuccess;
  kern<<<grid, UG * RG, smem, st>>>(a);
  return cudaGetLastError();
}

template <typename T, int DH, int DIM>
static cudaError_t fwd_dim(const RecDesc &d, int mode, FwdArgs<T> a, int max_grid, cudaStream_t st) {
  constexpr int ERT = eloc_rt<T>(DIM, DH);
  if (mode == MODE_SAMPLE)
    return fwd_one<T, DH, DIM, Rows<T>::SAMPLE_RT, Rows<T>::SAMPLE_RG, MODE_SAMPLE,
                   sample_groups<T, DH>()>(d, a, max_grid, st);
  if (mode == MODE_GIVEN)
    return fwd_one<T, DH, DIM, Rows<T>::SAMPLE_RT, Rows<T>::SAMPLE_RG, MODE_GIVEN,
                   sample_groups<T, DH>()>(d, a, max_grid, st);
  return fwd_one<T, DH, DIM, ERT, Rows<T>::ELOC_RG, MODE_ELOC>(d, a, max_grid, st);
}

template <typename T>
cudaError_t run_forward(const RecDesc &d, int mode, FwdArgs<T> a, int max_grid, cudaStream_t st) {
  NQS_DISPATCH_DH(d.dh, {
    if (d.dim == 1) return fwd_dim<T, DH, 1>(d, mode, a, max_grid, st);
    return fwd_dim<T, DH, 2>(d, mode, a, max_grid, st);
  });
  return cudaSuccess;
}

template <typename T, int DH, int DIM>
static int eloc_grid_dim(const RecDesc &d) {
  constexpr int RT = eloc_rt<T>(DIM, DH);
  constexpr int RG = Rows<T>::ELOC_RG;
  auto kern = k_forward<T, DH, DIM, RT, RG, MODE_ELOC, true>;
  size_t smem = fwd_smem_bytes<T, DH, DIM, RT * RG>(d.N, true);
  if constexpr (DH >= 96) {
    if (smem > SMEM_STAGE_LIMIT) {
      smem = fwd_smem_bytes<T, DH, DIM, RT * RG>(d.N, false);
      kern = k_forward<T, DH, DIM, RT, RG, MODE_ELOC, false>;
    }
  }
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 0;
  int per = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, Tile<DH>::UG * RG, smem) != cudaSuccess)
    return 0;
  return per * d.sm_count;
}

template <typename T> int eloc_max_grid(const RecDesc &d) {
  switch (d.dh) {
    case 8: return d.dim == 1 ? eloc_grid_dim<T, 8, 1>(d) : eloc_grid_dim<T, 8, 2>(d);
    case 16: return d.dim == 1 ? eloc_grid_dim<T, 16, 1>(d) : eloc_grid_dim<T, 16, 2>(d);
    case 32: return d.dim == 1 ? eloc_grid_dim<T, 32, 1>(d) : eloc_grid_dim<T, 32, 2>(d);
    case 64: return d.dim == 1 ? eloc_grid_dim<T, 64, 1>(d) : eloc_grid_dim<T, 64, 2>(d);
    case 96: return d.dim == 1 ? eloc_grid_dim<T, 96, 1>(d) : eloc_grid_dim<T, 96, 2>(d);
    case 128: return d.dim == 1 ? eloc_grid_dim<T, 128, 1>(d) : eloc_grid_dim<T, 128, 2>(d);
    case 200: return d.dim == 1 ? eloc_grid_dim<T, 200, 1>(d) : eloc_grid_dim<T, 200, 2>(d);
    case 256: return d.dim == 1 ? eloc_grid_dim<T, 256, 1>(d) : eloc_grid_dim<T, 256, 2>(d);
  }
  return 0;
}

template <typename T, int DH, int DIM>
static cudaError_t bwd_dim(const RecDesc &d, BwdArgs<T> a, cudaStream_t st) {
  constexpr int RT = Rows<T>::BWD_RT, RG = Rows<T>::BWD_RG, R = RT * RG;
  auto kern = k_jac_bwd<T, DH, DIM, RT, RG, true>;
  size_t smem = bwd_smem_bytes<T, DH, DIM, R, RT>(d.N, true);
  if constexpr (DH >= 96) {
    if (smem > SMEM_STAGE_LIMIT) {
      smem = bwd_smem_bytes<T, DH, DIM, R, RT>(d.N, false);
      kern = k_jac_bwd<T, DH, DIM, RT, RG, false>;
    }
  }
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  a.ntiles = (int)((a.nrows + R - 1) / R);
  if (a.ntiles <= 0) return cudaSuccess;
  kern<<<a.ntiles, BTile<DH>::UG * RG, smem, st>>>(a);
  return cudaGetLastError();
}

template <typename T> cudaError_t run_bwd(const RecDesc &d, BwdArgs<T> a, cudaStream_t st) {
  NQS_DISPATCH_DH(d.dh, {
    if (d.dim == 1) return bwd_dim<T, DH, 1>(d, a, st);
    return bwd_dim<T, DH, 2>(d, a, st);
  });
  return cudaSuccess;
}

template <typename T> cudaError_t run_grad(const RecDesc &d, GradArgs<T, T> a, cudaStream_t st) {
  if (a.nrows <= 0) return cudaSuccess;
  NQS_DISPATCH_DH(d.dh, {
    if (d.dim == 1) k_jac_grad<T, T, DH, 1><<<(unsigned)a.nrows, 256, 0, st>>>(a);
    else k_jac_grad<T, T, DH, 2><<<(unsigned)a.nrows, 256, 0, st>>>(a);
  });
  return cudaGetLastError();
}

}  // namespace nqs
