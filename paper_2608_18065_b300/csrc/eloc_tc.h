// eloc_tc.h -- tensor-core engine for the connected-configuration suffixes
// (mixed precision, 1D chains, hidden size 64, or 32 run with zero-padded
// units).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace nqs {

struct ElocTcArgs {
  const float *pack;      // packed FP32 weights
  int oWgT, oxw, obias, ohead, ohc;  // their offsets (PackOff)
  const uint8_t *spins;   // [ns][N] samples
  const float *hcache;    // [ns][N][dhm], or [ns][nck][dhm] checkpoints
  const float *lccache;   // [ns][N][2]
  int N, cplx, zmask;
  int64_t ns;
  int tiles_per_op, ntiles;  // 128-row tiles per operator, total tiles
  const int *op_f;        // [n_off][4]: flip sites f1, f2, first changed site, rank order
  const int *item_s;      // [n_off][ns] connected samples
  const double *item_e;   // [n_off][ns] matrix elements
  const int *item_cnt;    // [n_off]
  double *contrib;        // [n_off][ns][2]
  int *err;               // device status word
  int ck, nck;            // checkpoints: hcache holds h_{m ck - 1} in slot m - 1 (ck > 0)
  int dhm;                // the model's hidden size (64, or 32 padded with zero units)
  int *tile_ctr;          // zeroed before the launch: tiles handed out in rank order
                          // (op_f[4 i + 3] = the operator of rank i, longest suffix first)
};

bool eloc_tc_supported(int dim, int dh);
cudaError_t eloc_tc_run(const ElocTcArgs &args, int sm_count, cudaStream_t st);

}  // namespace nqs
