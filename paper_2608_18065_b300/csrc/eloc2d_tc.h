// eloc2d_tc.h -- tensor-core engines for the connected-configuration
// suffixes of 2D lattices (mixed precision, zig-zag path, every state
// cached): weights resident in shared memory for hidden size 64 and 32
// (padded to 64; eloc2d_tc.cu), streamed from L2 for hidden sizes 96 and
// 128 (eloc2d_tcs.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace nqs {

struct Eloc2dTcArgs {
  const float *pack;      // packed FP32 weights
  int oWgT, oxw, obias, ohead, ohc, oU12T;  // their offsets (PackOff)
  const uint8_t *spins;   // [ns][N] samples
  const float *hcache;    // [ns][N][64]: h_k of every sample
  const float *lccache;   // [ns][N][2]
  int N, Lx, cplx, zmask;
  int64_t ns;
  int tiles_per_op, ntiles;  // 128-row tiles per operator, total tiles
  const int *op_f;        // [n_off][4]: flip sites f1, f2, first changed site, rank order
  const int *item_s;      // [n_off][ns] connected samples
  const double *item_e;   // [n_off][ns] matrix elements
  const int *item_cnt;    // [n_off]
  double *contrib;        // [n_off][ns][2]
  float *colbuf;          // [grid][128][Lx][max(dh, 64)]: recomputed states (U2 h in
                          // the streamed engine) by lattice column
  int *err;               // device status word (NQS_ERR_TIMEOUT on a wait that ran out)
  int *tile_ctr;          // zeroed before the launch: tiles handed out in rank order
                          // (op_f[4 i + 3] = the operator of rank i, longest suffix first)
  const unsigned char *wimg;  // streamed engine: its weight image (eloc2d_tcs_image_bytes),
                              // written from pack by eloc2d_tcs_run before the engine runs
  // streamed engine, tests of failure detection: polls per bounded wait
  // (0: the default, about half a second) and, if set, a producer that never
  // publishes the first tile, so that every consumer's wait runs out
  unsigned long long spin_limit;
  int test_drop_tile;
  // streamed engine, sampling (Sec. II.A, eloc2d_tcs_sample): tiles of 128
  // samples from site 0, sigma_k drawn with the Philox uniforms of sample
  // s0 + s, step *step_dev, key seed; outputs as the sampler of the
  // recurrence kernels
  uint64_t seed;
  uint64_t step;           // used when step_dev is null
  const int64_t *step_dev;
  int64_t s0;
  int marshall;
  uint8_t *spins_out;      // [ns][N]
  double *logpsi;          // [ns][2]
  float *hcache_out;       // [ns][N][dh]: h_k
  float *lccache_out;      // [ns][N][2]: 1/2 log p(sigma_k), phi_k
  float *gcache;           // [ns][N][5 dh]: u, r, c, W_h h' + b_h, h' (or null)
};

constexpr int ELOC2D_TC_ROWS = 128;  // rows per tile (the MMA's M)

bool eloc2d_tc_supported(int dim, int dh);
// dh = the model's hidden size (64, or 32 padded to 64); grid <= sm_count;
// the column buffer must hold grid x 128 rows of Lx x 64 floats
cudaError_t eloc2d_tc_run(const Eloc2dTcArgs &args, int dh, int sm_count, cudaStream_t st);

// Streamed-weight engine, hidden sizes 96 and 128: column buffer [grid][128]
// [Lx][dh] of U2 h (FP32); grid <= sm_count.
bool eloc2d_tcs_supported(int dim, int dh);
size_t eloc2d_tcs_image_bytes(int dh);
cudaError_t eloc2d_tcs_run(const Eloc2dTcArgs &args, int dh, int sm_count, cudaStream_t st);
// The same in two parts, for a grouped launch: the weight image of one
// instance, then one launch over several instances of hidden size dh (each
// with its image written, its counter zeroed and cta0[i + 1] - cta0[i] CTAs,
// at most its tile count; the column buffer of instance i must hold that
// many CTAs' slices; grid = cta0[n] <= the SM count).
constexpr int ELOC2D_GROUP_MAX = 32;
struct Eloc2dTcGroup {
  int n;
  int cta0[ELOC2D_GROUP_MAX + 1];
  Eloc2dTcArgs inst[ELOC2D_GROUP_MAX];
};
cudaError_t eloc2d_tcs_image(const Eloc2dTcArgs &args, int dh, cudaStream_t st);
cudaError_t eloc2d_tcs_group_run(const Eloc2dTcGroup &g, int dh, cudaStream_t st);
// Sampling of ns configurations with the same engine (args.ns, ntiles =
// ceil(ns / 128), Lx <= 16, the column buffer and counter as above).
bool eloc2d_tcs_sample_supported(int dim, int dh, int Lx);
cudaError_t eloc2d_tcs_sample(const Eloc2dTcArgs &args, int dh, int sm_count, cudaStream_t st);

}  // namespace nqs
