// jac_tc.h -- tensor-core assembly of the per-sample Jacobian rows O (mixed
// precision, 1D chains, hidden size 64 or 32, every state cached).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace nqs {

struct JacTcArgs {
  int N, cplx, dh;          // chain length, complex head, hidden size (64 or 32)
  int64_t ns, nrows;        // samples; rows of O (ns, or 2 ns for the complex head)
  const uint8_t *spins;     // [ns][N]
  const float *hcache;      // [ns][N][dh]: h_k of every sample
  const float *adj;         // [nrows][N][adjw]: per site dau, dar, dg, dac (dh each), dz (4)
  int adjw;
  float *O;                 // [nrows][np]
  int64_t np;
  int64_t Wu, bu, Wr, br, Wh, bh, Win, bin, Uo, co, Up, cp;  // parameter offsets (App. A)
  int *err;                 // device status word (NQS_ERR_TIMEOUT on a wait that ran out)
};

bool jac_tc_supported(int dim, int dh);
cudaError_t jac_tc_run(const JacTcArgs &args, int sm_count, cudaStream_t st);

// 2D lattices (hidden size 32, 64, 96 or 128, every state cached): every
// row of O (jac2d_tc.cu).
struct Jac2dTcArgs {
  int N, Lx, cplx, dh;
  int64_t ns, nrows;        // samples; rows of O (ns, or 2 ns for the complex head)
  const uint8_t *spins;     // [ns][N]
  const float *hcache;      // [ns][N][dh]: h_k of every sample
  const float *adj;         // [nrows][N][adjw]: dau dar dg dac (dh each), the head
                            // adjoints (4), dh' (dh), h' (dh)
  int adjw, odz, odhp, ohp; // record width; offsets of the head adjoints, dh' and h'
  float *O;                 // [nrows][np]
  int64_t np;
  int64_t U1, U2, Wu, bu, Wr, br, Wh, bh, Win, bin, Uo, co, Up, cp;  // parameter offsets (App. A)
  int *err;                 // device status word (NQS_ERR_TIMEOUT on a wait that ran out)
};

bool jac2d_tc_supported(int dim, int dh);
cudaError_t jac2d_tc_run(const Jac2dTcArgs &args, int sm_count, cudaStream_t st);

}  // namespace nqs
