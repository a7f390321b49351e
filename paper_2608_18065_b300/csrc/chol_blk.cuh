// chol_blk.cuh -- (T + lambda I) x = eps' (Eq. minsrR) at large R: FP32
// Cholesky in 128-wide panels and FP64 iterative refinement by 128-block
// substitution, one cooperative launch (sm_103a).
//
// With 32-wide panels (k_chol_ir) every panel streams the whole remaining
// FP32 matrix through DRAM at 8 flops per byte; at R = 8192 that is 17 GB
// per solve.  Here the trailing update of a panel is a rank-128 product in
// 128 x 128 tiles, four times the arithmetic per byte and a quarter of the
// panels (and grid barriers).  Per panel p (columns c0 .. c0 + 127), with
// the factor L_pp of its diagonal block and D_p = L_pp^{-1} published:
//   panel rows   L_ip = A_ip D_p^T    one 128 x 128 x 128 product per row block
//   trailing     A_ij -= L_ip L_jp^T  tiles of the lower triangle, K = 128
// Both are the same shared-memory tile product C = X Y^T (8 x 8 outputs per
// thread, K in four 32-column pieces whose copies are all in flight at
// once).  With look-ahead, CTA 0 alone takes the next diagonal tile: it
// updates it, factors it in shared memory (32-wide sub-panels: a warp
// factors each 32 x 32 block, the CTA solves the rows below and updates the
// rest of the tile), forms D by block inversion, and publishes both before
// the panel's second grid barrier.  The FP32 panel solve by an explicit
// inverse multiplies its rounding by kappa(L_pp) = sqrt(kappa(A_pp)) at
// most, well inside what the FP64 refinement corrects whenever the FP32
// factor is usable at all.
//
// Refinement, as k_chol_ir: x_0 = 0, r_0 = b; per sweep, in FP32,
//   forward   w_p = D_p (r_p - sum_{q<p} L_pq w_q)
//   backward  d_p = D_p^T (w_p - sum_{q>p} L_qp^T d_q),
// one grid barrier per block step (every CTA forms the block's product with
// D_p itself); then x += d and r = b - A x in FP64, until LAPACK's dsposv
// backward-error test holds.  A non-positive FP32 pivot, or no convergence
// within maxit sweeps, sets *need_fp64 (the FP64 Cholesky follows on the
// stream).  Needs n % 4 == 0 (16-byte rows).  Grid barriers are bounded.
#pragma once
#include "chol_ir.cuh"

namespace nqs {

constexpr int BKB = 128;                 // panel width and tile side
constexpr int BKB_THREADS = 256;
constexpr int BKB_LD = BKB + 4;          // shared row stride (floats)

struct CholBlkArgs {
  const double *A;    // [n][n], both triangles: T + lambda I (not modified)
  int64_t n;          // n % 4 == 0
  const double *b;    // [n]
  double *x;          // [n] out
  float *L;           // [n][n] scratch: FP32 factor (lower triangle)
  float *Dinv;        // [ceil(n / 128)][128][128] scratch: inverses of the diagonal blocks
  float *t;           // [n] scratch: forward right-hand side, updated in place
  float *w;           // [n] scratch: forward solution, then the backward right-hand side
  double *r;          // [n] scratch: FP64 residual
  double *part;       // [2][gridDim][4] scratch: partial norms (by sweep parity)
  unsigned *bar;      // barrier arrival counter (zeroed before launch)
  int32_t *status;    // NQS_ERR_TIMEOUT on a barrier timeout
  int32_t *need_fp64; // out: 1 when the FP64 factorisation must run
  int maxit;
};

// Shared memory: X, Y and C tiles [128][BKB_LD], a [32][BKB_LD] scratch,
// two 128-vectors, the warp Cholesky's column buffer (216 KB).
inline size_t chol_blk_smem() {
  return sizeof(float) * (3 * (size_t)BKB * BKB_LD + 32 * (size_t)BKB_LD + 2 * BKB + 2 * 32);
}

inline bool chol_blk_supported(int64_t n) { return n % 4 == 0 && n >= 2 * BKB; }

namespace blk {

// Copies of K piece ch (columns 32 ch .. 32 ch + 31) of a 128-row block
// whose row 0 is at src (row stride ld, `rows` rows valid, zeros below).
__device__ __forceinline__ void stage_piece(float *S, const float *src, int64_t ld, int64_t rows,
                                            int ch, int tid) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int e = tid + q * BKB_THREADS;  // 128 rows x 8 16-byte pieces
    const int row = e >> 3, col = 32 * ch + 4 * (e & 7);
    const bool ok = row < rows;
    cp_async16(S + row * BKB_LD + col, ok ? src + row * ld + col : src, ok ? 16 : 0);
  }
}

// The 128 x 128 block at src (row stride ld, rows x cols valid, zeros
// outside; cols % 4 == 0 or cols >= 128), all four pieces at once.
__device__ __forceinline__ void stage_block(float *S, const float *src, int64_t ld, int64_t rows,
                                            int64_t cols, int tid) {
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int e = tid + q * BKB_THREADS;  // 128 rows x 32 16-byte pieces
    const int row = e >> 5, col = 4 * (e & 31);
    const bool ok = row < rows && col < cols;
    cp_async16(S + row * BKB_LD + col, ok ? src + row * ld + col : src, ok ? 16 : 0);
  }
}

template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// acc[a][b] = sum_k X[ty + 16 a][k] Y[tx + 16 b][k] over k = k0 .. k0 + 31.
// A warp reads two rows of X (broadcasts) and sixteen rows of Y (row
// stride 132 floats: eight consecutive rows fall in distinct banks).  The
// 64 accumulators take k, then k + 1, ... in turn, so that consecutive FMAs
// are independent (measured: 11.3 against 12.7 us per 128-cube tile with
// each accumulator's four k in a row; the same sums in the same order).
__device__ __forceinline__ void mac_piece(const float *X, const float *Y, int k0, int tx, int ty,
                                          float (&acc)[8][8]) {
#pragma unroll 2
  for (int k = k0; k < k0 + 32; k += 4) {
    float4 xa[8], yb[8];
#pragma unroll
    for (int a = 0; a < 8; ++a) xa[a] = *reinterpret_cast<const float4 *>(X + (ty + 16 * a) * BKB_LD + k);
#pragma unroll
    for (int b = 0; b < 8; ++b) yb[b] = *reinterpret_cast<const float4 *>(Y + (tx + 16 * b) * BKB_LD + k);
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(xa[a].x, yb[b].x, acc[a][b]);
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(xa[a].y, yb[b].y, acc[a][b]);
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(xa[a].z, yb[b].z, acc[a][b]);
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(xa[a].w, yb[b].w, acc[a][b]);
  }
}

// acc = X Y^T for two 128 x 128 blocks in global memory (Y = X when ysrc is
// null); the four K pieces are requested at once and multiplied as they
// land.  If csrc is set, the block of C to be updated comes into Cs behind
// them (crows x ccols valid), in place when the product is done.
__device__ __forceinline__ void tile_product(float *Xs, float *Ys, float *Cs, const float *xsrc,
                                             int64_t xld, int64_t xrows, const float *ysrc,
                                             int64_t yld, int64_t yrows, const float *csrc,
                                             int64_t cld, int64_t crows, int64_t ccols, int tid,
                                             float (&acc)[8][8]) {
  const int tx = tid & 15, ty = tid >> 4;
  __syncthreads();  // the previous product's readers are done with Xs, Ys, Cs
#pragma unroll
  for (int ch = 0; ch < 4; ++ch) {
    stage_piece(Xs, xsrc, xld, xrows, ch, tid);
    if (ysrc) stage_piece(Ys, ysrc, yld, yrows, ch, tid);
    cp_async_commit();
  }
  if (csrc) stage_block(Cs, csrc, cld, crows, ccols, tid);
  cp_async_commit();  // (possibly empty) group 4: C
  const float *Y = ysrc ? Ys : Xs;
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;
  cp_async_wait<4>();
  __syncthreads();
  mac_piece(Xs, Y, 0, tx, ty, acc);
  cp_async_wait<3>();
  __syncthreads();
  mac_piece(Xs, Y, 32, tx, ty, acc);
  cp_async_wait<2>();
  __syncthreads();
  mac_piece(Xs, Y, 64, tx, ty, acc);
  cp_async_wait<1>();
  __syncthreads();
  mac_piece(Xs, Y, 96, tx, ty, acc);
  cp_async_wait<0>();
  __syncthreads();
}

// y = D v for a 128 x 128 block D in global memory (row stride ld, rows
// from `rows` on zero) and v in shared memory: thread (row tid / 2, half
// tid % 2) with its 16 loads in flight together; y (or sub - D v) to shared
// memory.  Ends with a barrier.
__device__ __forceinline__ void matvec(const float *D, const float *v, float *y, int tid,
                                       int64_t ld = BKB, int rows = BKB,
                                       const float *sub = nullptr) {
  const int j = tid >> 1, h = tid & 1;
  const float4 *dr = reinterpret_cast<const float4 *>(D + j * ld + 64 * h);
  const float4 *vr = reinterpret_cast<const float4 *>(v + 64 * h);
  float4 d[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) d[q] = j < rows ? __ldcg(dr + q) : make_float4(0.f, 0.f, 0.f, 0.f);
  float s = 0.f;
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const float4 x = vr[q];
    s = fmaf(d[q].x, x.x, s);
    s = fmaf(d[q].y, x.y, s);
    s = fmaf(d[q].z, x.z, s);
    s = fmaf(d[q].w, x.w, s);
  }
  s += __shfl_xor_sync(0xffffffffu, s, 1);
  if (h == 0) y[j] = sub ? sub[j] - s : s;  // in place (y = sub) is allowed
  __syncthreads();
}

// y = D^T v (or sub - D^T v) for a 128-column block D (row stride ld, rows
// from `rows` on zero): thread (four columns 4 (tid % 32) .., sixteen rows
// 16 (tid / 32) ..) with its 16 loads in flight together, the eight row
// groups summed through part ([8][128] floats).  Ends with a barrier.
__device__ __forceinline__ void matvec_t(const float *D, const float *v, float *y, float *part,
                                         int tid, int64_t ld = BKB, int rows = BKB,
                                         const float *sub = nullptr) {
  const int k4 = tid & 31, r8 = tid >> 5;
  float4 d[16];
#pragma unroll
  for (int q = 0; q < 16; ++q)
    d[q] = 16 * r8 + q < rows ? __ldcg(reinterpret_cast<const float4 *>(D + (16 * r8 + q) * ld) + k4)
                              : make_float4(0.f, 0.f, 0.f, 0.f);
  float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const float x = v[16 * r8 + q];
    s.x = fmaf(d[q].x, x, s.x);
    s.y = fmaf(d[q].y, x, s.y);
    s.z = fmaf(d[q].z, x, s.z);
    s.w = fmaf(d[q].w, x, s.w);
  }
  reinterpret_cast<float4 *>(part + r8 * BKB)[k4] = s;
  __syncthreads();
  if (tid < BKB) {
    float t = 0.f;
#pragma unroll
    for (int r = 0; r < 8; ++r) t += part[r * BKB + tid];
    y[tid] = sub ? sub[tid] - t : t;  // in place (y = sub) is allowed
  }
  __syncthreads();
}

// C = (acc ? C : 0) + alpha A B for an M x N block in shared memory (M, N,
// K multiples of 4; row-major, B and C 16-byte aligned rows), 4 x 4 outputs
// per thread: per k four broadcast loads of A and one float4 of B for 16
// FMAs.  lower: only the lower triangle (j <= i) is formed and written.  C
// must not overlap A or B.  No barrier.
__device__ __forceinline__ void cta_gemm(float *C, int ldc, const float *A, int lda, const float *B,
                                         int ldb, int M, int N, int K, float alpha, bool acc,
                                         bool lower, int tid) {
  const int tn = N >> 2, ntile = (M >> 2) * tn;
  for (int t = tid; t < ntile; t += BKB_THREADS) {
    const int i0 = 4 * (t / tn), j0 = 4 * (t - (t / tn) * tn);
    if (lower && j0 > i0 + 3) continue;
    float c[4][4];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int r = 0; r < 4; ++r) c[q][r] = 0.f;
#pragma unroll 4
    for (int k = 0; k < K; ++k) {
      const float4 b = *reinterpret_cast<const float4 *>(B + k * ldb + j0);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float a = A[(i0 + q) * lda + k];
        c[q][0] = fmaf(a, b.x, c[q][0]);
        c[q][1] = fmaf(a, b.y, c[q][1]);
        c[q][2] = fmaf(a, b.z, c[q][2]);
        c[q][3] = fmaf(a, b.w, c[q][3]);
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        if (lower && j0 + r > i0 + q) continue;
        float *d = C + (i0 + q) * ldc + j0 + r;
        *d = (acc ? *d : 0.f) + alpha * c[q][r];
      }
  }
}

// Cholesky of the 128 x 128 block in S (lower triangle; rows and columns
// from m on hold the identity) and its inverse into Dv; the whole CTA, with
// W ([128][BKB_LD] floats) and PT as scratch.  Sub-panel s (columns
// o = 32 s .. o + 31): warp 0 factors the diagonal 32 x 32 block and
// inverts it; the rows below are solved with that inverse, X = S_r,o Dv_ss^T;
// the rest of the block takes the rank-32 update S -= X X^T.  Then the
// inverse by recursive doubling: for each pair of inverted diagonal blocks
// (32 wide, then 64), D_21 = -D_22 (L_21 D_11).  Returns nonzero (uniform
// over the CTA) for a pivot that is not positive.
__device__ __noinline__ int diag_factor(float *S, float *Dv, float *PT, float *W, float *colb,
                                        int *bad_s, int tid) {
  const int lane = tid & 31, warp = tid >> 5;
  for (int e = tid; e < BKB * BKB_LD; e += BKB_THREADS) Dv[e] = 0.f;
  if (tid == 0) *bad_s = 0;
  __syncthreads();
  for (int s = 0; s < 4; ++s) {
    const int o = 32 * s;
    if (warp == 0) {
      float rr[IR_B];
#pragma unroll
      for (int k = 0; k < IR_B; ++k) rr[k] = k <= lane ? S[(o + lane) * BKB_LD + o + k] : 0.f;
      float rinv = 1.f;
      const int bad = warp_chol32(rr, colb, lane, rinv);
#pragma unroll
      for (int k = 0; k < IR_B; ++k) S[(o + lane) * BKB_LD + o + k] = rr[k];
      __syncwarp();
      // inverse of the 32 x 32 factor: lane j forms column j
      float xc[IR_B];
#pragma unroll
      for (int i = 0; i < IR_B; ++i) {
        float acc = i == lane ? 1.f : 0.f;
#pragma unroll
        for (int k = 0; k < i; ++k) acc = fmaf(-S[(o + i) * BKB_LD + o + k], xc[k], acc);
        xc[i] = i >= lane ? acc / S[(o + i) * BKB_LD + o + i] : 0.f;
      }
#pragma unroll
      for (int i = 0; i < IR_B; ++i) {
        Dv[(o + i) * BKB_LD + o + lane] = xc[i];
        PT[lane * BKB_LD + i] = xc[i];  // Dv_ss^T
      }
      if (lane == 0 && bad) *bad_s = 1;
    }
    __syncthreads();
    const int rb = o + 32, nrow = BKB - rb;
    if (nrow > 0) {
      // X = S_r,o.. Dv_ss^T into W, then back into S and transposed into PT
      cta_gemm(W, BKB_LD, S + rb * BKB_LD + o, BKB_LD, PT, BKB_LD, nrow, 32, 32, 1.f, false,
               false, tid);
      __syncthreads();
      for (int e = tid; e < nrow * 32; e += BKB_THREADS) {
        const int r = e >> 5, k = e & 31;
        const float v = W[r * BKB_LD + k];
        S[(rb + r) * BKB_LD + o + k] = v;
        PT[k * BKB_LD + r] = v;
      }
      __syncthreads();
      // S_rr -= X X^T, lower triangle
      cta_gemm(S + rb * BKB_LD + rb, BKB_LD, W, BKB_LD, PT, BKB_LD, nrow, nrow, 32, -1.f, true,
               true, tid);
      __syncthreads();
    }
  }
  // recursive doubling: M = L_21 D_11 into W, then D_21 = -D_22 M
  for (int h = 32; h < BKB; h *= 2) {
    for (int q = 0; q < BKB / (2 * h); ++q) {
      const int b1 = 2 * h * q, b2 = b1 + h;
      cta_gemm(W, BKB_LD, S + b2 * BKB_LD + b1, BKB_LD, Dv + b1 * BKB_LD + b1, BKB_LD, h, h, h,
               1.f, false, false, tid);
      __syncthreads();
      cta_gemm(Dv + b2 * BKB_LD + b1, BKB_LD, Dv + b2 * BKB_LD + b2, BKB_LD, W, BKB_LD, h, h, h,
               -1.f, false, false, tid);
      __syncthreads();
    }
  }
  return *bad_s;
}

// Publish a factored diagonal block at (r0, r0) (m x m valid): the factor
// into L, the inverse into D ([128][128], zeros outside the triangle).
__device__ __forceinline__ void publish_block(const float *S, const float *Dv, float *L, float *D,
                                              int64_t n, int64_t r0, int m, int tid) {
  for (int e = tid; e < BKB * BKB; e += BKB_THREADS) {
    const int i = e >> 7, j = e & (BKB - 1);
    if (i < m && j <= i) __stcg(L + (r0 + i) * n + r0 + j, S[i * BKB_LD + j]);
    __stcg(D + e, Dv[i * BKB_LD + j]);
  }
}

// Stage the (already updated) diagonal block at (r0, r0) into S from L,
// lower triangle, identity outside the m x m block.
__device__ __forceinline__ void stage_diag(float *S, const float *L, int64_t n, int64_t r0, int m,
                                           int tid) {
  for (int e = tid; e < BKB * BKB; e += BKB_THREADS) {
    const int i = e >> 7, j = e & (BKB - 1);
    float v;
    if (i < m && j < m) v = j <= i ? __ldcg(L + (r0 + i) * n + r0 + j) : 0.f;
    else v = i == j ? 1.f : 0.f;
    S[i * BKB_LD + j] = v;
  }
}

}  // namespace blk

// The solve of one instance by CTAs g = 0 .. G-1 of the launch (all of a
// k_chol_blk grid, or the instance's range of a grouped grid).
__device__ __forceinline__ void chol_blk_run(const CholBlkArgs &a, const int g, const int G) {
  extern __shared__ __align__(16) float blk_smem[];
  float *Xs = blk_smem, *Ys = Xs + BKB * BKB_LD, *Cs = Ys + BKB * BKB_LD, *PT = Cs + BKB * BKB_LD;
  float *vx = PT + 32 * BKB_LD, *vy = vx + BKB, *colb = vy + BKB;
  float *vz = PT + 2048, *vw = PT + 2048 + BKB;  // refinement: the second block of a pair
  __shared__ int bad_s;
  __shared__ double red_s[BKB_THREADS / 32][3];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int tx = tid & 15, ty = tid >> 4;
  const int64_t n = a.n;
  const int nb = (int)((n + BKB - 1) / BKB);
  float *L = a.L;
  unsigned ep = 0;
  auto gsync = [&]() -> bool { ++ep; return cc_sync_ep(a.bar, a.status, ep * (unsigned)G); };
  auto fail = [&]() { return *reinterpret_cast<volatile int32_t *>(a.need_fp64) != 0; };

  // (0) FP32 copy of the lower triangle, x = 0; then CTA 0 factors block 0
  for (int64_t i = g; i < n; i += G) {
    const double *Ai = a.A + i * n;
    float *Lr = L + i * n;
    for (int64_t j = tid; j <= i; j += BKB_THREADS) __stcg(Lr + j, (float)Ai[j]);
  }
  for (int64_t i = (int64_t)g * BKB_THREADS + tid; i < n; i += (int64_t)G * BKB_THREADS) a.x[i] = 0.0;
  if (!gsync()) return;
  if (g == 0) {
    const int m0 = (int)min64(BKB, n);
    blk::stage_diag(Xs, L, n, 0, m0, tid);
    __syncthreads();
    const int bad = blk::diag_factor(Xs, Ys, PT, Cs, colb, &bad_s, tid);
    blk::publish_block(Xs, Ys, L, a.Dinv, n, 0, m0, tid);
    if (bad && tid == 0) *a.need_fp64 = 1;
  }
  if (!gsync()) return;
  if (fail()) return;

  // (1) panels
  for (int p = 0; p + 1 < nb; ++p) {
    const int64_t c0 = (int64_t)p * BKB, r0 = c0 + BKB;
    const int nr = (int)((n - r0 + BKB - 1) / BKB);  // row blocks below the panel
    const float *Dp = a.Dinv + (size_t)p * BKB * BKB;
    // panel rows: L_ip = A_ip D_p^T
    for (int rb = g; rb < nr; rb += G) {
      const int64_t i0 = r0 + (int64_t)rb * BKB;
      float acc[8][8];
      blk::tile_product(Xs, Ys, Cs, L + i0 * n + c0, n, n - i0, Dp, BKB, BKB, nullptr, 0, 0, 0,
                        tid, acc);
#pragma unroll
      for (int aa = 0; aa < 8; ++aa) {
        const int64_t i = i0 + ty + 16 * aa;
        if (i < n)
#pragma unroll
          for (int bb = 0; bb < 8; ++bb) __stcg(L + i * n + c0 + tx + 16 * bb, acc[aa][bb]);
      }
    }
    if (!gsync()) return;
    // trailing update; CTA 0 takes the next diagonal tile and factors it
    const int ntiles = nr * (nr + 1) / 2;
    const bool la = G > 1;
    if (g == 0) {
      const int m1 = (int)min64(BKB, n - r0);
      float acc[8][8];
      blk::tile_product(Xs, Ys, Cs, L + r0 * n + c0, n, m1, nullptr, 0, 0, L + r0 * n + r0, n, m1,
                        m1, tid, acc);
      // every thread is done reading Xs (the product ends with a barrier)
#pragma unroll
      for (int aa = 0; aa < 8; ++aa)
#pragma unroll
        for (int bb = 0; bb < 8; ++bb) {
          const int i = ty + 16 * aa, j = tx + 16 * bb;
          float v;
          if (i < m1 && j < m1) v = j <= i ? Cs[i * BKB_LD + j] - acc[aa][bb] : 0.f;
          else v = i == j ? 1.f : 0.f;
          Xs[i * BKB_LD + j] = v;
        }
      __syncthreads();
      const int bad = blk::diag_factor(Xs, Ys, PT, Cs, colb, &bad_s, tid);
      blk::publish_block(Xs, Ys, L, a.Dinv + (size_t)(p + 1) * BKB * BKB, n, r0, m1, tid);
      if (bad && tid == 0) *a.need_fp64 = 1;
    }
    if (!la || g > 0) {
      const int gr = la ? g - 1 : 0, Gr = la ? G - 1 : 1;
      for (int t = 1 + gr; t < ntiles; t += Gr) {
        int ti = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
        while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
        while (ti * (ti + 1) / 2 > t) --ti;
        const int tj = t - ti * (ti + 1) / 2;
        const int64_t i0 = r0 + (int64_t)ti * BKB, j0 = r0 + (int64_t)tj * BKB;
        float acc[8][8];
        blk::tile_product(Xs, Ys, Cs, L + i0 * n + c0, n, n - i0,
                          ti == tj ? nullptr : L + j0 * n + c0, n, n - j0, L + i0 * n + j0, n, n - i0,
                          n - j0, tid, acc);
#pragma unroll
        for (int aa = 0; aa < 8; ++aa) {
          const int64_t i = i0 + ty + 16 * aa;
          if (i >= n) continue;
#pragma unroll
          for (int bb = 0; bb < 8; ++bb) {
            const int64_t j = j0 + tx + 16 * bb;
            if (j <= i)
              __stcg(L + i * n + j, Cs[(ty + 16 * aa) * BKB_LD + tx + 16 * bb] - acc[aa][bb]);
          }
        }
      }
    }
    if (!gsync()) return;
    if (fail()) return;
  }

  // (2) refinement sweeps
  const int nwarps = G * (BKB_THREADS / 32), gw = g * (BKB_THREADS / 32) + warp;
  double normA = 0.0;
  bool converged = false;
  for (int it = 0; it < a.maxit && !converged; ++it) {
    // t = r (b on the first sweep)
    const double *rs = it == 0 ? a.b : a.r;
    for (int64_t i = (int64_t)g * BKB_THREADS + tid; i < n; i += (int64_t)G * BKB_THREADS)
      __stcg(a.t + i, (float)__ldcg(rs + i));
    if (!gsync()) return;
    // forward, two blocks per grid barrier: w_p = D_p t_p, w_{p+1} =
    // D_{p+1} (t_{p+1} - L_{p+1,p} w_p) in every CTA; t_i -= L_ip w_p +
    // L_i,p+1 w_{p+1} below the pair
    for (int p = 0; p < nb; p += 2) {
      const int64_t c0 = (int64_t)p * BKB, c1 = c0 + BKB;
      const int m = (int)min64(BKB, n - c0);
      const bool two = p + 1 < nb;
      const int m1 = two ? (int)min64(BKB, n - c1) : 0;
      if (tid < BKB) {
        vx[tid] = tid < m ? __ldcg(a.t + c0 + tid) : 0.f;
        vz[tid] = tid < m1 ? __ldcg(a.t + c1 + tid) : 0.f;
      }
      __syncthreads();
      blk::matvec(a.Dinv + (size_t)p * BKB * BKB, vx, vy, tid);
      if (two) {
        blk::matvec(L + c1 * n + c0, vy, vz, tid, n, m1, vz);
        blk::matvec(a.Dinv + (size_t)(p + 1) * BKB * BKB, vz, vw, tid);
      }
      if (g == 0 && tid < m) __stcg(a.w + c0 + tid, vy[tid]);
      if (g == 0 && tid < m1) __stcg(a.w + c1 + tid, vw[tid]);
      // rows below, four per warp with their loads in flight together
      for (int64_t i0 = c0 + (two ? 2 : 1) * BKB + 4 * (int64_t)gw; i0 < n; i0 += 4 * (int64_t)nwarps) {
        const float4 v = *reinterpret_cast<const float4 *>(vy + 4 * lane);
        const float4 v2 = *reinterpret_cast<const float4 *>(vw + 4 * lane);
        float4 l[4], l2[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const bool ok = i0 + q < n;
          l[q] = ok ? __ldcg(reinterpret_cast<const float4 *>(L + (i0 + q) * n + c0) + lane)
                    : make_float4(0.f, 0.f, 0.f, 0.f);
          l2[q] = ok && two ? __ldcg(reinterpret_cast<const float4 *>(L + (i0 + q) * n + c1) + lane)
                            : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        float sq[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          float s = l[q].x * v.x;
          s = fmaf(l[q].y, v.y, s);
          s = fmaf(l[q].z, v.z, s);
          s = fmaf(l[q].w, v.w, s);
          s = fmaf(l2[q].x, v2.x, s);
          s = fmaf(l2[q].y, v2.y, s);
          s = fmaf(l2[q].z, v2.z, s);
          s = fmaf(l2[q].w, v2.w, s);
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
          sq[q] = s;
        }
        if (lane < 4 && i0 + lane < n) {
          const float s = lane == 0 ? sq[0] : lane == 1 ? sq[1] : lane == 2 ? sq[2] : sq[3];
          __stcg(a.t + i0 + lane, __ldcg(a.t + i0 + lane) - s);
        }
      }
      if (!gsync()) return;
    }
    // backward, two blocks per grid barrier: d_p = D_p^T w_p, d_{p-1} =
    // D_{p-1}^T (w_{p-1} - L_{p,p-1}^T d_p); x += d; w_j -= L_pj d_p +
    // L_{p-1},j d_{p-1} left of the pair
    for (int p = nb - 1; p >= 0; p -= 2) {
      const int64_t c0 = (int64_t)p * BKB, cm = c0 - BKB;
      const int m = (int)min64(BKB, n - c0);
      const bool two = p >= 1;
      if (tid < BKB) {
        vx[tid] = tid < m ? __ldcg(a.w + c0 + tid) : 0.f;
        vz[tid] = two ? __ldcg(a.w + cm + tid) : 0.f;
      }
      __syncthreads();
      blk::matvec_t(a.Dinv + (size_t)p * BKB * BKB, vx, vy, PT, tid);
      if (g == 0 && tid < m) __stcg(a.x + c0 + tid, __ldcg(a.x + c0 + tid) + (double)vy[tid]);
      if (two) {
        blk::matvec_t(L + c0 * n + cm, vy, vz, PT, tid, n, m, vz);
        blk::matvec_t(a.Dinv + (size_t)(p - 1) * BKB * BKB, vz, vw, PT, tid);
        if (g == 0 && tid < BKB) __stcg(a.x + cm + tid, __ldcg(a.x + cm + tid) + (double)vw[tid]);
      }
      // columns left of the pair: 64 columns x 4 quarters of each block's
      // rows per CTA pass, 32 loads per thread in flight together
      const int64_t cl = two ? cm : c0;
      for (int64_t jb = (int64_t)g * 64; jb < cl; jb += (int64_t)G * 64) {
        const int jj = tid & 63, q = tid >> 6;
        const int64_t j = jb + jj;
        float s = 0.f;
        if (j < cl) {
          float lv[32];
#pragma unroll
          for (int i = 0; i < 32; ++i)
            lv[i] = 32 * q + i < m ? __ldcg(L + (c0 + 32 * q + i) * n + j) : 0.f;
#pragma unroll
          for (int i = 0; i < 32; ++i) s = fmaf(lv[i], vy[32 * q + i], s);
          if (two) {
#pragma unroll
            for (int i = 0; i < 32; ++i) lv[i] = __ldcg(L + (cm + 32 * q + i) * n + j);
#pragma unroll
            for (int i = 0; i < 32; ++i) s = fmaf(lv[i], vw[32 * q + i], s);
          }
        }
        PT[BKB * 8 + q * 64 + jj] = s;
        __syncthreads();
        if (q == 0 && j < cl) {
          const float *ps = PT + BKB * 8 + jj;
          __stcg(a.w + j, __ldcg(a.w + j) - (((ps[0] + ps[64]) + ps[128]) + ps[192]));
        }
        __syncthreads();
      }
      if (!gsync()) return;
    }
    // r = b - A x in FP64; partial max |r_i|, max |x_i| and (first sweep) max row sum |A|
    double rmax = 0.0, xmax = 0.0, amax = 0.0;
    for (int64_t i = gw; i < n; i += nwarps) {
      const double *Ai = a.A + i * n;
      double sacc = 0.0, sa = 0.0;
#pragma unroll 8
      for (int64_t j = lane; j < n; j += 32) {
        const double aij = Ai[j];
        sacc = fma(aij, __ldcg(a.x + j), sacc);
        if (it == 0) sa += fabs(aij);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        sacc += __shfl_xor_sync(0xffffffffu, sacc, o);
        sa += __shfl_xor_sync(0xffffffffu, sa, o);
      }
      const double ri = a.b[i] - sacc;
      if (lane == 0) __stcg(a.r + i, ri);
      rmax = fmax(rmax, fabs(ri));
      xmax = fmax(xmax, fabs(__ldcg(a.x + i)));
      amax = fmax(amax, sa);
    }
    if (lane == 0) { red_s[warp][0] = rmax; red_s[warp][1] = xmax; red_s[warp][2] = amax; }
    __syncthreads();
    if (tid == 0) {
      double m0 = 0.0, m1 = 0.0, m2 = 0.0;
      for (int q = 0; q < BKB_THREADS / 32; ++q) {
        m0 = fmax(m0, red_s[q][0]); m1 = fmax(m1, red_s[q][1]); m2 = fmax(m2, red_s[q][2]);
      }
      double *pt = a.part + (size_t)(it & 1) * G * 4;
      __stcg(pt + (size_t)g * 4 + 0, m0);
      __stcg(pt + (size_t)g * 4 + 1, m1);
      __stcg(pt + (size_t)g * 4 + 2, m2);
    }
    if (!gsync()) return;
    double q0 = 0.0, q1 = 0.0, q2 = 0.0;
    for (int q = lane; q < G; q += 32) {
      const double *pt = a.part + (size_t)(it & 1) * G * 4 + (size_t)q * 4;
      q0 = fmax(q0, __ldcg(pt)); q1 = fmax(q1, __ldcg(pt + 1)); q2 = fmax(q2, __ldcg(pt + 2));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      q0 = fmax(q0, __shfl_xor_sync(0xffffffffu, q0, o));
      q1 = fmax(q1, __shfl_xor_sync(0xffffffffu, q1, o));
      q2 = fmax(q2, __shfl_xor_sync(0xffffffffu, q2, o));
    }
    if (it == 0) normA = q2;
    converged = q0 <= sqrt((double)n) * 1.1102230246251565e-16 * normA * q1;
  }
  if (!converged && g == 0 && tid == 0) *a.need_fp64 = 1;
}

__global__ void __launch_bounds__(BKB_THREADS, 1) k_chol_blk(CholBlkArgs a) {
  chol_blk_run(a, blockIdx.x, gridDim.x);
}

// Several independent solves in one cooperative launch: instance i owns the
// CTAs [cta0[i], cta0[i + 1]) and its own barrier counter, so the instances'
// panel chains run side by side on disjoint SMs.
constexpr int BLK_GROUP_MAX = 32;
struct CholBlkGroup {
  int n;
  int cta0[BLK_GROUP_MAX + 1];
  CholBlkArgs inst[BLK_GROUP_MAX];
};

__global__ void __launch_bounds__(BKB_THREADS, 1) k_chol_blk_group(const __grid_constant__ CholBlkGroup gr) {
  int i = 0;
  while (i + 1 < gr.n && (int)blockIdx.x >= gr.cta0[i + 1]) ++i;
  chol_blk_run(gr.inst[i], (int)blockIdx.x - gr.cta0[i], gr.cta0[i + 1] - gr.cta0[i]);
}

}  // namespace nqs
