// chol_ir.cuh -- (T + lambda I) x = eps' (Eq. minsrR) to FP64 accuracy by
// iterative refinement on an FP32 Cholesky factor, one cooperative launch
// (sm_103a).
//
// B300's FP64 unit retires two lane-FMAs per clock per SM, 64x below FP32,
// and a Cholesky of this size is a chain of n dependent pivots; so the
// factor is computed in FP32 (same right-looking panel scheme as the FP64
// kernel: redundant warp-level diagonal blocks, grid-wide panel rows,
// trailing update in 32x32 tiles) and the solution is refined in FP64:
//   x_0 = 0, r_0 = b;  d = L^{-T} (L^{-1} r) (FP32);  x += d;
//   r = b - A x in FP64 on all SMs;  stop when the backward error satisfies
//   ||r||_inf <= sqrt(n) u64 ||A||_inf ||x||_inf  (LAPACK's dsposv test).
// Substitutions are a chain of dependent steps; instead the inverse L^{-1}
// is formed once by recursive doubling (32x32 diagonal blocks inverted in
// parallel, then per level X21 = -L22^{-1} (L21 L11^{-1}) as two tiled
// products over all SMs), and each sweep is two distributed products.
// A non-positive FP32 pivot, or no convergence within maxit sweeps, sets
// *need_fp64 and leaves x to the FP64 Cholesky that the host launches next
// (it returns at once when *need_fp64 is 0).  Grid barriers are bounded.
#pragma once
#include "chol_coop.cuh"

namespace nqs {

constexpr int IR_B = 32;
constexpr int IR_THREADS = 256;

struct CholIrArgs {
  const double *A;   // [n][n], both triangles: T + lambda I (not modified)
  int64_t n;
  const double *b;   // [n]
  double *x;         // [n] out
  float *L;          // [n][n] scratch: FP32 factor (lower triangle)
  float *Li;         // [n][n] scratch: FP32 inverse of the factor (lower)
  float *Tm;         // [n][n] scratch: products of the inversion levels
  float *wv;         // [n] scratch: L^{-1} r
  float *dpart;      // [chunks][n] scratch: partial sums of L^{-T} w
  double *r;         // [n] scratch: FP64 residual
  double *part;      // [2][gridDim][4] scratch: partial norms (by sweep parity)
  unsigned *bar;     // barrier arrival counter (zeroed before launch)
  int32_t *status;   // NQS_ERR_TIMEOUT on a barrier timeout
  int32_t *need_fp64;// out: 1 when the FP64 factorisation must run
  int maxit;
  float *dv;         // [n] scratch: L^{-T} w (substitution sweeps)
  int subst;         // 1: sweeps by block substitution with the inverted
                     // 32x32 diagonal blocks (no full inverse); 0: two
                     // products with the explicit inverse
  float *dg;         // [2][IR_DG] scratch: the next panel's factored
                     // diagonal block, 1/L_jj and its pivot flag
};

// published diagonal block: [32][32] factor (zero upper triangle), [32]
// reciprocal pivots, one pivot flag; padded to 128-byte rows
constexpr int IR_DG = IR_B * IR_B + 2 * IR_B;

// Per-warp 32x32 tile product in shared memory (row stride WS floats, a
// multiple of 4 so rows are 16-byte aligned): lane j owns column j of the
// tile, acc[i] += sum_k sA[i][k] * B(k, j) with B(k, j) = sB[j][k] (nt) or
// sB[k][j] (nn).  Row reads of sA are warp-wide broadcasts of 16 bytes.
constexpr int WS = IR_B + 4;
template <bool NT>
__device__ __forceinline__ void warp_tile_fma(const float *sA, const float *sB, int lane,
                                              float (&acc)[IR_B]) {
#pragma unroll 2
  for (int k = 0; k < IR_B; k += 4) {
    float b0, b1, b2, b3;
    if (NT) {
      const float4 bv = *reinterpret_cast<const float4 *>(sB + lane * WS + k);
      b0 = bv.x; b1 = bv.y; b2 = bv.z; b3 = bv.w;
    } else {
      b0 = sB[(k + 0) * WS + lane]; b1 = sB[(k + 1) * WS + lane];
      b2 = sB[(k + 2) * WS + lane]; b3 = sB[(k + 3) * WS + lane];
    }
#pragma unroll
    for (int i = 0; i < IR_B; ++i) {
      const float4 av = *reinterpret_cast<const float4 *>(sA + i * WS + k);
      acc[i] = fmaf(av.x, b0, acc[i]);
      acc[i] = fmaf(av.y, b1, acc[i]);
      acc[i] = fmaf(av.z, b2, acc[i]);
      acc[i] = fmaf(av.w, b3, acc[i]);
    }
  }
}

// Stage rows r0.. r0+31, columns c0.. c0+31 of M (row stride ld, nrow x ncol
// valid) into a warp's tile; zeros outside, and columns >= cmax.
__device__ __forceinline__ void warp_stage(float *sT, const float *M, int64_t ld, int64_t r0,
                                           int64_t c0, int64_t nrow, int64_t ncol, int64_t cmax,
                                           int lane) {
  const int64_t c = c0 + lane;
  const bool cok = c < ncol && c < cmax;
  float v[IR_B];  // all 32 row loads in flight before the first store
#pragma unroll
  for (int r = 0; r < IR_B; ++r) {
    const int64_t rr = r0 + r;
    v[r] = (cok && rr < nrow) ? M[rr * ld + c] : 0.f;
  }
#pragma unroll
  for (int r = 0; r < IR_B; ++r) sT[r * WS + lane] = v[r];
}

// Cholesky of one 32x32 diagonal block by one warp; lane i holds row i
// (identity outside the valid m x m block).  Column j is published through
// shared memory (one store per lane, read back as broadcast float4s; two
// buffers so one __syncwarp per column suffices) and every lane takes the
// pivot itself, so the dependent chain per column is one store/load round
// trip, a reciprocal square root and one FMA.  The updates run on every lane
// unconditionally: lanes i < k only touch the upper triangle, which is
// scratch and cleared column by column.  Returns nonzero (uniform over the
// warp) for a pivot that is not positive; lane j's rinv is 1/L_jj.
__device__ __forceinline__ int warp_chol32(float (&rr)[IR_B], float *colb, int lane,
                                           float &rinv) {
  int bad = 0;
#pragma unroll
  for (int j = 0; j < IR_B; ++j) {
    float *cb = colb + (j & 1) * IR_B;
    cb[lane] = rr[j];
    __syncwarp();
    float c[IR_B];
#pragma unroll
    for (int q = j / 4; q < IR_B / 4; ++q) {
      const float4 v = reinterpret_cast<const float4 *>(cb)[q];
      c[4 * q] = v.x; c[4 * q + 1] = v.y; c[4 * q + 2] = v.z; c[4 * q + 3] = v.w;
    }
    const float dj = c[j];
    bad |= !(dj > 0.f);
    const float inv = dj > 0.f ? rsqrtf(dj) : 0.f;
    const float lij = rr[j] * inv;  // L_ij for lane i > j
    const float t = lij * inv;      // L_ij / L_jj
#pragma unroll
    for (int k = j + 1; k < IR_B; ++k) rr[k] = fmaf(-t, c[k], rr[k]);
    rr[j] = lane == j ? dj * inv : (lane > j ? lij : 0.f);
    if (lane == j) rinv = inv;
  }
  return bad;
}

// Panel rows L_rp = A_rp L_pp^{-T} by substitution, NR rows per warp at
// once (lane k holds entry k of each row; the same operations per row
// whatever NR, so every CTA that solves a row gets the same values).
template <int NR>
__device__ __forceinline__ void panel_row_solve(float (&v)[NR], const float (*D)[IR_B + 1],
                                                const float *rinv, int m, int lane) {
  for (int k = 0; k < m; ++k) {
    const float rk = rinv[k], dk = D[lane][k];
    const bool upd = lane > k && lane < m;
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      if (lane == k) v[r] = v[r] * rk;
      const float lk = __shfl_sync(0xffffffffu, v[r], k);
      if (upd) v[r] = fmaf(-dk, lk, v[r]);
    }
  }
}

// Factor the diagonal block staged in S ([32][33], lower triangle valid for
// the first m rows and columns) and publish it: the factor into L (rows and
// columns c0..c0+m), the block with zero upper triangle, 1/L_jj and the pivot
// flag into dg.  One warp; S is overwritten.
__device__ __noinline__ void warp_factor_publish(float *S, int m, float *colb, float *L,
                                                    int64_t n, int64_t c0, float *dg, int lane) {
  constexpr int SS = IR_B + 1;
  float rr[IR_B];
#pragma unroll
  for (int k = 0; k < IR_B; ++k)
    rr[k] = (lane < m && k < m && k <= lane) ? S[lane * SS + k] : (k == lane ? 1.f : 0.f);
  float rinv = 1.f;
  const int bad = warp_chol32(rr, colb, lane, rinv);
  __syncwarp();
#pragma unroll
  for (int k = 0; k < IR_B; ++k) S[lane * SS + k] = rr[k];
  __syncwarp();
#pragma unroll 8
  for (int r = 0; r < IR_B; ++r) {
    const float v = S[r * SS + lane];
    dg[r * IR_B + lane] = v;
    if (r < m && lane <= r) L[(c0 + r) * n + c0 + lane] = v;
  }
  dg[IR_B * IR_B + lane] = rinv;
  if (lane == 0) dg[IR_B * IR_B + IR_B] = __int_as_float(bad);
}

// Inverse of the unit-padded lower-triangular block D ([32][33]) into the
// diagonal block of Li at c0 (m x m valid); lane j forms column j.
__device__ __noinline__ void warp_tri_inverse(const float (*D)[IR_B + 1], int m, float *Li,
                                                 int64_t n, int64_t c0, int lane) {
  const int j = lane;
  float xc[IR_B];
#pragma unroll
  for (int i = 0; i < IR_B; ++i) {
    float acc = (i == j) ? 1.f : 0.f;
#pragma unroll
    for (int k = 0; k < i; ++k) acc -= D[i][k] * xc[k];
    xc[i] = (i >= j) ? acc / D[i][i] : 0.f;
  }
#pragma unroll
  for (int i = 0; i < IR_B; ++i)
    if (i < m && j < m && i >= j) Li[(c0 + i) * n + c0 + j] = xc[i];
}

// Asynchronous global -> shared copies (cp.async, completion by groups);
// src_bytes < size fills the rest with zeros (0: nothing is read).
__device__ __forceinline__ void cp_async16(float *dst, const float *src, int src_bytes) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async4(float *dst, const float *src, int src_bytes) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all_but_one() {
  asm volatile("cp.async.wait_group 1;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// K pieces of the inversion-level products staged whole in shared memory:
// A rows [32][LV_KP + 4], B rows [LV_KP][36], two pieces in flight.
constexpr int LV_KP = 256;
constexpr int LV_AS = LV_KP + 4, LV_BS = IR_B + 4;
constexpr int LV_STAGE = IR_B * LV_AS + LV_KP * LV_BS;  // floats per piece

// Stage rows i0..i0+31, columns ac..ac+klen of Aop and rows br..br+klen,
// columns j0..j0+31 of Bop (n x n, row-major; zeros outside) into one piece.
// vec: n % 4 == 0, so every 16-byte chunk is aligned and wholly in or out.
__device__ __forceinline__ void lv_stage(float *sA, float *sB, const float *Aop, const float *Bop,
                                         int64_t n, int64_t i0, int64_t ac, int64_t br, int64_t j0,
                                         int klen, bool vec, int tid) {
  if (vec) {
    const int qa = klen / 4;
    for (int c = tid; c < IR_B * qa; c += IR_THREADS) {
      const int r = c / qa, q = c - r * qa;
      const int64_t row = i0 + r, col = ac + 4 * q;
      const bool ok = row < n && col < n;
      cp_async16(sA + r * LV_AS + 4 * q, ok ? Aop + row * n + col : Aop, ok ? 16 : 0);
    }
    for (int c = tid; c < klen * (IR_B / 4); c += IR_THREADS) {
      const int r = c >> 3, q = c & 7;
      const int64_t row = br + r, col = j0 + 4 * q;
      const bool ok = row < n && col < n;
      cp_async16(sB + r * LV_BS + 4 * q, ok ? Bop + row * n + col : Bop, ok ? 16 : 0);
    }
  } else {
    for (int c = tid; c < IR_B * klen; c += IR_THREADS) {
      const int r = c / klen, q = c - r * klen;
      const int64_t row = i0 + r, col = ac + q;
      const bool ok = row < n && col < n;
      cp_async4(sA + r * LV_AS + q, ok ? Aop + row * n + col : Aop, ok ? 4 : 0);
    }
    for (int c = tid; c < klen * IR_B; c += IR_THREADS) {
      const int r = c >> 5, q = c & 31;
      const int64_t row = br + r, col = j0 + q;
      const bool ok = row < n && col < n;
      cp_async4(sB + r * LV_BS + q, ok ? Bop + row * n + col : Bop, ok ? 4 : 0);
    }
  }
  cp_async_commit();
}

// WT: 32x32 tiles of the trailing update and of the inversion products are
// spread one per warp (more tiles in flight; better at large n), else one
// per CTA with four outputs per thread (shorter per-tile latency; better at
// small n).  The launch picks the variant (or the autotuner does).
template <bool WT>
__global__ void __launch_bounds__(IR_THREADS) k_chol_ir(CholIrArgs a) {
  extern __shared__ float ir_smem[];
  float (*D)[IR_B + 1] = reinterpret_cast<float (*)[IR_B + 1]>(ir_smem);  // [32][33]
  float *rinv = ir_smem + IR_B * (IR_B + 1);          // [32]
  float *wtile = rinv + IR_B;                          // [8 warps][2][32][WS]
  constexpr int TS = IR_B + 1;                         // CTA tiles: [32][33] each
  float *ta = wtile, *tb = wtile + IR_B * TS;
  __shared__ int flag_s;
  __shared__ double red_s[IR_THREADS / 32][3];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int G = gridDim.x, g = blockIdx.x;
  const int64_t n = a.n;
  const int nb = (int)((n + IR_B - 1) / IR_B);
  float *L = a.L;
  // grid barrier instances passed (the same sequence in every CTA)
  unsigned ep = 0;
  auto gsync = [&]() -> bool { ++ep; return cc_sync_ep(a.bar, a.status, ep * (unsigned)G); };

  // (0) FP32 copy of the lower triangle (diagonal block 0 excepted) and
  // Li cleared; CTA 0 factors diagonal block 0 straight from A and publishes
  // it.  From here on the factor is right-looking with look-ahead: while the
  // other CTAs update the trailing matrix of panel p, CTA 0 updates the
  // next diagonal block alone, factors and publishes it, so the factor of a
  // diagonal block is never on the path between the two grid barriers of a
  // panel.
  __shared__ __align__(16) float colb_s[2 * IR_B];
  float *S = wtile + 2 * IR_B * TS;  // [32][33] staging of a diagonal block
  const int m0 = (int)min64(IR_B, n);
  for (int64_t i = g; i < n; i += G) {  // one row per CTA at a time, no division
    const double *Ai = a.A + i * n;
    float *Lr = L + i * n, *Lir = a.Li + i * n;
    if (i >= m0) {
#pragma unroll 4
      for (int64_t j = tid; j <= i; j += IR_THREADS) Lr[j] = (float)Ai[j];
    }
#pragma unroll 4
    for (int64_t j = tid; j < n; j += IR_THREADS) Lir[j] = 0.f;
  }
  if (g == 0 && warp == 0) {
    float v[IR_B];
#pragma unroll
    for (int r = 0; r < IR_B; ++r) v[r] = (r < m0 && lane <= r) ? (float)a.A[r * n + lane] : 0.f;
#pragma unroll
    for (int r = 0; r < IR_B; ++r) S[r * TS + lane] = v[r];
    __syncwarp();
    warp_factor_publish(S, m0, colb_s, L, n, 0, a.dg, lane);
  }
  if (!gsync()) return;

  // (1) FP32 right-looking Cholesky.  With look-ahead CTA 0 solves the
  // panel rows of the next diagonal block itself and writes them, joins the
  // first barrier of the panel without waiting at it, updates and factors
  // that block and publishes it before the second barrier; the other CTAs
  // solve the panel rows below that block and update the rest of the
  // trailing matrix.  (CTA 0 alone writes the rows it reads at the start of
  // the panel, so no other CTA can overwrite them before it has read them.)
  const bool la = G > 1;
  const int Gr = la ? G - 1 : G;               // CTAs that solve panel rows
  const int gr = la ? g - 1 : g;
  for (int p = 0; p < nb; ++p) {
    const int64_t c0 = (int64_t)p * IR_B;
    const int m = (int)min64(IR_B, n - c0);
    const int64_t r0 = c0 + m;
    const int64_t tr = n - r0;
    const int m1 = (int)min64(IR_B, tr);     // size of the next diagonal block
    const bool look = la && g == 0;
    // panel rows are requested before the published block
    float v[4] = {0.f, 0.f, 0.f, 0.f};
    const int64_t rfirst = r0 + (la ? m1 : 0) + (int64_t)gr * (IR_THREADS / 32) + warp;
    if (look) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int row = warp + 8 * q;
        v[q] = (row < m1 && lane < m) ? L[(r0 + row) * n + c0 + lane] : 0.f;
      }
    } else {
      v[0] = (rfirst < n && lane < m) ? L[rfirst * n + c0 + lane] : 0.f;
    }
    {
      const float *dgp = a.dg + (p & 1) * IR_DG;
      float dv[IR_B * IR_B / IR_THREADS];
#pragma unroll
      for (int q = 0; q < IR_B * IR_B / IR_THREADS; ++q) dv[q] = __ldcg(dgp + tid + q * IR_THREADS);
      const float rv = tid < IR_B ? __ldcg(dgp + IR_B * IR_B + tid) : 0.f;
      const float fv = tid == 0 ? __ldcg(dgp + IR_B * IR_B + IR_B) : 0.f;
#pragma unroll
      for (int q = 0; q < IR_B * IR_B / IR_THREADS; ++q) {
        const int e = tid + q * IR_THREADS;
        D[e >> 5][e & 31] = dv[q];
      }
      if (tid < IR_B) rinv[tid] = rv;
      if (tid == 0) flag_s = __float_as_int(fv);
    }
    __syncthreads();
    if (flag_s) {  // identical in every CTA: the FP64 factorisation takes over
      if (g == 0 && tid == 0) *a.need_fp64 = 1;
      return;
    }
    if (look) {
      const int tx = tid % 32, ty = tid / 32;
      float old[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i = ty + 8 * q;
        old[q] = (i < m1 && tx <= i) ? L[(r0 + i) * n + r0 + tx] : 0.f;
      }
      if (tr > 0) {
        panel_row_solve<4>(v, D, rinv, m, lane);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int row = warp + 8 * q;
          ta[row * TS + lane] = v[q];
          if (row < m1 && lane < m) L[(r0 + row) * n + c0 + lane] = v[q];
        }
      }
      ++ep;
      cc_arrive(a.bar);  // first barrier of the panel (publishes those rows), not awaited
      if (tr > 0) {
        // tile (0, 0) of the trailing matrix from the rows just solved
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 8
        for (int k = 0; k < IR_B; ++k) {
          const float bv = ta[tx * TS + k];
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[q] = fmaf(ta[(ty + 8 * q) * TS + k], bv, acc[q]);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) S[(ty + 8 * q) * TS + tx] = old[q] - acc[q];
        __syncthreads();
        if (warp == 0)
          warp_factor_publish(S, m1, colb_s, L, n, r0, a.dg + ((p + 1) & 1) * IR_DG, lane);
      }
      // the first barrier must be complete before CTA 0 joins the second
      if (!cc_wait_ep(a.bar, a.status, ep * (unsigned)G)) return;
    } else {
      // panel rows below the diagonal block: L_rp = A_rp L_pp^{-T}
      for (int64_t r = rfirst; r < n; r += (int64_t)Gr * (IR_THREADS / 32)) {
        float w[1] = {r == rfirst ? v[0] : (lane < m ? L[r * n + c0 + lane] : 0.f)};
        panel_row_solve<1>(w, D, rinv, m, lane);
        if (lane < m) L[r * n + c0 + lane] = w[0];
      }
      if (!gsync()) return;
      if (tr > 0) {
        const int nt = (int)((tr + IR_B - 1) / IR_B);
        const int ntiles = nt * (nt + 1) / 2;
        const int cta0 = la ? 1 : 0;  // with look-ahead tile 0 is CTA 0's
        if constexpr (!WT) {
          // trailing update A_ij -= L_ip L_jp^T, one 32x32 tile per CTA at a
          // time; a CTA's tiles go in batches of TB whose loads (operands
          // and the outputs' old values) are all in flight together, then
          // are multiplied back to back
          constexpr int TB = 4;
          constexpr int TU = IR_B + 4;  // row stride: 16-byte rows, float4 reads conflict-free
          const int tx = tid % 32, ty = tid / 32;
          for (int tb0 = gr + cta0; tb0 < ntiles; tb0 += TB * Gr) {
            float va[TB][4], vb[TB][4], vc[TB][4];
            int64_t i0s[TB], j0s[TB];
#pragma unroll
            for (int b = 0; b < TB; ++b) {
              const int t = tb0 + b * Gr;
              int ti = 0, tj = 0;
              if (t < ntiles) {
                ti = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
                while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
                while (ti * (ti + 1) / 2 > t) --ti;
                tj = t - ti * (ti + 1) / 2;
              }
              const int64_t i0 = r0 + (int64_t)ti * IR_B, j0 = r0 + (int64_t)tj * IR_B;
              i0s[b] = t < ntiles ? i0 : n;  // n: nothing to do
              j0s[b] = j0;
#pragma unroll
              for (int q = 0; q < 4; ++q) {
                const int rr = ty + 8 * q, k = tx;
                va[b][q] = (t < ntiles && i0 + rr < n && k < m) ? L[(i0 + rr) * n + c0 + k] : 0.f;
                vb[b][q] = (t < ntiles && j0 + rr < n && k < m) ? L[(j0 + rr) * n + c0 + k] : 0.f;
                const int64_t i = i0 + rr, j = j0 + k;
                vc[b][q] = (t < ntiles && i < n && j < n && j <= i) ? L[i * n + j] : 0.f;
              }
            }
            __syncthreads();  // the previous batch is no longer read
#pragma unroll
            for (int b = 0; b < TB; ++b) {
              float *sa = wtile + b * 2 * IR_B * TU, *sb = sa + IR_B * TU;
#pragma unroll
              for (int q = 0; q < 4; ++q) {
                sa[(ty + 8 * q) * TU + tx] = va[b][q];
                sb[(ty + 8 * q) * TU + tx] = vb[b][q];
              }
            }
            __syncthreads();
#pragma unroll
            for (int b = 0; b < TB; ++b) {
              if (i0s[b] >= n) continue;  // uniform over the CTA
              const float *sa = wtile + b * 2 * IR_B * TU, *sb = sa + IR_B * TU;
              // 4 outputs per thread: rows ty + 8q, column tx; four k per
              // 16-byte load (the sums still run over k in order)
              float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 2
              for (int k = 0; k < IR_B; k += 4) {
                const float4 bv = *reinterpret_cast<const float4 *>(sb + tx * TU + k);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                  const float4 av = *reinterpret_cast<const float4 *>(sa + (ty + 8 * q) * TU + k);
                  acc[q] = fmaf(av.x, bv.x, acc[q]);
                  acc[q] = fmaf(av.y, bv.y, acc[q]);
                  acc[q] = fmaf(av.z, bv.z, acc[q]);
                  acc[q] = fmaf(av.w, bv.w, acc[q]);
                }
              }
#pragma unroll
              for (int q = 0; q < 4; ++q) {
                const int64_t i = i0s[b] + ty + 8 * q, j = j0s[b] + tx;
                if (i < n && j < n && j <= i) L[i * n + j] = vc[b][q] - acc[q];
              }
            }
          }
        } else {
          // trailing update A_ij -= L_ip L_jp^T, one 32x32 tile of the lower
          // triangle per warp
          float *sA = wtile + warp * 2 * IR_B * WS, *sB = sA + IR_B * WS;
          const int64_t gwarp = (int64_t)gr * (IR_THREADS / 32) + warp + cta0;
          for (int64_t t = gwarp; t < ntiles; t += (int64_t)Gr * (IR_THREADS / 32)) {
            int ti = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
            while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
            while (ti * (ti + 1) / 2 > t) --ti;
            const int tj = (int)(t - ti * (ti + 1) / 2);
            const int64_t i0 = r0 + (int64_t)ti * IR_B, j0 = r0 + (int64_t)tj * IR_B;
            __syncwarp();
            warp_stage(sA, L, n, i0, c0, n, n, c0 + m, lane);
            warp_stage(sB, L, n, j0, c0, n, n, c0 + m, lane);
            __syncwarp();
            float acc[IR_B];
#pragma unroll
            for (int i = 0; i < IR_B; ++i) acc[i] = 0.f;
            warp_tile_fma<true>(sA, sB, lane, acc);
            const int64_t j = j0 + lane;
#pragma unroll
            for (int i = 0; i < IR_B; ++i) {
              const int64_t ii = i0 + i;
              if (ii < n && j < n && j <= ii) L[ii * n + j] -= acc[i];
            }
          }
        }
        if (!la) {  // one CTA: it updated the next diagonal block itself
          __syncthreads();
          if (warp == 0) {
            float st[IR_B];
#pragma unroll
            for (int r = 0; r < IR_B; ++r)
              st[r] = (r < m1 && lane <= r) ? L[(r0 + r) * n + r0 + lane] : 0.f;
#pragma unroll
            for (int r = 0; r < IR_B; ++r) S[r * TS + lane] = st[r];
            __syncwarp();
            warp_factor_publish(S, m1, colb_s, L, n, r0, a.dg + ((p + 1) & 1) * IR_DG, lane);
          }
        }
      }
    }
    if (!gsync()) return;
  }
  // diagonal blocks of the inverse, one block per CTA
  for (int blk = g; blk < nb; blk += G) {
    const int64_t c0 = (int64_t)blk * IR_B;
    const int m = (int)min64(IR_B, n - c0);
    __syncthreads();
    for (int e = tid; e < IR_B * IR_B; e += IR_THREADS) {
      const int i = e / IR_B, j = e % IR_B;
      D[i][j] = (i < m && j <= i) ? L[(c0 + i) * n + c0 + j] : (i == j ? 1.f : 0.f);
    }
    __syncthreads();
    if (warp == 0) warp_tri_inverse(D, m, a.Li, n, c0, lane);
  }
  if (!gsync()) return;

  // (2) explicit inverse of the FP32 factor by recursive doubling: the
  //     diagonal 32x32 blocks are inverted above; per level, for every pair
  //     of inverted s x s blocks, X21 = -L22^{-1} (L21 L11^{-1}).
  float *Li = a.Li;
  for (int64_t sz = IR_B; sz < n && !a.subst; sz *= 2) {
    // Tm[pair block] = L21 Li11 ; then Li21 = -Li22 Tm
    for (int phase = 0; phase < 2; ++phase) {
      const int64_t pairs = (n + 2 * sz - 1) / (2 * sz);
      const int64_t tps = (sz + IR_B - 1) / IR_B;  // tiles per side of a pair block
      const int64_t ntile = pairs * tps * tps;
      if constexpr (!WT) {
        // one 32x32 output tile per CTA; the triangular operand (Li11 in
        // phase 0, Li22 in phase 1) makes leading or trailing K chunks zero,
        // which are skipped (each output still sums its nonzero terms in
        // ascending k).  Tiles go out by decreasing K length, round-robin
        // in alternating directions, to balance the CTAs.
        const bool vec = (n & 3) == 0;
        float *stg = wtile;  // two pieces of LV_STAGE floats
        for (int64_t rnd = 0; rnd * G < ntile; ++rnd) {
          const int64_t t = rnd * G + ((rnd & 1) ? (G - 1 - g) : g);
          if (t >= ntile) continue;                   // uniform over the CTA
          const int64_t pr = t % pairs, u = t / pairs;
          const int64_t ti = phase == 0 ? u % tps : tps - 1 - u / tps;
          const int64_t tj = phase == 0 ? u / tps : u % tps;
          const int64_t base = pr * 2 * sz;
          const int64_t i0 = base + sz + ti * IR_B;   // rows of the lower-left block
          const int64_t j0 = base + tj * IR_B;        // columns
          if (i0 >= n) continue;                      // uniform over the CTA
          const float *Aop; const float *Bop;
          int64_t acol0, brow0, kb, ke;
          if (phase == 0) {  // Tm = L21 Li11: Li11 rows below j0 only
            Aop = L; acol0 = base; Bop = Li; brow0 = base; kb = tj * IR_B; ke = sz;
          } else {           // Li21 = -Li22 Tm: Li22 columns up to row i0 + 31
            Aop = Li; acol0 = base + sz; Bop = a.Tm; brow0 = base + sz; kb = 0;
            ke = (ti + 1) * IR_B;
          }
          const int tx = tid % 32, ty = tid / 32;
          float acc[4] = {0.f, 0.f, 0.f, 0.f};
          const int np = (int)((ke - kb + LV_KP - 1) / LV_KP);
          __syncthreads();  // the previous tile's pieces are no longer read
          for (int q = 0; q < np && q < 2; ++q) {
            const int64_t k0 = kb + (int64_t)q * LV_KP;
            float *sA = stg + q * LV_STAGE;
            lv_stage(sA, sA + IR_B * LV_AS, Aop, Bop, n, i0, acol0 + k0, brow0 + k0, j0,
                     (int)min64(LV_KP, ke - k0), vec, tid);
          }
          for (int q = 0; q < np; ++q) {
            if (q + 1 < np) cp_async_wait_all_but_one(); else cp_async_wait_all();
            __syncthreads();
            const int64_t k0 = kb + (int64_t)q * LV_KP;
            const int klen = (int)min64(LV_KP, ke - k0);
            const float *sA = stg + (q & 1) * LV_STAGE, *sB = sA + IR_B * LV_AS;
#pragma unroll 2
            for (int kk = 0; kk < klen; kk += 4) {
              const float b0 = sB[(kk + 0) * LV_BS + tx], b1 = sB[(kk + 1) * LV_BS + tx];
              const float b2 = sB[(kk + 2) * LV_BS + tx], b3 = sB[(kk + 3) * LV_BS + tx];
#pragma unroll
              for (int r = 0; r < 4; ++r) {
                const float4 av = *reinterpret_cast<const float4 *>(sA + (ty + 8 * r) * LV_AS + kk);
                acc[r] = fmaf(av.x, b0, acc[r]);
                acc[r] = fmaf(av.y, b1, acc[r]);
                acc[r] = fmaf(av.z, b2, acc[r]);
                acc[r] = fmaf(av.w, b3, acc[r]);
              }
            }
            if (q + 2 < np) {
              __syncthreads();  // piece q is no longer read
              const int64_t k2 = kb + (int64_t)(q + 2) * LV_KP;
              float *sA2 = stg + (q & 1) * LV_STAGE;
              lv_stage(sA2, sA2 + IR_B * LV_AS, Aop, Bop, n, i0, acol0 + k2, brow0 + k2, j0,
                       (int)min64(LV_KP, ke - k2), vec, tid);
            }
          }
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int64_t i = i0 + ty + 8 * q, j = j0 + tx;
            if (i < n && j < n && j < base + sz) {
              if (phase == 0) a.Tm[i * n + j] = acc[q];
              else Li[i * n + j] = -acc[q];
            }
          }
        }
      } else {
      float *sA = wtile + warp * 2 * IR_B * WS, *sB = sA + IR_B * WS;
      const int64_t gwarp = (int64_t)g * (IR_THREADS / 32) + warp;
      for (int64_t t = gwarp; t < ntile; t += (int64_t)G * (IR_THREADS / 32)) {
        const int64_t pr = t / (tps * tps), tt = t % (tps * tps);
        const int64_t ti = tt / tps, tj = tt % tps;
        const int64_t base = pr * 2 * sz;
        const int64_t i0 = base + sz + ti * IR_B;   // rows of the lower-left block
        const int64_t j0 = base + tj * IR_B;        // columns
        if (i0 >= n) continue;                      // uniform over the warp
        const float *Aop; const float *Bop;
        int64_t acol0, brow0;
        if (phase == 0) {  // Tm = L21 * Li11: A = L rows i, cols base..; B = Li11
          Aop = L; acol0 = base; Bop = Li; brow0 = base;
        } else {           // Li21 = -Li22 * Tm: A = Li22 rows i, cols base+sz..; B = Tm
          Aop = Li; acol0 = base + sz; Bop = a.Tm; brow0 = base + sz;
        }
        float acc[IR_B];
#pragma unroll
        for (int i = 0; i < IR_B; ++i) acc[i] = 0.f;
        for (int64_t k0 = 0; k0 < sz; k0 += IR_B) {
          __syncwarp();
          warp_stage(sA, Aop, n, i0, acol0 + k0, n, n, n, lane);
          warp_stage(sB, Bop, n, brow0 + k0, j0, n, n, n, lane);
          __syncwarp();
          warp_tile_fma<false>(sA, sB, lane, acc);
        }
        const int64_t j = j0 + lane;
#pragma unroll
        for (int i = 0; i < IR_B; ++i) {
          const int64_t ii = i0 + i;
          if (ii < n && j < n && j < base + sz) {
            if (phase == 0) a.Tm[ii * n + j] = acc[i];
            else Li[ii * n + j] = -acc[i];
          }
        }
      }
      }
      if (!gsync()) return;
    }
  }

  // (3) refinement: d = Li^T (Li r) on all SMs, residual in FP64
  for (int64_t i = (int64_t)g * IR_THREADS + tid; i < n; i += (int64_t)G * IR_THREADS) {
    a.r[i] = a.b[i];
    a.x[i] = 0.0;
  }
  if (!gsync()) return;
  const int64_t nwarps = (int64_t)G * (IR_THREADS / 32);
  const int64_t gw = (int64_t)g * (IR_THREADS / 32) + warp;
  constexpr int CH = 64;  // rows per partial sum of the transposed product
  const int64_t nch = (n + CH - 1) / CH;
  double normA = 0.0;
  int converged = 0;
  __shared__ float sw_s[IR_B];
  for (int it = 0; it < a.maxit && !converged; ++it) {
    if (a.subst) {
      // d = L^{-T} L^{-1} r by block substitution: per 32-block one grid
      // barrier; every CTA forms the block's solution from the inverted
      // diagonal block, CTA 0 stores it, all warps fold it into the rows
      // (forward) or columns (backward) still to come.
      for (int64_t i = (int64_t)g * IR_THREADS + tid; i < n; i += (int64_t)G * IR_THREADS)
        a.wv[i] = (float)a.r[i];
      if (!gsync()) return;
      for (int p = 0; p < nb; ++p) {  // forward: L w = r
        const int64_t c0 = (int64_t)p * IR_B;
        const int m = (int)min64(IR_B, n - c0);
        if (warp == 0) {
          float acc = 0.f;
          if (lane < m)
            for (int j = 0; j <= lane; ++j) acc = fmaf(Li[(c0 + lane) * n + c0 + j], a.wv[c0 + j], acc);
          sw_s[lane] = acc;
        }
        __syncthreads();
        if (g == 0 && tid < m) a.dv[c0 + tid] = sw_s[tid];
        for (int64_t i = c0 + m + gw; i < n; i += nwarps) {
          float t = lane < m ? L[i * n + c0 + lane] * sw_s[lane] : 0.f;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
          if (lane == 0) a.wv[i] -= t;
        }
        if (!gsync()) return;
      }
      for (int p = nb - 1; p >= 0; --p) {  // backward: L^T d = w (w in dv)
        const int64_t c0 = (int64_t)p * IR_B;
        const int m = (int)min64(IR_B, n - c0);
        if (warp == 0) {
          float acc = 0.f;
          if (lane < m)
            for (int k = lane; k < m; ++k) acc = fmaf(Li[(c0 + k) * n + c0 + lane], a.dv[c0 + k], acc);
          sw_s[lane] = acc;
        }
        __syncthreads();
        // the block's correction goes straight into x (dv of this block is
        // not read again)
        if (g == 0 && tid < m) a.x[c0 + tid] += (double)sw_s[tid];
        for (int64_t j = (int64_t)g * IR_THREADS + tid; j < c0; j += (int64_t)G * IR_THREADS) {
          float t = 0.f;
          for (int i = 0; i < m; ++i) t = fmaf(L[(c0 + i) * n + j], sw_s[i], t);
          a.dv[j] -= t;
        }
        if (!gsync()) return;
      }
    } else {
    // w = Li r (one warp per row)
    for (int64_t i = gw; i < n; i += nwarps) {
      const float *row = Li + i * n;
      float sacc = 0.f;
#pragma unroll 8
      for (int64_t j = lane; j <= i; j += 32) sacc = fmaf(row[j], (float)a.r[j], sacc);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sacc += __shfl_xor_sync(0xffffffffu, sacc, o);
      if (lane == 0) a.wv[i] = sacc;
    }
    if (!gsync()) return;
    // partial sums of Li^T w over 64-row chunks: (chunk, 32-column block) per warp
    const int64_t ncb = (n + 31) / 32;
    for (int64_t u = gw; u < nch * ncb; u += nwarps) {
      const int64_t ch = u / ncb, cb = u % ncb;
      const int64_t j = cb * 32 + lane;
      float sacc = 0.f;
      const int64_t r1 = min64(n, (ch + 1) * CH);
      if (j < n) {
        const int64_t i1 = max64(ch * CH, j);
#pragma unroll 16
        for (int64_t i = i1; i < r1; ++i) sacc = fmaf(Li[i * n + j], a.wv[i], sacc);
      }
      if (j < n) a.dpart[ch * n + j] = sacc;
    }
    if (!gsync()) return;
    for (int64_t j = (int64_t)g * IR_THREADS + tid; j < n; j += (int64_t)G * IR_THREADS) {
      float d = 0.f;
#pragma unroll 8
      for (int64_t ch = j / CH; ch < nch; ++ch) d += a.dpart[ch * n + j];
      a.x[j] += (double)d;
    }
    if (!gsync()) return;
    }
    // r = b - A x in FP64; partial max |r_i|, max |x_i| and (first sweep) max
    // row sum |A|
    double rmax = 0.0, xmax = 0.0, amax = 0.0;
    for (int64_t i = gw; i < n; i += nwarps) {
      const double *Ai = a.A + i * n;
      double sacc = 0.0, sa = 0.0;
#pragma unroll 8
      for (int64_t j = lane; j < n; j += 32) {
        const double aij = Ai[j];
        sacc = fma(aij, a.x[j], sacc);
        if (it == 0) sa += fabs(aij);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        sacc += __shfl_xor_sync(0xffffffffu, sacc, o);
        sa += __shfl_xor_sync(0xffffffffu, sa, o);
      }
      const double ri = a.b[i] - sacc;
      if (lane == 0) a.r[i] = ri;
      rmax = fmax(rmax, fabs(ri));
      xmax = fmax(xmax, fabs(a.x[i]));
      amax = fmax(amax, sa);
    }
    if (lane == 0) { red_s[warp][0] = rmax; red_s[warp][1] = xmax; red_s[warp][2] = amax; }
    __syncthreads();
    if (tid == 0) {
      double m0 = 0.0, m1 = 0.0, m2 = 0.0;
      for (int q = 0; q < IR_THREADS / 32; ++q) {
        m0 = fmax(m0, red_s[q][0]); m1 = fmax(m1, red_s[q][1]); m2 = fmax(m2, red_s[q][2]);
      }
      double *pt = a.part + (size_t)(it & 1) * G * 4;  // two buffers by sweep parity
      pt[(size_t)g * 4 + 0] = m0; pt[(size_t)g * 4 + 1] = m1; pt[(size_t)g * 4 + 2] = m2;
    }
    if (!gsync()) return;
    // maxima over the CTAs' partials: all loads in flight at once (max is
    // exact, so the grouping does not matter)
    {
      double q0 = 0.0, q1 = 0.0, q2 = 0.0;
      for (int q = tid; q < G; q += IR_THREADS) {
        const double *pt = a.part + (size_t)(it & 1) * G * 4;
        q0 = fmax(q0, pt[(size_t)q * 4]); q1 = fmax(q1, pt[(size_t)q * 4 + 1]);
        q2 = fmax(q2, pt[(size_t)q * 4 + 2]);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        q0 = fmax(q0, __shfl_xor_sync(0xffffffffu, q0, o));
        q1 = fmax(q1, __shfl_xor_sync(0xffffffffu, q1, o));
        q2 = fmax(q2, __shfl_xor_sync(0xffffffffu, q2, o));
      }
      __syncthreads();  // red_s of the sweep's own maxima has been read
      if (lane == 0) { red_s[warp][0] = q0; red_s[warp][1] = q1; red_s[warp][2] = q2; }
      __syncthreads();
    }
    double rn = 0.0, xn = 0.0, an = 0.0;
#pragma unroll
    for (int q = 0; q < IR_THREADS / 32; ++q) {
      rn = fmax(rn, red_s[q][0]); xn = fmax(xn, red_s[q][1]); an = fmax(an, red_s[q][2]);
    }
    if (it == 0) normA = an;
    converged = rn <= sqrt((double)n) * 1.1102230246251565e-16 * normA * xn;
    // the next sweep writes the other buffer; the one after that comes only
    // after that sweep's barriers, which every CTA passes after this read
  }
  if (!converged && g == 0 && tid == 0) *a.need_fp64 = 1;
}

inline size_t chol_ir_smem(int64_t) {
  const size_t tiles = (IR_THREADS / 32) * 2 * (size_t)IR_B * WS;  // warp tiles
  const size_t pieces = 2 * (size_t)LV_STAGE;                      // level pieces
  return sizeof(float) * ((size_t)IR_B * (IR_B + 1) + IR_B + (tiles > pieces ? tiles : pieces));
}

}  // namespace nqs
