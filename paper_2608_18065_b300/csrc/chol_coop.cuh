// chol_coop.cuh -- FP64 Cholesky solve of (T + lambda I) x = eps' (Eq. minsrR)
// in one cooperative, persistent launch (sm_103a).
//
// B300 runs FP64 at roughly 1.5 lane-FMAs per clock per SM, so a solve of
// this size is bound by the serial chain of panel factorisations and by the
// number of kernel boundaries, not by the total flop count.  One CTA per SM
// walks the 32-wide panels of a right-looking Cholesky:
//   (1) every CTA factors the 32x32 diagonal block in shared memory
//       (identical redundant work, no barrier needed to share it) and solves
//       its piece of the forward substitution L y = b;
//   (2) the rows below the panel are spread over all warps of the grid: each
//       warp solves one row of L_ip = A_ip L_pp^{-T} with a lane per column
//       and folds the row into the forward substitution;
//   (3) the trailing lower triangle is updated in 16x16 tiles spread over
//       all CTAs.
// Then the backward substitution L^T x = y runs one 32-block at a time:
// partial sums over rows on all warps, one grid barrier, and every CTA
// finishes the block redundantly into its own shared copy of x.
// Grid barriers spin with an iteration limit; a barrier that runs out sets
// NQS_ERR_TIMEOUT and every CTA returns.
#pragma once
#include "common.cuh"
#include "grid_sync.cuh"

namespace nqs {

constexpr int CC_B = 32;   // panel width
constexpr int CC_T = 16;   // trailing-update tile edge
constexpr int CC_THREADS = 256;

struct CholCoopArgs {
  double *A;          // [n][n], lower triangle holds T + lambda I, overwritten by L
  int64_t n;
  const double *b;    // [n]
  double *x;          // [n] out
  double *rhs;        // [n] scratch: right-hand side being reduced
  double *y;          // [n] scratch: forward-substitution result
  double *part;       // [2][gridDim][32] scratch: backward partial sums
  unsigned *bar;      // barrier arrival counter (zeroed before launch)
  int32_t *status;    // 0, NQS_ERR_NOT_SPD or NQS_ERR_TIMEOUT
  const int32_t *gate;// optional: run only when *gate != 0
};

__global__ void __launch_bounds__(CC_THREADS) k_chol_coop(CholCoopArgs a) {
  extern __shared__ double cc_smem[];
  double (*D)[CC_B + 1] = reinterpret_cast<double (*)[CC_B + 1]>(cc_smem);  // [32][33]
  double *rinv = cc_smem + CC_B * (CC_B + 1);        // [32]
  double *yp = rinv + CC_B;                          // [32]
  double *red = yp + CC_B;                           // [8 warps][32]
  constexpr int TS = CC_B + 1;                        // padded row stride of the tiles
  double *ta = red + 8 * CC_B;                       // [16][33] update tile rows i
  double *tb = ta + CC_T * TS;                       // [16][33] update tile rows j
  double *xs = tb + CC_T * TS;                       // [n] backward solution copy

  if (a.gate && *a.gate == 0) return;  // the refinement already produced x
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int G = gridDim.x, g = blockIdx.x;
  const int64_t n = a.n;
  const int nb = (int)((n + CC_B - 1) / CC_B);
  double *A = a.A;

  for (int64_t i = (int64_t)g * CC_THREADS + tid; i < n; i += (int64_t)G * CC_THREADS)
    a.rhs[i] = a.b[i];
  if (!cc_grid_sync(a.bar, a.status)) return;

  for (int p = 0; p < nb; ++p) {
    const int64_t c0 = (int64_t)p * CC_B;
    const int m = (int)min64(CC_B, n - c0);
    // (1) diagonal block, factored by warp 0 in registers: lane i holds row i;
    //     per pivot one rsqrt on its own lane, the rank-1 update by shuffles.
    __shared__ int bad_s;
    if (warp == 0) {
      double r[CC_B];
#pragma unroll
      for (int k = 0; k < CC_B; ++k)
        r[k] = (lane < m && k < m && k <= lane) ? A[(c0 + lane) * n + c0 + k]
                                                : (k == lane ? 1.0 : 0.0);
      int bad = 0;
#pragma unroll
      for (int j = 0; j < CC_B; ++j) {
        if (j < m) {
          const double dj = __shfl_sync(0xffffffffu, r[j], j);
          bad |= !(dj > 0.0);
          double inv = 0.0;
          if (lane == j && dj > 0.0) inv = rsqrt(dj);
          inv = __shfl_sync(0xffffffffu, inv, j);
          if (lane == j) { r[j] = dj * inv; rinv[j] = inv; }
          else if (lane > j) r[j] *= inv;
#pragma unroll
          for (int k = j + 1; k < CC_B; ++k) {
            const double lkj = __shfl_sync(0xffffffffu, r[j], k);
            if (lane >= k) r[k] -= r[j] * lkj;
          }
        }
      }
#pragma unroll
      for (int k = 0; k < CC_B; ++k) D[lane][k] = (k <= lane) ? r[k] : 0.0;
      if (lane == 0) bad_s = bad;
    }
    __syncthreads();
    if (bad_s) {  // identical in every CTA
      if (g == 0 && tid == 0) atomicExch(reinterpret_cast<int *>(a.status), (int)NQS_ERR_NOT_SPD);
      return;
    }
    // forward substitution of the block: L_pp y_p = rhs_p (warp 0)
    if (warp == 0) {
      double v = lane < m ? a.rhs[c0 + lane] : 0.0;
      for (int k = 0; k < m; ++k) {
        if (lane == k) v *= rinv[k];
        const double yk = __shfl_sync(0xffffffffu, v, k);
        if (lane > k && lane < m) v -= D[lane][k] * yk;
      }
      if (lane < m) yp[lane] = v;
    }
    __syncthreads();
    // (2) panel rows: one warp per row over the whole grid
    const int64_t r0 = c0 + m;
    for (int64_t r = r0 + (int64_t)g * 8 + warp; r < n; r += (int64_t)G * 8) {
      double v = lane < m ? A[r * n + c0 + lane] : 0.0;
      for (int k = 0; k < m; ++k) {
        if (lane == k) v *= rinv[k];
        const double lk = __shfl_sync(0xffffffffu, v, k);
        if (lane > k && lane < m) v -= D[lane][k] * lk;
      }
      if (lane < m) A[r * n + c0 + lane] = v;
      double t = lane < m ? v * yp[lane] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (lane == 0) a.rhs[r] -= t;
    }
    if (!cc_grid_sync(a.bar, a.status)) return;
    // every CTA has read A_pp and rhs_p by now: CTA 0 stores L_pp and y_p
    if (g == 0) {
      for (int e = tid; e < m * m; e += CC_THREADS) {
        const int i = e / m, j = e % m;
        if (j <= i) A[(c0 + i) * n + c0 + j] = D[i][j];
      }
      if (tid < m) a.y[c0 + tid] = yp[tid];
    }
    // (3) trailing update A_ij -= L_ip L_jp^T on 16x16 tiles of the lower triangle
    const int64_t tr = n - r0;
    if (tr > 0) {
      const int nt = (int)((tr + CC_T - 1) / CC_T);
      const int ntiles = nt * (nt + 1) / 2;
      for (int t = g; t < ntiles; t += G) {
        // t -> (ti, tj), tj <= ti, row-major over the lower triangle (FP32
        // estimate, integer correction: no FP64 on this path)
        int ti = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
        while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
        while (ti * (ti + 1) / 2 > t) --ti;
        const int tj = t - ti * (ti + 1) / 2;
        const int64_t i0 = r0 + (int64_t)ti * CC_T, j0 = r0 + (int64_t)tj * CC_T;
        __syncthreads();
        for (int e = tid; e < CC_T * CC_B; e += CC_THREADS) {
          const int rr = e / CC_B, k = e % CC_B;
          ta[rr * TS + k] = (i0 + rr < n && k < m) ? A[(i0 + rr) * n + c0 + k] : 0.0;
          tb[rr * TS + k] = (j0 + rr < n && k < m) ? A[(j0 + rr) * n + c0 + k] : 0.0;
        }
        __syncthreads();
        const int ty = tid / CC_T, tx = tid % CC_T;
        const int64_t i = i0 + ty, j = j0 + tx;
        if (i < n && j < n && j <= i) {
          double acc = 0.0;
#pragma unroll 8
          for (int k = 0; k < CC_B; ++k) acc = fma(ta[ty * TS + k], tb[tx * TS + k], acc);
          A[i * n + j] -= acc;
        }
      }
    }
    if (!cc_grid_sync(a.bar, a.status)) return;
  }

  // backward substitution L^T x = y, one block at a time from the last
  for (int p = nb - 1; p >= 0; --p) {
    const int64_t c0 = (int64_t)p * CC_B;
    const int m = (int)min64(CC_B, n - c0);
    const int64_t r0 = c0 + m;
    double acc = 0.0;  // lane = column of the block
    for (int64_t r = r0 + (int64_t)g * 8 + warp; r < n; r += (int64_t)G * 8)
      if (lane < m) acc += A[r * n + c0 + lane] * xs[r];
    red[warp * CC_B + lane] = acc;
    __syncthreads();
    double *part = a.part + (size_t)(p & 1) * G * CC_B;
    if (tid < CC_B) {
      double s = 0.0;
      for (int w = 0; w < 8; ++w) s += red[w * CC_B + tid];
      part[(size_t)g * CC_B + tid] = s;
    }
    if (!cc_grid_sync(a.bar, a.status)) return;
    // diagonal block of L into shared memory for the substitution
    for (int e = tid; e < CC_B * CC_B; e += CC_THREADS) {
      const int i = e / CC_B, j = e % CC_B;
      D[i][j] = (i < m && j <= i) ? A[(c0 + i) * n + c0 + j] : 0.0;
    }
    {  // the CTAs' partial sums, eight strided groups in flight
      double s = 0.0;
#pragma unroll 4
      for (int q = warp; q < G; q += 8) s += part[(size_t)q * CC_B + lane];
      red[warp * CC_B + lane] = s;
    }
    __syncthreads();
    if (warp == 0) {
      double s = 0.0;
      for (int w = 0; w < 8; ++w) s += red[w * CC_B + lane];
      double v = lane < m ? a.y[c0 + lane] - s : 0.0;
      const double dinv = lane < m ? 1.0 / D[lane][lane] : 0.0;
      for (int k = m - 1; k >= 0; --k) {
        if (lane == k) v *= dinv;
        const double xk = __shfl_sync(0xffffffffu, v, k);
        if (lane < k) v -= D[k][lane] * xk;
      }
      if (lane < m) {
        xs[c0 + lane] = v;
        if (g == 0) a.x[c0 + lane] = v;
      }
    }
    __syncthreads();
  }
}

inline size_t chol_coop_smem(int64_t n) {
  return sizeof(double) * ((size_t)CC_B * (CC_B + 1) + 2 * CC_B + 8 * CC_B + 2 * CC_T * (CC_B + 1) + (size_t)n);
}

}  // namespace nqs
