// gram_tc.cu -- T = A A^T (Algorithm 1, Gram step, Eq. minsrR) for FP32 A with
// split BF16 products on the 5th-generation tensor cores (sm_103a).
//
// A = hi + lo with hi = bf16(A), lo = bf16(A - hi), so hi + lo carries 16
// significant bits of A and T ~ (hi + lo)(hi + lo)^T = hi hi^T + hi lo^T +
// lo hi^T + lo lo^T.  All four products are issued: dropping lo lo^T (a
// positive semi-definite term of relative size 2^-18) biases every
// eigenvalue of T downwards and makes T + lambda I indefinite once lambda is
// below that bias.  The tensor core accumulates in FP32; summing thousands of
// MMAs into one FP32 accumulator loses about one unit in the last place of
// the running sum per MMA (2e-4 relative at K = 22k, always downwards), so
// each 64-wide k-block (16 MMAs) starts a fresh accumulator and the k-block
// results are added in registers with ordinary round-to-nearest FP32
// additions, whose errors do not drift in one direction.  Each CTA owns one 128x128 tile of the
// upper triangle and one slice of the K = Np reduction:
//   warp 0 lane 0  TMA producer: 4 operand tiles (hi/lo of the row block and
//                  of the column block, 128 x 64 bf16 each, 128B swizzle)
//                  per k-block into a 3-stage shared-memory ring;
//   warp 1 lane 0  MMA issuer: 4 k-steps x 4 tcgen05.mma (M=N=128, K=16)
//                  per k-block, alternating between two FP32 accumulators;
//   warps 2-9      add each finished accumulator into register sums (two
//                  warps per lane quarter, 64 columns each), then write the
//                  slice's FP64 partial tile.
// Tensor memory: the two accumulators at columns 0 and 128.  A second kernel sums the K-slices in FP64 and writes both
// triangles, so T is deterministic and exactly symmetric.  Every mbarrier
// wait has an iteration limit; on expiry the CTA raises an error flag, drains
// its own copies and MMAs (again with a limit), frees its tensor memory and
// exits.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <algorithm>
#include <cmath>
#include <cuda_bf16.h>

#include "common.cuh"
#include "gram_tc.h"
#include "tc_common.cuh"

namespace nqs {
namespace {

constexpr int BM = 128;                    // tile edge (M = N)
constexpr int BK = 64;                     // bf16 per k-block = one 128-byte swizzle row
constexpr int STAGES = 3;
constexpr int TILE_BYTES = BM * BK * 2;    // 16 KB
constexpr int STAGE_BYTES = 4 * TILE_BYTES;
constexpr int EPI_WARPS = 8;
constexpr int THREADS = 64 + 32 * EPI_WARPS;
constexpr int TMEM_COLS = 256;
constexpr int NBARS = 2 * STAGES + 5;      // full[S] empty[S] accfull[2] accfree[2] done
constexpr size_t SMEM_BYTES = (size_t)STAGES * STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/;

struct GramArgs {
  int R, kblocks, splits, nT;
  double *part;  // [tiles*splits][128][128]
  int *err;
};

__device__ __forceinline__ void tmem_ld16u(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
        "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}

__global__ void __launch_bounds__(THREADS, 1)
k_gram_tc(const __grid_constant__ CUtensorMap tm_hi, const __grid_constant__ CUtensorMap tm_lo,
              GramArgs g) {
  extern __shared__ __align__(1024) unsigned char gsm_raw[];
  unsigned char *gsm = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(gsm_raw) + 1023) & ~uintptr_t(1023));
  uint64_t *bars = reinterpret_cast<uint64_t *>(gsm + STAGES * STAGE_BYTES);
  uint64_t *full = bars, *empty = bars + STAGES, *accfull = bars + 2 * STAGES;
  uint64_t *accfree = accfull + 2, *done = accfree + 2;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + NBARS);
  int *abort_flag = reinterpret_cast<int *>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = blockIdx.x / g.splits, split = blockIdx.x % g.splits;
  // tile index -> (bi, bj), bi <= bj, row-major over the upper triangle
  int bi = 0, rem = t;
  while (rem >= g.nT - bi) { rem -= g.nT - bi; ++bi; }
  const int bj = bi + rem;
  const int kb0 = (int)((int64_t)split * g.kblocks / g.splits);
  const int kb1 = (int)((int64_t)(split + 1) * g.kblocks / g.splits);
  const int nk = kb1 - kb0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < 2 * STAGES + 2; ++s) mbar_init(smem_u32(&bars[s]), 1);
    for (int b = 0; b < 2; ++b) mbar_init(smem_u32(&accfree[b]), 32 * EPI_WARPS);
    mbar_init(smem_u32(done), 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------------------------------------------- TMA producer
      int issued = 0;
      for (int i = 0; i < nk; ++i) {
        const int s = i % STAGES;
        if (!mbar_wait(smem_u32(&empty[s]), ((i / STAGES) & 1) ^ 1)) {
          atomicExch(abort_flag, 1);
          break;
        }
        if (*reinterpret_cast<volatile int *>(abort_flag)) break;
        const uint32_t fb = smem_u32(&full[s]);
        mbar_expect_tx(fb, STAGE_BYTES);
        const uint32_t base = smem_u32(gsm + (size_t)s * STAGE_BYTES);
        const int x = (kb0 + i) * BK;
        tma_load_2d(base + 0 * TILE_BYTES, &tm_hi, fb, x, bi * BM);
        tma_load_2d(base + 1 * TILE_BYTES, &tm_lo, fb, x, bi * BM);
        tma_load_2d(base + 2 * TILE_BYTES, &tm_hi, fb, x, bj * BM);
        tma_load_2d(base + 3 * TILE_BYTES, &tm_lo, fb, x, bj * BM);
        ++issued;
      }
      // drain: every issued stage's copies have landed before the CTA may exit
      for (int i = (issued > STAGES ? issued - STAGES : 0); i < issued; ++i)
        if (!mbar_wait(smem_u32(&full[i % STAGES]), (i / STAGES) & 1)) atomicExch(abort_flag, 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ----------------------------------------------------- MMA issuer
      constexpr uint32_t idesc = idesc_bf16(BM, BM);
      for (int i = 0; i < nk; ++i) {
        const int s = i % STAGES, buf = i & 1;
        // accumulator buf is free once chunk i - 2 has been folded
        if (i >= 2 && !mbar_wait(smem_u32(&accfree[buf]), ((i >> 1) - 1) & 1)) {
          atomicExch(abort_flag, 1);
          break;
        }
        if (!mbar_wait(smem_u32(&full[s]), (i / STAGES) & 1)) {
          atomicExch(abort_flag, 1);
          break;
        }
        if (*reinterpret_cast<volatile int *>(abort_flag)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t base = smem_u32(gsm + (size_t)s * STAGE_BYTES);
        const uint64_t ah = sw128_desc(base), al = sw128_desc(base + TILE_BYTES);
        const uint64_t bh = sw128_desc(base + 2 * TILE_BYTES), bl = sw128_desc(base + 3 * TILE_BYTES);
        const uint32_t d = tmem + (uint32_t)(buf * BM);
#pragma unroll
        for (int kk = 0; kk < BK / 16; ++kk) {
          const uint64_t adv = (uint64_t)(kk * 32) >> 4;  // 16 bf16 = 32 bytes along K
          mma_bf16(d, ah + adv, bh + adv, idesc, kk > 0 ? 1u : 0u);
          mma_bf16(d, ah + adv, bl + adv, idesc, 1u);
          mma_bf16(d, al + adv, bh + adv, idesc, 1u);
          mma_bf16(d, al + adv, bl + adv, idesc, 1u);
        }
        mma_commit(smem_u32(&empty[s]));      // stage free once these MMAs finish
        mma_commit(smem_u32(&accfull[buf]));  // chunk i ready to fold
      }
      mma_commit(smem_u32(done));             // every MMA issued has completed
    }
  } else {
    // ----------------------------------------------- fold and epilogue
    // each thread keeps the running sums of its 64 columns in registers;
    // these are ordinary round-to-nearest FP32 additions, one per k-block
    const int ew = warp - 2;                      // 0..7
    const int quarter = warp & 3, half = ew >> 2;
    const int row = quarter * 32 + lane;
    const uint32_t lanebase = tmem + ((uint32_t)(quarter * 32) << 16);
    const uint32_t c0 = (uint32_t)(half * 64);
    float sum[64];
#pragma unroll
    for (int e = 0; e < 64; ++e) sum[e] = 0.f;
    bool ok = true;
    for (int i = 0; i < nk && ok; ++i) {
      const int buf = i & 1;
      if (!mbar_wait(smem_u32(&accfull[buf]), (i >> 1) & 1)) { ok = false; break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int cg = 0; cg < 4; ++cg) {
        uint32_t x[16];
        tmem_ld16u(lanebase + (uint32_t)(buf * BM) + c0 + (uint32_t)(cg * 16), x);
        tmem_wait_ld();
#pragma unroll
        for (int e = 0; e < 16; ++e) sum[cg * 16 + e] += __uint_as_float(x[e]);
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(smem_u32(&accfree[buf]));
    }
    if (!ok) atomicExch(abort_flag, 1);
    if (ok && *reinterpret_cast<volatile int *>(abort_flag) == 0) {
      double2 *dst = reinterpret_cast<double2 *>(
          g.part + ((size_t)t * g.splits + split) * BM * BM + (size_t)row * BM + c0);
#pragma unroll
      for (int q = 0; q < 32; ++q)
        dst[q] = make_double2((double)sum[2 * q], (double)sum[2 * q + 1]);
    }
  }
  __syncwarp();
  // every MMA this CTA issued has completed before the tensor memory goes
  const bool drained = mbar_wait(smem_u32(done), 0);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  __syncthreads();
  if (threadIdx.x == 0 && (!drained || *reinterpret_cast<volatile int *>(abort_flag)))
    atomicExch(g.err, (int)NQS_ERR_TIMEOUT);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS)
                 : "memory");
}

// Sum of the K-slices in FP64; T[i][j] and T[j][i] for i <= j.
__global__ void k_gram_reduce(const double *__restrict__ part, int R, int splits, int nT,
                              double *__restrict__ T) {
  const int t = blockIdx.y;
  int bi = 0, rem = t;
  while (rem >= nT - bi) { rem -= nT - bi; ++bi; }
  const int bj = bi + rem;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < BM * BM; e += gridDim.x * blockDim.x) {
    const int r = e / BM, c = e % BM;
    const int i = bi * BM + r, j = bj * BM + c;
    if (i >= R || j >= R || j < i) continue;
    double acc = 0.0;
    for (int s = 0; s < splits; ++s) acc += part[((size_t)t * splits + s) * BM * BM + e];
    T[(size_t)i * R + j] = acc;
    T[(size_t)j * R + i] = acc;
  }
}

// hi = bf16(A), lo = bf16(A - hi); columns np..Kpad-1 are zero.
__global__ void k_split_bf16(const float *__restrict__ A, int64_t R, int64_t np, int64_t Kpad,
                             __nv_bfloat16 *hi, __nv_bfloat16 *lo) {
  const int64_t tot = R * Kpad;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / Kpad, k = e - r * Kpad;
    const float v = k < np ? A[r * np + k] : 0.f;
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    hi[e] = h;
    lo[e] = __float2bfloat16_rn(v - __bfloat162float(h));
  }
}

// Centring and split in one pass (Algorithm 1, log-derivative step): v = (O - mean)/sqrt(Ns)
// with the difference O - mean formed from the column mean as an FP32 pair
// (hi, lo) by an error-free TwoSum, i.e. the exact difference rounded to FP32
// within one unit in the last place, without the FP64 pipe; then
// hi = bf16(v), lo = bf16(v - hi) (v - hi is exact in FP32); columns up to
// Kpad are zero.  Grid (column chunks, rows); each thread owns 8 consecutive
// columns of one row and writes them as one 16-byte store per plane.
constexpr int CS_THREADS = 256, CS_COLS = 8;

__device__ __forceinline__ uint32_t bf16x2_rn(float x0, float x1) {
  uint32_t u;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(u) : "f"(x1), "f"(x0));
  return u;
}

__global__ void __launch_bounds__(CS_THREADS) k_center_split(
    const float *__restrict__ O, int64_t ns, int64_t np, int64_t Kpad,
    const float2 *__restrict__ mean, float isq, __nv_bfloat16 *hi, __nv_bfloat16 *lo) {
  const int64_t r = blockIdx.y;
  const int64_t k0 = ((int64_t)blockIdx.x * CS_THREADS + threadIdx.x) * CS_COLS;
  if (k0 >= Kpad) return;
  const float *orow = O + r * np;
  const float2 *mrow = mean + (r / ns) * np;
  float v[CS_COLS];
#pragma unroll
  for (int j = 0; j < CS_COLS; ++j) {
    const int64_t k = k0 + j;
    float d = 0.f;
    if (k < np) {
      // o - (m_hi + m_lo): TwoSum of o and -m_hi (exact error e), then the
      // low-order terms: the FP32 rounding of the exact difference to within
      // one unit in the last place, on the FP32 pipe
      const float o = orow[k];
      const float2 m = mrow[k];
      const float s = o - m.x, bb = s - o;
      const float e = (o - (s - bb)) + (-m.x - bb);
      d = s + (e - m.y);
    }
    v[j] = d * isq;
  }
  uint32_t hp[4], lp[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    hp[q] = bf16x2_rn(v[2 * q], v[2 * q + 1]);
    const float h0 = __uint_as_float(hp[q] << 16), h1 = __uint_as_float(hp[q] & 0xffff0000u);
    lp[q] = bf16x2_rn(v[2 * q] - h0, v[2 * q + 1] - h1);
  }
  *reinterpret_cast<uint4 *>(hi + r * Kpad + k0) = make_uint4(hp[0], hp[1], hp[2], hp[3]);
  *reinterpret_cast<uint4 *>(lo + r * Kpad + k0) = make_uint4(lp[0], lp[1], lp[2], lp[3]);
}

// Partial sums of O'x from the split planes: part[c][p] = sum over the rows r
// of chunk c of (hi + lo)[r][p] x[r].  hi + lo is exact in FP32; the products
// are accumulated in FP32 within a chunk of rows_per rows (x rounded to FP32)
// and the chunks are summed in FP64 by the caller.  Each thread owns 2
// adjacent columns (one 4-byte load per plane and row).
__global__ void __launch_bounds__(256) k_gemv_split_part(
    const __nv_bfloat16 *__restrict__ hi, const __nv_bfloat16 *__restrict__ lo, int64_t R,
    int64_t np, int64_t Kpad, const double *__restrict__ x, int rows_per, double *part) {
  const int64_t p = 2 * (blockIdx.x * (int64_t)blockDim.x + threadIdx.x);
  if (p >= np) return;
  const int64_t r0 = (int64_t)blockIdx.y * rows_per;
  const int64_t r1 = min64(R, r0 + rows_per);
  float a0 = 0.f, a1 = 0.f;
  for (int64_t r = r0; r < r1; ++r) {
    const uint32_t h = *reinterpret_cast<const uint32_t *>(hi + r * Kpad + p);
    const uint32_t l = *reinterpret_cast<const uint32_t *>(lo + r * Kpad + p);
    const float xr = (float)x[r];
    a0 = fmaf(__uint_as_float(h << 16) + __uint_as_float(l << 16), xr, a0);
    a1 = fmaf(__uint_as_float(h & 0xffff0000u) + __uint_as_float(l & 0xffff0000u), xr, a1);
  }
  double *out = part + (int64_t)blockIdx.y * np + p;
  out[0] = a0;
  if (p + 1 < np) out[1] = a1;
}

// T = (hi + lo)(hi + lo)^T in FP64 from the split planes, run only when
// *gate != 0 (the FP64 Cholesky of the tensor-core T found a non-positive
// pivot).  hi + lo is exact in FP64, so this T is the Gram matrix of the
// stored vectors up to FP64 rounding, positive semi-definite to that
// accuracy.  64x64 output tiles of the upper triangle over a persistent
// grid, K in chunks of 32 through shared memory, 4x4 outputs per thread.
__global__ void __launch_bounds__(256) k_gram_split_f64(
    const __nv_bfloat16 *__restrict__ hi, const __nv_bfloat16 *__restrict__ lo, int64_t R,
    int64_t Kpad, const int32_t *gate, double *__restrict__ T) {
  if (*gate == 0) return;
  __shared__ double sa[32][65], sb[32][65];
  const int nt = (int)((R + 63) / 64);
  const int ntiles = nt * (nt + 1) / 2;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    int bi = 0, rem = t;
    while (rem >= nt - bi) { rem -= nt - bi; ++bi; }
    const int bj = bi + rem;
    const int64_t i0 = (int64_t)bi * 64, j0 = (int64_t)bj * 64;
    double acc[4][4] = {};
    for (int64_t k0 = 0; k0 < Kpad; k0 += 32) {
      __syncthreads();
      for (int e = threadIdx.x; e < 32 * 64; e += 256) {
        const int kk = e % 32, r = e / 32;
        const int64_t ia = i0 + r, ib = j0 + r, k = k0 + kk;
        sa[kk][r] = ia < R ? (double)__bfloat162float(hi[ia * Kpad + k]) +
                                 (double)__bfloat162float(lo[ia * Kpad + k]) : 0.0;
        sb[kk][r] = ib < R ? (double)__bfloat162float(hi[ib * Kpad + k]) +
                                 (double)__bfloat162float(lo[ib * Kpad + k]) : 0.0;
      }
      __syncthreads();
#pragma unroll 4
      for (int kk = 0; kk < 32; ++kk) {
        double av[4], bv[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) { av[q] = sa[kk][ty + 16 * q]; bv[q] = sb[kk][tx + 16 * q]; }
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[p][q] = fma(av[p], bv[q], acc[p][q]);
      }
    }
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int64_t i = i0 + ty + 16 * p, j = j0 + tx + 16 * q;
        if (i < R && j < R && j >= i) {
          T[i * R + j] = acc[p][q];
          T[j * R + i] = acc[p][q];
        }
      }
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

bool make_map(CUtensorMap *m, const void *base, int64_t R, int64_t Kpad) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)Kpad, (cuuint64_t)R};
  cuuint64_t strides[1] = {(cuuint64_t)Kpad * 2};
  cuuint32_t box[2] = {BK, BM};
  cuuint32_t es[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box,
            es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int64_t kpad_of(int64_t np) { return (np + BK - 1) / BK * BK; }

void plan(int64_t R, int64_t np, int sms, int *nT, int *tiles, int *kblocks, int *splits) {
  *nT = (int)((R + BM - 1) / BM);
  *tiles = *nT * (*nT + 1) / 2;
  *kblocks = (int)(kpad_of(np) / BK);
  int s = (2 * sms + *tiles - 1) / *tiles;  // about two CTAs per SM
  if (s > *kblocks / 4) s = *kblocks / 4;
  if (s < 1) s = 1;
  *splits = s;
}

int g_sms = 0;
int sm_count() {
  if (!g_sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_sms <= 0) g_sms = 148;
  }
  return g_sms;
}

}  // namespace

bool gram_tc_available() {
  static int avail = -1;
  if (avail < 0) {
    int dev = 0, major = 0, minor = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    avail = (major == 10 && minor == 3 && encode_fn() != nullptr) ? 1 : 0;
  }
  return avail == 1;
}

int gram_tc_launches() { return 3; }

size_t gram_tc_split_bytes(int64_t R, int64_t np) {
  // any plan with R' <= R, np' <= np has tiles' * splits' <= tiles + 2 * SMs
  int nT, tiles, kb, splits;
  plan(R, np, sm_count(), &nT, &tiles, &kb, &splits);
  const size_t hl = 2 * (size_t)R * kpad_of(np) * 2;
  const size_t part = ((size_t)tiles + 2 * (size_t)sm_count()) * BM * BM * 8;
  return ((hl + 255) & ~size_t(255)) + part + 256;
}

int64_t gram_tc_kpad(int64_t np) { return kpad_of(np); }

int gram_tc_max_splits(int64_t R, int64_t np) {
  int nT, tiles, kb, splits;
  plan(R, np, sm_count(), &nT, &tiles, &kb, &splits);
  const int cap = (tiles + 2 * sm_count()) / tiles;  // partials the scratch holds
  return std::max(1, std::min(cap, kb));
}

int gram_tc_default_splits(int64_t R, int64_t np) {
  int nT, tiles, kb, splits;
  plan(R, np, sm_count(), &nT, &tiles, &kb, &splits);
  return splits;
}

cudaError_t gram_tc_from_split(const void *hi, const void *lo, int64_t R, int64_t np, double *T,
                               void *scratch_part, int *err, cudaStream_t st, int want_splits = 0) {
  int nT, tiles, kb, splits;
  plan(R, np, sm_count(), &nT, &tiles, &kb, &splits);
  if (want_splits > 0) splits = std::min(want_splits, gram_tc_max_splits(R, np));
  const int64_t Kpad = kpad_of(np);
  CUtensorMap mh, ml;
  if (!make_map(&mh, hi, R, Kpad) || !make_map(&ml, lo, R, Kpad)) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k_gram_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)SMEM_BYTES);
  if (e != cudaSuccess) return e;
  GramArgs g{(int)R, kb, splits, nT, static_cast<double *>(scratch_part), err};
  k_gram_tc<<<tiles * splits, THREADS, SMEM_BYTES, st>>>(mh, ml, g);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_gram_reduce<<<dim3(16, tiles), 256, 0, st>>>(static_cast<const double *>(scratch_part), (int)R,
                                                 splits, nT, T);
  return cudaGetLastError();
}

cudaError_t center_split(const float *O, int64_t ns, int64_t np, int64_t R, const float2 *mean,
                         void *scratch, cudaStream_t st) {
  const int64_t Kpad = kpad_of(np);
  __nv_bfloat16 *hi = static_cast<__nv_bfloat16 *>(scratch);
  __nv_bfloat16 *lo = hi + R * Kpad;
  dim3 g((unsigned)((Kpad + CS_THREADS * CS_COLS - 1) / (CS_THREADS * CS_COLS)), (unsigned)R);
  k_center_split<<<g, CS_THREADS, 0, st>>>(O, ns, np, Kpad, mean, (float)(1.0 / std::sqrt((double)ns)),
                                            hi, lo);
  return cudaGetLastError();
}

cudaError_t gemv_split(const void *scratch, int64_t R, int64_t np, const double *x, int rows_per,
                       double *part, cudaStream_t st) {
  const int64_t Kpad = kpad_of(np);
  const __nv_bfloat16 *hi = static_cast<const __nv_bfloat16 *>(scratch);
  const __nv_bfloat16 *lo = hi + R * Kpad;
  dim3 g((unsigned)((np + 511) / 512), (unsigned)((R + rows_per - 1) / rows_per));
  k_gemv_split_part<<<g, 256, 0, st>>>(hi, lo, R, np, Kpad, x, rows_per, part);
  return cudaGetLastError();
}

cudaError_t gram_from_center_split(const void *scratch, int64_t R, int64_t np, double *T, int *err,
                                   cudaStream_t st, int splits) {
  const int64_t Kpad = kpad_of(np);
  const __nv_bfloat16 *hi = static_cast<const __nv_bfloat16 *>(scratch);
  const __nv_bfloat16 *lo = hi + R * Kpad;
  const size_t hl = 2 * (size_t)R * Kpad * 2;
  void *part = static_cast<char *>(const_cast<void *>(scratch)) + ((hl + 255) & ~size_t(255));
  return gram_tc_from_split(hi, lo, R, np, T, part, err, st, splits);
}

cudaError_t gram_split_f64(const void *scratch, int64_t R, int64_t np, double *T,
                           const int32_t *gate, cudaStream_t st) {
  const int64_t Kpad = kpad_of(np);
  const __nv_bfloat16 *hi = static_cast<const __nv_bfloat16 *>(scratch);
  const __nv_bfloat16 *lo = hi + R * Kpad;
  const int64_t nt = (R + 63) / 64;
  const int grid = (int)std::min<int64_t>(nt * (nt + 1) / 2, 4 * (int64_t)sm_count());
  k_gram_split_f64<<<grid, 256, 0, st>>>(hi, lo, R, Kpad, gate, T);
  return cudaGetLastError();
}

cudaError_t gram_tc_bf16x3(const float *A, int64_t R, int64_t np, double *T, void *scratch,
                           int *err, cudaStream_t st) {
  const int64_t Kpad = kpad_of(np);
  __nv_bfloat16 *hi = static_cast<__nv_bfloat16 *>(scratch);
  __nv_bfloat16 *lo = hi + R * Kpad;
  const size_t hl = 2 * (size_t)R * Kpad * 2;
  void *part = static_cast<char *>(scratch) + ((hl + 255) & ~size_t(255));
  const int64_t tot = R * Kpad;
  const int blocks = (int)min64((tot + 255) / 256, 148 * 32);
  k_split_bf16<<<blocks, 256, 0, st>>>(A, R, np, Kpad, hi, lo);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return gram_tc_from_split(hi, lo, R, np, T, part, err, st);
}

}  // namespace nqs
