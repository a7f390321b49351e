// jac_tc.cu -- the rows of O (Alg. 1, log-derivative step, App. A) on the tensor cores.
//
// For one row (sample, adjoint seed) every entry of O is a sum over the
// sites k of an adjoint component times a state component:
//   W_u[a][b] = sum_k dau_k[a] h_{k-1}[b],  b_u[a] = sum_k dau_k[a],
//   W_u x-column d: sum_k dau_k[a] [sigma_{k-1} = d]   (likewise W_r, dar),
//   W_h[a][b] = sum_k dg_k[a] h_{k-1}[b],   b_h[a] = sum_k dg_k[a],
//   W_in[a][d] = sum_k dac_k[a] [sigma_{k-1} = d], b_in[a] = sum_k dac_k[a],
//   U[o][b] = sum_k dz_k[o] h_k[b],         c[o] = sum_k dz_k[o].
// With the site index shifted by one for the heads (k' = k + 1) all of these
// are one product D = A B^T over k' = 0..N:
//   A rows (three M = 128 tiles): [dau | dar], [dg | dac], dz_{k'-1} (4 rows);
//   B rows (N = dh + 3, padded to 16): h_{k'-1}, ones, the one-hot of
//   sigma_{k'-1} (0 outside the chain),
// which the kernel forms per row from the adjoint records of the reverse
// sweep and the cached states: each FP32 value is split into BF16 hi + lo
// (the ones and one-hots are exact), staged in the non-swizzled K-major
// layout 16 sites at a time (two buffers), and accumulated in tensor memory
// as hi.hi + hi.lo + lo.hi (FP32), the same three products as the Gram.  The
// result goes back through shared memory so that the row of O is written
// coalesced.  Two CTAs per SM walk the rows.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "nqs.h"
#include "jac_tc.h"
#include "tc_common.cuh"

namespace nqs {
namespace {

constexpr int JT_THREADS = 256;
constexpr int JT_TILES = 3;                   // A tiles of 128 rows
constexpr int JT_KC = 16;                     // sites per staged chunk
constexpr int JT_KS = JT_KC / 16;             // K = 16 steps per chunk
constexpr int JT_ASUB = (128 / 8) * 256;      // one K = 16 block of a 128-row tile (4 KB)
constexpr int JT_TMEM_COLS = 256;

template <int DH> struct JtShape {
  static constexpr int NB = ((DH + 3) + 15) / 16 * 16;  // B rows: h, ones, one-hot (2)
  static constexpr int BSUB = (NB / 8) * 256;           // one K = 16 block of B
  static constexpr int A_BYTES = JT_KS * 2 * JT_TILES * JT_ASUB;
  static constexpr int STAGE = (A_BYTES + JT_KS * 2 * BSUB + 1023) / 1024 * 1024;
  static constexpr int TRS = NB + 1;                    // transpose stride (floats)
  static constexpr size_t SMEM = 1024 + 2 * (size_t)STAGE + sizeof(float) * 128 * TRS + 64;
};

// Stage layout: A block (ks, plane, tile) at ((ks * 2 + plane) * 3 + tile)
// * JT_ASUB, then B block (ks, plane) at A_BYTES + (ks * 2 + plane) * BSUB.
template <int DH>
__device__ __forceinline__ void put_a(unsigned char *stage, int tile, int r, int kk, float v) {
  const int ks = kk >> 4, k = kk & 15;
  const __nv_bfloat16 h = __float2bfloat16_rn(v);
  const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
  const uint32_t o = kmaj_off(r, k);
  *reinterpret_cast<__nv_bfloat16 *>(stage + ((ks * 2 + 0) * JT_TILES + tile) * JT_ASUB + o) = h;
  *reinterpret_cast<__nv_bfloat16 *>(stage + ((ks * 2 + 1) * JT_TILES + tile) * JT_ASUB + o) = l;
}

template <int DH>
__device__ __forceinline__ void put_b(unsigned char *stage, int n, int kk, float v) {
  using S = JtShape<DH>;
  const int ks = kk >> 4, k = kk & 15;
  const __nv_bfloat16 h = __float2bfloat16_rn(v);
  const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
  const uint32_t o = kmaj_off(n, k);
  *reinterpret_cast<__nv_bfloat16 *>(stage + S::A_BYTES + (ks * 2 + 0) * S::BSUB + o) = h;
  *reinterpret_cast<__nv_bfloat16 *>(stage + S::A_BYTES + (ks * 2 + 1) * S::BSUB + o) = l;
}

// One chunk's values in registers: chunk c (sites k' = 16 c .. 16 c + 15) of
// row `row` (sample s).  The loads of the next chunk are issued right after
// the current one is stored, so they overlap the barrier, the products and,
// at the end of a row, the epilogue.
// Each thread owns pairs of consecutive sites (k', k' + 1) of one column m
// (or unit n), so that the two BF16 values of a plane go out as one 4-byte
// store.
template <int DH> struct ChunkRegs {
  static constexpr int AW = 4 * DH;                        // dau, dar, dg, dac
  static constexpr int NA = JT_KC * AW / JT_THREADS / 2;   // site pairs of gate adjoints
  static constexpr int NH = JT_KC * DH / JT_THREADS / 2;   // site pairs of states
  float va[NA][2], vh[NH][2], vz;
  int sp;
};

// hi, lo planes of the pair (v0, v1) at sites kk, kk + 1 (kk even) of a row
__device__ __forceinline__ void put_pair(unsigned char *hi, unsigned char *lo, int r, int kk,
                                         float v0, float v1) {
  const __nv_bfloat16 h0 = __float2bfloat16_rn(v0), h1 = __float2bfloat16_rn(v1);
  const __nv_bfloat16 l0 = __float2bfloat16_rn(v0 - __bfloat162float(h0));
  const __nv_bfloat16 l1 = __float2bfloat16_rn(v1 - __bfloat162float(h1));
  const uint32_t o = kmaj_off(r, kk & 15);
  *reinterpret_cast<__nv_bfloat162 *>(hi + o) = __halves2bfloat162(h0, h1);
  *reinterpret_cast<__nv_bfloat162 *>(lo + o) = __halves2bfloat162(l0, l1);
}

template <int DH>
__device__ __forceinline__ void fetch_chunk(const JacTcArgs &a, ChunkRegs<DH> &r, int64_t row,
                                            int64_t s, int c, int tid) {
  using CR = ChunkRegs<DH>;
  const int N = a.N;
  const int k0 = c * JT_KC;
  const float *arow = a.adj + row * (int64_t)N * a.adjw;
  const float *hrow = a.hcache + s * (int64_t)N * DH;
#pragma unroll
  for (int q = 0; q < CR::NA; ++q) {
    const int e = tid + q * JT_THREADS;
    const int kp = e / CR::AW, m = e - kp * CR::AW, k = k0 + 2 * kp;
    r.va[q][0] = k < N ? __ldcg(arow + (int64_t)k * a.adjw + m) : 0.f;
    r.va[q][1] = k + 1 < N ? __ldcg(arow + (int64_t)(k + 1) * a.adjw + m) : 0.f;
  }
  r.vz = 0.f;
  if (tid < 4 * JT_KC) {  // dz of site k' - 1: the heads' shifted index
    const int kk = tid >> 2, o = tid & 3, k = k0 + kk - 1;
    r.vz = (k >= 0 && k < N) ? __ldcg(arow + (int64_t)k * a.adjw + CR::AW + o) : 0.f;
  }
#pragma unroll
  for (int q = 0; q < CR::NH; ++q) {
    const int e = tid + q * JT_THREADS;
    const int kp = e / DH, n = e - kp * DH, k = k0 + 2 * kp - 1;
    r.vh[q][0] = (k >= 0 && k < N) ? __ldcg(hrow + (int64_t)k * DH + n) : 0.f;
    r.vh[q][1] = (k + 1 >= 0 && k + 1 < N) ? __ldcg(hrow + (int64_t)(k + 1) * DH + n) : 0.f;
  }
  r.sp = -1;
  if (tid < JT_KC) {
    const int k = k0 + tid - 1;
    r.sp = (k >= 0 && k < N) ? (int)__ldcg(a.spins + s * (int64_t)N + k) : -1;
  }
}

template <int DH>
__device__ __forceinline__ void store_chunk(const ChunkRegs<DH> &r, unsigned char *stage, int N,
                                            int c, int tid) {
  using CR = ChunkRegs<DH>;
  const int k0 = c * JT_KC;
#pragma unroll
  for (int q = 0; q < CR::NA; ++q) {
    const int e = tid + q * JT_THREADS;
    const int kp = e / CR::AW, m = e - kp * CR::AW, kk = 2 * kp;
    const int t = m / (2 * DH), ks = kk >> 4;
    put_pair(stage + ((ks * 2 + 0) * JT_TILES + t) * JT_ASUB,
             stage + ((ks * 2 + 1) * JT_TILES + t) * JT_ASUB, m % (2 * DH), kk, r.va[q][0],
             r.va[q][1]);
  }
  if (tid < 4 * JT_KC) put_a<DH>(stage, 2, tid & 3, tid >> 2, r.vz);
#pragma unroll
  for (int q = 0; q < CR::NH; ++q) {
    const int e = tid + q * JT_THREADS;
    const int kp = e / DH, n = e - kp * DH, kk = 2 * kp, ks = kk >> 4;
    using S = JtShape<DH>;
    put_pair(stage + S::A_BYTES + (ks * 2 + 0) * S::BSUB, stage + S::A_BYTES + (ks * 2 + 1) * S::BSUB,
             n, kk, r.vh[q][0], r.vh[q][1]);
  }
  if (tid < JT_KC) {
    put_b<DH>(stage, DH, tid, k0 + tid <= N ? 1.f : 0.f);  // ones over k' = 0..N
    put_b<DH>(stage, DH + 1, tid, r.sp == 0 ? 1.f : 0.f);
    put_b<DH>(stage, DH + 2, tid, r.sp == 1 ? 1.f : 0.f);
  }
}

// Row m of tile t (in the transpose buffer) into its entries of O.
template <int DH>
__device__ __forceinline__ void write_tile(const JacTcArgs &a, const float *tr, int64_t row, int t,
                                           int warp, int lane) {
  using S = JtShape<DH>;
  float *orow = a.O + row * a.np;
  const int w = DH + 2;  // row length of W_u and W_r: h part, then the two x-columns
  if (t < 2) {
    for (int m = warp; m < 2 * DH; m += JT_THREADS / 32) {
      const float *v = tr + m * S::TRS;
      const int blk = m / DH, q = m - blk * DH;
      if (t == 0) {  // dau -> W_u, b_u; dar -> W_r, b_r
        const int64_t base = (blk ? a.Wr : a.Wu) + (int64_t)q * w;
        for (int b = lane; b < DH; b += 32) orow[base + b] = v[b];
        if (lane < 2) orow[base + DH + lane] = v[DH + 1 + lane];
        if (lane == 0) orow[(blk ? a.br : a.bu) + q] = v[DH];
      } else if (blk == 0) {  // dg -> W_h, b_h
        for (int b = lane; b < DH; b += 32) orow[a.Wh + (int64_t)q * DH + b] = v[b];
        if (lane == 0) orow[a.bh + q] = v[DH];
      } else {  // dac -> W_in, b_in
        if (lane < 2) orow[a.Win + (int64_t)q * 2 + lane] = v[DH + 1 + lane];
        if (lane == 0) orow[a.bin + q] = v[DH];
      }
    }
  } else {
    for (int o = warp; o < 4; o += JT_THREADS / 32) {
      if (o >= 2 && !a.cplx) continue;
      const float *v = tr + o * S::TRS;
      const int64_t base = o < 2 ? a.Uo + (int64_t)o * DH : a.Up + (int64_t)(o - 2) * DH;
      for (int b = lane; b < DH; b += 32) orow[base + b] = v[b];
      if (lane == 0) orow[o < 2 ? a.co + o : a.cp + (o - 2)] = v[DH];
    }
  }
}

template <int DH>
__global__ void __launch_bounds__(JT_THREADS, 2) k_jac_tc(const JacTcArgs a) {
  using S = JtShape<DH>;
  extern __shared__ __align__(1024) unsigned char jraw[];
  unsigned char *sm = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(jraw) + 1023) & ~uintptr_t(1023));
  unsigned char *stg[2] = {sm, sm + S::STAGE};
  float *tr = reinterpret_cast<float *>(sm + 2 * S::STAGE);           // [128][TRS]
  uint64_t *bars = reinterpret_cast<uint64_t *>(tr + 128 * S::TRS);   // MMA done, per stage
  uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 2);
  __shared__ int flag_s;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // rows that are never written (padding of the tiles) stay zero
  for (int e = tid; e < 2 * S::STAGE / 16; e += JT_THREADS)
    reinterpret_cast<uint4 *>(sm)[e] = make_uint4(0u, 0u, 0u, 0u);
  if (tid == 0) {
    mbar_init(smem_u32(&bars[0]), 1);
    mbar_init(smem_u32(&bars[1]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tslot)),
                 "r"(JT_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  constexpr uint32_t idesc = idesc_bf16(128, S::NB);
  const int NC = (a.N + 1 + JT_KC - 1) / JT_KC;  // chunks of k' = 0..N
  uint32_t ph[2] = {0u, 0u};
  int pending[2] = {0, 0};  // commits on each stage's barrier not yet waited for
  bool ok = true;

  // wait (thread 0, bounded) for the commit pending on stage st; uniform result
  auto drain = [&](int st) -> bool {
    if (tid == 0) flag_s = mbar_wait(smem_u32(&bars[st]), ph[st]) ? 0 : 1;
    ph[st] ^= 1u;
    pending[st] = 0;
    __syncthreads();
    return flag_s == 0;
  };

  ChunkRegs<DH> cr;
  if ((int64_t)blockIdx.x < a.nrows) fetch_chunk<DH>(a, cr, blockIdx.x, blockIdx.x % a.ns, 0, tid);
  for (int64_t row = blockIdx.x; row < a.nrows && ok; row += gridDim.x) {
    const int64_t s = row % a.ns;
    for (int c = 0; c < NC; ++c) {
      const int st = c & 1;
      if (pending[st] && !drain(st)) { ok = false; break; }
      store_chunk<DH>(cr, stg[st], a.N, c, tid);
      // the next chunk's loads, or the next row's first, fly during the rest
      if (c + 1 < NC) {
        fetch_chunk<DH>(a, cr, row, s, c + 1, tid);
      } else if (row + gridDim.x < a.nrows) {
        const int64_t nrow = row + gridDim.x;
        fetch_chunk<DH>(a, cr, nrow, nrow % a.ns, 0, tid);
      }
      fence_async_smem();
      __syncthreads();
      if (tid == 0) {
        tc_fence_after();
        const uint32_t base = smem_u32(stg[st]);
#pragma unroll
        for (int ks = 0; ks < JT_KS; ++ks) {
          const uint64_t bh = kmaj_desc(base + S::A_BYTES + (ks * 2 + 0) * S::BSUB);
          const uint64_t bl = kmaj_desc(base + S::A_BYTES + (ks * 2 + 1) * S::BSUB);
#pragma unroll
          for (int t = 0; t < JT_TILES; ++t) {
            const uint64_t ah = kmaj_desc(base + ((ks * 2 + 0) * JT_TILES + t) * JT_ASUB);
            const uint64_t al = kmaj_desc(base + ((ks * 2 + 1) * JT_TILES + t) * JT_ASUB);
            const uint32_t d = tmem + (uint32_t)(t * S::NB);
            mma_bf16(d, ah, bh, idesc, (c == 0 && ks == 0) ? 0u : 1u);
            mma_bf16(d, ah, bl, idesc, 1u);
            mma_bf16(d, al, bh, idesc, 1u);
          }
        }
        mma_commit(smem_u32(&bars[st]));
      }
      pending[st] = 1;
    }
    if (!ok) break;
    // the row's products are complete once both stages' last commits are
    if ((pending[0] && !drain(0)) || (pending[1] && !drain(1))) { ok = false; break; }
    tc_fence_after();
    for (int t = 0; t < JT_TILES; ++t) {
      if (warp < 4) {  // warp w reads tensor-memory lanes 32 w .. 32 w + 31
        const int m = warp * 32 + lane;
#pragma unroll
        for (int cc = 0; cc < S::NB; cc += 16) {
          float v[16];
          tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(t * S::NB + cc), v);
          tmem_wait_ld();
#pragma unroll
          for (int j = 0; j < 16; ++j) tr[m * S::TRS + cc + j] = v[j];
        }
      }
      __syncthreads();
      write_tile<DH>(a, tr, row, t, warp, lane);
      __syncthreads();
    }
    tc_fence_before();  // the next row's first products overwrite the accumulators
  }
  if (!ok) {
    if (tid == 0) atomicCAS(a.err, 0, (int)NQS_ERR_TIMEOUT);
    // let products still in flight finish (bounded) before the memory goes
    if (tid == 0) {
      if (pending[0]) mbar_wait(smem_u32(&bars[0]), ph[0]);
      if (pending[1]) mbar_wait(smem_u32(&bars[1]), ph[1]);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(JT_TMEM_COLS)
                 : "memory");
}

}  // namespace

bool jac_tc_supported(int dim, int dh) { return dim == 1 && (dh == 64 || dh == 32); }

cudaError_t jac_tc_run(const JacTcArgs &args, int sm_count, cudaStream_t st) {
  if (args.nrows <= 0) return cudaSuccess;
  if (args.dh != 64 && args.dh != 32) return cudaErrorInvalidValue;
  const bool d64 = args.dh == 64;
  const void *kern = d64 ? (const void *)k_jac_tc<64> : (const void *)k_jac_tc<32>;
  const size_t smem = d64 ? JtShape<64>::SMEM : JtShape<32>::SMEM;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // two CTAs per SM (about 104 KB of shared memory and 256 tensor-memory
  // columns each): one row's loads overlap the other's products and epilogue
  const int64_t g2 = 2 * (int64_t)sm_count;
  const int grid = (int)(args.nrows < g2 ? args.nrows : g2);
  if (d64)
    k_jac_tc<64><<<grid, JT_THREADS, smem, st>>>(args);
  else
    k_jac_tc<32><<<grid, JT_THREADS, smem, st>>>(args);
  return cudaGetLastError();
}

}  // namespace nqs
