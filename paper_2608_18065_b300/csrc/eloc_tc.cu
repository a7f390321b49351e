// eloc_tc.cu -- log Psi of every connected configuration (Sec. II.C) for 1D
// chains with hidden size 64, mixed precision, on the tensor cores (sm_103a).
//
// A connected configuration sigma' differs from its sample sigma from site j
// on, so its suffix k = j..N-1 is recomputed from the cached state h_{j-1}.
// Rows of one operator share j; 128 of them form a tile.  Per site the gate
// pre-activations of the tile are one product [128 x 64] x [64 x 192] (App. A):
// the FP32 states are split h = hi + lo into BF16 planes in shared memory and
// tcgen05.mma accumulates hi W_hi + hi W_lo + lo W_hi in FP32 in tensor memory
// (the weights are split once per CTA).  Each epilogue thread owns one row:
// it reads its 192 accumulator columns with tcgen05.ld, applies the GRU cell
// and the heads in FP32 registers, accumulates the change of log Psi in FP64
// and writes the next BF16 planes.  Two tiles per CTA (two epilogue
// warpgroups, two accumulators) alternate so that the tensor core works on
// one tile while the other runs its epilogue; one extra warp issues the MMAs.
// Every mbarrier wait is bounded; on expiry the CTA flags NQS_ERR_TIMEOUT,
// drains its MMAs, frees its tensor memory and exits.
#include <cuda_bf16.h>

#include "common.cuh"
#include "eloc_tc.h"
#include "tc_common.cuh"

namespace nqs {
namespace {

constexpr int DH = 64;
constexpr int NG = 3 * DH;                   // gate columns, n = 3a + g
constexpr int TR = 128;                      // rows per tile (MMA M)
constexpr int SLOTS = 2;
constexpr int EPI = TR * SLOTS;              // epilogue threads
constexpr int THREADS = EPI + 32;            // + MMA warp
constexpr int TMEM_COLS = 512;
constexpr int ACC_STRIDE = 256;              // tensor-memory columns per slot
constexpr int ATILE = TR * DH * 2;           // one BF16 plane of a row tile (16 KB)
constexpr int BTILE = NG * DH * 2;           // one BF16 plane of the weights (24 KB)
constexpr size_t SMEM_BYTES = 1024 + 2 * (size_t)BTILE + 2 * SLOTS * (size_t)ATILE +
                              sizeof(float) * (DH * 4 + 2 * NG + 4 * DH + 8) + 128;

// Two floats rounded to BF16 and packed, x0 in the low half (lower address).
__device__ __forceinline__ uint32_t pack_bf16x2(float x0, float x1) {
  uint32_t u;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(u) : "f"(x1), "f"(x0));
  return u;
}

__device__ __forceinline__ float sigm_f(float x) { return __fdividef(1.0f, 1.0f + __expf(-x)); }
__device__ __forceinline__ float tanh_f(float x) { return 2.0f * sigm_f(2.0f * x) - 1.0f; }

__global__ void __launch_bounds__(THREADS, 1) k_eloc_tc(const ElocTcArgs a) {
  extern __shared__ __align__(1024) unsigned char eraw[];
  unsigned char *sm = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(eraw) + 1023) & ~uintptr_t(1023));
  unsigned char *Bhi = sm, *Blo = sm + BTILE;
  unsigned char *Abase = sm + 2 * BTILE;     // A(slot, plane) = Abase + (2 slot + plane) ATILE
  float *sbias = reinterpret_cast<float *>(Abase + 2 * SLOTS * ATILE);  // [DH][4]
  float *sxw = sbias + DH * 4;               // [2][NG]
  float *shead = sxw + 2 * NG;               // [4][DH]
  float *shc = shead + 4 * DH;               // [4]
  uint64_t *bars = reinterpret_cast<uint64_t *>(shc + 8);  // hready[2] accfull[2] drain
  int *cmd = reinterpret_cast<int *>(bars + 5);            // [2]
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(cmd + 2);
  int *abort_flag = reinterpret_cast<int *>(tmem_slot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int N = a.N;

  // weights B[n][k] = W_g[a][k] (n = 3a+g) split into BF16 planes, 128B swizzle
  for (int e = tid; e < NG * DH; e += THREADS) {
    const int n = e / DH, k = e % DH;
    const float w = a.pack[a.oWgT + k * NG + n];
    const __nv_bfloat16 h = __float2bfloat16_rn(w);
    *reinterpret_cast<__nv_bfloat16 *>(Bhi + sw128_off(n, k)) = h;
    *reinterpret_cast<__nv_bfloat16 *>(Blo + sw128_off(n, k)) =
        __float2bfloat16_rn(w - __bfloat162float(h));
  }
  for (int e = tid; e < DH * 4; e += THREADS) sbias[e] = a.pack[a.obias + e];
  for (int e = tid; e < 2 * NG; e += THREADS) sxw[e] = a.pack[a.oxw + e];
  for (int e = tid; e < 4 * DH; e += THREADS) shead[e] = a.pack[a.ohead + e];
  if (tid < 4) shc[tid] = a.pack[a.ohc + tid];
  if (tid == 0) {
    for (int t = 0; t < SLOTS; ++t) {
      mbar_init(smem_u32(&bars[t]), TR);       // hready[t]: all rows of the tile
      mbar_init(smem_u32(&bars[2 + t]), 1);    // accfull[t]: one commit
      cmd[t] = 1;
    }
    mbar_init(smem_u32(&bars[4]), 1);          // drain
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_async_smem();
  if (warp == SLOTS * 4) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == SLOTS * 4) {
    // ------------------------------------------------------- MMA issuer
    if (lane == 0) {
      int alive[SLOTS] = {1, 1};
      uint32_t ph[SLOTS] = {0, 0};
      constexpr uint32_t idesc = idesc_bf16(TR, NG);
      const uint64_t bh = sw128_desc(smem_u32(Bhi)), bl = sw128_desc(smem_u32(Blo));
      bool ok = true;
      while (ok && (alive[0] || alive[1])) {
        for (int t = 0; t < SLOTS && ok; ++t) {
          if (!alive[t]) continue;
          if (!mbar_wait(smem_u32(&bars[t]), ph[t])) { ok = false; break; }
          ph[t] ^= 1;
          if (*reinterpret_cast<volatile int *>(&cmd[t]) == 0) { alive[t] = 0; continue; }
          if (*reinterpret_cast<volatile int *>(abort_flag)) { ok = false; break; }
          tc_fence_after();
          const uint64_t ah = sw128_desc(smem_u32(Abase + (2 * t) * ATILE));
          const uint64_t al = sw128_desc(smem_u32(Abase + (2 * t + 1) * ATILE));
          const uint32_t d = tmem + (uint32_t)(t * ACC_STRIDE);
#pragma unroll
          for (int kk = 0; kk < DH / 16; ++kk) {
            const uint64_t adv = (uint64_t)(kk * 32) >> 4;
            mma_bf16(d, ah + adv, bh + adv, idesc, kk > 0 ? 1u : 0u);
            mma_bf16(d, ah + adv, bl + adv, idesc, 1u);
            mma_bf16(d, al + adv, bh + adv, idesc, 1u);
          }
          mma_commit(smem_u32(&bars[2 + t]));
        }
      }
      if (!ok) {
        atomicExch(abort_flag, 1);
        atomicExch(a.err, (int)NQS_ERR_TIMEOUT);
      }
      mma_commit(smem_u32(&bars[4]));   // all MMAs issued so far
      mbar_wait(smem_u32(&bars[4]), 0);
    }
  } else {
    // ---------------------------------------------------------- epilogue
    const int t = warp / 4;
    const int row = (warp % 4) * 32 + lane;
    unsigned char *Ahi = Abase + (2 * t) * ATILE, *Alo = Abase + (2 * t + 1) * ATILE;
    const uint32_t dcol = tmem + ((uint32_t)((warp % 4) * 32) << 16) + (uint32_t)(t * ACC_STRIDE);
    uint32_t acc_ph = 0;
    bool ok = true;
    for (int tile = blockIdx.x * SLOTS + t; tile < a.ntiles && ok; tile += gridDim.x * SLOTS) {
      const int op = tile / a.tiles_per_op;
      const int base = (tile - op * a.tiles_per_op) * TR;
      const int cnt = a.item_cnt[op];
      if (base >= cnt) continue;  // uniform over the warpgroup
      const int f1 = a.op_f[4 * op], f2 = a.op_f[4 * op + 1], j0 = a.op_f[4 * op + 2];
      const bool valid = base + row < cnt;
      const int64_t item = (int64_t)op * a.ns + base + row;
      const int s = valid ? a.item_s[item] : 0;
      const uint8_t *sp = a.spins + (int64_t)s * N;
      float h[DH];
#pragma unroll
      for (int q = 0; q < DH; ++q)
        h[q] = (valid && j0 > 0) ? a.hcache[((int64_t)s * N + j0 - 1) * DH + q] : 0.f;
      int n_up = 0, n_dn = 0;
      if (a.zmask)
        for (int k = 0; k < j0; ++k) { if (sp[k] == 0) ++n_up; else ++n_dn; }
      double dre = 0.0, dimg = 0.0;
      for (int k = j0; k < N; ++k) {
        // BF16 planes of h_{k-1} for this row, then hand the tile to the MMA warp
#pragma unroll
        for (int c = 0; c < DH / 8; ++c) {
          uint32_t hp[4], lp[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float x0 = h[8 * c + 2 * q], x1 = h[8 * c + 2 * q + 1];
            hp[q] = pack_bf16x2(x0, x1);
            const float h0 = __uint_as_float(hp[q] << 16), h1 = __uint_as_float(hp[q] & 0xffff0000u);
            lp[q] = pack_bf16x2(x0 - h0, x1 - h1);
          }
          const uint32_t off = sw128_off(row, 8 * c);
          *reinterpret_cast<uint4 *>(Ahi + off) = make_uint4(hp[0], hp[1], hp[2], hp[3]);
          *reinterpret_cast<uint4 *>(Alo + off) = make_uint4(lp[0], lp[1], lp[2], lp[3]);
        }
        fence_async_smem();
        tc_fence_before();
        mbar_arrive(smem_u32(&bars[t]));
        if (!mbar_wait(smem_u32(&bars[2 + t]), acc_ph)) { ok = false; break; }
        acc_ph ^= 1;
        tc_fence_after();
        const int d0 = k > 0 ? (sp[k - 1] ^ ((k - 1 == f1 || k - 1 == f2) ? 1 : 0)) : -1;
        const int sk = sp[k] ^ ((k == f1 || k == f2) ? 1 : 0);
        float z0 = shc[0], z1 = shc[1], y0 = shc[2], y1 = shc[3];
#pragma unroll
        for (int ch = 0; ch < DH / 8; ++ch) {
          float v0[8], v1[8], v2[8];  // columns 24 ch .. 24 ch + 23 = units 8 ch .. 8 ch + 7
          tmem_ld8(dcol + (uint32_t)(ch * 24), v0);
          tmem_ld8(dcol + (uint32_t)(ch * 24 + 8), v1);
          tmem_ld8(dcol + (uint32_t)(ch * 24 + 16), v2);
          tmem_wait_ld();
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int q = ch * 8 + u;
            const int c0 = 3 * u, c1 = 3 * u + 1, c2 = 3 * u + 2;
            const float pu = c0 < 8 ? v0[c0] : (c0 < 16 ? v1[c0 - 8] : v2[c0 - 16]);
            const float pr = c1 < 8 ? v0[c1] : (c1 < 16 ? v1[c1 - 8] : v2[c1 - 16]);
            const float pg = c2 < 8 ? v0[c2] : (c2 < 16 ? v1[c2 - 8] : v2[c2 - 16]);
            float au = pu + sbias[4 * q];
            float ar = pr + sbias[4 * q + 1];
            const float gg = pg + sbias[4 * q + 2];
            float ai = sbias[4 * q + 3];
            if (d0 >= 0) {
              au += sxw[d0 * NG + 3 * q];
              ar += sxw[d0 * NG + 3 * q + 1];
              ai += sxw[d0 * NG + 3 * q + 2];
            }
            const float uu = sigm_f(au), rr = sigm_f(ar);
            const float cc = tanh_f(rr * gg + ai);
            const float hn = (1.0f - uu) * h[q] + uu * cc;
            h[q] = hn;
            z0 = fmaf(shead[q], hn, z0);
            z1 = fmaf(shead[DH + q], hn, z1);
            if (a.cplx) {
              y0 = fmaf(shead[2 * DH + q], hn, y0);
              y1 = fmaf(shead[3 * DH + q], hn, y1);
            }
          }
        }
        tc_fence_before();
        // head of site k (Sec. II.A) and the change against sigma's cached term
        float lp0, lp1;
        log_softmax2<float>(z0, z1, lp0, lp1);
        int forced = -1;
        if (a.zmask) {
          if (n_up >= N / 2) forced = 1;
          else if (n_dn >= N / 2) forced = 0;
        }
        double lps;
        if (forced >= 0) lps = (sk == forced) ? 0.0 : -INFINITY;
        else lps = (double)(sk == 0 ? lp0 : lp1);
        double ph = 0.0;
        if (a.cplx) ph = NQS_PI * (double)softsign(sk == 0 ? y0 : y1);
        if (valid) {
          const float *lc = a.lccache + ((int64_t)s * N + k) * 2;
          dre += 0.5 * lps - (double)lc[0];
          dimg += ph - (double)lc[1];
        }
        if (sk == 0) ++n_up; else ++n_dn;
      }
      if (ok && valid) {
        const double e = a.item_e[item];
        const double mag = exp(dre);
        double *c = a.contrib + ((int64_t)op * a.ns + s) * 2;
        c[0] = e * mag * cos(dimg);
        c[1] = e * mag * sin(dimg);
      }
    }
    // slot finished (or failed): tell the MMA warp
    if (row == 0) cmd[t] = 0;
    if (!ok) atomicExch(abort_flag, 1);
    mbar_arrive(smem_u32(&bars[t]));
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == SLOTS * 4)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS)
                 : "memory");
}

}  // namespace

bool eloc_tc_supported(int dim, int dh) { return dim == 1 && dh == DH; }

cudaError_t eloc_tc_run(const ElocTcArgs &args, int sm_count, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(k_eloc_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)SMEM_BYTES);
  if (e != cudaSuccess) return e;
  const int needed = (args.ntiles + SLOTS - 1) / SLOTS;
  const int grid = needed < sm_count ? needed : sm_count;
  if (grid <= 0) return cudaSuccess;
  k_eloc_tc<<<grid, THREADS, SMEM_BYTES, st>>>(args);
  return cudaGetLastError();
}

}  // namespace nqs
