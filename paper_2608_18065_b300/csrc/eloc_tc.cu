// eloc_tc.cu -- log Psi of every connected configuration (Sec. II.C) for 1D
// chains with hidden size 64, mixed precision, on the tensor cores (sm_103a).
//
// A connected configuration sigma' differs from its sample sigma from site j
// on, so its suffix k = j..N-1 is recomputed from the cached state h_{j-1}.
// Rows of one operator share j; 128 of them form a tile.  Per round the tile's
// FP32 states are split h = hi + lo into BF16 planes in shared memory and one
// product [128 x 80] x [80 x 208] is accumulated in FP32 in tensor memory as
// hi W_hi + hi W_lo + lo W_hi (App. A).  K = 64 state columns plus a 16-wide
// block holding (1, one-hot of sigma'_{k-1}) exactly in BF16, so the gate
// biases and the one-hot input weights of W_u, W_r and the bias of W_h come
// out of the MMA too.  Output columns 0..191 are the gate pre-activations of
// the next site (n = 3a + g: [W_u|W_r][h;x] + b, W_h h + b_h), columns
// 192..195 the output heads U h, U_phi h of the state itself (Sec. II.A):
// round r yields the gates of site j + r and the conditional of site
// j + r - 1, and one extra round after the last site reads the last head.
// Only W_in x + b_in (outside the reset gate) comes from a small table.
// The 64 units of a row are split over two warps that read the same
// tensor-memory lanes, so 16 warps (two tiles x two halves x four lane
// quarters) share the epilogue; the tensor core alternates between the two
// tiles.  After a named barrier of its 256 threads one thread of each tile
// issues the tile's MMAs and commits them to the tile's mbarrier.  Every
// mbarrier wait is bounded and its outcome is OR-reduced over the tile at
// the next barrier, so all threads of a tile leave together; on expiry the
// CTA flags NQS_ERR_TIMEOUT, drains its MMAs, frees its tensor memory and
// exits.
#include <cuda_bf16.h>

#include "common.cuh"
#include "eloc_tc.h"
#include "tc_common.cuh"

namespace nqs {
namespace {

constexpr int DH = 64;
constexpr int NG = 3 * DH;                   // gate columns, n = 3a + g
constexpr int NHD = 16;                      // head columns (4 used)
constexpr int NB = NG + NHD;                 // MMA N
constexpr int TR = 128;                      // rows per tile (MMA M)
constexpr int SLOTS = 2;
constexpr int HALVES = 2;                    // warps sharing one row's units
constexpr int UH = DH / HALVES;              // units per thread
constexpr int THREADS = TR * SLOTS * HALVES;  // 16 warps
constexpr int TMEM_COLS = 512;
constexpr int ACC_STRIDE = 256;              // tensor-memory columns per slot
constexpr int ATILE = TR * 64 * 2;           // one 128-byte-swizzle atom column of A (16 KB)
constexpr int BTILE = NB * 64 * 2;           // one atom column of B (26 KB)
// the augmented K = 16 block in the non-swizzled K-major layout: core
// matrices of 8 rows x 16 bytes, the two K halves 128 bytes apart, 8-row
// groups 256 bytes apart
constexpr int XLBO = 128, XSBO = 256;
constexpr int XTILE_B = (NB / 8) * XSBO;     // 6.5 KB
constexpr int XTILE_A = (TR / 8) * XSBO;     // 4 KB
constexpr int SLOT_BYTES = 2 * ATILE + XTILE_A;
constexpr int HSTATE = TR * DH;              // FP32 states of one tile
constexpr int XS = DH + 1;                   // padded stride of the W_in x + b_in table
// B: hi, lo (128-byte swizzle), augmented hi, lo; per slot A: hi, lo,
// augmented; per slot the FP32 states; barriers and small tables
constexpr size_t SMEM_BYTES = 1024 + 2 * (size_t)BTILE + 2 * (size_t)XTILE_B +
                              SLOTS * (size_t)SLOT_BYTES + SLOTS * (size_t)HSTATE * 4 + 4 * 8 +
                              2 * 4 + sizeof(float) * (3 * XS + 4) + 64;
static_assert(BTILE % 1024 == 0 && ATILE % 1024 == 0, "swizzle atoms stay 1024-aligned");
static_assert((2 * BTILE + 2 * XTILE_B) % 1024 == 0 && SLOT_BYTES % 1024 == 0,
              "the A atoms of every slot stay 1024-aligned");
static_assert(SMEM_BYTES <= 227 * 1024, "fits one CTA per SM");

// Byte offset of element k (< 16) of row r in the augmented block.
__device__ __forceinline__ uint32_t xoff(int r, int k) {
  return (uint32_t)(r >> 3) * XSBO + (uint32_t)(k >> 3) * XLBO + (uint32_t)(r & 7) * 16u +
         (uint32_t)(k & 7) * 2u;
}

// Shared-memory matrix descriptor of a K-major bf16 tile without swizzle.
__device__ __forceinline__ uint64_t noswz_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);        // start address
  d |= (uint64_t)(XLBO >> 4) << 16;             // leading byte offset: next core matrix in K
  d |= (uint64_t)(XSBO >> 4) << 32;             // stride byte offset: next 8-row group
  d |= (uint64_t)1 << 46;                       // descriptor version (tcgen05)
  return d;                                     // layout 0: no swizzle
}

constexpr uint16_t BF16_ONE = 0x3F80;

// Two floats rounded to BF16 and packed, x0 in the low half (lower address).
__device__ __forceinline__ uint32_t pack_bf16x2(float x0, float x1) {
  uint32_t u;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(u) : "f"(x1), "f"(x0));
  return u;
}

__device__ __forceinline__ float sigm_f(float x) { return __fdividef(1.0f, 1.0f + __expf(-x)); }
__device__ __forceinline__ float tanh_f(float x) { return 2.0f * sigm_f(2.0f * x) - 1.0f; }

// BF16 hi/lo planes of units k0 .. k0 + 7 of row `row`.
__device__ __forceinline__ void write_planes8(unsigned char *Ahi, unsigned char *Alo, int row,
                                              int k0, const float (&h)[8]) {
  uint32_t hp[4], lp[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float x0 = h[2 * q], x1 = h[2 * q + 1];
    hp[q] = pack_bf16x2(x0, x1);
    const float h0 = __uint_as_float(hp[q] << 16), h1 = __uint_as_float(hp[q] & 0xffff0000u);
    lp[q] = pack_bf16x2(x0 - h0, x1 - h1);
  }
  const uint32_t off = sw128_off(row, k0);
  *reinterpret_cast<uint4 *>(Ahi + off) = make_uint4(hp[0], hp[1], hp[2], hp[3]);
  *reinterpret_cast<uint4 *>(Alo + off) = make_uint4(lp[0], lp[1], lp[2], lp[3]);
}

// The FP32 state of a row lives in shared memory, 64 floats in 16 chunks of
// 4; chunk c of row r sits at position c ^ (r mod 8) (within its half), so
// the 8 rows a quarter-warp reads with one 16-byte load hit distinct banks.
__device__ __forceinline__ float4 *hchunk(float *hrow, int row, int c) {
  return reinterpret_cast<float4 *>(hrow) + (c ^ (row & 7));
}

// Augmented columns of row `row`: (1, [d == 0], [d == 1], 0 ...); d = 2: no input.
__device__ __forceinline__ void write_aug(unsigned char *Aaug, int row, int d) {
  const uint32_t w0 = BF16_ONE | ((d == 0 ? (uint32_t)BF16_ONE : 0u) << 16);
  const uint32_t w1 = d == 1 ? (uint32_t)BF16_ONE : 0u;
  *reinterpret_cast<uint4 *>(Aaug + xoff(row, 0)) = make_uint4(w0, w1, 0u, 0u);
}

// Named barrier of n threads whose result is the OR of pred over them.
__device__ __forceinline__ bool bar_any(int id, int n, bool pred) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, %2, %3, p;\n"
      " selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)pred), "r"(id), "r"(n)
      : "memory");
  return r != 0;
}

// One round of the tile's product into tensor memory d, committed to bar.
// a0: shared address of the tile's A atoms (hi, lo, augmented); b0: of the
// B atoms (hi, lo, augmented hi, augmented lo).
__device__ __forceinline__ void issue_round(uint32_t d, uint32_t a0, uint32_t b0, uint32_t bar) {
  constexpr uint32_t idesc = idesc_bf16(TR, NB);
  const uint64_t ah = sw128_desc(a0), al = sw128_desc(a0 + ATILE), ax = noswz_desc(a0 + 2 * ATILE);
  const uint64_t bh = sw128_desc(b0), bl = sw128_desc(b0 + BTILE);
  tc_fence_after();
#pragma unroll
  for (int kk = 0; kk < DH / 16; ++kk) {
    const uint64_t adv = (uint64_t)(kk * 32) >> 4;
    mma_bf16(d, ah + adv, bh + adv, idesc, kk > 0 ? 1u : 0u);
    mma_bf16(d, ah + adv, bl + adv, idesc, 1u);
    mma_bf16(d, al + adv, bh + adv, idesc, 1u);
  }
  // augmented block: exact in BF16, so two products suffice
  mma_bf16(d, ax, noswz_desc(b0 + 2 * BTILE), idesc, 1u);
  mma_bf16(d, ax, noswz_desc(b0 + 2 * BTILE + XTILE_B), idesc, 1u);
  mma_commit(bar);
}

// w split into BF16 hi + lo at byte offset off of the two planes.
__device__ __forceinline__ void put_split(unsigned char *hi, unsigned char *lo, uint32_t off,
                                          float w) {
  const __nv_bfloat16 h = __float2bfloat16_rn(w);
  *reinterpret_cast<__nv_bfloat16 *>(hi + off) = h;
  *reinterpret_cast<__nv_bfloat16 *>(lo + off) = __float2bfloat16_rn(w - __bfloat162float(h));
}

// DHM: the model's hidden size (64, or 32 run with zero-padded units)
template <int DHM>
__global__ void __launch_bounds__(THREADS, 1) k_eloc_tc(const ElocTcArgs a) {
  extern __shared__ __align__(1024) unsigned char eraw[];
  unsigned char *sm = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(eraw) + 1023) & ~uintptr_t(1023));
  unsigned char *Bhi = sm, *Blo = sm + BTILE, *Bxh = sm + 2 * BTILE, *Bxl = Bxh + XTILE_B;
  unsigned char *Abase = Bxl + XTILE_B;      // slot t: Abase + t SLOT_BYTES: hi, lo, augmented
  float *hstate = reinterpret_cast<float *>(Abase + SLOTS * SLOT_BYTES);  // [SLOTS][TR][DH]
  // mbarriers next: they need 8-byte alignment (this address is 1024-aligned)
  uint64_t *bars = reinterpret_cast<uint64_t *>(hstate + SLOTS * HSTATE);  // accfull[2] drain[2]
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 4);
  float *sxi = reinterpret_cast<float *>(tmem_slot + 2);  // [3][XS]
  float *shc = sxi + 3 * XS;                 // [4]

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int N = a.N;
  const int nh = a.cplx ? 4 : 2;
  __shared__ int s_tile[SLOTS][2];  // the slot's next tile, double-buffered

  // zero the augmented blocks (columns 3..15 stay zero)
  for (int e = tid; e < 2 * XTILE_B / 16; e += THREADS)
    reinterpret_cast<uint4 *>(Bxh)[e] = make_uint4(0u, 0u, 0u, 0u);
  for (int t = 0; t < SLOTS; ++t)
    for (int e = tid; e < XTILE_A / 16; e += THREADS)
      reinterpret_cast<uint4 *>(Abase + t * SLOT_BYTES + 2 * ATILE)[e] = make_uint4(0u, 0u, 0u, 0u);
  __syncthreads();
  // weights B[n][k], split into BF16 planes with the 128-byte swizzle:
  // n < 192: W_g[a][k] (n = 3a + g); 192 + j: head row j; rest zero
  // a model of hidden size dhm < 64 runs with its units padded by zero
  // weights: a padded unit's state stays 0 (c = tanh(0), h' = 0) and adds
  // nothing to the other units or the heads, so the values are unchanged
  constexpr int dhm = DHM, ngm = 3 * DHM;
  for (int e = tid; e < NB * DH; e += THREADS) {
    const int n = e / DH, k = e % DH;
    float w = 0.f;
    if (n < NG) {
      if (n / 3 < dhm && k < dhm) w = a.pack[a.oWgT + k * ngm + n];
    } else if (n - NG < nh && k < dhm) {
      w = a.pack[a.ohead + (n - NG) * dhm + k];
    }
    put_split(Bhi, Blo, sw128_off(n, k), w);
  }
  // augmented rows: column 0 the bias of gate n, columns 1, 2 the one-hot
  // input weights of the update and reset gates
  for (int n = tid; n < NG; n += THREADS) {
    const int q = n / 3, g = n % 3;
    const bool u = q < dhm;
    put_split(Bxh, Bxl, xoff(n, 0), u ? a.pack[a.obias + 4 * q + g] : 0.f);
    put_split(Bxh, Bxl, xoff(n, 1), u && g < 2 ? a.pack[a.oxw + n] : 0.f);
    put_split(Bxh, Bxl, xoff(n, 2), u && g < 2 ? a.pack[a.oxw + ngm + n] : 0.f);
  }
  // W_in x + b_in per previous spin d (0, 1; 2 = none at site 0)
  for (int e = tid; e < 3 * DH; e += THREADS) {
    const int d = e / DH, q = e % DH;
    sxi[d * XS + q] = q < dhm ? a.pack[a.obias + 4 * q + 3] +
                                    (d < 2 ? a.pack[a.oxw + d * ngm + 3 * q + 2] : 0.f)
                              : 0.f;
  }
  if (tid < 4) shc[tid] = a.pack[a.ohc + tid];
  if (tid == 0) {
    for (int t = 0; t < 2 * SLOTS; ++t) mbar_init(smem_u32(&bars[t]), 1);  // one commit each
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_async_smem();
  if (warp == 0) {
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

  {
    const int t = warp / 8, half = (warp / 4) & 1, quarter = warp & 3;
    const int row = quarter * 32 + lane;
    const bool issuer = (warp & 7) == 0 && lane == 0;
    unsigned char *Ahi = Abase + t * SLOT_BYTES, *Alo = Ahi + ATILE, *Aaug = Ahi + 2 * ATILE;
    float *hrow = hstate + (t * TR + row) * DH;
    const uint32_t a0 = smem_u32(Ahi), b0 = smem_u32(Bhi);
    const uint32_t dacc = tmem + (uint32_t)(t * ACC_STRIDE);
    const uint32_t accbar = smem_u32(&bars[t]);
    const uint32_t dcol = dacc + ((uint32_t)(quarter * 32) << 16);
    const uint32_t gcol = dcol + (uint32_t)(3 * UH * half);  // this half's gate columns
    uint32_t acc_ph = 0;
    bool ok = true;
    // tiles in rank order (longest suffixes first) from the launch's counter:
    // the slot's issuer takes one and publishes it at a barrier of the slot,
    // which also makes ok uniform over the slot
    int par = 0;
    auto grab = [&]() -> int {
      if (issuer) s_tile[t][par] = atomicAdd(a.tile_ctr, 1);
      if (bar_any(1 + t, 2 * TR, !ok)) ok = false;
      const int v = s_tile[t][par];
      par ^= 1;
      return v;
    };
    for (int tile = grab(); tile < a.ntiles && ok; tile = grab()) {
      const int rk = tile / a.tiles_per_op;
      const int op = a.op_f[4 * rk + 3];
      const int base = (tile - rk * a.tiles_per_op) * TR;
      const int cnt = a.item_cnt[op];
      if (base >= cnt) continue;  // uniform over the tile's 256 threads
      const int f1 = a.op_f[4 * op], f2 = a.op_f[4 * op + 1], j0 = a.op_f[4 * op + 2];
      const bool valid = base + row < cnt;
      const int64_t item = (int64_t)op * a.ns + base + row;
      const int s = valid ? __ldcg(a.item_s + item) : 0;
      const uint8_t *sp = a.spins + (int64_t)s * N;
      const float *lcrow = a.lccache + (int64_t)s * N * 2;
      // streamed operands bypass L1 (ld.global.cg), which keeps the small L1
      // left beside the 202 KB of shared memory for register spills
      auto spin_at = [&](int k) { return (int)__ldcg(sp + k) ^ ((k == f1 || k == f2) ? 1 : 0); };
      // first recomputed site: j0, or with checkpoints the site after the
      // last checkpoint before it (its sites up to j0 - 1 add nothing)
      const int kr = a.ck > 0 ? (j0 / a.ck) * a.ck : j0;
      // h_{kr-1}: this half's 32 units into the shared state and the planes
      {
        const float4 *src = nullptr;
        if (valid && kr > 0 && UH * half < dhm) {
          const int64_t slot =
              a.ck > 0 ? (int64_t)s * a.nck + (kr / a.ck - 1) : (int64_t)s * N + kr - 1;
          src = reinterpret_cast<const float4 *>(a.hcache + slot * dhm + UH * half);
        }
#pragma unroll
        for (int g8 = 0; g8 < UH / 8; ++g8) {
          float h8[8];
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            const float4 v = src ? __ldcg(src + 2 * g8 + q) : make_float4(0.f, 0.f, 0.f, 0.f);
            *hchunk(hrow, row, (UH / 4) * half + 2 * g8 + q) = v;
            h8[4 * q] = v.x; h8[4 * q + 1] = v.y; h8[4 * q + 2] = v.z; h8[4 * q + 3] = v.w;
          }
          write_planes8(Ahi, Alo, row, UH * half + 8 * g8, h8);
        }
      }
      int n_up = 0, n_dn = 0;
      if (a.zmask && half == 0)
        for (int k = 0; k < kr; ++k) { if (__ldcg(sp + k) == 0) ++n_up; else ++n_dn; }
      // round 0: planes of h_{kr-1} and the input of site kr
      int sprev = kr > 0 ? spin_at(kr - 1) : 2;
      if (half == 0) write_aug(Aaug, row, sprev);
      fence_async_smem();
      tc_fence_before();
      if (bar_any(1 + t, 2 * TR, !ok)) { ok = false; break; }
      if (issuer) issue_round(dacc, a0, b0, accbar);
      // log |psi(sigma')/psi(sigma)| and the phase difference as error-free
      // FP32 TwoSum pairs (each term's parts added exactly, off the slow FP64
      // pipe); dead: the mask forces the amplitude of sigma' to zero
      float sre = 0.f, cre = 0.f, sim = 0.f, cim = 0.f;
      bool dead = false;
      const int L = N - kr;
      for (int r = 0; r <= L; ++r) {
        const int k = kr + r;  // gates of site k (r < L), head of site k - 1 (r > 0)
        // loads for after the wait: sigma'_k and sigma's cached terms at k - 1
        const int sraw = k < N ? (int)__ldcg(sp + k) : 0;  // flipped when used, after it lands
        float2 lc = make_float2(0.f, 0.f);
        if (half == 0 && r > 0 && valid) lc = __ldcg(reinterpret_cast<const float2 *>(lcrow + 2 * (k - 1)));
        if (!mbar_wait(accbar, acc_ph)) ok = false;
        acc_ph ^= 1;
        tc_fence_after();
        if (half == 0 && r > 0) {
          // conditional of site k - 1 from U h_{k-1} (Sec. II.A); sprev = sigma'_{k-1}
          float hv[8];
          tmem_ld8(dcol + (uint32_t)NG, hv);
          tmem_wait_ld();
          float lp0, lp1;
          log_softmax2<float>(hv[0] + shc[0], hv[1] + shc[1], lp0, lp1);
          int forced = -1;
          if (a.zmask) {
            if (n_up >= N / 2) forced = 1;
            else if (n_dn >= N / 2) forced = 0;
          }
          const bool kill = forced >= 0 && sprev != forced;
          const float hl = forced >= 0 ? 0.f : 0.5f * (sprev == 0 ? lp0 : lp1);
          float pp = 0.f, pe = 0.f;
          if (a.cplx) pi_times(softsign(sprev == 0 ? hv[2] + shc[2] : hv[3] + shc[3]), pp, pe);
          if (valid && k - 1 >= j0) {
            dead |= kill;
            two_add(sre, cre, hl);
            two_add(sre, cre, -lc.x);
            two_add(sim, cim, pp);
            two_add(sim, cim, pe - lc.y);
          }
          if (sprev == 0) ++n_up; else ++n_dn;
        }
        if (r < L) {
          // GRU cell of site k (App. A) on this half's units, 8 at a time:
          // state from shared memory, gate pre-activations from tensor memory
          const float *xi = sxi + (k > 0 ? sprev : 2) * XS + UH * half;
#pragma unroll
          for (int g8 = 0; g8 < UH / 8; ++g8) {
            // columns 3q + g of units 8 g8 .. 8 g8 + 7: 24 columns, loads of 4
            // starting at multiples of 4
            float v[24];
#pragma unroll
            for (int q = 0; q < 6; ++q) {
              float t4[4];
              tmem_ld4(gcol + (uint32_t)(g8 * 24 + 4 * q), t4);
#pragma unroll
              for (int e = 0; e < 4; ++e) v[4 * q + e] = t4[e];
            }
            float h8[8];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
              const float4 c4 = *hchunk(hrow, row, (UH / 4) * half + 2 * g8 + q);
              h8[4 * q] = c4.x; h8[4 * q + 1] = c4.y; h8[4 * q + 2] = c4.z; h8[4 * q + 3] = c4.w;
            }
            tmem_wait_ld();
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              const float uu = sigm_f(v[3 * u]), rr = sigm_f(v[3 * u + 1]);
              const float cc = tanh_f(fmaf(rr, v[3 * u + 2], xi[8 * g8 + u]));
              h8[u] = fmaf(uu, cc - h8[u], h8[u]);
            }
#pragma unroll
            for (int q = 0; q < 2; ++q)
              *hchunk(hrow, row, (UH / 4) * half + 2 * g8 + q) =
                  make_float4(h8[4 * q], h8[4 * q + 1], h8[4 * q + 2], h8[4 * q + 3]);
            write_planes8(Ahi, Alo, row, UH * half + 8 * g8, h8);
          }
          sprev = sraw ^ ((k == f1 || k == f2) ? 1 : 0);
          if (half == 0) write_aug(Aaug, row, sprev);
          fence_async_smem();
          tc_fence_before();
          if (bar_any(1 + t, 2 * TR, !ok)) { ok = false; break; }
          if (issuer) issue_round(dacc, a0, b0, accbar);
        } else {
          tc_fence_before();
          if (bar_any(1 + t, 2 * TR, !ok)) { ok = false; break; }
        }
      }
      if (ok && valid && half == 0) {
        const double e = a.item_e[item];
        const double dre = (double)sre + (double)cre, dimg = (double)sim + (double)cim;
        const double mag = dead ? 0.0 : exp(dre);
        double *c = a.contrib + ((int64_t)op * a.ns + s) * 2;
        c[0] = e * mag * cos(dimg);
        c[1] = e * mag * sin(dimg);
      }
    }
    // drain this tile's MMAs before the tensor memory is freed
    if (issuer) {
      mma_commit(smem_u32(&bars[SLOTS + t]));
      if (!mbar_wait(smem_u32(&bars[SLOTS + t]), 0)) ok = false;
    }
    if (!ok) atomicExch(a.err, (int)NQS_ERR_TIMEOUT);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS)
                 : "memory");
}

}  // namespace

// hidden size 64, or 32 padded to 64 (dhm must be a multiple of UH = 32 so
// that each half's cached units are whole or absent)
bool eloc_tc_supported(int dim, int dh) { return dim == 1 && (dh == DH || dh == DH / 2); }

cudaError_t eloc_tc_run(const ElocTcArgs &args, int sm_count, cudaStream_t st) {
  if (args.dhm != DH && args.dhm != DH / 2) return cudaErrorInvalidValue;
  const void *kern = args.dhm == DH ? (const void *)k_eloc_tc<DH> : (const void *)k_eloc_tc<DH / 2>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)SMEM_BYTES);
  if (e != cudaSuccess) return e;
  const int needed = (args.ntiles + SLOTS - 1) / SLOTS;
  const int grid = needed < sm_count ? needed : sm_count;
  if (grid <= 0) return cudaSuccess;
  if (args.dhm == DH)
    k_eloc_tc<DH><<<grid, THREADS, SMEM_BYTES, st>>>(args);
  else
    k_eloc_tc<DH / 2><<<grid, THREADS, SMEM_BYTES, st>>>(args);
  return cudaGetLastError();
}

}  // namespace nqs
