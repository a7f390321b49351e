// eloc2d_tcs.cu -- log Psi of every connected configuration (Sec. II.C) for
// 2D lattices on the zig-zag path (Sec. II.B) with hidden size 96 or 128,
// mixed precision, on the tensor cores (sm_103a), with the weights streamed
// from L2.
//
// At these sizes the BF16 hi/lo planes of the weights (240 KB at d_h = 96,
// 320 KB at 128) do not fit in shared memory beside a tile's states, so they
// are kept in global memory as ready-swizzled K atoms (an image written once
// per step from the packed weights) and streamed through a ring of shared-
// memory slots by cp.async.bulk; they stay resident in L2.
//
// The vertical input of the 2D cell (App. A) enters as U2 h_ver.  Instead of
// staging h_ver as a second operand, each site's first product also forms
// U2 h_{k-1}, which is kept (FP32) in a per-CTA column buffer until the site
// above k-1 reads it.  So per site k, with M = 128 connected configurations
// of one operator (a tile, sharing the first changed site kst) and the BF16x3
// split (hi.hi + lo.hi + hi.lo) of both operands, FP32 accumulation:
//   D1 = [U1; U2] h_{k-1}   N = 2 d_h, K = d_h     (X = U1 h_{k-1}, Y = U2 h_{k-1})
//   h' = X [if a horizontal neighbour] + (Y at a row start | U2 h_ver from the
//        column buffer | 0)
//   D2 = W h'               N = 3 d_h in chunks of units (u, r, c gate
//                           columns of a chunk's units side by side), K = d_h
// Before a tile's first site, one D1 pass per cached state of the row
// frontier (the last cached state of each lattice column: not simply the last
// Lx sites, since the path visits a column twice in a row where it turns)
// puts U2 h of those states into the column buffer.  K is padded to two 64-wide atoms; the
// padded k-steps are not issued.
//
// The A operand of both products (h_{k-1}, then h', as BF16 hi and lo
// planes, two K per 32-bit column) lives in tensor memory beside the
// accumulators, written by the compute threads with tcgen05.st (a thread's
// row is its lane), so that the MMAs read only B from shared memory and the
// ring holds six slots at d_h 128, eight at 96 (measured: local energies of
// the 12 x 12 d_h 128 instance 88.5 -> 85.3 ms, of the d_h 96 one 22.2 ->
// 21.0 ms against A planes in shared memory with four and five slots).
//
// Warp roles: 4 d_h / UT compute warps (thread (quarter q, part p) owns row
// 32 q + lane, its tensor-memory lane, and units UT p .. UT p + UT - 1; UT =
// 64 at d_h = 128, 32 at 96, so that no register spills), one MMA
// warp (one thread issues every tcgen05.mma and commit) and one producer warp
// (one thread hands out tiles and streams the weight stages).  The producer
// takes tiles from the launch's counter, longest suffixes first, and
// publishes them in a two-slot queue; all three roles derive the same stage
// schedule from the tile.  Every wait is bounded; a wait that runs out sets a
// CTA-wide abort flag that ends every role's loop, the MMAs are drained, the
// producer waits for its copies in flight, the tensor memory is freed and
// NQS_ERR_TIMEOUT goes to the status word.
#include <cuda_bf16.h>

#include "common.cuh"
#include "eloc2d_tc.h"
#include "tc_common.cuh"

namespace nqs {
namespace {

template <int DH>
struct Tcs {
  static constexpr int TR = ELOC2D_TC_ROWS;         // rows per tile (the MMA's M)
  static constexpr int UT = DH == 128 ? 64 : 32;    // hidden units per compute thread
  static constexpr int P = DH / UT;                 // unit parts per row
  static constexpr int NCW = 4 * P;                 // compute warps
  static constexpr int NCT = 32 * NCW;              // compute threads
  static constexpr int THREADS = NCT + 64;          // + MMA warp + producer warp
  // registers per thread: each of the 4 SM sub-partitions holds 16 K of
  // them and ceil(warps / 4) of the CTA's warps
  static constexpr int REGS = (16384 / (32 * ((THREADS / 32 + 3) / 4))) & ~7;
  static constexpr int NA = 2;                      // 64-wide K atoms (K padded to 128)
  static constexpr int KS_LAST = (DH - 64) / 16;    // k-steps issued in the last atom
  static constexpr int CU = DH == 128 ? 64 : 32;    // units per gate chunk
  static constexpr int NCH = DH / CU;               // gate chunks
  static constexpr int N1 = 2 * DH;                 // first product: [U1; U2]
  static constexpr int N2 = 3 * CU;                 // second product, per chunk
  static constexpr int SB1 = N1 * 128, SB2 = N2 * 128;    // stage bytes (one atom, one plane)
  static constexpr int NS1 = 2 * NA, NS2 = NCH * 2 * NA;  // stages per product
  static constexpr int SLOT = SB1 > SB2 ? SB1 : SB2;
  static constexpr int NSLOT = DH == 128 ? 6 : 8;
  static constexpr int TS = 3 * DH + 4;             // bias / input table row stride (floats)
  // tensor memory: accumulators in columns [0, 3 d_h), the A operand (BF16
  // hi, lo planes, two K per column) in [TA_HI, TA_HI + 64), [TA_LO, TA_LO + 64)
  static constexpr int TA_HI = 384, TA_LO = TA_HI + 64;
  static constexpr int OFF_RING = 0;
  static constexpr int OFF_TAB = OFF_RING + NSLOT * SLOT;  // float [9][TS]
  static constexpr int OFF_BH = OFF_TAB + 9 * TS * 4;      // float [DH]: b_h
  static constexpr int OFF_HEAD = OFF_BH + DH * 4;         // float [4][DH]: head rows
  static constexpr int OFF_HC = OFF_HEAD + 4 * DH * 4;     // float [4]: head biases
  static constexpr int OFF_ZX = OFF_HC + 16;               // float4 [P-1][TR]: head partials
  static constexpr int OFF_SPR = OFF_ZX + (P - 1) * TR * 16;  // uint8 [TR][32]: sampled spins
  static constexpr int OFF_BAR = OFF_SPR + TR * 32;
  // mbarriers: full[NSLOT], empty[NSLOT], a, d1, d2[NCH], z, tfull[2], tempty[2], drain
  static constexpr int B_FULL = 0, B_EMPTY = NSLOT, B_A = 2 * NSLOT, B_D1 = B_A + 1,
                       B_D2 = B_D1 + 1, B_Z = B_D2 + NCH, B_TF = B_Z + 1, B_TE = B_TF + 2,
                       B_DRAIN = B_TE + 2, NBAR = B_DRAIN + 1;
  static constexpr int OFF_MISC = OFF_BAR + NBAR * 8;      // int tile[2], abort, tmem base
  static constexpr size_t SMEM = 1024 + OFF_MISC + 32;
  static constexpr int IMG = NS1 * SB1 + NS2 * SB2;        // weight image bytes
  static_assert(OFF_RING % 1024 == 0 && SLOT % 1024 == 0, "atom alignment");
  static_assert(OFF_ZX % 16 == 0 && OFF_BAR % 8 == 0, "vector and barrier alignment");
  static_assert(SMEM <= 227 * 1024, "one CTA per SM");
  static_assert(3 * DH <= TA_HI && N1 <= 256 && N2 <= 256 && N2 % 16 == 0 && DH <= 128,
                "MMA shapes, TMEM");
};

__device__ __forceinline__ uint32_t pack2(float x0, float x1) {
  uint32_t u;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(u) : "f"(x1), "f"(x0));
  return u;
}
__device__ __forceinline__ float sigm_f(float x) { return __fdividef(1.0f, 1.0f + __expf(-x)); }
__device__ __forceinline__ float tanh_f(float x) { return 2.0f * sigm_f(2.0f * x) - 1.0f; }

// BF16 hi/lo planes of units k0 .. k0 + 7 (k0 % 8 == 0, the same in the
// whole warp) of this thread's row into the A operand in tensor memory
// (`lanes`: the warp's lane quarter); columns k0 / 2 .. k0 / 2 + 3 of each
// plane.  The MMA reads them after tmem_wait_st and the arrival on a.
template <int DH>
__device__ __forceinline__ void planes8(uint32_t lanes, int k0, const float *h) {
  uint32_t hp[4], lp[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float x0 = h[2 * q], x1 = h[2 * q + 1];
    hp[q] = pack2(x0, x1);
    lp[q] = pack2(x0 - __uint_as_float(hp[q] << 16), x1 - __uint_as_float(hp[q] & 0xffff0000u));
  }
  tmem_st4(lanes + (uint32_t)(Tcs<DH>::TA_HI + (k0 >> 1)), hp);
  tmem_st4(lanes + (uint32_t)(Tcs<DH>::TA_LO + (k0 >> 1)), lp);
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes,
                                         uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

// Bounded wait that also gives up once another role of the CTA has aborted;
// running out sets the abort flag.
__device__ __forceinline__ bool wait_ab(uint32_t bar, uint32_t parity, volatile int *abort,
                                        unsigned long long limit = SPIN_LIMIT) {
  for (unsigned long long it = 0; it < limit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (*abort) return false;
    __nanosleep(20);
  }
  *abort = 1;
  return false;
}

// Stage schedule of a tile: F frontier passes (first product only) and S
// sites (both products); zero for a tile past its operator's row count.
template <bool SMP>
__device__ __forceinline__ void tile_sched(const Eloc2dTcArgs &a, int tile, int &F, int &S) {
  if (SMP) { F = 0; S = a.N; return; }  // sampling: every site from the first
  const int rk = tile / a.tiles_per_op;
  const int op = a.op_f[4 * rk + 3];
  const int base = (tile - rk * a.tiles_per_op) * ELOC2D_TC_ROWS;
  if (base >= a.item_cnt[op]) { F = S = 0; return; }
  const int kst = a.op_f[4 * op + 2];
  F = kst >= 1 ? min(a.Lx, kst) - 1 : 0;
  S = a.N - kst;
}

// SMP: sampling mode (tiles of 128 samples from site 0, sigma_k drawn from
// the conditionals) instead of the connected configurations' suffixes.  The
// engine of one instance as CTA `cta` of those that share its tile counter
// (its column buffer slice is the CTA's).
template <int DH, bool SMP>
__device__ __forceinline__ void tcs_body(const Eloc2dTcArgs &a, const int cta) {
  using C = Tcs<DH>;
  extern __shared__ __align__(1024) unsigned char eraw[];
  unsigned char *sm = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(eraw) + 1023) & ~uintptr_t(1023));
  unsigned char *ring = sm + C::OFF_RING;
  float *tab = reinterpret_cast<float *>(sm + C::OFF_TAB);
  float *sbh = reinterpret_cast<float *>(sm + C::OFF_BH);
  float *shead = reinterpret_cast<float *>(sm + C::OFF_HEAD);
  float *shc = reinterpret_cast<float *>(sm + C::OFF_HC);
  float4 *zx = reinterpret_cast<float4 *>(sm + C::OFF_ZX);
  uint8_t *spr = sm + C::OFF_SPR;  // [row][32]: sampled spins, by site mod 32
  uint64_t *bars = reinterpret_cast<uint64_t *>(sm + C::OFF_BAR);
  int *s_tile = reinterpret_cast<int *>(sm + C::OFF_MISC);
  volatile int *s_abort = reinterpret_cast<volatile int *>(sm + C::OFF_MISC + 8);
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sm + C::OFF_MISC + 16);
  auto bar = [&](int i) { return smem_u32(&bars[i]); };

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  constexpr int NG = 3 * DH;
  // additive terms per input pair (d0, d1), 2 = no input: update and reset
  // gates b + W_x x, candidate input W_in x + b_in (outside the reset gate)
  for (int e = tid; e < 9 * NG; e += C::THREADS) {
    const int c = e / NG, r = e % NG, j = r / DH, q = r % DH, d0 = c / 3, d1 = c % 3;
    float v = a.pack[a.obias + 4 * q + (j == 2 ? 3 : j)];
    if (d0 < 2) v += a.pack[a.oxw + d0 * NG + 3 * q + j];
    if (d1 < 2) v += a.pack[a.oxw + (2 + d1) * NG + 3 * q + j];
    tab[c * C::TS + r] = v;
  }
  for (int e = tid; e < DH; e += C::THREADS) sbh[e] = a.pack[a.obias + 4 * e + 2];
  for (int e = tid; e < 4 * DH; e += C::THREADS) shead[e] = a.pack[a.ohead + e];
  if (tid < 4) shc[tid] = a.pack[a.ohc + tid];
  if (tid == 0) {
    for (int i = 0; i < C::NSLOT; ++i) {
      mbar_init(bar(C::B_FULL + i), 1);   // the producer's expect_tx arrive
      mbar_init(bar(C::B_EMPTY + i), 1);  // the MMA thread's commit
    }
    mbar_init(bar(C::B_A), C::NCT);       // every compute thread: operand written
    mbar_init(bar(C::B_D1), 1);
    for (int c = 0; c < C::NCH; ++c) mbar_init(bar(C::B_D2 + c), 1);
    mbar_init(bar(C::B_Z), C::NCT);       // end of a tile: head partials written
    for (int i = 0; i < 2; ++i) {
      mbar_init(bar(C::B_TF + i), 1);             // the producer publishes a tile
      mbar_init(bar(C::B_TE + i), C::NCW + 1);    // compute warps and the MMA warp are done
    }
    mbar_init(bar(C::B_DRAIN), 1);
    *s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int N = a.N, Lx = a.Lx;
  const unsigned long long lim = a.spin_limit ? a.spin_limit : SPIN_LIMIT;

  if (warp == C::NCW + 1) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      uint32_t q = 0;  // stages issued so far
      for (int it = 0;; ++it) {
        const int slot = it & 1;
        if (it >= 2 && !wait_ab(bar(C::B_TE + slot), ((it >> 1) - 1) & 1, s_abort, lim)) break;
        const int tile = *s_abort ? a.ntiles : atomicAdd(a.tile_ctr, 1);
        s_tile[slot] = tile;
        if (a.test_drop_tile && it == 0) break;  // (test) the first tile is never published
        mbar_arrive(bar(C::B_TF + slot));
        if (tile >= a.ntiles) break;
        int F, S;
        tile_sched<SMP>(a, tile, F, S);
        bool stop = false;
        for (int f = 0; f < F + S && !stop; ++f) {
          const int len = f < F ? C::NS1 : C::NS1 + C::NS2;
          for (int si = 0; si < len; ++si, ++q) {
            const uint32_t sl = q % C::NSLOT, round = q / C::NSLOT;
            if (round > 0 && !wait_ab(bar(C::B_EMPTY + sl), (round - 1) & 1, s_abort, lim)) {
              stop = true;
              break;
            }
            const uint32_t bytes = si < C::NS1 ? C::SB1 : C::SB2;
            const uint32_t off = si < C::NS1 ? si * C::SB1 : C::NS1 * C::SB1 + (si - C::NS1) * C::SB2;
            mbar_expect_tx(bar(C::B_FULL + sl), bytes);
            bulk_g2s(smem_u32(ring + sl * C::SLOT), a.wimg + off, bytes, bar(C::B_FULL + sl));
          }
        }
        if (stop) break;
      }
      // no copy outlives the kernel: wait for the last one issued into each slot
      const uint32_t q0 = q > (uint32_t)C::NSLOT ? q - C::NSLOT : 0;
      for (uint32_t r = q0; r < q; ++r) {
        volatile int never = 0;
        wait_ab(bar(C::B_FULL + r % C::NSLOT), (r / C::NSLOT) & 1, &never);
      }
    }
    __syncwarp();
  } else if (warp == C::NCW) {
    // ---------------------------------------------------------- MMA issuer
    if (lane == 0) {
      constexpr uint32_t id1 = idesc_bf16(C::TR, C::N1), id2 = idesc_bf16(C::TR, C::N2);
      const uint32_t aH = tmem + (uint32_t)C::TA_HI, aL = tmem + (uint32_t)C::TA_LO;
      uint32_t q = 0, pa = 0;
      bool stop = false;
      for (int it = 0; !stop; ++it) {
        const int slot = it & 1;
        if (!wait_ab(bar(C::B_TF + slot), (it >> 1) & 1, s_abort, lim)) break;
        const int tile = s_tile[slot];
        if (tile >= a.ntiles) break;
        int F, S;
        tile_sched<SMP>(a, tile, F, S);
        for (int f = 0; f < F + S && !stop; ++f) {
          for (int prod = 0; prod < (f < F ? 1 : 2) && !stop; ++prod) {
            if (!wait_ab(bar(C::B_A), pa & 1, s_abort, lim)) { stop = true; break; }
            ++pa;
            tc_fence_after();
            const int nst = prod == 0 ? C::NS1 : C::NS2;
            for (int si = 0; si < nst; ++si, ++q) {
              const uint32_t sl = q % C::NSLOT;
              if (!wait_ab(bar(C::B_FULL + sl), (q / C::NSLOT) & 1, s_abort, lim)) { stop = true; break; }
              tc_fence_after();
              const int at = (si >> 1) % C::NA, plane = si & 1, chunk = si / (2 * C::NA);
              const uint64_t bd = sw128_desc(smem_u32(ring + sl * C::SLOT));
              const uint32_t ah = aH + (uint32_t)(32 * at), al = aL + (uint32_t)(32 * at);
              const uint32_t d = prod == 0 ? tmem : tmem + (uint32_t)(chunk * C::N2);
              const uint32_t idn = prod == 0 ? id1 : id2;
              const int ks = at == C::NA - 1 ? C::KS_LAST : 4;
              for (int kk = 0; kk < ks; ++kk) {
                // B: 16 K = 32 bytes along the swizzled row; A: 8 columns
                const uint64_t adv = (uint64_t)(kk * 32) >> 4;
                const uint32_t ac = (uint32_t)(8 * kk);
                if (plane == 0) {
                  mma_bf16_ts(d, ah + ac, bd + adv, idn, (at == 0 && kk == 0) ? 0u : 1u);
                  mma_bf16_ts(d, al + ac, bd + adv, idn, 1u);
                } else {
                  mma_bf16_ts(d, ah + ac, bd + adv, idn, 1u);
                }
              }
              mma_commit(bar(C::B_EMPTY + sl));
              if (prod == 1 && si % (2 * C::NA) == 2 * C::NA - 1) mma_commit(bar(C::B_D2 + chunk));
            }
            if (prod == 0 && !stop) mma_commit(bar(C::B_D1));
          }
        }
        if (!stop) mbar_arrive(bar(C::B_TE + slot));
      }
      // drain the MMAs before the tensor memory is freed
      mma_commit(bar(C::B_DRAIN));
      volatile int never = 0;
      if (!wait_ab(bar(C::B_DRAIN), 0, &never)) *s_abort = 1;
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------ compute warps
    const int quarter = warp & 3, part = warp >> 2;
    constexpr int UT = C::UT, G8 = UT / 8;
    // A thread's units, 8 at a time.  Where the units divide evenly, a part
    // takes CU / P units of every gate chunk (group g8 in chunk g8 / GPC), so
    // that every part starts its cell update as soon as the first chunk of
    // the gate product lands; otherwise part p takes units UT p .. UT p + UT - 1.
    constexpr bool SPLIT = C::NCH > 1 && UT % (8 * C::NCH) == 0;
    constexpr int GPC = SPLIT ? G8 / C::NCH : G8;
    const int row = 32 * quarter + lane, u0 = UT * part;
    auto unit_of = [&](int g8) {
      return SPLIT ? (g8 / GPC) * C::CU + part * (C::CU / C::P) + 8 * (g8 % GPC) : u0 + 8 * g8;
    };
    const uint32_t lanes = tmem + ((uint32_t)(32 * quarter) << 16);
    // gate j of unit un in the second product's accumulator
    auto gcol = [&](int un) {
      return lanes + (uint32_t)((un / C::CU) * C::N2 + un % C::CU);
    };
    const int chunk = u0 / C::CU;  // the chunk of a part's units when not split
    uint32_t na = 0, pd1 = 0, pd2 = 0, pz = 0;  // arrivals on a; phases of d1, d2, z waited
    bool ok = true;
    auto arrive_a = [&]() {
      tmem_wait_st();  // this thread's A-operand stores have landed
      fence_async_smem();
      tc_fence_before();
      mbar_arrive(bar(C::B_A));
      ++na;
    };
    for (int it = 0; ok; ++it) {
      const int slot = it & 1;
      if (!wait_ab(bar(C::B_TF + slot), (it >> 1) & 1, s_abort, lim)) { ok = false; break; }
      const int tile = s_tile[slot];
      if (tile >= a.ntiles) break;
      int op = 0, base, cnt;
      if (SMP) {
        base = tile * C::TR;
        cnt = (int)a.ns;
      } else {
        const int rk = tile / a.tiles_per_op;
        op = a.op_f[4 * rk + 3];
        base = (tile - rk * a.tiles_per_op) * C::TR;
        cnt = a.item_cnt[op];
      }
      if (base >= cnt) {
        __syncwarp();
        if (lane == 0) mbar_arrive(bar(C::B_TE + slot));
        continue;
      }
      const int f1 = SMP ? -1 : a.op_f[4 * op], f2 = SMP ? -1 : a.op_f[4 * op + 1];
      const int kst = SMP ? 0 : a.op_f[4 * op + 2];
      const bool valid = base + row < cnt;
      const int64_t item = (int64_t)op * a.ns + base + row;
      const int s = SMP ? (valid ? base + row : 0) : (valid ? __ldcg(a.item_s + item) : 0);
      const uint8_t *sp = a.spins + (int64_t)s * N;
      const float *lcrow = a.lccache + (int64_t)s * N * 2;
      const float *hrow = a.hcache + (int64_t)s * N * DH;
      float *cb = a.colbuf + ((int64_t)cta * C::TR + row) * Lx * DH;
      auto colof = [&](int k) {
        const int jr = k / Lx, m = k - jr * Lx;
        return (jr & 1) ? (Lx - 1 - m) : m;
      };
      auto spin_at = [&](int k) { return (int)__ldcg(sp + k) ^ ((k == f1 || k == f2) ? 1 : 0); };
      // cached state h_k (this thread's units) into the A planes, zero if k < 0
      auto cached_planes = [&](int k) {
#pragma unroll
        for (int g8 = 0; g8 < G8; ++g8) {
          float h8[8];
          if (valid && k >= 0) {
            ld_global_cg_v8(hrow + (int64_t)k * DH + unit_of(g8), h8);
          } else {
#pragma unroll
            for (int i = 0; i < 8; ++i) h8[i] = 0.f;
          }
          planes8<DH>(lanes, unit_of(g8), h8);
        }
      };
      // Y = U2 h (columns DH + units) of the last first product into the
      // column buffer at lattice column col
      auto store_y = [&](int col) {
#pragma unroll
        for (int g8 = 0; g8 < G8; ++g8) {
          float y[8];
          tmem_ld8(lanes + (uint32_t)(DH + unit_of(g8)), y);
          tmem_wait_ld();
          if (valid) st_global_v8(cb + col * DH + unit_of(g8), y);
        }
      };

      // frontier passes: U2 h of the last cached state of every lattice
      // column but that of kst - 1 (the first site's product forms it).  With
      // kst at position m0 of row j0 these are row j0 - 1's first Lx - m0
      // sites (its others lie below row j0's first m0 sites, in the same
      // columns) and row j0's sites before kst - 1.
      const int F = kst >= 1 ? min(Lx, kst) - 1 : 0;
      const int j0 = kst / Lx, m0 = kst - j0 * Lx;
      for (int fi = 0; fi < F && ok; ++fi) {
        const int f = j0 == 0 ? fi : (fi < Lx - m0 ? (j0 - 1) * Lx + fi : kst - m0 + fi - (Lx - m0));
        cached_planes(f);
        arrive_a();
        if (!wait_ab(bar(C::B_D1), pd1 & 1, s_abort, lim)) { ok = false; break; }
        ++pd1;
        tc_fence_after();
        store_y(colof(f));
      }
      if (!ok) break;
      cached_planes(kst - 1);

      // spins of the first site: sigma'_{k-1} (horizontal input), sigma'_k, vertical input
      int s_prev = 2, s_cur = 2, s_ver = 2;
      if (!SMP) {
        s_prev = kst > 0 ? spin_at(kst - 1) : 2;
        s_cur = spin_at(kst);
        const int m = kst % Lx;
        s_ver = kst >= Lx ? spin_at(kst - 2 * m - 1) : 2;
      }
      int n_up = 0, n_dn = 0, nA = 0;
      if (!SMP && a.zmask && part == 0)
        for (int k = 0; k < kst; ++k) { if (__ldcg(sp + k) == 0) ++n_up; else ++n_dn; }
      // log |psi(sigma')/psi(sigma)| and the phase difference as error-free
      // FP32 TwoSum pairs; dead: the mask forces the amplitude of sigma' to zero
      float sre = 0.f, cre = 0.f, sim = 0.f, cim = 0.f;
      bool dead = false;
      float zp[4] = {0.f, 0.f, 0.f, 0.f};
      int sgp = -1, kr = -1;  // pending row work: spin (or to draw), site
      float2 lcp = make_float2(0.f, 0.f);
      const uint64_t stp = SMP ? (a.step_dev ? (uint64_t)*a.step_dev : a.step) : 0;
      auto row_work = [&]() {
        float4 zo = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int p = 0; p < C::P - 1; ++p) {
          const float4 v = zx[p * C::TR + row];
          zo.x += v.x; zo.y += v.y; zo.z += v.z; zo.w += v.w;
        }
        float lp0, lp1;
        log_softmax2<float>(zp[0] + zo.x + shc[0], zp[1] + zo.y + shc[1], lp0, lp1);
        int forced = -1;  // value forced by the mask, or -1
        if (a.zmask) {
          if (n_up >= N / 2) forced = 1;
          else if (n_dn >= N / 2) forced = 0;
        }
        if (SMP) {  // draw sigma_k: 0 iff u < p_k(0) (FP32, 24-bit uniform)
          const float p0 = forced == 0 ? 1.f : (forced == 1 ? 0.f : ex(lp0));
          sgp = uniform24(a.seed, stp, (uint32_t)(s + a.s0), (uint32_t)kr) < p0 ? 0 : 1;
          spr[row * 32 + (kr & 31)] = (uint8_t)sgp;
        }
        const bool kill = forced >= 0 && sgp != forced;
        const float hl = forced >= 0 ? 0.f : 0.5f * (sgp == 0 ? lp0 : lp1);
        float pp = 0.f, pe = 0.f;
        if (a.cplx)
          pi_times(softsign(sgp == 0 ? zp[2] + zo.z + shc[2] : zp[3] + zo.w + shc[3]), pp, pe);
        dead |= kill;
        two_add(sre, cre, hl);
        two_add(sre, cre, -lcp.x);
        two_add(sim, cim, pp);
        two_add(sim, cim, pe - lcp.y);
        if (sgp == 0) ++n_up; else ++n_dn;
        if (SMP && valid) {
          a.spins_out[(int64_t)s * N + kr] = (uint8_t)sgp;
          reinterpret_cast<float2 *>(a.lccache_out)[(int64_t)s * N + kr] =
              make_float2(kill ? -INFINITY : hl, pp + pe);
          if (a.marshall && sgp == 1 && (((kr / Lx) & 1 ? Lx - 1 - kr % Lx : kr % Lx) + kr / Lx) & 1)
            ++nA;
        }
      };

      for (int k = kst; k < N; ++k) {
        const int jr = k / Lx, m = k - jr * Lx;
        const int col = (jr & 1) ? (Lx - 1 - m) : m;
        const bool hor = m != 0;
        const int ver = k >= Lx ? k - 2 * m - 1 : -1;
        int d0 = hor ? s_prev : 2, d1 = ver >= 0 ? s_ver : 2;
        arrive_a();  // A = h_{k-1}
        // the vertical term from the column buffer (in flight during the product)
        float hp[UT];
        const bool vbuf = valid && ver >= 0 && ver != k - 1;
#pragma unroll
        for (int g8 = 0; g8 < G8; ++g8) {
          float v[8];
          if (vbuf) {
            ld_global_v8(cb + col * DH + unit_of(g8), v);
          } else {
#pragma unroll
            for (int i = 0; i < 8; ++i) v[i] = 0.f;
          }
#pragma unroll
          for (int i = 0; i < 8; ++i) hp[8 * g8 + i] = v[i];
        }
        // next site's raw spins (flipped when used) and this site's cached terms
        int r_next = 0, r_vnext = 0, k_v = -1;
        if (!SMP && k + 1 < N) {
          const int m1 = (k + 1) % Lx;
          r_next = __ldcg(sp + k + 1);
          if (k + 1 >= Lx) {
            k_v = k + 1 - 2 * m1 - 1;
            r_vnext = __ldcg(sp + k_v);
          }
        }
        float2 lc = make_float2(0.f, 0.f);
        if (!SMP && part == 0 && valid) lc = __ldcg(reinterpret_cast<const float2 *>(lcrow + 2 * k));
        // the previous site's row work overlaps the first product (the other
        // parts' head partials are published by their arrival on a)
        if (part == 0 && (SMP ? k > 0 : sgp >= 0)) {
          if (!wait_ab(bar(C::B_A), (na - 1) & 1, s_abort, lim)) { ok = false; break; }
          row_work();
        }
        if (!wait_ab(bar(C::B_D1), pd1 & 1, s_abort, lim)) { ok = false; break; }
        ++pd1;
        tc_fence_after();
        // h' = X [horizontal] + (Y at a row start | U2 h_ver | 0); Y to the
        // buffer; h' to the planes, 8 units at a time (the next group's
        // tensor-memory loads in flight while this one is used)
        {
          float x[2][8], y[2][8];
          tmem_ld8(lanes + (uint32_t)unit_of(0), x[0]);
          tmem_ld8(lanes + (uint32_t)(DH + unit_of(0)), y[0]);
#pragma unroll
          for (int g8 = 0; g8 < G8; ++g8) {
            const int cu = g8 & 1;
            tmem_wait_ld();
            if (g8 + 1 < G8) {
              tmem_ld8(lanes + (uint32_t)unit_of(g8 + 1), x[cu ^ 1]);
              tmem_ld8(lanes + (uint32_t)(DH + unit_of(g8 + 1)), y[cu ^ 1]);
            }
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              const float v = ver == k - 1 ? y[cu][i] : hp[8 * g8 + i];
              hp[8 * g8 + i] = hor ? x[cu][i] + v : v;
            }
            if (valid && k >= 1) st_global_v8(cb + colof(k - 1) * DH + unit_of(g8), y[cu]);
            planes8<DH>(lanes, unit_of(g8), hp + 8 * g8);
          }
        }
        arrive_a();  // A = h'
        // sampling: part 0 drew sigma_{k-1} before its arrival on a
        if (SMP && part > 0 && !wait_ab(bar(C::B_A), (na - 1) & 1, s_abort, lim)) { ok = false; break; }
        if (!SPLIT && !wait_ab(bar(C::B_D2 + chunk), pd2 & 1, s_abort, lim)) { ok = false; break; }
        tc_fence_after();
        if (SMP) {
          d0 = hor ? spr[row * 32 + ((k - 1) & 31)] : 2;
          d1 = ver >= 0 ? spr[row * 32 + (ver & 31)] : 2;
        }
        // GRU cell (App. A) on this thread's units, 8 at a time; h_k overwrites
        // h' in registers and goes to the planes once every chunk is done
        const float *tb = tab + (d0 * 3 + d1) * C::TS;
        float *grow = SMP && a.gcache ? a.gcache + ((int64_t)s * N + k) * 5 * DH : nullptr;
        float z0 = 0.f, z1 = 0.f, z2 = 0.f, z3 = 0.f;
        bool dok = true;
        // gate values of group g8 in slot g8 % 2; the next group's loads are
        // issued before this one is used, within a chunk of the product
        float gq[2][3][8];
        auto gate_ld = [&](int g, int sl) {
          const int ugl = unit_of(g);
          tmem_ld8(gcol(ugl), gq[sl][0]);
          tmem_ld8(gcol(ugl) + (uint32_t)C::CU, gq[sl][1]);
          tmem_ld8(gcol(ugl) + (uint32_t)(2 * C::CU), gq[sl][2]);
        };
#pragma unroll
        for (int g8 = 0; g8 < G8; ++g8) {
          const int ug = unit_of(g8), cu = g8 & 1;
          if (g8 % GPC == 0) {  // the first group of a chunk: its loads are issued here
            if (SPLIT) {  // the next chunk of the gate product
              dok = dok && wait_ab(bar(C::B_D2 + g8 / GPC), pd2 & 1, s_abort, lim);
              tc_fence_after();
            }
            gate_ld(g8, cu);
          }
          tmem_wait_ld();
          if (g8 + 1 < G8 && (g8 + 1) % GPC != 0) gate_ld(g8 + 1, cu ^ 1);
          float *gu = gq[cu][0], *gr = gq[cu][1], *gg = gq[cu][2];
          float su[8], sr[8], sc[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int i = 8 * g8 + u, un = ug + u;
            const float uu = sigm_f(gu[u] + tb[un]), rr = sigm_f(gr[u] + tb[DH + un]);
            const float cc = tanh_f(fmaf(rr, gg[u] + sbh[un], tb[2 * DH + un]));
            const float hn = fmaf(uu, cc - hp[i], hp[i]);
            if (SMP) { su[u] = uu; sr[u] = rr; sc[u] = cc; gg[u] += sbh[un]; gu[u] = hp[i]; }
            hp[i] = hn;
            z0 = fmaf(shead[un], hn, z0);
            z1 = fmaf(shead[DH + un], hn, z1);
            if (a.cplx) {
              z2 = fmaf(shead[2 * DH + un], hn, z2);
              z3 = fmaf(shead[3 * DH + un], hn, z3);
            }
          }
          if (SMP && valid) {  // gate cache (u, r, c, W_h h' + b_h, h') and h_k
            // (rows are 5 d_h and d_h floats, units in groups of 8: every
            // store starts on a 32-byte boundary)
            if (grow) {
              st_global_v8(grow + ug, su);
              st_global_v8(grow + DH + ug, sr);
              st_global_v8(grow + 2 * DH + ug, sc);
              st_global_v8(grow + 3 * DH + ug, gg);
              st_global_v8(grow + 4 * DH + ug, gu);
            }
            st_global_v8(a.hcache_out + ((int64_t)s * N + k) * DH + ug, hp + 8 * g8);
          }
        }
        if (!dok) { ok = false; break; }
        // every chunk of the gate product has read the planes before h_k goes in
        if (!SPLIT && chunk != C::NCH - 1 &&
            !wait_ab(bar(C::B_D2 + C::NCH - 1), pd2 & 1, s_abort, lim)) { ok = false; break; }
        ++pd2;
#pragma unroll
        for (int g8 = 0; g8 < G8; ++g8) planes8<DH>(lanes, unit_of(g8), hp + 8 * g8);
        if (part > 0) {
          zx[(part - 1) * C::TR + row] = make_float4(z0, z1, z2, z3);
        } else {
          zp[0] = z0; zp[1] = z1; zp[2] = z2; zp[3] = z3;
          sgp = s_cur;
          lcp = lc;
          kr = k;
        }
        s_prev = s_cur;
        s_cur = k + 1 < N ? r_next ^ ((k + 1 == f1 || k + 1 == f2) ? 1 : 0) : 2;
        s_ver = k_v >= 0 ? r_vnext ^ ((k_v == f1 || k_v == f2) ? 1 : 0) : 2;
      }
      if (!ok) break;
      // the last site's row work, then the row's contribution
      tc_fence_before();
      mbar_arrive(bar(C::B_Z));
      if (!wait_ab(bar(C::B_Z), pz & 1, s_abort, lim)) { ok = false; break; }
      ++pz;
      if (part == 0 && SMP) {
        row_work();
        if (valid) {
          a.logpsi[2 * (int64_t)s] = dead ? -INFINITY : (double)sre + (double)cre;
          a.logpsi[2 * (int64_t)s + 1] =
              (double)sim + (double)cim + (a.marshall && (nA & 1) ? NQS_PI : 0.0);
        }
      } else if (part == 0) {
        if (sgp >= 0) row_work();
        if (valid) {
          const double e = a.item_e[item];
          const double dre = (double)sre + (double)cre, dimg = (double)sim + (double)cim;
          const double mag = dead ? 0.0 : exp(dre);
          double *c = a.contrib + ((int64_t)op * a.ns + s) * 2;
          c[0] = e * mag * cos(dimg);
          c[1] = e * mag * sin(dimg);
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(C::B_TE + slot));
    }
    if (!ok) *s_abort = 1;
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (tid == 0 && *s_abort) atomicExch(a.err, (int)NQS_ERR_TIMEOUT);
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512)
                 : "memory");
}

template <int DH, bool SMP>
__global__ void __launch_bounds__(Tcs<DH>::THREADS) __maxnreg__(Tcs<DH>::REGS)
    k_eloc2d_tcs(const __grid_constant__ Eloc2dTcArgs a) {
  tcs_body<DH, SMP>(a, (int)blockIdx.x);
}

// The local energies of several instances of one hidden size in one
// launch: instance i owns the CTAs [cta0[i], cta0[i + 1]) and its own tile
// counter, so the instances' tiles run side by side instead of one launch
// after another.
template <int DH>
__global__ void __launch_bounds__(Tcs<DH>::THREADS) __maxnreg__(Tcs<DH>::REGS)
    k_eloc2d_tcs_group(const __grid_constant__ Eloc2dTcGroup g) {
  // the instance's arguments in shared memory (uniform loads, no indexed
  // parameter reads in the loops)
  __shared__ Eloc2dTcArgs s_args;
  int i = 0;
  while (i + 1 < g.n && (int)blockIdx.x >= g.cta0[i + 1]) ++i;
  static_assert(sizeof(Eloc2dTcArgs) % 8 == 0, "argument copy");
  for (int e = threadIdx.x; e < (int)(sizeof(Eloc2dTcArgs) / 8); e += blockDim.x)
    reinterpret_cast<uint64_t *>(&s_args)[e] = reinterpret_cast<const uint64_t *>(&g.inst[i])[e];
  __syncthreads();
  tcs_body<DH, false>(s_args, (int)blockIdx.x - g.cta0[i]);
}

// The weight image: every stage of the two products as a K atom (64 k, 128 B
// rows, 128-byte swizzle) of BF16 hi then lo, in the order the MMAs use them:
// [U1; U2] atom 0 hi, lo, atom 1 hi, lo; then per gate chunk the same four.
// Row n of a chunk is gate n / CU of unit chunk * CU + n % CU.
template <int DH>
__global__ void k_eloc2d_tcs_image(const float *__restrict__ pack, int oWgT, int oU12T,
                                   unsigned char *__restrict__ img) {
  using C = Tcs<DH>;
  const int e1 = C::NA * C::N1 * 64, e2 = C::NCH * C::NA * C::N2 * 64;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < e1 + e2; e += gridDim.x * blockDim.x) {
    float w = 0.f;
    unsigned char *hi;
    int n, kk;
    if (e < e1) {
      const int at = e / (C::N1 * 64), r = e % (C::N1 * 64);
      n = r / 64; kk = r % 64;
      const int k = 64 * at + kk;
      if (k < DH) w = n < DH ? pack[oU12T + k * DH + n] : pack[oU12T + (DH + k) * DH + (n - DH)];
      hi = img + (2 * at) * C::SB1;
    } else {
      const int f = e - e1, c = f / (C::NA * C::N2 * 64), r = f % (C::NA * C::N2 * 64);
      const int at = r / (C::N2 * 64), r2 = r % (C::N2 * 64);
      n = r2 / 64; kk = r2 % 64;
      const int k = 64 * at + kk, j = n / C::CU, q = c * C::CU + n % C::CU;
      if (k < DH) w = pack[oWgT + k * 3 * DH + 3 * q + j];
      hi = img + C::NS1 * C::SB1 + ((c * C::NA + at) * 2) * C::SB2;
    }
    const int sb = e < e1 ? C::SB1 : C::SB2;
    const __nv_bfloat16 h = __float2bfloat16_rn(w);
    const uint32_t off = sw128_off(n, kk);
    *reinterpret_cast<__nv_bfloat16 *>(hi + off) = h;
    *reinterpret_cast<__nv_bfloat16 *>(hi + sb + off) = __float2bfloat16_rn(w - __bfloat162float(h));
  }
}

template <int DH>
cudaError_t image_dh(const Eloc2dTcArgs &args, cudaStream_t st) {
  using C = Tcs<DH>;
  k_eloc2d_tcs_image<DH><<<C::IMG / 2 / 256 / 4 + 1, 256, 0, st>>>(
      args.pack, args.oWgT, args.oU12T, const_cast<unsigned char *>(args.wimg));
  return cudaGetLastError();
}

template <int DH, bool SMP>
cudaError_t run_dh(const Eloc2dTcArgs &args, int sm_count, cudaStream_t st) {
  using C = Tcs<DH>;
  cudaError_t e = image_dh<DH>(args, st);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_eloc2d_tcs<DH, SMP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)C::SMEM);
  if (e != cudaSuccess) return e;
  const int grid = args.ntiles < sm_count ? args.ntiles : sm_count;
  if (grid <= 0) return cudaSuccess;
  k_eloc2d_tcs<DH, SMP><<<grid, C::THREADS, C::SMEM, st>>>(args);
  return cudaGetLastError();
}

}  // namespace

bool eloc2d_tcs_supported(int dim, int dh) { return dim == 2 && (dh == 96 || dh == 128); }

size_t eloc2d_tcs_image_bytes(int dh) {
  return dh == 128 ? (size_t)Tcs<128>::IMG : dh == 96 ? (size_t)Tcs<96>::IMG : 0;
}

cudaError_t eloc2d_tcs_run(const Eloc2dTcArgs &args, int dh, int sm_count, cudaStream_t st) {
  if (dh == 128) return run_dh<128, false>(args, sm_count, st);
  if (dh == 96) return run_dh<96, false>(args, sm_count, st);
  return cudaErrorInvalidValue;
}

cudaError_t eloc2d_tcs_image(const Eloc2dTcArgs &args, int dh, cudaStream_t st) {
  if (dh == 128) return image_dh<128>(args, st);
  if (dh == 96) return image_dh<96>(args, st);
  return cudaErrorInvalidValue;
}

namespace {
template <int DH>
cudaError_t group_dh(const Eloc2dTcGroup &g, cudaStream_t st) {
  using C = Tcs<DH>;
  cudaError_t e = cudaFuncSetAttribute(k_eloc2d_tcs_group<DH>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
  if (e != cudaSuccess) return e;
  k_eloc2d_tcs_group<DH><<<g.cta0[g.n], C::THREADS, C::SMEM, st>>>(g);
  return cudaGetLastError();
}
}  // namespace

cudaError_t eloc2d_tcs_group_run(const Eloc2dTcGroup &g, int dh, cudaStream_t st) {
  if (g.n < 1 || g.n > ELOC2D_GROUP_MAX || g.cta0[0] != 0) return cudaErrorInvalidValue;
  for (int i = 0; i < g.n; ++i)
    if (g.cta0[i + 1] <= g.cta0[i] || g.cta0[i + 1] - g.cta0[i] > g.inst[i].ntiles)
      return cudaErrorInvalidValue;
  if (dh == 128) return group_dh<128>(g, st);
  if (dh == 96) return group_dh<96>(g, st);
  return cudaErrorInvalidValue;
}

// The sampled spins of a row are kept in a 32-site ring: the vertical
// neighbour of site k is at most 2 Lx - 1 sites back.
bool eloc2d_tcs_sample_supported(int dim, int dh, int Lx) {
  return eloc2d_tcs_supported(dim, dh) && Lx >= 1 && 2 * Lx - 1 <= 31;
}

cudaError_t eloc2d_tcs_sample(const Eloc2dTcArgs &args, int dh, int sm_count, cudaStream_t st) {
  if (!eloc2d_tcs_sample_supported(2, dh, args.Lx) || !args.spins_out || !args.logpsi ||
      !args.hcache_out || !args.lccache_out || !args.colbuf || !args.tile_ctr || !args.err)
    return cudaErrorInvalidValue;
  if (dh == 128) return run_dh<128, true>(args, sm_count, st);
  if (dh == 96) return run_dh<96, true>(args, sm_count, st);
  return cudaErrorInvalidValue;
}

}  // namespace nqs
