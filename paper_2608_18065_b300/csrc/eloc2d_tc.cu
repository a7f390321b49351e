// eloc2d_tc.cu -- log Psi of every connected configuration (Sec. II.C) for
// 2D lattices on the zig-zag path (Sec. II.B), hidden size 64 (and 32, run
// with its units padded to 64 by zero weights, biases and head columns: a
// padded unit keeps h' = 0, c = tanh(0) = 0, h = 0 and adds nothing), mixed
// precision, on the tensor cores (sm_103a).
//
// A connected configuration sigma' first differs from its sample at site
// kstart; its suffix is recomputed from the sample's cached h_{kstart-1} and
// cached vertical neighbours (sites before kstart), the recomputed ones
// coming from a per-CTA column buffer.  Rows of one operator share kstart;
// 128 of them form a tile.  Per site the 2D cell (App. A) has two dependent
// products, both on tcgen05 with FP32 accumulation in tensor memory and the
// BF16x3 split (hi.hi + hi.lo + lo.hi) of both operands:
//   h'    = U1 h_hor + U2 h_ver   M = 128, N = 64,  K = 64 + 64 (columns 0..63)
//   gates = W [h']                M = 128, N = 192, K = 64      (columns 64..255,
//                                 gate j of unit a at 64 + 64 j + a)
// The gate biases and the one-hot input weights of the horizontal and
// vertical spins come from a table indexed by the row's two inputs.  One
// pair of BF16 planes cycles h_{k-1} -> h' -> h_k (each product has
// finished reading it before the next value is written), a second pair
// holds the vertical neighbour.  Thread (quarter q, half f) of the 8 warps
// owns row 32 q + lane (its tensor-memory lane) and units 32 f .. 32 f + 31:
// it splits its own states into the planes, reads h' back from tensor
// memory for the update (the columns hold it until the next site's first
// product), and writes h_k to the column buffer.  The next site's vertical
// states are staged by cp.async into a per-thread FP32 area while a site
// runs.  Tiles come from a per-launch counter, longest suffixes first.  The
// MMAs are issued by a half-1 thread, which has no row work.  The output
// heads run in FP32 on the SIMT side; a row's log-softmax, mask and
// log-amplitude sums of site k run on its half-0 thread during the next
// site's first product.  Every
// mbarrier wait is bounded and its outcome OR-reduced at the next barrier;
// on expiry the CTA flags NQS_ERR_TIMEOUT, drains its MMAs, frees its tensor
// memory and exits.
#include <cuda_bf16.h>

#include "common.cuh"
#include "eloc2d_tc.h"
#include "tc_common.cuh"

namespace nqs {
namespace {

constexpr int DH = 64, NG = 3 * DH, TR = ELOC2D_TC_ROWS, THREADS = 256, UH = 32;
constexpr int TMEM_COLS = 256;          // h' (64) | gates (192)
constexpr int ATOM = TR * 128;          // one 128-byte-swizzle K atom of a 128-row A tile
constexpr int BW = NG * 128;            // the W atom, N = 192 rows
constexpr int BU = DH * 128;            // one K atom of [U1 | U2], N = 64 rows
constexpr int TS = NG + 4;              // stride of the bias / input table rows (floats)
// B: W hi, lo; U hi (atoms hor, ver), U lo (hor, ver); A: S hi, lo, V hi, lo
constexpr int OFF_BW = 0, OFF_BU = 2 * BW, OFF_S = OFF_BU + 4 * BU, OFF_V = OFF_S + 2 * ATOM;
constexpr int VSS = DH + 4;                     // staging row stride (floats): rows on distinct banks
constexpr int OFF_VS = OFF_V + 2 * ATOM;        // float [128][VSS]: next vertical states (FP32)
constexpr int OFF_TAB = OFF_VS + TR * VSS * 4;  // float [9][TS]: per input pair (d0, d1)
constexpr int OFF_BH = OFF_TAB + 9 * TS * 4;    // float [64]: b_h
constexpr int OFF_HEAD = OFF_BH + DH * 4;       // float [4][64]: head rows
constexpr int OFF_HC = OFF_HEAD + 4 * DH * 4;   // float [4]: head biases
constexpr int OFF_ZX = OFF_HC + 16;             // float [128][4]: half-1 head partials
constexpr int OFF_BAR = OFF_ZX + TR * 4 * 4;    // mbarriers: h', gates, drain
constexpr int OFF_TM = OFF_BAR + 3 * 8;         // tensor-memory base address
constexpr size_t SMEM_BYTES = 1024 + OFF_TM + 16;
static_assert(OFF_BU % 1024 == 0 && OFF_S % 1024 == 0 && OFF_V % 1024 == 0 && ATOM % 1024 == 0 &&
                  BU % 1024 == 0,
              "swizzle atoms stay 1024-aligned");
static_assert(OFF_ZX % 16 == 0 && OFF_BAR % 8 == 0, "vector and barrier alignment");
static_assert(SMEM_BYTES <= 227 * 1024, "fits one CTA per SM");

__device__ __forceinline__ uint32_t pack2(float x0, float x1) {
  uint32_t u;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(u) : "f"(x1), "f"(x0));
  return u;
}

__device__ __forceinline__ float sigm_f(float x) { return __fdividef(1.0f, 1.0f + __expf(-x)); }
__device__ __forceinline__ float tanh_f(float x) { return 2.0f * sigm_f(2.0f * x) - 1.0f; }

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
}

// BF16 hi/lo planes of units k0 .. k0 + 7 of row `row`.
__device__ __forceinline__ void planes8(unsigned char *hi, unsigned char *lo, int row, int k0,
                                        const float *h) {
  uint32_t hp[4], lp[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float x0 = h[2 * q], x1 = h[2 * q + 1];
    hp[q] = pack2(x0, x1);
    lp[q] = pack2(x0 - __uint_as_float(hp[q] << 16), x1 - __uint_as_float(hp[q] & 0xffff0000u));
  }
  const uint32_t off = sw128_off(row, k0);
  *reinterpret_cast<uint4 *>(hi + off) = make_uint4(hp[0], hp[1], hp[2], hp[3]);
  *reinterpret_cast<uint4 *>(lo + off) = make_uint4(lp[0], lp[1], lp[2], lp[3]);
}

// w split into BF16 hi + lo at byte offset off of the two planes.
__device__ __forceinline__ void split_at(unsigned char *hi, unsigned char *lo, uint32_t off, float w) {
  const __nv_bfloat16 h = __float2bfloat16_rn(w);
  *reinterpret_cast<__nv_bfloat16 *>(hi + off) = h;
  *reinterpret_cast<__nv_bfloat16 *>(lo + off) = __float2bfloat16_rn(w - __bfloat162float(h));
}

// D (+)= A B^T over one 64-wide K atom: a = A hi atom (lo one ATOM after),
// b = B hi atom (lo blo bytes after); first: the first product overwrites D.
template <int N_>
__device__ __forceinline__ void issue_atom(uint32_t d, uint32_t a, uint32_t b, uint32_t blo,
                                           bool first) {
  constexpr uint32_t id = idesc_bf16(TR, N_);
  const uint64_t ah = sw128_desc(a), al = sw128_desc(a + ATOM);
  const uint64_t bh = sw128_desc(b), bl = sw128_desc(b + blo);
#pragma unroll
  for (int kk = 0; kk < DH / 16; ++kk) {
    const uint64_t adv = (uint64_t)(kk * 32) >> 4;
    mma_bf16(d, ah + adv, bh + adv, id, (first && kk == 0) ? 0u : 1u);
    mma_bf16(d, ah + adv, bl + adv, id, 1u);
    mma_bf16(d, al + adv, bh + adv, id, 1u);
  }
}

// DHM: the model's hidden size (64, or 32 padded to 64); it fixes only how
// the weights and the cached states are read.
template <int DHM>
__global__ void __launch_bounds__(THREADS, 1) k_eloc2d_tc(const Eloc2dTcArgs a) {
  extern __shared__ __align__(1024) unsigned char eraw[];
  unsigned char *sm = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(eraw) + 1023) & ~uintptr_t(1023));
  unsigned char *Wh = sm + OFF_BW, *Wl = Wh + BW;
  unsigned char *Uh = sm + OFF_BU, *Ul = Uh + 2 * BU;
  unsigned char *Sh = sm + OFF_S, *Sl = Sh + ATOM, *Vh = sm + OFF_V, *Vl = Vh + ATOM;
  float *tab = reinterpret_cast<float *>(sm + OFF_TAB);
  float *sbh = reinterpret_cast<float *>(sm + OFF_BH);
  float *shead = reinterpret_cast<float *>(sm + OFF_HEAD);
  float *shc = reinterpret_cast<float *>(sm + OFF_HC);
  float4 *zx = reinterpret_cast<float4 *>(sm + OFF_ZX);
  float *vsrow = reinterpret_cast<float *>(sm + OFF_VS);  // + row * VSS + UH * half below
  uint64_t *bars = reinterpret_cast<uint64_t *>(sm + OFF_BAR);
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sm + OFF_TM);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int quarter = warp & 3, half = warp >> 2;
  const int row = 32 * quarter + lane;
  const int N = a.N, Lx = a.Lx;
  float4 *vs = reinterpret_cast<float4 *>(vsrow + row * VSS + UH * half);  // this thread's staging

  // weights as B[n][k] planes: W row n = 64 j + unit (gate j), U atoms
  // B[unit][k] over the horizontal (atom 0) and vertical (atom 1) inputs
  constexpr int ngm = 3 * DHM;
  for (int e = tid; e < NG * DH; e += THREADS) {
    const int n = e / DH, k = e % DH, j = n / DH, q = n % DH;
    split_at(Wh, Wl, sw128_off(n, k),
             q < DHM && k < DHM ? a.pack[a.oWgT + k * ngm + 3 * q + j] : 0.f);
  }
  for (int e = tid; e < 2 * DH * DH; e += THREADS) {
    const int at = e / (DH * DH), r = e % (DH * DH), n = r / DH, k = r % DH;
    split_at(Uh + at * BU, Ul + at * BU, sw128_off(n, k),
             n < DHM && k < DHM ? a.pack[a.oU12T + (DHM * at + k) * DHM + n] : 0.f);
  }
  // additive terms per input pair (d0, d1), 2 = no input: update and reset
  // gates b + W_x x, candidate input W_in x + b_in (outside the reset gate)
  for (int e = tid; e < 9 * NG; e += THREADS) {
    const int c = e / NG, r = e % NG, j = r / DH, q = r % DH, d0 = c / 3, d1 = c % 3;
    float v = 0.f;
    if (q < DHM) {
      v = a.pack[a.obias + 4 * q + (j == 2 ? 3 : j)];
      if (d0 < 2) v += a.pack[a.oxw + d0 * ngm + 3 * q + j];
      if (d1 < 2) v += a.pack[a.oxw + (2 + d1) * ngm + 3 * q + j];
    }
    tab[c * TS + r] = v;
  }
  for (int e = tid; e < DH; e += THREADS) sbh[e] = e < DHM ? a.pack[a.obias + 4 * e + 2] : 0.f;
  for (int e = tid; e < 4 * DH; e += THREADS)
    shead[e] = e % DH < DHM ? a.pack[a.ohead + (e / DH) * DHM + e % DH] : 0.f;
  if (tid < 4) shc[tid] = a.pack[a.ohc + tid];
  if (tid == 0) {
    for (int t = 0; t < 3; ++t) mbar_init(smem_u32(&bars[t]), 1);  // one commit each
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
  const uint32_t lanes = tmem + ((uint32_t)(32 * quarter) << 16);
  const uint32_t hcol = lanes + (uint32_t)(UH * half);       // h' of this half's units
  const uint32_t gcol = lanes + (uint32_t)(DH + UH * half);  // gate j at + 64 j
  const bool issuer = tid == 128;  // a half-1 thread (no row work)
  const uint32_t bar_h = smem_u32(&bars[0]), bar_g = smem_u32(&bars[1]);
  const uint32_t aS = smem_u32(Sh), aV = smem_u32(Vh), bW = smem_u32(Wh), bU = smem_u32(Uh);
  uint32_t ph_h = 0, ph_g = 0;
  bool ok = true;
  // tiles in rank order (longest suffixes first) from the launch's counter,
  // taken by one thread and published at a barrier that also makes ok uniform
  __shared__ int s_tile[2];
  int par = 0;
  auto grab = [&]() -> int {
    if (issuer) s_tile[par] = atomicAdd(a.tile_ctr, 1);
    if (__syncthreads_or(!ok)) ok = false;
    const int v = s_tile[par];
    par ^= 1;
    return v;
  };

  for (int tile = grab(); tile < a.ntiles && ok; tile = grab()) {
    const int rk = tile / a.tiles_per_op;
    const int op = a.op_f[4 * rk + 3];
    const int base = (tile - rk * a.tiles_per_op) * TR;
    const int cnt = a.item_cnt[op];
    if (base >= cnt) continue;  // uniform over the CTA
    const int f1 = a.op_f[4 * op], f2 = a.op_f[4 * op + 1], kst = a.op_f[4 * op + 2];
    const bool valid = base + row < cnt;
    const int64_t item = (int64_t)op * a.ns + base + row;
    const int s = valid ? __ldcg(a.item_s + item) : 0;
    const uint8_t *sp = a.spins + (int64_t)s * N;
    const float *lcrow = a.lccache + (int64_t)s * N * 2;
    float *cb = a.colbuf + ((int64_t)blockIdx.x * TR + row) * Lx * DH + UH * half;
    auto spin_at = [&](int k) { return (int)__ldcg(sp + k) ^ ((k == f1 || k == f2) ? 1 : 0); };
    // vertical-neighbour state of site k for this thread's units into its
    // staging slots, in flight until the next wait: recomputed (>= kst) from
    // the column buffer, else from the sample's cache; zero without one
    auto fetch_ver = [&](int k) {
      const int jr = k / Lx, m = k - jr * Lx;
      const int col = (jr & 1) ? (Lx - 1 - m) : m;
      const int ver = k >= Lx ? k - 2 * m - 1 : -1;
      // (units of a padded half have no cached state: zero)
      if (valid && ver >= 0 && (ver >= kst || UH * half < DHM)) {
        const float4 *src = reinterpret_cast<const float4 *>(
            ver >= kst ? cb + col * DH : a.hcache + ((int64_t)s * N + ver) * DHM + UH * half);
#pragma unroll
        for (int q = 0; q < UH / 4; ++q) cp_async16(vs + q, src + q);
      } else {
#pragma unroll
        for (int q = 0; q < UH / 4; ++q) vs[q] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    };
    // h_{kst-1} of this thread's units into the S planes
    {
      const float4 *src = valid && kst > 0 && UH * half < DHM
          ? reinterpret_cast<const float4 *>(a.hcache + ((int64_t)s * N + kst - 1) * DHM + UH * half)
          : nullptr;
#pragma unroll
      for (int g8 = 0; g8 < UH / 8; ++g8) {
        float h8[8];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const float4 v = src ? __ldcg(src + 2 * g8 + q) : make_float4(0.f, 0.f, 0.f, 0.f);
          h8[4 * q] = v.x; h8[4 * q + 1] = v.y; h8[4 * q + 2] = v.z; h8[4 * q + 3] = v.w;
        }
        planes8(Sh, Sl, row, UH * half + 8 * g8, h8);
      }
    }
    fetch_ver(kst);
    // spins of the first site: sigma'_{k-1} (horizontal input), sigma'_k, vertical input
    int s_prev = kst > 0 ? spin_at(kst - 1) : 2;
    int s_cur = spin_at(kst);
    int s_ver;
    {
      const int m = kst % Lx;
      s_ver = kst >= Lx ? spin_at(kst - 2 * m - 1) : 2;
    }
    int n_up = 0, n_dn = 0;
    if (a.zmask && half == 0)
      for (int k = 0; k < kst; ++k) { if (__ldcg(sp + k) == 0) ++n_up; else ++n_dn; }
    // log |psi(sigma')/psi(sigma)| and the phase difference as error-free
    // FP32 TwoSum pairs; dead: the mask forces the amplitude of sigma' to zero
    float sre = 0.f, cre = 0.f, sim = 0.f, cim = 0.f;
    bool dead = false;
    // a site whose row work is pending: own head partials, sigma', cached terms
    float zp[4] = {0.f, 0.f, 0.f, 0.f};
    int sgp = -1;
    float2 lcp = make_float2(0.f, 0.f);
    auto row_work = [&]() {
      const float4 zo = zx[row];
      float lp0, lp1;
      log_softmax2<float>(zp[0] + zo.x + shc[0], zp[1] + zo.y + shc[1], lp0, lp1);
      int forced = -1;  // value forced by the mask, or -1
      if (a.zmask) {
        if (n_up >= N / 2) forced = 1;
        else if (n_dn >= N / 2) forced = 0;
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
    };

    for (int k = kst; k < N; ++k) {
      const int jr = k / Lx, m = k - jr * Lx;
      const int col = (jr & 1) ? (Lx - 1 - m) : m;
      const bool hor = m != 0;
      const int ver = k >= Lx ? k - 2 * m - 1 : -1;
      const int d0 = hor ? s_prev : 2, d1 = ver >= 0 ? s_ver : 2;
      if (ver >= 0) {
        cp_async_wait_all();  // this thread's staging copies
#pragma unroll
        for (int g8 = 0; g8 < UH / 8; ++g8) {
          const float4 v0 = vs[2 * g8], v1 = vs[2 * g8 + 1];
          const float h8[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
          planes8(Vh, Vl, row, UH * half + 8 * g8, h8);
        }
      }
      fence_async_smem();
      tc_fence_before();
      if (__syncthreads_or(!ok)) { ok = false; break; }
      // h' = U1 h_hor + U2 h_ver into columns 0..63
      const bool any = hor || ver >= 0;
      if (issuer && any) {
        tc_fence_after();
        if (hor) issue_atom<DH>(tmem, aS, bU, 2 * BU, true);
        if (ver >= 0) issue_atom<DH>(tmem, aV, bU + BU, 2 * BU, !hor);
        mma_commit(bar_h);
      }
      // the previous site's row work overlaps the product
      if (half == 0 && sgp >= 0) row_work();
      // loads for the next site: its vertical states (unless they are this
      // site's own, at the first site of a lattice row), spins, and this
      // site's cached terms
      bool turn = false;
      int r_next = 0, r_vnext = 0, k_v = -1;  // raw spins: flipped at the end of the site,
      if (k + 1 < N) {                        // when the loads have landed
        const int m1 = (k + 1) % Lx;
        if (m1 == 0) turn = true;
        else fetch_ver(k + 1);
        r_next = __ldcg(sp + k + 1);
        if (k + 1 >= Lx) {
          k_v = k + 1 - 2 * m1 - 1;
          r_vnext = __ldcg(sp + k_v);
        }
      }
      float2 lc = make_float2(0.f, 0.f);
      if (half == 0 && valid) lc = __ldcg(reinterpret_cast<const float2 *>(lcrow + 2 * k));
      // h' of this thread's units into the S planes (tensor memory keeps it
      // for the update: the next write of these columns is the next site's)
      if (any) {
        if (!mbar_wait(bar_h, ph_h)) ok = false;
        ph_h ^= 1;
        tc_fence_after();
#pragma unroll
        for (int h16 = 0; h16 < 2; ++h16) {
          float t16[16];
          tmem_ld16(hcol + (uint32_t)(16 * h16), t16);
          tmem_wait_ld();
          planes8(Sh, Sl, row, UH * half + 16 * h16, t16);
          planes8(Sh, Sl, row, UH * half + 16 * h16 + 8, t16 + 8);
        }
      } else {
        const float z8[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int g8 = 0; g8 < UH / 8; ++g8) planes8(Sh, Sl, row, UH * half + 8 * g8, z8);
      }
      fence_async_smem();
      tc_fence_before();
      if (__syncthreads_or(!ok)) { ok = false; break; }
      if (issuer) {
        tc_fence_after();
        issue_atom<NG>(tmem + DH, aS, bW, BW, true);
        mma_commit(bar_g);
      }
      if (!mbar_wait(bar_g, ph_g)) ok = false;
      ph_g ^= 1;
      tc_fence_after();
      // GRU cell (App. A) on this thread's units, 8 at a time; h_k to the
      // S planes, the column buffer and the head partials
      const float *tb = tab + (d0 * 3 + d1) * TS + UH * half;
      float z0 = 0.f, z1 = 0.f, z2 = 0.f, z3 = 0.f;
#pragma unroll
      for (int g8 = 0; g8 < UH / 8; ++g8) {
        float gu[8], gr[8], gg[8], hp[8];
        tmem_ld8(gcol + (uint32_t)(8 * g8), gu);
        tmem_ld8(gcol + (uint32_t)(DH + 8 * g8), gr);
        tmem_ld8(gcol + (uint32_t)(2 * DH + 8 * g8), gg);
        if (any) tmem_ld8(hcol + (uint32_t)(8 * g8), hp);
        else {
#pragma unroll
          for (int u = 0; u < 8; ++u) hp[u] = 0.f;
        }
        tmem_wait_ld();
        float h8[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int i = 8 * g8 + u, un = UH * half + i;
          const float uu = sigm_f(gu[u] + tb[i]), rr = sigm_f(gr[u] + tb[DH + i]);
          const float cc = tanh_f(fmaf(rr, gg[u] + sbh[un], tb[2 * DH + i]));
          h8[u] = fmaf(uu, cc - hp[u], hp[u]);
          z0 = fmaf(shead[un], h8[u], z0);
          z1 = fmaf(shead[DH + un], h8[u], z1);
          if (a.cplx) {
            z2 = fmaf(shead[2 * DH + un], h8[u], z2);
            z3 = fmaf(shead[3 * DH + un], h8[u], z3);
          }
        }
        planes8(Sh, Sl, row, UH * half + 8 * g8, h8);
        if (valid) st_global_v8(cb + col * DH + 8 * g8, h8);  // 32-byte aligned: whole sectors
        if (turn) {  // the next site's vertical input is this state
          vs[2 * g8] = valid ? make_float4(h8[0], h8[1], h8[2], h8[3]) : make_float4(0.f, 0.f, 0.f, 0.f);
          vs[2 * g8 + 1] = valid ? make_float4(h8[4], h8[5], h8[6], h8[7]) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
      if (half == 1) {
        zx[row] = make_float4(z0, z1, z2, z3);
      } else {
        zp[0] = z0; zp[1] = z1; zp[2] = z2; zp[3] = z3;
        sgp = s_cur;
        lcp = lc;
      }
      s_prev = s_cur;
      s_cur = k + 1 < N ? r_next ^ ((k + 1 == f1 || k + 1 == f2) ? 1 : 0) : 2;
      s_ver = k_v >= 0 ? r_vnext ^ ((k_v == f1 || k_v == f2) ? 1 : 0) : 2;
    }
    // the last site's row work, then the row's contribution
    tc_fence_before();
    if (__syncthreads_or(!ok)) ok = false;
    if (ok && half == 0) {
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
  }
  cp_async_wait_all();  // no staging copy outlives the kernel (early exit)
  // drain the MMAs before the tensor memory is freed
  if (issuer) {
    mma_commit(smem_u32(&bars[2]));
    if (!mbar_wait(smem_u32(&bars[2]), 0)) ok = false;
  }
  if (!ok) atomicExch(a.err, (int)NQS_ERR_TIMEOUT);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS)
                 : "memory");
}

}  // namespace

bool eloc2d_tc_supported(int dim, int dh) { return dim == 2 && (dh == DH || dh == DH / 2); }

cudaError_t eloc2d_tc_run(const Eloc2dTcArgs &args, int dh, int sm_count, cudaStream_t st) {
  if (dh != DH && dh != DH / 2) return cudaErrorInvalidValue;
  const void *kern = dh == DH ? (const void *)k_eloc2d_tc<DH> : (const void *)k_eloc2d_tc<DH / 2>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)SMEM_BYTES);
  if (e != cudaSuccess) return e;
  const int grid = args.ntiles < sm_count ? args.ntiles : sm_count;
  if (grid <= 0) return cudaSuccess;
  if (dh == DH)
    k_eloc2d_tc<DH><<<grid, THREADS, SMEM_BYTES, st>>>(args);
  else
    k_eloc2d_tc<DH / 2><<<grid, THREADS, SMEM_BYTES, st>>>(args);
  return cudaGetLastError();
}

}  // namespace nqs
