// jac2d_tc.cu -- the rows of O (Alg. 1, log-derivative step, App. A) for 2D
// lattices on the tensor cores.
//
// For one row (sample, adjoint seed) of a 2D model (the cell input is
// h' = U1 h_hor + U2 h_ver; the one-hot inputs are the horizontal spin
// x_0, x_1 and the vertical one x_2, x_3) every entry of O is a sum over the
// sites k of an adjoint component times a state component:
//   W_u[a][b] = sum_k dau_k[a] h'_k[b],  W_u x-column d: sum_k dau_k[a] x_d(k),
//   b_u[a] = sum_k dau_k[a]              (W_r, b_r with dar; W_h, b_h with dg),
//   W_in[a][d] = sum_k dac_k[a] x_d(k),  b_in[a] = sum_k dac_k[a],
//   U1[a][b] = sum_k dh'_k[a] h_{k-1}[b] (sites with a left neighbour),
//   U2[a][b] = sum_k dh'_k[a] h_ver(k)[b] (sites with a neighbour above),
//   U[o][b] = sum_k dz_k[o] h_k[b],      c[o] = sum_k dz_k[o]  (and the phase head).
// A row is two work items, each a set of products D = A B^T over K = sites:
//   gates: A = [dau; dar; dg] (3 d_h rows, tiles of 128), B = [h'; 1; x_0..x_3]
//   rest:  A tile 0 = dh' with B = [h_hor; h_ver], tile 1 = dac with
//          B = [1; x_0..x_3], tile 2 = dz (4 rows) with B = [h_k; 1].
// The adjoints and h' come from the reverse sweep's records, the states
// from the cache, the one-hots from the spins.  Each FP32 value is split
// into BF16 hi + lo, staged in the non-swizzled K-major layout 16 sites at a
// time (two stages; the next chunk's loads are in flight while the current
// one is multiplied) and accumulated in tensor memory as hi.hi + hi.lo +
// lo.hi (FP32), the same three products as the Gram; the one-hots and ones
// are exact.  The accumulators go back through shared memory, 128 columns at
// a time, so that the row of O is written coalesced.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "nqs.h"
#include "jac_tc.h"
#include "tc_common.cuh"

namespace nqs {
namespace {

constexpr int J2_THREADS = 256;
constexpr int J2_KC = 16;          // sites per staged chunk (one K step)
constexpr int J2_ASUB = 16 * 256;  // one K = 16 block of a 128-row tile (bytes)
constexpr int J2_TRS = 128 + 1;    // transpose stride (floats)

template <int DH> struct J2 {
  static constexpr int TG = (3 * DH + 127) / 128;      // A tiles of the gate item
  static constexpr int NG = DH + 16;                   // its B rows: h', 1, x_0..x_3, zeros
  // rest item: B rows [h_hor; h_ver] (2 dh), [1; x] (16), [h_k; 1] (dh + 16)
  static constexpr int NU0 = 2 * DH, NU1 = 16, NU2 = DH + 16;
  static constexpr int BROWS = NU0 + NU1 + NU2;        // >= NG
  static constexpr int BSUB = (BROWS / 8) * 256;       // one plane of B (bytes)
  static constexpr int A_BYTES = 2 * 3 * J2_ASUB;      // hi, lo planes of three tiles
  static constexpr int STAGE = (A_BYTES + 2 * BSUB + 1023) / 1024 * 1024;
  static constexpr int COLS = TG * NG > BROWS ? TG * NG : BROWS;
  static constexpr int TCOLS = COLS > 256 ? 512 : 256;
  static constexpr size_t SMEM = 1024 + 2 * (size_t)STAGE + sizeof(float) * 128 * J2_TRS + 64;
  static_assert(TG <= 3 && COLS <= 512 && NU0 <= 256, "MMA shapes, tensor memory");
  static_assert(SMEM <= 227 * 1024, "one CTA per SM");
};

// BF16 hi and lo of (x0, x1) as packed pairs (x0 in the low half)
__device__ __forceinline__ void split2(float x0, float x1, uint32_t &hi, uint32_t &lo) {
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(hi) : "f"(x1), "f"(x0));
  const float r0 = x0 - __uint_as_float(hi << 16), r1 = x1 - __uint_as_float(hi & 0xffff0000u);
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(lo) : "f"(r1), "f"(r0));
}

// rows r .. r + 3 of a K-major block at sites kk, kk + 1 (kk even): the
// values of site kk in v0, of site kk + 1 in v1
__device__ __forceinline__ void put_quad(unsigned char *hi, unsigned char *lo, int r, int kk,
                                         float4 v0, float4 v1) {
  const float a0[4] = {v0.x, v0.y, v0.z, v0.w}, a1[4] = {v1.x, v1.y, v1.z, v1.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    uint32_t h, l;
    split2(a0[i], a1[i], h, l);
    const uint32_t o = kmaj_off(r + i, kk & 15);
    *reinterpret_cast<uint32_t *>(hi + o) = h;
    *reinterpret_cast<uint32_t *>(lo + o) = l;
  }
}

// an exact value (0 or 1): lo plane zero
__device__ __forceinline__ void put_exact(unsigned char *hi, unsigned char *lo, int r, int kk,
                                          float v) {
  const uint32_t o = kmaj_off(r, kk & 15);
  *reinterpret_cast<__nv_bfloat16 *>(hi + o) = __float2bfloat16_rn(v);
  *reinterpret_cast<__nv_bfloat16 *>(lo + o) = __float2bfloat16_rn(0.f);
}

// Work units of a chunk: (site pair, four consecutive columns) of a column
// range of C values per site, the site pair fastest over the threads (so that
// a warp's stores of one row quad fall in eight banks, not two); unit counts
// per thread.
template <int C> struct Units {
  static constexpr int N = 8 * (C / 4), PER = (N + J2_THREADS - 1) / J2_THREADS;
  static_assert(C % 4 == 0, "column quads");
};

// One chunk (sites 16 c .. 16 c + 15) of an item in registers: per work
// unit the four columns at the two sites (coalesced 16-byte loads; zero past
// the chain), the one-hot word of one site, one head adjoint.
template <int DH> struct Chunk2 {
  static constexpr int UA = Units<3 * DH>::PER > Units<2 * DH>::PER ? Units<3 * DH>::PER : Units<2 * DH>::PER;
  static constexpr int UB = Units<3 * DH>::PER;
  float4 a[UA][2];  // gates: dau | dar | dg;  rest: dh' | dac
  float4 b[UB][2];  // gates: h';  rest: h_hor | h_ver | h_k
  float z;          // rest: dz of (site, component) tid / 4, tid % 4
  int x;            // one-hot bits of site tid / 16 (bit 4: inside the chain)
};

template <int DH>
__device__ __forceinline__ void fetch2(const Jac2dTcArgs &a, Chunk2<DH> &r, int64_t row, int pass,
                                       int c, int tid) {
  const int N = a.N, Lx = a.Lx, k0 = c * J2_KC;
  const int64_t s = row % a.ns;
  const float *arow = a.adj + row * (int64_t)N * a.adjw;
  const float *hrow = a.hcache + s * (int64_t)N * DH;
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  auto rec = [&](int k, int off) {
    return k < N ? __ldcg(reinterpret_cast<const float4 *>(arow + (int64_t)k * a.adjw + off)) : zero;
  };
  auto hst = [&](int k, int b) {
    return k >= 0 && k < N ? __ldcg(reinterpret_cast<const float4 *>(hrow + (int64_t)k * DH + b)) : zero;
  };
  if (pass == 0) {
    using UA = Units<3 * DH>;
#pragma unroll
    for (int q = 0; q < UA::PER; ++q) {  // dau | dar | dg: record columns 0 .. 3 dh
      const int e = tid + q * J2_THREADS, kp = e & 7, m = 4 * (e >> 3);
      const int k = k0 + 2 * kp;
      r.a[q][0] = e < UA::N ? rec(k, m) : zero;
      r.a[q][1] = e < UA::N ? rec(k + 1, m) : zero;
    }
    using UB = Units<DH>;
#pragma unroll
    for (int q = 0; q < UB::PER; ++q) {  // h'
      const int e = tid + q * J2_THREADS, kp = e & 7, n = 4 * (e >> 3);
      const int k = k0 + 2 * kp;
      r.b[q][0] = e < UB::N ? rec(k, a.ohp + n) : zero;
      r.b[q][1] = e < UB::N ? rec(k + 1, a.ohp + n) : zero;
    }
  } else {
    using UA = Units<2 * DH>;
#pragma unroll
    for (int q = 0; q < UA::PER; ++q) {  // dh' | dac
      const int e = tid + q * J2_THREADS, kp = e & 7, m = 4 * (e >> 3);
      const int k = k0 + 2 * kp, off = m < DH ? a.odhp + m : 3 * DH + (m - DH);
      r.a[q][0] = e < UA::N ? rec(k, off) : zero;
      r.a[q][1] = e < UA::N ? rec(k + 1, off) : zero;
    }
    using UB = Units<3 * DH>;
#pragma unroll
    for (int q = 0; q < UB::PER; ++q) {  // h_hor | h_ver | h_k
      const int e = tid + q * J2_THREADS, kp = e & 7, n = 4 * (e >> 3);
      const int part = n / DH, b = n - part * DH;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int k = k0 + 2 * kp + h;
        int src = -1;
        if (e < UB::N && k < N) {
          const int m = k % Lx;
          src = part == 0 ? (m != 0 ? k - 1 : -1) : part == 1 ? (k >= Lx ? k - 2 * m - 1 : -1) : k;
        }
        r.b[q][h] = hst(src, b);
      }
    }
    r.z = 0.f;
    if (tid < 4 * J2_KC) {
      const int k = k0 + (tid >> 2);
      r.z = k < N ? __ldcg(arow + (int64_t)k * a.adjw + a.odz + (tid & 3)) : 0.f;
    }
  }
  r.x = 0;
  if ((tid & 15) == 0) {  // one-hot word of site tid / 16
    const int k = k0 + (tid >> 4);
    if (k < N) {
      const uint8_t *sp = a.spins + s * (int64_t)N;
      const int m = k % Lx;
      int x = 16;
      if (m != 0) x |= 1 << (int)__ldcg(sp + k - 1);
      if (k >= Lx) x |= 1 << (2 + (int)__ldcg(sp + k - 2 * m - 1));
      r.x = x;
    }
  }
}

template <int DH>
__device__ __forceinline__ void store2(const Chunk2<DH> &r, unsigned char *stage, int pass, int tid) {
  using S = J2<DH>;
  unsigned char *bh = stage + S::A_BYTES, *bl = bh + S::BSUB;
  // the one-hot word of each site goes from its thread to the whole warp set
  const int xk = __shfl_sync(0xffffffffu, r.x, (tid & 16));  // site tid / 16 (two sites per warp)
  const int kk = tid >> 4, j = tid & 15;
  const float sv = j == 0 ? (float)((xk >> 4) & 1) : (j <= 4 ? (float)((xk >> (j - 1)) & 1) : 0.f);
  if (pass == 0) {
    using UA = Units<3 * DH>;
#pragma unroll
    for (int q = 0; q < UA::PER; ++q) {
      const int e = tid + q * J2_THREADS, kp = e & 7, m = 4 * (e >> 3);
      const int t = m >> 7;
      if (e < UA::N)
        put_quad(stage + t * J2_ASUB, stage + (3 + t) * J2_ASUB, m & 127, 2 * kp, r.a[q][0], r.a[q][1]);
    }
    using UB = Units<DH>;
#pragma unroll
    for (int q = 0; q < UB::PER; ++q) {
      const int e = tid + q * J2_THREADS, kp = e & 7, n = 4 * (e >> 3);
      if (e < UB::N) put_quad(bh, bl, n, 2 * kp, r.b[q][0], r.b[q][1]);
    }
    put_exact(bh, bl, DH + j, kk, sv);  // [1, x_0 .. x_3, 0 ..]
  } else {
    using UA = Units<2 * DH>;
#pragma unroll
    for (int q = 0; q < UA::PER; ++q) {
      const int e = tid + q * J2_THREADS, kp = e & 7, m = 4 * (e >> 3);
      const int t = m < DH ? 0 : 1, rr = m < DH ? m : m - DH;
      if (e < UA::N)
        put_quad(stage + t * J2_ASUB, stage + (3 + t) * J2_ASUB, rr, 2 * kp, r.a[q][0], r.a[q][1]);
    }
    if (tid < 4 * J2_KC) {  // dz into rows 0..3 of tile 2
      const __nv_bfloat16 h = __float2bfloat16_rn(r.z);
      const __nv_bfloat16 l = __float2bfloat16_rn(r.z - __bfloat162float(h));
      const uint32_t o = kmaj_off(tid & 3, tid >> 2);
      *reinterpret_cast<__nv_bfloat16 *>(stage + 2 * J2_ASUB + o) = h;
      *reinterpret_cast<__nv_bfloat16 *>(stage + 5 * J2_ASUB + o) = l;
    }
    using UB = Units<3 * DH>;
#pragma unroll
    for (int q = 0; q < UB::PER; ++q) {
      const int e = tid + q * J2_THREADS, kp = e & 7, n = 4 * (e >> 3);
      // rows: h_hor, h_ver at 0 .. 2 dh; h_k after the 16 one-hot rows
      const int rr = n < 2 * DH ? n : n + S::NU1;
      if (e < UB::N) put_quad(bh, bl, rr, 2 * kp, r.b[q][0], r.b[q][1]);
    }
    put_exact(bh, bl, S::NU0 + j, kk, sv);                                   // [1; x]
    put_exact(bh, bl, S::NU0 + S::NU1 + DH + j, kk, j == 0 ? sv : 0.f);     // h_k's [1]
  }
}

// Row r of tile t of an item into the row of O: its nc accumulator entries
// from column cb on (a block of the transpose buffer at v), one warp.
template <int DH>
__device__ __forceinline__ void write_row2(const Jac2dTcArgs &a, float *orow, int pass, int t,
                                           int r, int cb, int nc, const float *v, int lane) {
  using S = J2<DH>;
  const int w = DH + 4;  // row length of W_u and W_r: h part, then the four input columns
  if (pass == 0) {
    const int m = 128 * t + r;
    if (m >= 3 * DH) return;
    const int blk = m / DH, q = m - blk * DH;
    float *hb = orow + (blk == 0 ? a.Wu + (int64_t)q * w : blk == 1 ? a.Wr + (int64_t)q * w
                                                                  : a.Wh + (int64_t)q * DH);
    float *bias = orow + (blk == 0 ? a.bu : blk == 1 ? a.br : a.bh) + q;
    for (int cc = lane; cc < nc; cc += 32) {
      const int c = cb + cc;
      if (c < DH) hb[c] = v[cc];
      else if (c == DH) *bias = v[cc];
      else if (c <= DH + 4 && blk < 2) hb[c - 1] = v[cc];  // x-column c - DH - 1 at DH + (c - DH - 1)
    }
  } else if (t == 0) {
    if (r >= DH) return;
    float *u1 = orow + a.U1 + (int64_t)r * DH, *u2 = orow + a.U2 + (int64_t)r * DH - DH;
    for (int cc = lane; cc < nc; cc += 32) {
      const int c = cb + cc;
      if (c < DH) u1[c] = v[cc];
      else u2[c] = v[cc];
    }
  } else if (t == 1) {
    if (r >= DH) return;
    if (lane == 0) orow[a.bin + r] = v[0];
    if (lane >= 1 && lane <= 4) orow[a.Win + (int64_t)r * 4 + (lane - 1)] = v[lane];
  } else {
    if (r >= (a.cplx ? 4 : 2)) return;
    float *hd = orow + (r < 2 ? a.Uo + (int64_t)r * DH : a.Up + (int64_t)(r - 2) * DH);
    for (int cc = lane; cc < nc; cc += 32) {
      const int c = cb + cc;
      if (c < DH) hd[c] = v[cc];
      else if (c == DH) orow[r < 2 ? a.co + r : a.cp + (r - 2)] = v[cc];
    }
  }
  (void)S::NU0;
}

template <int DH>
__global__ void __launch_bounds__(J2_THREADS, 1) k_jac2d_tc(const Jac2dTcArgs a) {
  using S = J2<DH>;
  extern __shared__ __align__(1024) unsigned char j2raw[];
  unsigned char *sm = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(j2raw) + 1023) & ~uintptr_t(1023));
  unsigned char *stg[2] = {sm, sm + S::STAGE};
  float *tr = reinterpret_cast<float *>(sm + 2 * S::STAGE);           // [128][J2_TRS]
  uint64_t *bars = reinterpret_cast<uint64_t *>(tr + 128 * J2_TRS);   // products done, per stage
  uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 2);
  __shared__ int flag_s;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // rows of a tile that no item writes feed only accumulator rows that are
  // never read; they start (and stay) finite
  for (int e = tid; e < 2 * S::STAGE / 16; e += J2_THREADS)
    reinterpret_cast<uint4 *>(sm)[e] = make_uint4(0u, 0u, 0u, 0u);
  if (tid == 0) {
    mbar_init(smem_u32(&bars[0]), 1);
    mbar_init(smem_u32(&bars[1]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tslot)),
                 "r"(S::TCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  constexpr uint32_t id_g = idesc_bf16(128, S::NG), id_u0 = idesc_bf16(128, S::NU0),
                     id_u1 = idesc_bf16(128, S::NU1), id_u2 = idesc_bf16(128, S::NU2);
  const int NC = (a.N + J2_KC - 1) / J2_KC;
  const int64_t nitems = 2 * a.nrows;
  uint32_t ph[2] = {0u, 0u};
  int pending[2] = {0, 0};  // commits on each stage's barrier not yet waited for
  bool ok = true;

  auto drain = [&](int st) -> bool {
    if (tid == 0) flag_s = mbar_wait(smem_u32(&bars[st]), ph[st]) ? 0 : 1;
    ph[st] ^= 1u;
    pending[st] = 0;
    __syncthreads();
    return flag_s == 0;
  };

  // This CTA's (item, chunk) sequence, q = 0 .. Q - 1; the loads of chunk
  // q + 2 are issued as soon as chunk q is staged (two chunks in flight,
  // across item boundaries), into the register set chunk q used.
  const int64_t nmy = (int64_t)blockIdx.x < nitems ? (nitems - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int64_t Q = nmy * NC;
  auto fetch_q = [&](Chunk2<DH> &r, int64_t q) {
    const int64_t it = blockIdx.x + (q / NC) * gridDim.x;
    fetch2<DH>(a, r, it >> 1, (int)(it & 1), (int)(q % NC), tid);
  };
  // the accumulators of an item into its row of O
  auto epilogue = [&](int64_t row, int pass) {
    float *orow = a.O + row * a.np;
    const int ntile = pass == 0 ? S::TG : 3;
    for (int t = 0; t < ntile; ++t) {
      const int coff = pass == 0 ? t * S::NG : (t == 0 ? 0 : t == 1 ? S::NU0 : S::NU0 + S::NU1);
      const int ncol = pass == 0 ? S::NG : (t == 0 ? S::NU0 : t == 1 ? S::NU1 : S::NU2);
      for (int cb = 0; cb < ncol; cb += 128) {
        const int nc = ncol - cb < 128 ? ncol - cb : 128;  // a multiple of 16
        {  // warp w: tensor-memory lanes 32 (w % 4) .., columns of half w / 4
          const int r = (warp & 3) * 32 + lane;
          for (int cc = (warp >> 2) * 16; cc < nc; cc += 32) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(coff + cb + cc), v);
            tmem_wait_ld();
#pragma unroll
            for (int jj = 0; jj < 16; ++jj) tr[r * J2_TRS + cc + jj] = v[jj];
          }
        }
        __syncthreads();
        for (int r = warp; r < 128; r += J2_THREADS / 32)
          write_row2<DH>(a, orow, pass, t, r, cb, nc, tr + r * J2_TRS, lane);
        __syncthreads();
      }
    }
  };
  auto body = [&](int64_t q, Chunk2<DH> &r) -> bool {
    const int c = (int)(q % NC);
    const int64_t item = blockIdx.x + (q / NC) * gridDim.x;
    const int64_t row = item >> 1;
    const int pass = (int)(item & 1), st = (int)(q & 1);
    if (pending[st] && !drain(st)) return false;
    store2<DH>(r, stg[st], pass, tid);
    if (q + 2 < Q) fetch_q(r, q + 2);
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t base = smem_u32(stg[st]), bb = base + S::A_BYTES;
      const uint32_t acc = c == 0 ? 0u : 1u;
      auto mma3 = [&](int t, uint32_t d, uint32_t brow, uint32_t id) {
        const uint64_t ah = kmaj_desc(base + t * J2_ASUB), al = kmaj_desc(base + (3 + t) * J2_ASUB);
        const uint64_t bh = kmaj_desc(bb + (brow / 8) * 256), bl = kmaj_desc(bb + S::BSUB + (brow / 8) * 256);
        mma_bf16(d, ah, bh, id, acc);
        mma_bf16(d, ah, bl, id, 1u);
        mma_bf16(d, al, bh, id, 1u);
      };
      if (pass == 0) {
#pragma unroll
        for (int t = 0; t < S::TG; ++t) mma3(t, tmem + (uint32_t)(t * S::NG), 0u, id_g);
      } else {
        mma3(0, tmem, 0u, id_u0);
        mma3(1, tmem + (uint32_t)S::NU0, (uint32_t)S::NU0, id_u1);
        mma3(2, tmem + (uint32_t)(S::NU0 + S::NU1), (uint32_t)(S::NU0 + S::NU1), id_u2);
      }
      mma_commit(smem_u32(&bars[st]));
    }
    pending[st] = 1;
    if (c == NC - 1) {  // the item's products are complete once both stages' commits are
      if ((pending[0] && !drain(0)) || (pending[1] && !drain(1))) return false;
      tc_fence_after();
      epilogue(row, pass);
      tc_fence_before();  // the next item's first products overwrite the accumulators
    }
    return true;
  };
  Chunk2<DH> cr0, cr1;
  if (Q > 0) fetch_q(cr0, 0);
  if (Q > 1) fetch_q(cr1, 1);
  for (int64_t q = 0; q < Q && ok; q += 2) {
    if (!body(q, cr0)) { ok = false; break; }
    if (q + 1 < Q && !body(q + 1, cr1)) { ok = false; break; }
  }
  if (!ok) {
    if (tid == 0) atomicCAS(a.err, 0, (int)NQS_ERR_TIMEOUT);
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
                 "r"(S::TCOLS)
                 : "memory");
}

template <int DH>
cudaError_t run2(const Jac2dTcArgs &args, int sm_count, cudaStream_t st) {
  using S = J2<DH>;
  cudaError_t e = cudaFuncSetAttribute(k_jac2d_tc<DH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)S::SMEM);
  if (e != cudaSuccess) return e;
  const int64_t items = 2 * args.nrows;
  const int grid = (int)(items < sm_count ? items : sm_count);
  k_jac2d_tc<DH><<<grid, J2_THREADS, S::SMEM, st>>>(args);
  return cudaGetLastError();
}

}  // namespace

bool jac2d_tc_supported(int dim, int dh) {
  return dim == 2 && (dh == 32 || dh == 64 || dh == 96 || dh == 128);
}

cudaError_t jac2d_tc_run(const Jac2dTcArgs &args, int sm_count, cudaStream_t st) {
  if (args.nrows <= 0) return cudaSuccess;
  switch (args.dh) {
    case 32: return run2<32>(args, sm_count, st);
    case 64: return run2<64>(args, sm_count, st);
    case 96: return run2<96>(args, sm_count, st);
    case 128: return run2<128>(args, sm_count, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace nqs
