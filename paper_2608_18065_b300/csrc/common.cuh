// common.cuh -- device helpers shared by the kernels of libnqs (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/nqs.h"

#ifndef NQS_PI
#define NQS_PI 3.14159265358979323846
#endif

namespace nqs {

__host__ __device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }
__host__ __device__ __forceinline__ int64_t max64(int64_t a, int64_t b) { return a > b ? a : b; }

// ---------------------------------------------------------------- Philox
// Philox4x32-10 of Salmon et al. (SC'11): ten rounds of two 32x32->64-bit
// multiplies on lanes 0 and 2 with a Weyl-sequence key schedule.
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint32_t hi0 = __umulhi(M0, c[0]), lo0 = M0 * c[0];
    uint32_t hi1 = __umulhi(M1, c[2]), lo1 = M1 * c[2];
    uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    k0 += W0; k1 += W1;
  }
}

// u(seed, step, s, k) in [0,1) with 53 random bits.
__device__ __forceinline__ double uniform53(uint64_t seed, uint64_t step, uint32_t s, uint32_t k) {
  uint32_t c[4] = {k, s, (uint32_t)step, (uint32_t)(step >> 32)};
  philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  uint64_t bits = ((uint64_t)c[1] << 32) | (uint64_t)c[0];
  return (double)(bits >> 11) * 0x1.0p-53;
}

// The top 24 of those 53 bits as an FP32 uniform: u24 <= u53 < u24 + 2^-24,
// so a comparison with a probability differs from the FP64 one only within
// 2^-24 of a tie.
__device__ __forceinline__ float uniform24(uint64_t seed, uint64_t step, uint32_t s, uint32_t k) {
  uint32_t c[4] = {k, s, (uint32_t)step, (uint32_t)(step >> 32)};
  philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  return (float)(c[1] >> 8) * 0x1.0p-24f;
}

// Error-free FP32 accumulation (Knuth's TwoSum): sum + err carries the
// running sum to about twice FP32's precision without the FP64 pipe (64
// times slower than FP32 on this part).
__device__ __forceinline__ void two_add(float &sum, float &err, float x) {
  const float t = sum + x, z = t - sum;
  err += (sum - (t - z)) + (x - z);
  sum = t;
}
// pi s as the pair (p, e) with p + e = pi s to about 2^-46 relative: p the
// rounded product, e its exact error (FMA) plus the error of pi in FP32.
__device__ __forceinline__ void pi_times(float s, float &p, float &e) {
  const float pi_hi = 3.14159274101257324f;        // pi rounded to FP32
  const float pi_lo = -8.742277657347586e-08f;     // pi - pi_hi, rounded to FP32
  p = pi_hi * s;
  e = fmaf(pi_hi, s, -p) + pi_lo * s;
}

// ------------------------------------------------- warp-level BF16 MMA
// Two floats rounded to BF16 and packed, x0 in the low half.
__device__ __forceinline__ uint32_t bf16x2_pack(float x0, float x1) {
  uint32_t u;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(u) : "f"(x1), "f"(x0));
  return u;
}
// hi = bf16(x), lo = bf16(x - hi) of a pair, packed as above.
__device__ __forceinline__ void bf16x2_split(float x0, float x1, uint32_t &hi, uint32_t &lo) {
  hi = bf16x2_pack(x0, x1);
  lo = bf16x2_pack(x0 - __uint_as_float(hi << 16), x1 - __uint_as_float(hi & 0xffff0000u));
}
// D += A B on one warp: m16n8k16, BF16 inputs, FP32 accumulation.
__device__ __forceinline__ void mma_m16n8k16(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                             uint32_t a3, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// --------------------------------------------------------- activations
__device__ __forceinline__ float sigm(float x) { return 1.0f / (1.0f + __expf(-x)); }
__device__ __forceinline__ double sigm(double x) { return 1.0 / (1.0 + exp(-x)); }
__device__ __forceinline__ float tnh(float x) { return tanhf(x); }
__device__ __forceinline__ double tnh(double x) { return tanh(x); }
__device__ __forceinline__ float ex(float x) { return expf(x); }
__device__ __forceinline__ double ex(double x) { return exp(x); }
__device__ __forceinline__ float lg1p(float x) { return log1pf(x); }
__device__ __forceinline__ double lg1p(double x) { return log1p(x); }

// log-softmax of two logits: returns (lp0, lp1) with lp = z - logsumexp(z).
template <typename T>
__device__ __forceinline__ void log_softmax2(T z0, T z1, T &lp0, T &lp1) {
  T d = z1 - z0;
  T ad = d < T(0) ? -d : d;
  T sp = (d > T(0) ? d : T(0)) + lg1p(ex(-ad));  // softplus(d) = log(1+e^d)
  lp0 = -sp;
  lp1 = d - sp;
}

// Softsign and its derivative.
template <typename T> __device__ __forceinline__ T softsign(T y) {
  return y / (T(1) + (y < T(0) ? -y : y));
}

// -------------------------------------------------------- model layout
// Offsets of the parameter blocks in the flat FP64 theta (layout of nqs.h).
struct Layout {
  int N, Lx, Ly, dim, dh, din, cplx, marshall, zmask;
  int64_t U1, U2, Wu, bu, Wr, br, Wh, bh, Win, bin, Uo, co, Up, cp, np;
};

inline Layout make_layout(const nqs_model_desc &m) {
  Layout L;
  L.N = m.Lx * m.Ly; L.Lx = m.Lx; L.Ly = m.Ly; L.dim = m.dim; L.dh = m.dh;
  L.din = m.dim == 2 ? 4 : 2;
  L.cplx = m.cplx; L.marshall = m.marshall; L.zmask = m.zmask;
  const int64_t dh = m.dh, w = dh + L.din;
  int64_t o = 0;
  L.U1 = L.U2 = -1;
  if (m.dim == 2) { L.U1 = o; o += dh * dh; L.U2 = o; o += dh * dh; }
  L.Wu = o; o += dh * w;  L.bu = o; o += dh;
  L.Wr = o; o += dh * w;  L.br = o; o += dh;
  L.Wh = o; o += dh * dh; L.bh = o; o += dh;
  L.Win = o; o += dh * L.din; L.bin = o; o += dh;
  L.Uo = o; o += 2 * dh; L.co = o; o += 2;
  L.Up = L.cp = -1;
  if (m.cplx) { L.Up = o; o += 2 * dh; L.cp = o; o += 2; }
  L.np = o;
  return L;
}

// Packed copy of theta in the recurrence precision T.  Gate index g: 0 = u,
// 1 = r, 2 = candidate (W_h on h', W_in on x).  Interleaved column n = 3a+g.
//   WgT  [dh][3dh]   WgT[k][3a+g] = W_g[a][k]       (forward, K-major)
//   Wg   [3dh][dh]   Wg[3a+g][b]  = W_g[a][b]        (backward)
//   xw   [din][3dh]  xw[d][3a+g]  = W_g[a][dh+d] (g<2), W_in[a][d] (g=2)
//   bias [dh][4]     (b_u, b_r, b_h, b_in)
//   head [4][dh]     (U row 0, U row 1, Uphi row 0, Uphi row 1), hc[4]
//   U12T [2dh][dh]   U12T[k][a] = U1[a][k] | U2[a][k-dh]  (2D forward)
//   U12  [dh][2dh]   U12[a][b]  = U1[a][b] | U2[a][b-dh]  (2D backward)
struct PackOff {
  int64_t WgT, Wg, xw, bias, head, hc, U12T, U12, total;
};

inline PackOff pack_offsets(const Layout &L) {
  PackOff P;
  const int64_t dh = L.dh;
  int64_t o = 0;
  auto al = [](int64_t x) { return (x + 31) & ~int64_t(31); };
  P.WgT = o; o = al(o + dh * 3 * dh);
  P.Wg = o; o = al(o + 3 * dh * dh);
  P.xw = o; o = al(o + L.din * 3 * dh);
  P.bias = o; o = al(o + dh * 4);
  P.head = o; o = al(o + 4 * dh);
  P.hc = o; o = al(o + 4);
  P.U12T = P.U12 = -1;
  if (L.dim == 2) {
    P.U12T = o; o = al(o + 2 * dh * dh);
    P.U12 = o; o = al(o + 2 * dh * dh);
  }
  P.total = o;
  return P;
}

}  // namespace nqs
