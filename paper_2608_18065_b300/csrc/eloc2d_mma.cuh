// eloc2d_mma.cuh -- connected-configuration engine for 2D lattices, FP32
// state, hidden size 64, with the two per-site products on warp-level MMAs.
//
// A connected configuration sigma' of sample sigma first differs from it at
// site kstart of the zig-zag path (Sec. II.B); log psi(sigma') - log
// psi(sigma) is recomputed from the sample's cached h_{kstart-1} and the
// cached vertical neighbours (Sec. II.C).  Per site and tile of 64 rows the
// 2D cell (App. A) has two dependent products,
//   h'    = U1 h_hor + U2 h_ver      [64 x 128] x [128 x 64]
//   gates = [W_u; W_r; W_h] h'       [64 x 64]  x [64 x 192]
// which run as mma.sync m16n8k16 on BF16 hi/lo splits of both operands
// (hi.hi + hi.lo + lo.hi, FP32 accumulation).  Warp w owns hidden units
// 8w .. 8w + 7: its B fragments ([U1 | U2] and the three gate columns of
// those units, split once per CTA) stay in registers, and lane (g, t) =
// (lane / 4, lane % 4) finishes with h' and the three gate pre-activations
// of units 8w + 2t, 8w + 2t + 1 for rows 16m + g + 8h (m = 0..3, h = 0..1),
// which is exactly what its GRU update needs.  The states that feed the
// next product are split into BF16 hi/lo planes once, by their owner, and
// read back with ldmatrix.  Output heads (FP32) are reduced over the lanes
// of a warp with shuffles and over the warps through shared memory; row
// 8w + g's log-softmax, mask and log-amplitude sums run on lane (g, 0) of
// warp w.
#pragma once
#include "recurrence.cuh"

namespace nqs {

namespace e2d {
constexpr int DH = 64, C3 = 3 * DH, R = 64, NW = 8, NTH = 32 * NW;
constexpr int LDW = DH / 2 + 4;  // 32-bit words per plane row (ldmatrix rows on distinct banks)
constexpr int PLANE = R * LDW;   // words per BF16x2 plane
// float offsets of the small blocks, then the planes
constexpr int F_XW = 0, F_BIAS = F_XW + 4 * C3, F_HEAD = F_BIAS + DH * 4, F_HC = F_HEAD + 4 * DH;
constexpr int F_Z = F_HC + 8, F_END = F_Z + 4 * NW * R;
static_assert(F_END % 4 == 0, "planes start on a 16-byte boundary");

__device__ __forceinline__ float sigm_fast(float x) { return __fdividef(1.0f, 1.0f + __expf(-x)); }
__device__ __forceinline__ float tanh_fast(float x) { return 2.0f * sigm_fast(2.0f * x) - 1.0f; }

// Four 8x8 BF16 matrices from shared memory: the A fragment of one
// m16n8k16 tile when lane L points at row (L & 7) + 8 ((L >> 3) & 1), word
// column 4 (L >> 4) of the tile.
__device__ __forceinline__ void ldsm4(const uint32_t *p, uint32_t (&r)[4]) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a)
               : "memory");
}

// Vertical-neighbour states of site k for a lane's rows 16m + g + 8h and
// units ua, ua + 1: recomputed ones (ver >= kstart) from the CTA's column
// buffer, the others from the sample's cache; zero without a neighbour.
__device__ __forceinline__ void fetch_ver(const FwdArgs<float> &A, int k, int kstart, int g, int ua,
                                          const int (&so)[8], float2 (&vv)[8]) {
  const int Lx = A.Lx, j = k / Lx, m = k - j * Lx;
  const int col = (j & 1) ? (Lx - 1 - m) : m;
  const int ver = k >= Lx ? k - 2 * m - 1 : -1;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int rho = 16 * (i >> 1) + g + 8 * (i & 1);
    vv[i] = make_float2(0.f, 0.f);
    if (ver >= 0 && so[i] >= 0) {
      const float *src = ver >= kstart
          ? A.colbuf + (((int64_t)blockIdx.x * R + rho) * Lx + col) * DH + ua
          : A.hcache + ((int64_t)so[i] * A.N + ver) * DH + ua;
      vv[i] = *reinterpret_cast<const float2 *>(src);
    }
  }
}
}  // namespace e2d

inline size_t eloc2d_mma_smem_bytes(int N) {
  const size_t NP = (size_t)((N + 15) & ~15);
  const size_t b = (size_t)e2d::F_END * 4 + (size_t)6 * e2d::PLANE * 4 + e2d::R * NP + e2d::R * 4;
  return (b + 127) & ~size_t(127);
}

template <int DHX>
__global__ void __launch_bounds__(e2d::NTH, 1) k_eloc2d_mma(const FwdArgs<float> A) {
  static_assert(DHX == e2d::DH, "hidden size 64");
  using namespace e2d;
  extern __shared__ __align__(16) unsigned char smraw[];
  float *sf = reinterpret_cast<float *>(smraw);
  float *sxw = sf + F_XW;      // [4][C3]: input rows (horizontal 0/1, vertical 2/3)
  float *sbias = sf + F_BIAS;  // [DH][4]: b_u, b_r, b_h, b_in
  float *shead = sf + F_HEAD;  // [4][DH]
  float *shc = sf + F_HC;      // [4]
  float *sz = sf + F_Z;        // [4 heads][NW][R]: per-warp head partials
  uint32_t *pl = reinterpret_cast<uint32_t *>(sf + F_END);
  uint32_t *sHh = pl, *sHl = pl + PLANE;              // h_{k-1}
  uint32_t *sVh = pl + 2 * PLANE, *sVl = pl + 3 * PLANE;  // vertical neighbour
  uint32_t *sPh = pl + 4 * PLANE, *sPl = pl + 5 * PLANE;  // h'
  const int N = A.N, Lx = A.Lx, NP = (N + 15) & ~15;
  uint8_t *ssp = reinterpret_cast<uint8_t *>(pl + 6 * PLANE);
  int *srow = reinterpret_cast<int *>(ssp + R * NP);

  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
  const int ua = 8 * w + 2 * t;  // first of the lane's two units
  const int kpo = 4 * w + t;     // its word in a plane row
  // ldmatrix lane offset inside a 16-row tile
  const int lrow = (lane & 7) + 8 * ((lane >> 3) & 1), lcol = 4 * (lane >> 4);

  // packed-weight offsets (the library's pack layout for hidden size 64, 2D)
  const float *p = A.pack;
  auto al = [](int x) { return (x + 31) & ~31; };
  const int oWgT = 0, oWg = al(DH * C3), oxw = al(oWg + C3 * DH);
  const int obias = al(oxw + 4 * C3), ohead = al(obias + DH * 4), ohc = al(ohead + 4 * DH);
  const int oU12T = al(ohc + 4);
  for (int e = tid; e < 4 * C3; e += NTH) sxw[e] = p[oxw + e];
  for (int e = tid; e < DH * 4; e += NTH) sbias[e] = p[obias + e];
  for (int e = tid; e < 4 * DH; e += NTH) shead[e] = p[ohead + e];
  if (tid < 4) shc[tid] = p[ohc + tid];
  // B fragments: gate j of unit 8w + g is column 3 (8w + g) + j of W^T;
  // unit 8w + g is column 8w + g of [U1 | U2]^T
  uint32_t bgh[24], bgl[24], buh[16], bul[16];
#pragma unroll
  for (int st = 0; st < 4; ++st)
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        const int k = 16 * st + 2 * t + 8 * hh, n = 3 * (8 * w + g) + j;
        bf16x2_split(__ldg(p + oWgT + k * C3 + n), __ldg(p + oWgT + (k + 1) * C3 + n),
                     bgh[(st * 3 + j) * 2 + hh], bgl[(st * 3 + j) * 2 + hh]);
      }
#pragma unroll
  for (int st = 0; st < 8; ++st)
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
      const int k = 16 * st + 2 * t + 8 * hh, n = 8 * w + g;
      bf16x2_split(__ldg(p + oU12T + k * DH + n), __ldg(p + oU12T + (k + 1) * DH + n),
                   buh[2 * st + hh], bul[2 * st + hh]);
    }

  const int rr = 8 * w + g;  // row of this lane's scalar work (t == 0)
  const bool rowt = t == 0;

  for (int tile = blockIdx.x; tile < A.ntiles; tile += gridDim.x) {
    const int op = tile / A.tiles_per_op;
    const int base = (tile - op * A.tiles_per_op) * R;
    const int cnt = A.item_cnt[op];
    if (base >= cnt) continue;  // uniform over the CTA
    const int f1 = A.op_f[4 * op + 0], f2 = A.op_f[4 * op + 1], kstart = A.op_f[4 * op + 2];
    __syncthreads();  // the previous tile is done with shared memory
    if (tid < R) srow[tid] = base + tid < cnt ? A.item_s[(int64_t)op * A.nrows + base + tid] : -1;
    __syncthreads();
    for (int e = tid; e < R * N; e += NTH) {
      const int r = e / N, k = e - r * N, s = srow[r];
      uint8_t v = 0;
      if (s >= 0) {
        v = A.spins[(int64_t)s * N + k];
        if (k == f1 || k == f2) v ^= 1;
      }
      ssp[r * NP + k] = v;
    }
    int so[8];  // samples of the lane's rows 16m + g + 8h, index 2m + h
#pragma unroll
    for (int i = 0; i < 8; ++i) so[i] = srow[16 * (i >> 1) + g + 8 * (i & 1)];
    // h_{kstart-1} of the lane's rows and units, split into the h planes
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int rho = 16 * (i >> 1) + g + 8 * (i & 1);
      float2 v = make_float2(0.f, 0.f);
      if (kstart > 0 && so[i] >= 0)
        v = *reinterpret_cast<const float2 *>(A.hcache + ((int64_t)so[i] * N + kstart - 1) * DH + ua);
      uint32_t hi, lo;
      bf16x2_split(v.x, v.y, hi, lo);
      sHh[rho * LDW + kpo] = hi;
      sHl[rho * LDW + kpo] = lo;
    }
    float2 vv[8];  // vertical-neighbour states of the next site to run
    e2d::fetch_ver(A, kstart, kstart, g, ua, so, vv);
    __syncthreads();  // spins and h planes written
    const int rs = srow[rr];
    float sre = 0.f, cre = 0.f, sim = 0.f, cim = 0.f;
    bool dead = false;
    int n_up = 0, n_dn = 0;
    if (rowt && rs >= 0)
      for (int k = 0; k < kstart; ++k) {
        if (ssp[rr * NP + k] == 0) ++n_up; else ++n_dn;
      }

    for (int k = kstart; k < N; ++k) {
      const int j = k / Lx, m_ = k - j * Lx;
      const int col = (j & 1) ? (Lx - 1 - m_) : m_;
      const bool hor_ok = m_ != 0;
      const int ver = k >= Lx ? k - 2 * m_ - 1 : -1;
      // vertical planes of this site
      if (ver >= 0) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int rho = 16 * (i >> 1) + g + 8 * (i & 1);
          uint32_t hi, lo;
          bf16x2_split(vv[i].x, vv[i].y, hi, lo);
          sVh[rho * LDW + kpo] = hi;
          sVl[rho * LDW + kpo] = lo;
        }
      }
      // next site's vertical states in flight during this site, unless they
      // are this site's own results (the first site of a lattice row sits
      // above the last site of the previous one)
      bool turn = false;
      if (k + 1 < N) {
        if ((k + 1) % Lx == 0) turn = true;
        else e2d::fetch_ver(A, k + 1, kstart, g, ua, so, vv);
      }
      float lc0 = 0.f, lc1 = 0.f;  // the sample's log-conditional terms of site k
      if (rowt && rs >= 0) {
        const float *lc = A.lccache + ((int64_t)rs * N + k) * 2;
        lc0 = lc[0];
        lc1 = lc[1];
      }
      __syncthreads();  // h and vertical planes complete

      // h' = U1 h_hor + U2 h_ver
      float cp[4][4];
#pragma unroll
      for (int m = 0; m < 4; ++m) cp[m][0] = cp[m][1] = cp[m][2] = cp[m][3] = 0.f;
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        if (half == 0 ? !hor_ok : ver < 0) continue;
        const uint32_t *Ph = half ? sVh : sHh, *Pl = half ? sVl : sHl;
#pragma unroll
        for (int st = 0; st < 4; ++st) {
          const int b = 2 * (4 * half + st);
          uint32_t ah[4][4], alo[4][4];
#pragma unroll
          for (int m = 0; m < 4; ++m) {
            const int off = (16 * m + lrow) * LDW + 8 * st + lcol;
            ldsm4(Ph + off, ah[m]);
            ldsm4(Pl + off, alo[m]);
          }
#pragma unroll
          for (int m = 0; m < 4; ++m)
            mma_m16n8k16(cp[m], ah[m][0], ah[m][1], ah[m][2], ah[m][3], buh[b], buh[b + 1]);
#pragma unroll
          for (int m = 0; m < 4; ++m)
            mma_m16n8k16(cp[m], ah[m][0], ah[m][1], ah[m][2], ah[m][3], bul[b], bul[b + 1]);
#pragma unroll
          for (int m = 0; m < 4; ++m)
            mma_m16n8k16(cp[m], alo[m][0], alo[m][1], alo[m][2], alo[m][3], buh[b], buh[b + 1]);
        }
      }
      // h' planes: cp[m][2h + uu] is row 16m + g + 8h, unit ua + uu
#pragma unroll
      for (int m = 0; m < 4; ++m)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int rho = 16 * m + g + 8 * h;
          uint32_t hi, lo;
          bf16x2_split(cp[m][2 * h], cp[m][2 * h + 1], hi, lo);
          sPh[rho * LDW + kpo] = hi;
          sPl[rho * LDW + kpo] = lo;
        }
      __syncthreads();  // h' planes complete

      // gate pre-activations [W_u; W_r; W_h] h'
      float cg[4][3][4];
#pragma unroll
      for (int m = 0; m < 4; ++m)
#pragma unroll
        for (int jj = 0; jj < 3; ++jj) cg[m][jj][0] = cg[m][jj][1] = cg[m][jj][2] = cg[m][jj][3] = 0.f;
#pragma unroll
      for (int st = 0; st < 4; ++st) {
        uint32_t ah[4][4], alo[4][4];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          const int off = (16 * m + lrow) * LDW + 8 * st + lcol;
          ldsm4(sPh + off, ah[m]);
          ldsm4(sPl + off, alo[m]);
        }
#pragma unroll
        for (int jj = 0; jj < 3; ++jj) {
          const int b = (st * 3 + jj) * 2;
#pragma unroll
          for (int m = 0; m < 4; ++m)
            mma_m16n8k16(cg[m][jj], ah[m][0], ah[m][1], ah[m][2], ah[m][3], bgh[b], bgh[b + 1]);
#pragma unroll
          for (int m = 0; m < 4; ++m)
            mma_m16n8k16(cg[m][jj], ah[m][0], ah[m][1], ah[m][2], ah[m][3], bgl[b], bgl[b + 1]);
#pragma unroll
          for (int m = 0; m < 4; ++m)
            mma_m16n8k16(cg[m][jj], alo[m][0], alo[m][1], alo[m][2], alo[m][3], bgh[b], bgh[b + 1]);
        }
      }

      // GRU update (App. A) of the lane's rows and units; the new state goes
      // to the column buffer (a later site's vertical input), to the h planes
      // (the next site's horizontal input) and into the head partials
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int m = i >> 1, h = i & 1, rho = 16 * m + g + 8 * h;
        const int d0 = hor_ok ? ssp[rho * NP + k - 1] : -1;
        const int d1 = ver >= 0 ? 2 + ssp[rho * NP + ver] : -1;
        float hn[2];
#pragma unroll
        for (int uu = 0; uu < 2; ++uu) {
          const int a = ua + uu, e = 2 * h + uu;
          float au = cg[m][0][e] + sbias[4 * a + 0];
          float ar = cg[m][1][e] + sbias[4 * a + 1];
          const float gg = cg[m][2][e] + sbias[4 * a + 2];
          float ai = sbias[4 * a + 3];
          if (d0 >= 0) {
            au += sxw[d0 * C3 + 3 * a + 0];
            ar += sxw[d0 * C3 + 3 * a + 1];
            ai += sxw[d0 * C3 + 3 * a + 2];
          }
          if (d1 >= 0) {
            au += sxw[d1 * C3 + 3 * a + 0];
            ar += sxw[d1 * C3 + 3 * a + 1];
            ai += sxw[d1 * C3 + 3 * a + 2];
          }
          const float u = sigm_fast(au), r = sigm_fast(ar);
          const float c = tanh_fast(r * gg + ai);
          hn[uu] = (1.f - u) * cp[m][e] + u * c;
        }
        if (so[i] >= 0)
          *reinterpret_cast<float2 *>(A.colbuf + (((int64_t)blockIdx.x * R + rho) * Lx + col) * DH + ua) =
              make_float2(hn[0], hn[1]);
        uint32_t hi, lo;
        bf16x2_split(hn[0], hn[1], hi, lo);
        sHh[rho * LDW + kpo] = hi;
        sHl[rho * LDW + kpo] = lo;
        if (turn) vv[i] = so[i] >= 0 ? make_float2(hn[0], hn[1]) : make_float2(0.f, 0.f);
        float z0 = shead[0 * DH + ua] * hn[0] + shead[0 * DH + ua + 1] * hn[1];
        float z1 = shead[1 * DH + ua] * hn[0] + shead[1 * DH + ua + 1] * hn[1];
        z0 += __shfl_xor_sync(0xffffffffu, z0, 1);
        z1 += __shfl_xor_sync(0xffffffffu, z1, 1);
        z0 += __shfl_xor_sync(0xffffffffu, z0, 2);
        z1 += __shfl_xor_sync(0xffffffffu, z1, 2);
        if (t == 0) {
          sz[(0 * NW + w) * R + rho] = z0;
          sz[(1 * NW + w) * R + rho] = z1;
        }
        if (A.cplx) {
          float z2 = shead[2 * DH + ua] * hn[0] + shead[2 * DH + ua + 1] * hn[1];
          float z3 = shead[3 * DH + ua] * hn[0] + shead[3 * DH + ua + 1] * hn[1];
          z2 += __shfl_xor_sync(0xffffffffu, z2, 1);
          z3 += __shfl_xor_sync(0xffffffffu, z3, 1);
          z2 += __shfl_xor_sync(0xffffffffu, z2, 2);
          z3 += __shfl_xor_sync(0xffffffffu, z3, 2);
          if (t == 0) {
            sz[(2 * NW + w) * R + rho] = z2;
            sz[(3 * NW + w) * R + rho] = z3;
          }
        }
      }
      __syncthreads();  // head partials complete

      // row rr: conditional of site k (Sec. II.A), mask, log-amplitude terms
      if (rowt && rs >= 0) {
        float z0 = shc[0], z1 = shc[1], z2 = shc[2], z3 = shc[3];
#pragma unroll
        for (int v = 0; v < NW; ++v) {
          z0 += sz[(0 * NW + v) * R + rr];
          z1 += sz[(1 * NW + v) * R + rr];
        }
        if (A.cplx) {
#pragma unroll
          for (int v = 0; v < NW; ++v) {
            z2 += sz[(2 * NW + v) * R + rr];
            z3 += sz[(3 * NW + v) * R + rr];
          }
        }
        float lp0, lp1;
        log_softmax2<float>(z0, z1, lp0, lp1);
        int forced = -1;  // value forced by the mask, or -1
        if (A.zmask) {
          if (n_up >= N / 2) forced = 1;
          else if (n_dn >= N / 2) forced = 0;
        }
        const int sg = ssp[rr * NP + k];
        const bool kill = forced >= 0 && sg != forced;  // log p = -inf
        const float hl = forced >= 0 ? 0.f : 0.5f * (sg == 0 ? lp0 : lp1);
        float pp = 0.f, pe = 0.f;  // pi softsign(y) as a pair
        if (A.cplx) pi_times(softsign(sg == 0 ? z2 : z3), pp, pe);
        dead |= kill;
        two_add(sre, cre, hl);
        two_add(sre, cre, -lc0);
        two_add(sim, cim, pp);
        two_add(sim, cim, pe - lc1);
        if (sg == 0) ++n_up; else ++n_dn;
      }
    }
    // row outputs: the operator's matrix element times psi(sigma')/psi(sigma)
    if (rowt && rs >= 0) {
      const double acc_re = dead ? -INFINITY : (double)sre + (double)cre;
      const double acc_im = (double)sim + (double)cim;
      const double e = A.item_e[(int64_t)op * A.nrows + base + rr];
      const double mag = exp(acc_re);
      double *c = A.contrib + ((int64_t)op * A.nrows + rs) * 2;
      c[0] = e * mag * cos(acc_im);
      c[1] = e * mag * sin(acc_im);
    }
  }
}

}  // namespace nqs
