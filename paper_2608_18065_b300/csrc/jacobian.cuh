// jacobian.cuh -- per-sample log-derivatives O = d log Psi / d theta.
//
// Stage 1 (k_jac_bwd): one reverse sweep per row (row = sample and adjoint
// seed: d(1/2 log P) for the real rows, d(phi) for the imaginary rows of a
// complex head) through the GRU of App. A.  The gate pre-activations of each
// site are recomputed from the cached hidden states, the adjoint of h' is
// one small GEMM [R x 3dh] x [3dh x dh] per site, and the per-site gate
// adjoints are written out.
// Stage 2 (k_jac_grad): the weight gradients of one row are sums over sites
// of outer products (adjoint of a gate) x (its input), assembled into the
// row of O in the flat parameter layout.
#pragma once
#include "recurrence.cuh"

namespace nqs {

template <typename T> struct BwdArgs {
  const T *pack;
  int N, Lx, cplx, zmask;
  int64_t ns, nrows;        // nrows = ns (real head) or 2 ns (complex head)
  int ntiles;
  const uint8_t *spins;     // [ns][N]
  const T *hcache;          // [ns][N][dh]
  const T *gcache;          // [ns][N][gw] gate activations of the forward pass
  int gw;
  const T *lccache;         // [ns][N][2]: 1/2 log p(sigma_k), phi_k
  T *adj;                   // [nrows][N][adjw]
  int adjw;
  T *adjcol;                // 2D: [nrows][Lx][dh] pending vertical adjoints
  // sites of this pass, [k_lo, k_hi) (0, N: the whole chain), and where
  // their inputs live: h_{k-1} at hcache[(s hN + k - 1 - hoff) dh], gates at
  // gcache[(s gN + k - goff) gw], records at adj[(row aN + k - aoff) adjw]
  int k_lo, k_hi, hN, hoff, gN, goff, aN, aoff;
  T *carry;                 // optional [nrows][dh]: adjoint of h_{k_hi-1} in, of h_{k_lo-1} out
};

// adjoint record of one site: dau | dar | dg | dac (4 dh) | dz0 dz1 dy0 dy1 |
// 2D: dhp (dh) | hp (dh)
template <int DH, int DIM> struct Adj {
  static constexpr int W = 4 * DH + 4 + (DIM == 2 ? 2 * DH : 0);
  static constexpr int DZ = 4 * DH, DHP = 4 * DH + 4, HP = 5 * DH + 4;
};

// Unit groups of the reverse sweep: two units per thread at dh >= 64.
template <int DH> struct BTile {
  static constexpr int UG = DH == 200 ? 8 : (DH >= 32 ? 32 : DH);
  static constexpr int UT = DH / UG;
};

// Row stride of the shared [unit][row] arrays of k_jac_bwd: padded by RT
// (the lanes of a warp, consecutive units, spread over the banks; a thread's
// RT rows stay aligned for its vector loads).
template <int R, int RT> __host__ __device__ constexpr int bwd_rp() { return R % 8 == 0 ? R + RT : R; }

template <typename T, int DH, int DIM, int R, int RT>
inline size_t bwd_smem_bytes(int N, bool wsmem = true) {
  constexpr int RP = bwd_rp<R, RT>();                       // padded row stride (see k_jac_bwd)
  size_t t = 4 * DH + 8;                                   // head, hc
  if (wsmem) t += 3 * (size_t)DH * DH + (DIM == 2 ? 2 * (size_t)DH * DH : 0);  // Wg, U12
  if (DIM == 2) t += (size_t)DH * RP;                      // sdp
  t += 3 * (size_t)DH * RP;                               // sda
  size_t b = t * sizeof(T) + (size_t)R * ((N + 15) & ~15) + R * 16;
  return (b + 127) & ~size_t(127);
}

// Reverse sweep of one row (sample, seed) through the GRU (App. A).  The
// forward pass stored u, r, c, W_h h' + b_h (and h' in 2D) per site, and the
// log-conditional of sigma_k, so per site only the adjoint of h',
// W^T (dau, dar, dg) -- one GEMM [R x 3dh] x [3dh x dh] -- is computed.  The
// head adjoint follows from the stored terms: p(sigma_k) = exp(2 lc_0),
// p(other) = 1 - p(sigma_k) (a site fixed by the mask has p = 1 and no
// gradient), and the softsign slope pi (1 - |phi_k/pi|)^2.
// WS: W and [U1|U2] staged in shared memory (otherwise read through L1).
template <typename T, int DH, int DIM, int RT, int RG, bool WS = true>
__global__ void __launch_bounds__(BTile<DH>::UG * RG)
k_jac_bwd(const BwdArgs<T> A) {
  constexpr int UG = BTile<DH>::UG, UT = BTile<DH>::UT;
  constexpr int R = RT * RG;
  constexpr int NTH = UG * RG;
  constexpr int C3 = 3 * DH;
  using AJ = Adj<DH, DIM>;
  extern __shared__ __align__(16) unsigned char smraw[];
  T *shead = reinterpret_cast<T *>(smraw);  // [4][dh]
  T *shc = shead + 4 * DH;
  T *swb = shc + 8;                        // staged Wg [3dh][dh] and U12 [dh][2dh] (wsmem)
  const T *sWg = swb;
  const T *sU12 = swb + C3 * DH;
  // the R rows of a unit are stored R + RT floats apart, so the lanes of a
  // warp (one row group, consecutive units) spread over the banks and every
  // thread's RT rows stay aligned for its vector loads (bwd_rp)
  constexpr int RP = bwd_rp<R, RT>();
  T *sdp = swb + (WS ? C3 * DH + (DIM == 2 ? 2 * DH * DH : 0) : 0);  // 2D: [dh][RP]
  T *sda = sdp + (DIM == 2 ? DH * RP : 0);  // gate adjoints [3dh][RP]
  const int NP = (A.N + 15) & ~15;
  uint8_t *ssp = reinterpret_cast<uint8_t *>(sda + C3 * RP);
  int *srow = reinterpret_cast<int *>(ssp + R * NP);

  const int tid = threadIdx.x;
  const int ug = tid % UG, rg = tid / UG;
  // FP32 d_h = 64 (1D and 2D): the per-site product dh1 = dpd + W_g^T
  // [dau; dar; dg] (K = 3 d_h; in 2D the adjoint of h') runs as warp-level MMAs, m16n8k16 with BF16 hi.hi + hi.lo +
  // lo.hi and FP32 accumulation, 8 of the 16 rows used.  These products are
  // a dependent chain of N small ones on 8 rows per CTA, which the register
  // operands of warp MMAs serve with the least latency.  Warp w owns units
  // 8w .. 8w + 7 of all 8 rows; lane (lane / 4, lane % 4) = (row g, t) owns
  // units 8w + 2t, 8w + 2t + 1 of row g, where the MMA leaves their sums.
  constexpr bool WMMA = sizeof(T) == 4 && DH == 64 && RT == 1 && RG == 8;
  const int r0 = WMMA ? (tid & 31) >> 2 : rg * RT;
  const int a0 = WMMA ? 8 * (tid >> 5) + 2 * (tid & 3) : ug * UT;
  const bool row_lead = WMMA ? (tid >> 5) == 0 && (tid & 3) == 0 : ug == 0;
  const int N = A.N, Lx = A.Lx;

  {
    const T *p = A.pack;
    auto al = [](int x) { return (x + 31) & ~31; };
    constexpr int DIN = DIM == 2 ? 4 : 2;
    const int oWg = al(DH * C3), oxw = al(oWg + C3 * DH);
    const int obias = al(oxw + DIN * C3), ohead = al(obias + DH * 4), ohc = al(ohead + 4 * DH);
    const int oU12T = al(ohc + 4), oU12 = al(oU12T + 2 * DH * DH);
    for (int e = tid; e < 4 * DH; e += NTH) shead[e] = p[ohead + e];
    if (tid < 4) shc[tid] = p[ohc + tid];
    if constexpr (WS) {
      for (int e = tid; e < C3 * DH; e += NTH) swb[e] = p[oWg + e];
      if (DIM == 2)
        for (int e = tid; e < 2 * DH * DH; e += NTH) swb[C3 * DH + e] = p[oU12 + e];
    } else {
      sWg = p + oWg;
      sU12 = p + oU12;
    }
  }

  // the MMA's B operand, W_g of this warp's 8 units split into BF16 hi / lo,
  // stays in registers for the whole sweep: [12 K steps][2 registers]
  uint32_t wbh[WMMA ? 24 : 1], wbl[WMMA ? 24 : 1];
  if constexpr (WMMA) {
    __syncthreads();  // W_g staged
    const int gq = (tid & 31) >> 2, tq = tid & 3, n = 8 * (tid >> 5) + gq;
#pragma unroll
    for (int st = 0; st < 12; ++st)
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        const int k = 16 * st + 2 * tq + 8 * hh;
        bf16x2_split((float)sWg[k * DH + n], (float)sWg[(k + 1) * DH + n], wbh[2 * st + hh],
                     wbl[2 * st + hh]);
      }
  }

  for (int tile = blockIdx.x; tile < A.ntiles; tile += gridDim.x) {
    __syncthreads();
    for (int r = tid; r < R; r += NTH) {
      int64_t g = (int64_t)tile * R + r;
      srow[r] = g < A.nrows ? (int)g : -1;
    }
    __syncthreads();
    for (int e = tid; e < R * N; e += NTH) {
      int r = e / N, k = e - r * N;
      int g = srow[r];
      ssp[r * NP + k] = g >= 0 ? A.spins[(g % A.ns) * (int64_t)N + k] : 0;
    }
    __syncthreads();
    if (DIM == 2) {
#pragma unroll
      for (int i = 0; i < RT; ++i) {
        int g = srow[r0 + i];
        if (g < 0) continue;
        for (int c = 0; c < Lx; ++c)
#pragma unroll
          for (int uu = 0; uu < UT; ++uu)
            A.adjcol[((int64_t)g * Lx + c) * DH + a0 + uu] = T(0);
      }
    }
    T carry[RT][UT];
#pragma unroll
    for (int i = 0; i < RT; ++i) {
      const int g = srow[r0 + i];
#pragma unroll
      for (int uu = 0; uu < UT; ++uu)
        carry[i][uu] = (A.carry && g >= 0) ? A.carry[(int64_t)g * DH + a0 + uu] : T(0);
    }

    // forward-pass values of site k for this thread's rows and units,
    // loaded one site ahead of their use
    T gu[RT][UT], gr[RT][UT], gc[RT][UT], gg[RT][UT], ghp[RT][UT], lc0[RT], lc1[RT];
    auto load_site = [&](int k) {
#pragma unroll
      for (int i = 0; i < RT; ++i) {
        const int g = srow[r0 + i];
        const int64_t s = g >= 0 ? g % A.ns : 0;
        const T *G = A.gcache + (s * A.gN + k - A.goff) * A.gw;
#pragma unroll
        for (int uu = 0; uu < UT; ++uu) {
          const int a = a0 + uu;
          gu[i][uu] = G[a]; gr[i][uu] = G[DH + a]; gc[i][uu] = G[2 * DH + a];
          gg[i][uu] = G[3 * DH + a];
          if (DIM == 2) ghp[i][uu] = G[4 * DH + a];
          else ghp[i][uu] = k > 0 ? A.hcache[(s * A.hN + k - 1 - A.hoff) * DH + a] : T(0);
        }
        lc0[i] = A.lccache[(s * N + k) * 2];
        lc1[i] = A.lccache[(s * N + k) * 2 + 1];
      }
    };
    load_site(A.k_hi - 1);

    for (int k = A.k_hi - 1; k >= A.k_lo; --k) {
      int hor_ok = k > 0, ver = -1, col = 0;
      if (DIM == 2) {
        int j = k / Lx, m = k - j * Lx;
        col = (j & 1) ? (Lx - 1 - m) : m;
        hor_ok = m != 0;
        ver = (k >= Lx) ? k - 2 * m - 1 : -1;
      }
      T dpd[RT][UT];  // (1-u) dh: the direct path of dh into h'
      T hpv[RT][UT];
#pragma unroll
      for (int i = 0; i < RT; ++i) {
        const int r = r0 + i, g = srow[r];
        const int which = g >= 0 ? (int)(g / A.ns) : 0;
        const int sk = ssp[r * NP + k];
        // head adjoint from the stored log-conditional and phase of sigma_k
        T dz0 = T(0), dz1 = T(0), dy = T(0);
        if (which == 0) {
          const T ps = ex(T(2) * lc0[i]);
          dz0 = sk == 0 ? T(0.5) * (T(1) - ps) : T(-0.5) * (T(1) - ps);
          dz1 = -dz0;
        } else {
          const T q = lc1[i] / T(NQS_PI);
          const T om = T(1) - (q < T(0) ? -q : q);
          dy = T(NQS_PI) * om * om;
        }
        T *rec = A.adj + ((int64_t)(g >= 0 ? g : 0) * A.aN + k - A.aoff) * A.adjw;
        if (g >= 0 && row_lead) {
          rec[AJ::DZ + 0] = dz0; rec[AJ::DZ + 1] = dz1;
          rec[AJ::DZ + 2] = sk == 0 ? dy : T(0);
          rec[AJ::DZ + 3] = sk == 1 ? dy : T(0);
        }
#pragma unroll
        for (int uu = 0; uu < UT; ++uu) {
          const int a = a0 + uu;
          T dh = carry[i][uu] + shead[a] * dz0 + shead[DH + a] * dz1;
          if (A.cplx) dh += shead[(2 + sk) * DH + a] * dy;
          if (DIM == 2 && g >= 0) dh += A.adjcol[((int64_t)g * Lx + col) * DH + a];
          const T u = gu[i][uu], rr = gr[i][uu], c = gc[i][uu], gv = gg[i][uu];
          const T hp = ghp[i][uu];
          hpv[i][uu] = hp;
          const T dc = dh * u;
          const T du = dh * (c - hp);
          dpd[i][uu] = dh * (T(1) - u);
          const T dac = dc * (T(1) - c * c);
          const T dr = dac * gv;
          const T dg = dac * rr;
          const T dar = dr * rr * (T(1) - rr);
          const T dau = du * u * (T(1) - u);
          sda[(3 * a + 0) * RP + r] = dau;
          sda[(3 * a + 1) * RP + r] = dar;
          sda[(3 * a + 2) * RP + r] = dg;
          if (g >= 0) {
            rec[a] = dau; rec[DH + a] = dar; rec[2 * DH + a] = dg; rec[3 * DH + a] = dac;
            if (DIM == 2) rec[AJ::HP + a] = hp;
          }
        }
      }
      if (k > A.k_lo) load_site(k - 1);  // in flight during the GEMM below
      __syncthreads();
      T dh1[RT][UT];
#pragma unroll
      for (int i = 0; i < RT; ++i)
#pragma unroll
        for (int uu = 0; uu < UT; ++uu) dh1[i][uu] = dpd[i][uu];
      if constexpr (WMMA) {
        if (DIM == 2 || k > 0) {
          const int gq = (tid & 31) >> 2, tq = tid & 3;
          float c[4] = {(float)dh1[0][0], (float)dh1[0][1], 0.f, 0.f};
#pragma unroll
          for (int st = 0; st < 12; ++st) {
            const int kb = 16 * st + 2 * tq;
            uint32_t h0, l0, h2, l2;
            bf16x2_split((float)sda[kb * RP + gq], (float)sda[(kb + 1) * RP + gq], h0, l0);
            bf16x2_split((float)sda[(kb + 8) * RP + gq], (float)sda[(kb + 9) * RP + gq], h2, l2);
            mma_m16n8k16(c, h0, 0u, h2, 0u, wbh[2 * st], wbh[2 * st + 1]);
            mma_m16n8k16(c, h0, 0u, h2, 0u, wbl[2 * st], wbl[2 * st + 1]);
            mma_m16n8k16(c, l0, 0u, l2, 0u, wbh[2 * st], wbh[2 * st + 1]);
          }
          dh1[0][0] = (T)c[0];
          dh1[0][1] = (T)c[1];
        }
      } else {
        if (DIM == 2 || k > 0) mm_acc<T, RT, UT, 8>(sda, RP, r0, sWg, DH, a0, C3, dh1);
      }
      if (DIM == 1) {
#pragma unroll
        for (int i = 0; i < RT; ++i)
#pragma unroll
          for (int uu = 0; uu < UT; ++uu) carry[i][uu] = dh1[i][uu];
      } else {
        // d h' -> record, then route to the horizontal and vertical inputs
#pragma unroll
        for (int i = 0; i < RT; ++i) {
          const int r = r0 + i, g = srow[r];
#pragma unroll
          for (int uu = 0; uu < UT; ++uu) {
            sdp[(a0 + uu) * RP + r] = dh1[i][uu];
            if (g >= 0) A.adj[((int64_t)g * A.aN + k - A.aoff) * A.adjw + AJ::DHP + a0 + uu] = dh1[i][uu];
          }
        }
        __syncthreads();
        T dhh[RT][UT], dhv[RT][UT];
#pragma unroll
        for (int i = 0; i < RT; ++i)
#pragma unroll
          for (int uu = 0; uu < UT; ++uu) { dhh[i][uu] = T(0); dhv[i][uu] = T(0); }
        mm_acc<T, RT, UT, 8>(sdp, RP, r0, sU12, 2 * DH, a0, DH, dhh);
        mm_acc<T, RT, UT, 8>(sdp, RP, r0, sU12 + DH, 2 * DH, a0, DH, dhv);
#pragma unroll
        for (int i = 0; i < RT; ++i) {
          const int g = srow[r0 + i];
#pragma unroll
          for (int uu = 0; uu < UT; ++uu) {
            carry[i][uu] = hor_ok ? dhh[i][uu] : T(0);
            if (g >= 0)
              A.adjcol[((int64_t)g * Lx + col) * DH + a0 + uu] = ver >= 0 ? dhv[i][uu] : T(0);
          }
        }
      }
      (void)hpv;
      __syncthreads();
    }
    if (A.carry) {
#pragma unroll
      for (int i = 0; i < RT; ++i) {
        const int g = srow[r0 + i];
        if (g < 0) continue;
#pragma unroll
        for (int uu = 0; uu < UT; ++uu) A.carry[(int64_t)g * DH + a0 + uu] = carry[i][uu];
      }
    }
  }
}

// ------------------------------------------------------------ stage 2
template <typename T, typename TO> struct GradArgs {
  int N, Lx, cplx, dim;
  int64_t ns, nrows;
  const uint8_t *spins;
  const T *hcache;
  const T *adj;
  int adjw;
  TO *O;                    // [nrows][np]
  int64_t np;
  // sites [k_lo, k_hi) of this pass; h_k at hcache[(s hN + k - hoff) dh],
  // records at adj[(row aN + k - aoff) adjw]; accumulate: O += (else O =)
  int k_lo, k_hi, hN, hoff, aN, aoff, accumulate;
  // layout offsets
  int64_t U1, U2, Wu, bu, Wr, br, Wh, bh, Win, bin, Uo, co, Up, cp;
};

template <int DH> struct GTile {
  // tile edge per thread, threads per edge (d_h = 200: 10 x 10 threads of
  // 10 x 10 tiles, 2 x 2 sub-blocks)
  static constexpr int TA = DH == 200 ? 10 : DH >= 16 ? (DH / 16 < 8 ? DH / 16 : 8) : 1;
  static constexpr int GT = DH == 200 ? 10 : (DH / TA < 16 ? DH / TA : 16);
  static constexpr int SB = DH / (GT * TA);  // sub-blocks per edge (one per pass above 128)
  static_assert(GT * TA * SB == DH, "tiles cover the block");
};

// Sites per shared-memory chunk of k_jac_grad: static shared memory <= ~45 KB.
template <typename T, int DH, int DIM> __host__ __device__ constexpr int grad_kc() {
  return (16 * (Adj<DH, DIM>::W + 4 * DH) * (int)sizeof(T) <= 45000) ? 16
       : (8 * (Adj<DH, DIM>::W + 4 * DH) * (int)sizeof(T) <= 45000) ? 8 : 4;
}

template <typename T, typename TO, int DH, int DIM>
__global__ void __launch_bounds__(256) k_jac_grad(const GradArgs<T, TO> A) {
  constexpr int TA = GTile<DH>::TA, GT = GTile<DH>::GT, SB = GTile<DH>::SB;
  constexpr int KC = grad_kc<T, DH, DIM>();
  constexpr int DIN = DIM == 2 ? 4 : 2;
  constexpr int NB = DIM == 2 ? 5 : 3;  // big blocks: Wu_h Wr_h Wh (U1 U2)
  // above dh = 64 the big blocks are accumulated one per pass (registers)
  constexpr int BPP = TA <= 4 ? NB : 1;
  // passes: groups of BPP big blocks, each block in SB x SB sub-blocks
  constexpr int NPASS = ((NB + BPP - 1) / BPP) * SB * SB;
  using AJ = Adj<DH, DIM>;
  const int row = blockIdx.x;
  const int64_t s = row % A.ns;
  const int N = A.N, Lx = A.Lx;
  const int tid = threadIdx.x;
  __shared__ T sadj[KC][AJ::W];
  __shared__ T sQ[KC][DH];      // input state of the gates: h_{k-1} (1D) or h' (2D)
  __shared__ T sH[KC][DH];      // h_k (heads)
  __shared__ T sHh[DIM == 2 ? KC : 1][DH];  // 2D: h_hor
  __shared__ T sHv[DIM == 2 ? KC : 1][DH];  // 2D: h_ver
  __shared__ int sx[KC][2];     // active one-hot input columns of site k (-1: none)

  const bool big = tid < GT * GT;
  constexpr int NA = (KC * AJ::W + 255) / 256;   // adjoint values per thread and chunk
  constexpr int NH = (KC * DH + 255) / 256;      // state values per thread and chunk
  const int ta0 = (tid / GT) * TA, tb0 = (tid % GT) * TA;
  // small entries: heads (4 dh), x-columns (3 dh din), biases (4 dh + 4)
  const int nsmall = 4 * DH + 3 * DH * DIN + 4 * DH + 4;
  constexpr int SPT = (4 * DH + 3 * DH * DIN + 4 * DH + 4 + 255) / 256;
  T accS[SPT];
#pragma unroll
  for (int q = 0; q < SPT; ++q) accS[q] = T(0);

  // record of site k, state h_k (k >= hoff) of this row
  auto adj_at = [&](int k) { return A.adj + ((int64_t)row * A.aN + (k - A.aoff)) * A.adjw; };
  auto h_at = [&](int k) { return A.hcache + (s * A.hN + (k - A.hoff)) * DH; };
  const uint8_t *sprow = A.spins + s * N;
  TO *Orow = A.O + (int64_t)row * A.np;
  auto put = [&](int64_t idx, TO v) { Orow[idx] = A.accumulate ? Orow[idx] + v : v; };
  const int w = DH + DIN;
  // big block qb: 0 Wu_h, 1 Wr_h, 2 Wh (adjoint x h'), 3 U1, 4 U2 (adjoint of h' x h_hor/h_ver)
  auto adj_off = [&](int qb) { return qb == 0 ? 0 : qb == 1 ? DH : qb == 2 ? 2 * DH : AJ::DHP; };
  for (int pass = 0; pass < NPASS; ++pass) {
    const int pgrp = pass / (SB * SB), psub = pass % (SB * SB);
    const int ta = ta0 + (psub / SB) * GT * TA, tb = tb0 + (psub % SB) * GT * TA;
    T accB[BPP][TA][TA];
#pragma unroll
    for (int q = 0; q < BPP; ++q)
#pragma unroll
      for (int i = 0; i < TA; ++i)
#pragma unroll
        for (int j = 0; j < TA; ++j) accB[q][i][j] = T(0);
    // chunks of KC sites through shared memory; the next chunk's values are
    // fetched into registers while the current one is multiplied
    T ra[NA], rh[NH], rq[NH], rhh[DIM == 2 ? NH : 1], rhv[DIM == 2 ? NH : 1];
    int rx0 = -1, rx1 = -1;
    auto fetch = [&](int k0) {
      const int kc = min(KC, A.k_hi - k0);
#pragma unroll
      for (int q = 0; q < NA; ++q) {
        const int e = tid + 256 * q;
        if (e < kc * AJ::W) {
          const int kk = e / AJ::W, wi = e - kk * AJ::W;
          ra[q] = adj_at(k0 + kk)[wi];
        }
      }
#pragma unroll
      for (int q = 0; q < NH; ++q) {
        const int e = tid + 256 * q;
        if (e < kc * DH) {
          const int kk = e / DH, a = e - kk * DH, k = k0 + kk;
          rh[q] = h_at(k)[a];
          if (DIM == 1) {
            rq[q] = k > 0 ? h_at(k - 1)[a] : T(0);
          } else {
            const int j = k / Lx, m = k - j * Lx;
            const int ver = k >= Lx ? k - 2 * m - 1 : -1;
            rhh[DIM == 2 ? q : 0] = m != 0 ? h_at(k - 1)[a] : T(0);
            rhv[DIM == 2 ? q : 0] = ver >= 0 ? h_at(ver)[a] : T(0);
            rq[q] = adj_at(k)[AJ::HP + a];
          }
        }
      }
      if (tid < kc) {
        const int k = k0 + tid;
        if (DIM == 1) {
          rx0 = k > 0 ? sprow[k - 1] : -1;
          rx1 = -1;
        } else {
          const int j = k / Lx, m = k - j * Lx;
          const int ver = k >= Lx ? k - 2 * m - 1 : -1;
          rx0 = m != 0 ? sprow[k - 1] : -1;
          rx1 = ver >= 0 ? 2 + sprow[ver] : -1;
        }
      }
    };
    auto commit = [&](int k0) {
      const int kc = min(KC, A.k_hi - k0);
#pragma unroll
      for (int q = 0; q < NA; ++q) {
        const int e = tid + 256 * q;
        if (e < kc * AJ::W) {
          const int kk = e / AJ::W, wi = e - kk * AJ::W;
          sadj[kk][wi] = ra[q];
        }
      }
#pragma unroll
      for (int q = 0; q < NH; ++q) {
        const int e = tid + 256 * q;
        if (e < kc * DH) {
          const int kk = e / DH, a = e - kk * DH;
          sH[kk][a] = rh[q];
          sQ[kk][a] = rq[q];
          if (DIM == 2) {
            sHh[kk][a] = rhh[DIM == 2 ? q : 0];
            sHv[kk][a] = rhv[DIM == 2 ? q : 0];
          }
        }
      }
      if (tid < kc) { sx[tid][0] = rx0; sx[tid][1] = rx1; }
    };
    fetch(A.k_lo);
    for (int k0 = A.k_lo; k0 < A.k_hi; k0 += KC) {
      const int kc = min(KC, A.k_hi - k0);
      __syncthreads();  // the previous chunk is no longer read
      commit(k0);
      __syncthreads();
      if (k0 + KC < A.k_hi) fetch(k0 + KC);
      if (big) {
        for (int kk = 0; kk < kc; ++kk) {
#pragma unroll
          for (int q = 0; q < BPP; ++q) {
            const int qb = pgrp * BPP + q;
            if (qb >= NB) break;
            const T *Qv = qb < 3 ? sQ[kk] : (qb == 3 ? sHh[kk] : sHv[kk]);
            const int po = adj_off(qb);
            T qv[TA];
#pragma unroll
            for (int j = 0; j < TA; ++j) qv[j] = Qv[tb + j];
#pragma unroll
            for (int i = 0; i < TA; ++i) {
              const T pv = sadj[kk][po + ta + i];
#pragma unroll
              for (int j = 0; j < TA; ++j) accB[q][i][j] = fma(pv, qv[j], accB[q][i][j]);
            }
          }
        }
      }
      if (pass == 0) {
#pragma unroll
        for (int q = 0; q < SPT; ++q) {
          const int e = tid + 256 * q;
          if (e >= nsmall) continue;
          T v = accS[q];
          if (e < 4 * DH) {  // heads: U (o<2) and Uphi (o>=2): sum_k dz/dy[k][o] h_k[b]
            const int o = e / DH, b2 = e - o * DH;
            for (int kk = 0; kk < kc; ++kk) v = fma(sadj[kk][AJ::DZ + o], sH[kk][b2], v);
          } else if (e < 4 * DH + 3 * DH * DIN) {  // x-columns of Wu, Wr, Win
            const int e2 = e - 4 * DH;
            const int gsel = e2 / (DH * DIN), rem = e2 - gsel * DH * DIN;
            const int a = rem / DIN, d = rem - a * DIN;
            const int off = gsel == 0 ? 0 : (gsel == 1 ? DH : 3 * DH);  // dau, dar, dac
            for (int kk = 0; kk < kc; ++kk)
              if (sx[kk][0] == d || sx[kk][1] == d) v += sadj[kk][off + a];
          } else {  // biases: bu br bh bin (sum of dau dar dg dac), then c, cphi
            const int e2 = e - 4 * DH - 3 * DH * DIN;
            if (e2 < 4 * DH) {
              for (int kk = 0; kk < kc; ++kk) v += sadj[kk][e2];
            } else {
              for (int kk = 0; kk < kc; ++kk) v += sadj[kk][AJ::DZ + (e2 - 4 * DH)];
            }
          }
          accS[q] = v;
        }
      }
    }
    // write this pass's big blocks into the row of O
    if (big) {
#pragma unroll
      for (int q = 0; q < BPP; ++q) {
        const int qb = pgrp * BPP + q;
        if (qb >= NB) break;
#pragma unroll
        for (int i = 0; i < TA; ++i)
#pragma unroll
          for (int j = 0; j < TA; ++j) {
            const int a = ta + i, b2 = tb + j;
            const TO v = (TO)accB[q][i][j];
            if (qb == 0) put(A.Wu + (int64_t)a * w + b2, v);
            else if (qb == 1) put(A.Wr + (int64_t)a * w + b2, v);
            else if (qb == 2) put(A.Wh + (int64_t)a * DH + b2, v);
            else if (qb == 3) put(A.U1 + (int64_t)a * DH + b2, v);
            else put(A.U2 + (int64_t)a * DH + b2, v);
          }
      }
    }
  }
#pragma unroll
  for (int q = 0; q < SPT; ++q) {
    const int e = tid + 256 * q;
    if (e >= nsmall) continue;
    const TO v = (TO)accS[q];
    if (e < 4 * DH) {
      const int o = e / DH, b2 = e - o * DH;
      if (o < 2) put(A.Uo + o * DH + b2, v);
      else if (A.cplx) put(A.Up + (o - 2) * DH + b2, v);
    } else if (e < 4 * DH + 3 * DH * DIN) {
      const int e2 = e - 4 * DH;
      const int gsel = e2 / (DH * DIN), rem = e2 - gsel * DH * DIN;
      const int a = rem / DIN, d = rem - a * DIN;
      if (gsel == 0) put(A.Wu + (int64_t)a * w + DH + d, v);
      else if (gsel == 1) put(A.Wr + (int64_t)a * w + DH + d, v);
      else put(A.Win + (int64_t)a * DIN + d, v);
    } else {
      const int e2 = e - 4 * DH - 3 * DH * DIN;
      if (e2 < DH) put(A.bu + e2, v);
      else if (e2 < 2 * DH) put(A.br + e2 - DH, v);
      else if (e2 < 3 * DH) put(A.bh + e2 - 2 * DH, v);
      else if (e2 < 4 * DH) put(A.bin + e2 - 3 * DH, v);
      else if (e2 < 4 * DH + 2) put(A.co + e2 - 4 * DH, v);
      else if (A.cplx) put(A.cp + e2 - 4 * DH - 2, v);
    }
  }
}

}  // namespace nqs
