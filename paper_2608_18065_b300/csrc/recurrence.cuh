// recurrence.cuh -- fused GRU recurrences of libnqs (sm_103a).
//
// One CTA advances a tile of R rows (configurations) through the sites of
// the zig-zag path together.  Per site the gate pre-activations of all rows
// are one small GEMM [R x dh] x [dh x 3dh] (App. A) with the packed weights
// resident in shared memory; each thread owns RT rows x UT hidden units of
// all three gates, so the gate non-linearities, the state update and the
// partial output-head dot products stay in registers.  The heads are reduced
// over the 16 unit-group lanes with warp shuffles; the log-softmax, the
// zero-magnetisation mask and the Philox draw of each row run on one lane.
#pragma once
#include "common.cuh"

namespace nqs {

template <int DH> struct Tile {
  // unit groups (lanes): a power of two dividing d_h (8 for d_h = 200)
  static constexpr int UG = DH == 200 ? 8 : DH >= 256 ? 32 : (DH >= 16 ? 16 : DH);
  static constexpr int UT = DH / UG;  // hidden units per thread
};

// n consecutive values from shared or global memory, as 16-byte vectors when
// the element offset is a multiple of the vector width, else as float pairs
// when n is even (callers guarantee it: row/column offsets and leading
// dimensions are multiples of 4 floats or 2 doubles whenever n is, and even
// whenever n is)
template <typename T, int n>
__device__ __forceinline__ void load_run(const T *__restrict__ p, T (&v)[n]) {
  constexpr int VW = 16 / (int)sizeof(T);
  if constexpr (sizeof(T) == 4 && n % VW != 0 && n % 2 == 0) {
#pragma unroll
    for (int q = 0; q < n / 2; ++q) {
      const float2 t = reinterpret_cast<const float2 *>(p)[q];
      v[2 * q] = t.x; v[2 * q + 1] = t.y;
    }
  } else if constexpr (n % VW == 0) {
#pragma unroll
    for (int q = 0; q < n / VW; ++q) {
      if constexpr (sizeof(T) == 4) {
        const float4 t = reinterpret_cast<const float4 *>(p)[q];
        v[4 * q] = t.x; v[4 * q + 1] = t.y; v[4 * q + 2] = t.z; v[4 * q + 3] = t.w;
      } else {
        const double2 t = reinterpret_cast<const double2 *>(p)[q];
        v[2 * q] = t.x; v[2 * q + 1] = t.y;
      }
    }
  } else {
#pragma unroll
    for (int i = 0; i < n; ++i) v[i] = p[i];
  }
}

// acc[i][j] += sum_k At[k*lda + r0 + i] * B[k*ldb + c0 + j]; U: k steps
// unrolled (loads of U steps in flight; the sums keep their order)
template <typename T, int RT, int CT, int U = 2>
__device__ __forceinline__ void mm_acc(const T *__restrict__ At, int lda, int r0,
                                       const T *__restrict__ B, int ldb, int c0,
                                       int K, T (&acc)[RT][CT]) {
#pragma unroll U
  for (int k = 0; k < K; ++k) {
    T a[RT], b[CT];
    load_run<T, RT>(At + k * lda + r0, a);
    load_run<T, CT>(B + k * ldb + c0, b);
#pragma unroll
    for (int i = 0; i < RT; ++i)
#pragma unroll
      for (int j = 0; j < CT; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
  }
}

// Shared-memory state arrays are unit-major, [a][r] for R rows, with the row
// index XOR-swizzled by the unit's lane group (a / UT) in steps of RT rows:
// the unit-group lanes of a warp that store or load the same rows of
// different units then fall in different banks, while every thread's RT
// consecutive rows stay contiguous for vector loads.
template <int R, int RT, int UT>
__device__ __forceinline__ int ssw(int a, int r) {
  static_assert((R & (R - 1)) == 0, "R is a power of two");
  constexpr int G = (R / RT) < 8 ? (R / RT) : 8;
  return a * R + (r ^ (((a / UT) & (G - 1)) * RT));
}

// mm_acc with the A operand in the swizzled [k][r] layout.
template <typename T, int RT, int CT, int R, int UT, int U = 2>
__device__ __forceinline__ void mm_acc_s(const T *__restrict__ At, int r0,
                                         const T *__restrict__ B, int ldb, int c0,
                                         int K, T (&acc)[RT][CT]) {
#pragma unroll U
  for (int k = 0; k < K; ++k) {
    T a[RT], b[CT];
    load_run<T, RT>(At + ssw<R, RT, UT>(k, r0), a);
    load_run<T, CT>(B + k * ldb + c0, b);
#pragma unroll
    for (int i = 0; i < RT; ++i)
#pragma unroll
      for (int j = 0; j < CT; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
  }
}

template <typename T, int UG>
__device__ __forceinline__ T group_sum(T v) {
#pragma unroll
  for (int o = UG / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Zig-zag path helpers (Sec. II.B): column i of path index k, and the path
// index of the vertical neighbour (i, j-1) = k - 2m - 1 with m = k mod Lx.
__device__ __forceinline__ int path_col(int k, int Lx) {
  int j = k / Lx, m = k - j * Lx;
  return (j & 1) ? (Lx - 1 - m) : m;
}
__device__ __forceinline__ bool on_sublattice_A(int k, int Lx) {
  return ((path_col(k, Lx) + k / Lx) & 1) != 0;
}

enum { MODE_SAMPLE = 0, MODE_GIVEN = 1, MODE_ELOC = 2 };

template <typename T> struct FwdArgs {
  const T *pack;           // packed weights (PackOff layout)
  int N, Lx, cplx, marshall, zmask;
  int64_t nrows;           // SAMPLE/GIVEN: rows; ELOC: Ns
  int ntiles;
  // SAMPLE
  uint64_t seed, step;
  const int64_t *step_dev; // optional: step counter on the device (overrides step)
  int64_t s0;              // Philox sample index of row 0 (a rank's range of a sharded draw)
  // SAMPLE/GIVEN/ELOC spins: SAMPLE writes, others read
  uint8_t *spins;
  double *logpsi;          // [rows*2]
  T *hcache;               // [rows][N][dh]  (SAMPLE/GIVEN write, ELOC read)
  T *lccache;              // [rows][N][2]
  T *gcache;               // optional [rows][N][gw]: u | r | c | W_h h'+b_h (| h' in 2D)
  int gw;
  // ELOC
  int tiles_per_op;
  const int *op_f;         // [n_off*4]: f1, f2, start, rank order (unused here)
  const int *item_s;       // [n_off*Ns]
  const double *item_e;    // [n_off*Ns]
  const int *item_cnt;     // [n_off]
  double *contrib;         // [n_off*Ns*2]
  T *colbuf;               // 2D ELOC: [gridDim][R][Lx][dh]
  // hidden-state checkpoints (1D): ck > 0 keeps h_k only for k = m ck - 1
  // (m = 1..nck), in slot m - 1 of hcache rows of nck slots; ck = 0 keeps
  // every h_k (hcache rows of N sites)
  int ck, nck;
  // segment recompute (MODE_GIVEN, ck > 0): sites [k_lo, k_hi) from the
  // checkpoint h_{k_lo-1}; states to hseg [rows][ck+1][dh] (slot 0 =
  // h_{k_lo-1}), gates to gcache [rows][ck][gw]; log Psi is not written
  int k_lo, k_hi;
  T *hseg;
};

// Shared-memory footprint of k_forward; wsmem = 0 leaves the two large
// weight blocks (W^T and, in 2D, [U1 | U2]^T) in global memory (read
// through L1), for hidden sizes whose weights exceed shared memory.
template <typename T, int DH, int DIM, int R>
inline size_t fwd_smem_bytes(int N, bool wsmem = true) {
  constexpr int DIN = DIM == 2 ? 4 : 2;
  size_t t = (size_t)DIN * 3 * DH + (size_t)DH * 4 + 4 * DH + 8;
  if (wsmem) t += (size_t)DH * 3 * DH + (DIM == 2 ? 2 * (size_t)DH * DH : 0);
  t += (size_t)(DIM == 2 ? 4 : 2) * DH * R;
  size_t b = t * sizeof(T) + (size_t)R * ((N + 15) & ~15) + R * 16;
  return (b + 127) & ~size_t(127);
}

// WS: the two large weight blocks are staged in shared memory (otherwise they
// are read through L1 from the packed copy in global memory).
// UGX: unit groups (lanes per row) when not Tile<DH>::UG; more groups give
// each thread fewer hidden units and the CTA more warps per site.
template <typename T, int DH, int DIM, int RT, int RG, int MODE, bool WS = true, int UGX = 0>
__global__ void __launch_bounds__((UGX ? UGX : Tile<DH>::UG) * RG)
k_forward(const FwdArgs<T> A) {
  constexpr int UG = UGX ? UGX : Tile<DH>::UG, UT = DH / UG;
  static_assert(UG * UT == DH && UG <= 32 && (UG & (UG - 1)) == 0, "unit groups");
  constexpr int R = RT * RG;
  constexpr int NTH = UG * RG;
  constexpr int DIN = DIM == 2 ? 4 : 2;
  constexpr int C3 = 3 * DH;
  // k steps of the per-site products unrolled: loads of several steps in
  // flight (fewer where the accumulators already fill the registers)
  constexpr int MMU = (RT * 3 * UT <= 12) ? 8 : 2;
  extern __shared__ __align__(16) unsigned char smraw[];
  T *sxw = reinterpret_cast<T *>(smraw);
  T *sbias = sxw + DIN * C3;
  T *shead = sbias + DH * 4;
  T *shc = shead + 4 * DH;
  T *sw = shc + 8;                         // staged W^T and [U1|U2]^T (WS)
  const T *sWgT = sw;
  const T *sU12T = sw + DH * C3;
  T *sh0 = sw + (WS ? DH * C3 + (DIM == 2 ? 2 * DH * DH : 0) : 0);
  T *sh1 = sh0 + DH * R;
  T *shv = sh1 + DH * R;                    // 2D: vertical neighbour states
  T *shp = shv + (DIM == 2 ? DH * R : 0);   // 2D: h'
  const int NP = (A.N + 15) & ~15;
  uint8_t *ssp = reinterpret_cast<uint8_t *>(shp + (DIM == 2 ? DH * R : 0));
  int *srow = reinterpret_cast<int *>(ssp + R * NP);  // sample id or -1

  const int tid = threadIdx.x;
  const int ug = tid % UG, rg = tid / UG;
  const int r0 = rg * RT, a0 = ug * UT;
  const int N = A.N, Lx = A.Lx;

  // stage the packed weights once per CTA
  {
    const T *p = A.pack;
    // offsets follow pack_offsets(): recomputed here for the compile-time dh
    auto al = [](int x) { return (x + 31) & ~31; };
    int oWgT = 0, oWg = al(oWgT + DH * C3), oxw = al(oWg + C3 * DH);
    int obias = al(oxw + DIN * C3), ohead = al(obias + DH * 4), ohc = al(ohead + 4 * DH);
    int oU12T = al(ohc + 4);
    for (int e = tid; e < DIN * C3; e += NTH) sxw[e] = p[oxw + e];
    for (int e = tid; e < DH * 4; e += NTH) sbias[e] = p[obias + e];
    for (int e = tid; e < 4 * DH; e += NTH) shead[e] = p[ohead + e];
    if (tid < 4) shc[tid] = p[ohc + tid];
    if constexpr (WS) {
      for (int e = tid; e < DH * C3; e += NTH) sw[e] = p[oWgT + e];
      if (DIM == 2)
        for (int e = tid; e < 2 * DH * DH; e += NTH) sw[DH * C3 + e] = p[oU12T + e];
    } else {
      sWgT = p + oWgT;
      sU12T = p + oU12T;
    }
  }

  // 1D FP32 d_h = 64 sampling / given-configuration sweeps: the per-site
  // gate product [8 rows x 64] x [64 x 192] runs as warp-level MMAs
  // (m16n8k16, BF16 hi.hi + hi.lo + lo.hi, FP32 accumulation, 8 of the 16
  // rows used) with W_g in registers: warp w computes gate j of units
  // 8w .. 8w + 7 for every row, and the results reach the threads that own
  // them (row = warp, units 2 lane, 2 lane + 1) through shared memory.
  constexpr bool WMMA = sizeof(T) == 4 && DIM == 1 && DH == 64 && UG == 32 && RT == 1 &&
                        RG == 8 && MODE != MODE_ELOC;
  __shared__ float sgate[WMMA ? 8 * DH * 3 : 1];
  uint32_t wbh[WMMA ? 24 : 1], wbl[WMMA ? 24 : 1];  // [4 K steps][3 gates][2 registers]
  if constexpr (WMMA) {
    __syncthreads();  // W_g staged
    const int gq = (tid & 31) >> 2, tq = tid & 3, w = tid >> 5;
#pragma unroll
    for (int st = 0; st < 4; ++st)
#pragma unroll
      for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          const int k = 16 * st + 2 * tq + 8 * hh, n = 3 * (8 * w + gq) + j;
          bf16x2_split((float)sWgT[k * C3 + n], (float)sWgT[(k + 1) * C3 + n],
                       wbh[(st * 3 + j) * 2 + hh], wbl[(st * 3 + j) * 2 + hh]);
        }
  }

  for (int tile = blockIdx.x; tile < A.ntiles; tile += gridDim.x) {
    // ------------------------------------------------------- tile setup
    int kstart = 0, op = 0, f1 = -1, f2 = -1, base = 0, cnt = 0;
    if (MODE == MODE_ELOC) {
      op = tile / A.tiles_per_op;
      base = (tile - op * A.tiles_per_op) * R;
      cnt = A.item_cnt[op];
      if (base >= cnt) continue;  // uniform over the CTA
      f1 = A.op_f[4 * op + 0];
      f2 = A.op_f[4 * op + 1];
      kstart = A.op_f[4 * op + 2];
    }
    __syncthreads();  // previous tile finished with smem
    for (int r = tid; r < R; r += NTH) {
      int s = -1;
      if (MODE == MODE_ELOC) {
        if (base + r < cnt) s = A.item_s[(int64_t)op * A.nrows + base + r];
      } else {
        int64_t g = (int64_t)tile * R + r;
        if (g < A.nrows) s = (int)g;
      }
      srow[r] = s;
    }
    __syncthreads();
    for (int e = tid; e < R * N; e += NTH) {
      int r = e / N, k = e - r * N;
      int s = srow[r];
      uint8_t v = 0;
      if (MODE != MODE_SAMPLE && s >= 0) {
        v = A.spins[(int64_t)s * N + k];
        if (MODE == MODE_ELOC && (k == f1 || k == f2)) v ^= 1;
      }
      ssp[r * NP + k] = v;
    }
    // first recomputed site: the op's first changed site, or with
    // checkpoints the site after the last checkpoint before it (sites in
    // between are recomputed but add nothing to log Psi(sigma') - log Psi)
    const bool seg = MODE == MODE_GIVEN && A.hseg != nullptr;
    int krec = 0, kend = N;
    if (MODE == MODE_ELOC) krec = A.ck > 0 ? (kstart / A.ck) * A.ck : kstart;
    if (seg) { krec = A.k_lo; kend = A.k_hi; }
    // initial state h_{krec-1} (zero at the chain start)
    for (int e = tid; e < R * DH; e += NTH) {
      int r = e / DH, a = e - r * DH;
      int s = srow[r];
      T v = T(0);
      if (krec > 0 && s >= 0) {
        if (A.ck > 0) v = A.hcache[((int64_t)s * A.nck + (krec / A.ck - 1)) * DH + a];
        else v = A.hcache[((int64_t)s * N + (krec - 1)) * DH + a];
      }
      sh0[ssw<R, RT, UT>(a, r)] = v;
      if (seg && s >= 0) A.hseg[((int64_t)s * (A.ck + 1)) * DH + a] = v;
    }
    __syncthreads();

    // per-row scalar state lives on lane ug == i of each row group; the
    // log-amplitude sums are FP64 for FP64 data and TwoSum pairs for FP32
    // data (each term's parts added exactly); dead: an amplitude the mask
    // forces to zero
    double acc_re = 0.0, acc_im = 0.0;
    float sre = 0.f, cre = 0.f, sim = 0.f, cim = 0.f;
    bool dead = false;
    constexpr bool F32 = sizeof(T) == 4;
    int n_up = 0, n_dn = 0, nA = 0;
    const int my_i = ug;  // row handled by this lane (if ug < RT)
    const int my_r = r0 + (my_i < RT ? my_i : 0);
    const int my_s = my_i < RT ? srow[my_r] : -1;
    if ((MODE == MODE_ELOC || seg) && my_s >= 0) {
      for (int k = 0; k < krec; ++k) {
        if (ssp[my_r * NP + k] == 0) ++n_up; else ++n_dn;
      }
    }

    T *hcur = sh0, *hnxt = sh1;
    for (int k = krec; k < kend; ++k) {
      const T *Ag = hcur;  // A operand of the gate GEMM: h_{k-1} or h'
      int hor_ok = k > 0, ver = -1, col = 0;
      if (DIM == 2) {
        int j = k / Lx, m = k - j * Lx;
        col = (j & 1) ? (Lx - 1 - m) : m;
        hor_ok = m != 0;
        ver = (k >= Lx) ? k - 2 * m - 1 : -1;
        // vertical neighbour states into shv[a][r]
#pragma unroll
        for (int i = 0; i < RT; ++i) {
          int r = r0 + i, s = srow[r];
#pragma unroll
          for (int uu = 0; uu < UT; ++uu) {
            int a = a0 + uu;
            T v = T(0);
            if (ver >= 0 && s >= 0) {
              if (MODE == MODE_ELOC && ver >= kstart)
                v = A.colbuf[(((int64_t)blockIdx.x * R + r) * Lx + col) * DH + a];
              else
                v = A.hcache[((int64_t)s * N + ver) * DH + a];
            }
            shv[ssw<R, RT, UT>(a, r)] = v;
          }
        }
        __syncthreads();
        T acc1[RT][UT];
#pragma unroll
        for (int i = 0; i < RT; ++i)
#pragma unroll
          for (int j2 = 0; j2 < UT; ++j2) acc1[i][j2] = T(0);
        if (hor_ok) mm_acc_s<T, RT, UT, R, UT, MMU>(hcur, r0, sU12T, DH, a0, DH, acc1);
        if (ver >= 0) mm_acc_s<T, RT, UT, R, UT, MMU>(shv, r0, sU12T + DH * DH, DH, a0, DH, acc1);
#pragma unroll
        for (int i = 0; i < RT; ++i)
#pragma unroll
          for (int uu = 0; uu < UT; ++uu) shp[ssw<R, RT, UT>(a0 + uu, r0 + i)] = acc1[i][uu];
        __syncthreads();
        Ag = shp;
      }
      T acc[RT][3 * UT];
#pragma unroll
      for (int i = 0; i < RT; ++i)
#pragma unroll
        for (int j2 = 0; j2 < 3 * UT; ++j2) acc[i][j2] = T(0);
      if constexpr (WMMA) {
        if (k > 0) {
          const int gq = (tid & 31) >> 2, tq = tid & 3, w = tid >> 5;
          float c[3][4];
#pragma unroll
          for (int j = 0; j < 3; ++j) c[j][0] = c[j][1] = c[j][2] = c[j][3] = 0.f;
#pragma unroll
          for (int st = 0; st < 4; ++st) {
            const int kb = 16 * st + 2 * tq;
            uint32_t h0, l0, h2, l2;
            bf16x2_split((float)Ag[ssw<R, RT, UT>(kb, gq)], (float)Ag[ssw<R, RT, UT>(kb + 1, gq)],
                         h0, l0);
            bf16x2_split((float)Ag[ssw<R, RT, UT>(kb + 8, gq)],
                         (float)Ag[ssw<R, RT, UT>(kb + 9, gq)], h2, l2);
#pragma unroll
            for (int j = 0; j < 3; ++j) {
              const int b = (st * 3 + j) * 2;
              mma_m16n8k16(c[j], h0, 0u, h2, 0u, wbh[b], wbh[b + 1]);
              mma_m16n8k16(c[j], h0, 0u, h2, 0u, wbl[b], wbl[b + 1]);
              mma_m16n8k16(c[j], l0, 0u, l2, 0u, wbh[b], wbh[b + 1]);
            }
          }
#pragma unroll
          for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int uu = 0; uu < 2; ++uu)
              sgate[(gq * DH + 8 * w + 2 * tq + uu) * 3 + j] = c[j][uu];
          __syncthreads();
#pragma unroll
          for (int uu = 0; uu < UT; ++uu)
#pragma unroll
            for (int j = 0; j < 3; ++j) acc[0][3 * uu + j] = (T)sgate[(r0 * DH + a0 + uu) * 3 + j];
        }
      } else {
        if (DIM == 2 || k > 0) mm_acc_s<T, RT, 3 * UT, R, UT, MMU>(Ag, r0, sWgT, C3, 3 * a0, DH, acc);
      }

      // epilogue: GRU cell (App. A), partial heads, then the row's head on
      // lane ug == i (log-softmax, mask, draw, accumulate)
#pragma unroll
      for (int i = 0; i < RT; ++i) {
        const int r = r0 + i;
        const int s = srow[r];
        int d0 = -1, d1 = -1;
        if (DIM == 1) {
          if (k > 0) d0 = ssp[r * NP + k - 1];
        } else {
          if (hor_ok) d0 = ssp[r * NP + k - 1];
          if (ver >= 0) d1 = 2 + ssp[r * NP + ver];
        }
        T z0 = T(0), z1 = T(0), z2 = T(0), z3 = T(0);
#pragma unroll
        for (int uu = 0; uu < UT; ++uu) {
          const int a = a0 + uu;
          T au = acc[i][3 * uu + 0] + sbias[4 * a + 0];
          T ar = acc[i][3 * uu + 1] + sbias[4 * a + 1];
          T gg = acc[i][3 * uu + 2] + sbias[4 * a + 2];
          T ai = sbias[4 * a + 3];
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
          const T u = sigm(au), rr = sigm(ar);
          const T c = tnh(rr * gg + ai);
          const T hp = (DIM == 2 || k > 0) ? Ag[ssw<R, RT, UT>(a, r)] : T(0);
          const T hn = (T(1) - u) * hp + u * c;
          hnxt[ssw<R, RT, UT>(a, r)] = hn;
          if (s >= 0) {
            if (seg) {
              A.hseg[((int64_t)s * (A.ck + 1) + (k - krec + 1)) * DH + a] = hn;
            } else if (MODE != MODE_ELOC && A.hcache) {
              if (A.ck == 0) A.hcache[((int64_t)s * N + k) * DH + a] = hn;
              else if ((k + 1) % A.ck == 0 && (k + 1) / A.ck <= A.nck)
                A.hcache[((int64_t)s * A.nck + ((k + 1) / A.ck - 1)) * DH + a] = hn;
            }
            if (MODE != MODE_ELOC && A.gcache) {
              T *gr = seg ? A.gcache + ((int64_t)s * A.ck + (k - krec)) * A.gw
                          : A.gcache + ((int64_t)s * N + k) * A.gw;
              gr[a] = u; gr[DH + a] = rr; gr[2 * DH + a] = c; gr[3 * DH + a] = gg;
              if (DIM == 2) gr[4 * DH + a] = hp;
            }
            if (DIM == 2 && MODE == MODE_ELOC)
              A.colbuf[(((int64_t)blockIdx.x * R + r) * Lx + col) * DH + a] = hn;
          }
          z0 += shead[0 * DH + a] * hn;
          z1 += shead[1 * DH + a] * hn;
          if (A.cplx) {
            z2 += shead[2 * DH + a] * hn;
            z3 += shead[3 * DH + a] * hn;
          }
        }
        z0 = group_sum<T, UG>(z0);
        z1 = group_sum<T, UG>(z1);
        if (A.cplx) {
          z2 = group_sum<T, UG>(z2);
          z3 = group_sum<T, UG>(z3);
        }
        if (i != my_i || my_s < 0) continue;
        T lp0, lp1;
        log_softmax2<T>(z0 + shc[0], z1 + shc[1], lp0, lp1);
        int forced = -1;  // value forced by the mask, or -1
        if (A.zmask) {
          if (n_up >= N / 2) forced = 1;
          else if (n_dn >= N / 2) forced = 0;
        }
        int sg;
        if (MODE == MODE_SAMPLE) {
          const uint64_t stp = A.step_dev ? (uint64_t)*A.step_dev : A.step;
          if constexpr (F32) {
            const float p0 = forced == 0 ? 1.f : (forced == 1 ? 0.f : (float)ex(lp0));
            sg = uniform24(A.seed, stp, (uint32_t)(my_s + A.s0), (uint32_t)k) < p0 ? 0 : 1;
          } else {
            double p0 = forced == 0 ? 1.0 : (forced == 1 ? 0.0 : (double)ex(lp0));
            double uu = uniform53(A.seed, stp, (uint32_t)(my_s + A.s0), (uint32_t)k);
            sg = uu < p0 ? 0 : 1;
          }
          ssp[r * NP + k] = (uint8_t)sg;
          A.spins[(int64_t)my_s * N + k] = (uint8_t)sg;
        } else {
          sg = ssp[r * NP + k];
        }
        if constexpr (F32) {
          const bool kill = forced >= 0 && sg != forced;  // log p = -inf
          const float hl = forced >= 0 ? 0.f : 0.5f * (float)(sg == 0 ? lp0 : lp1);
          float pp = 0.f, pe = 0.f;  // pi softsign(y) as a pair
          if (A.cplx) pi_times((float)softsign((sg == 0 ? z2 : z3) + shc[2 + sg]), pp, pe);
          if (MODE == MODE_ELOC) {
            if (k >= kstart) {
              const T *lc = A.lccache + ((int64_t)my_s * N + k) * 2;
              dead |= kill;
              two_add(sre, cre, hl);
              two_add(sre, cre, -(float)lc[0]);
              two_add(sim, cim, pp);
              two_add(sim, cim, pe - (float)lc[1]);
            }
          } else if (!seg) {
            dead |= kill;
            two_add(sre, cre, hl);
            two_add(sim, cim, pp);
            two_add(sim, cim, pe);
            if (A.lccache) {
              T *lc = A.lccache + ((int64_t)my_s * N + k) * 2;
              lc[0] = kill ? (T)-INFINITY : (T)hl;
              lc[1] = (T)(pp + pe);
            }
          }
        } else {
          double lps;
          if (forced >= 0) lps = (sg == forced) ? 0.0 : -INFINITY;
          else lps = (double)(sg == 0 ? lp0 : lp1);
          double ph = 0.0;
          if (A.cplx) {
            T y = (sg == 0 ? z2 : z3) + shc[2 + sg];
            ph = NQS_PI * (double)softsign(y);
          }
          if (MODE == MODE_ELOC) {
            if (k >= kstart) {
              const T *lc = A.lccache + ((int64_t)my_s * N + k) * 2;
              acc_re += 0.5 * lps - (double)lc[0];
              acc_im += ph - (double)lc[1];
            }
          } else if (!seg) {
            acc_re += 0.5 * lps;
            acc_im += ph;
            if (A.lccache) {
              T *lc = A.lccache + ((int64_t)my_s * N + k) * 2;
              lc[0] = (T)(0.5 * lps);
              lc[1] = (T)ph;
            }
          }
        }
        if (sg == 0) ++n_up; else ++n_dn;
        if (A.marshall && sg == 1 && on_sublattice_A(k, Lx)) ++nA;
      }
      __syncthreads();
      T *t = hcur; hcur = hnxt; hnxt = t;
    }
    if constexpr (F32) {
      acc_re = dead ? -INFINITY : (double)sre + (double)cre;
      acc_im = (double)sim + (double)cim;
    }
    // row outputs
    if (my_i < RT && my_s >= 0) {
      if (MODE == MODE_ELOC) {
        double e = A.item_e[(int64_t)op * A.nrows + base + my_i + r0];
        double mag = exp(acc_re);
        double* c = A.contrib + ((int64_t)op * A.nrows + my_s) * 2;
        c[0] = e * mag * cos(acc_im);
        c[1] = e * mag * sin(acc_im);
      } else if (!seg) {
        A.logpsi[2 * (int64_t)my_s] = acc_re;
        A.logpsi[2 * (int64_t)my_s + 1] = acc_im + (A.marshall ? NQS_PI * (double)(nA & 1) : 0.0);
      }
    }
  }
}

}  // namespace nqs
