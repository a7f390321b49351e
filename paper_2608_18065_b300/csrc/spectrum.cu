// spectrum.cu -- conditioning diagnostics of the damped minSR system
// (App. E): extreme eigenvalues of the sample-space matrix T by Lanczos in
// FP64, kappa_2(T + lambda I) and the digit estimate -log10(kappa eps).
//
// One cooperative launch (one CTA of 256 threads per SM, grid barriers
// between the phases of a Lanczos step):
//   w = T v_j                 one warp per row, coalesced FP64 row reads;
//   h = V^T w, w -= V h       twice (classical Gram-Schmidt applied twice,
//                             full reorthogonalisation), one warp per dot;
//   alpha_j = h_j, beta_j = |w|, v_{j+1} = w / beta_j.
// The step stops early when beta_j falls below 1e-14 |T|-scale (the Krylov
// space is invariant).  Warp 0 of CTA 0 then finds the largest and smallest
// eigenvalues of the tridiagonal matrix by 32-point multisection with Sturm
// counts, and the Ritz residual beta_m |s_m| of the top pair by inverse
// iteration on the tridiagonal.  Every sum has a fixed order, so the result
// is bit-reproducible for a given grid.
#include <cuda_runtime.h>
#include <math.h>

#include "nqs.h"
#include "grid_sync.cuh"
#include "common.cuh"

using namespace nqs;

namespace {

constexpr int LZ_THREADS = 256;
constexpr int LZ_MAX_GRID = 256;
constexpr int LZ_MAX_M = 512;

inline size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

// Scratch layout (byte offsets from the caller's work pointer).
struct LzLayout {
  size_t hdr, alpha, beta, h1, h2, part, w, V, total;
};

LzLayout lz_layout(int64_t R, int m) {
  LzLayout L{};
  size_t p = 0;
  auto take = [&](size_t b) { size_t at = p; p = al256(p + b); return at; };
  L.hdr = take(256);  // barrier counter (u32) and status (i32)
  L.alpha = take(sizeof(double) * (size_t)(m + 1));
  L.beta = take(sizeof(double) * (size_t)(m + 1));
  L.h1 = take(sizeof(double) * (size_t)(m + 1));
  L.h2 = take(sizeof(double) * (size_t)(m + 1));
  L.part = take(sizeof(double) * (size_t)LZ_MAX_GRID);
  L.w = take(sizeof(double) * (size_t)R);
  L.V = take(sizeof(double) * (size_t)R * (size_t)(m + 1));
  L.total = p;
  return L;
}

struct LzArgs {
  const double *T;
  int64_t R;
  double lam;
  int m;
  uint64_t seed;
  unsigned *bar;
  int32_t *status;
  double *alpha, *beta, *h1, *h2, *part, *w, *V;
  nqs_spectrum_stats *out;
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Number of eigenvalues of the symmetric tridiagonal (a, b) below x (Sturm
// sequence of the LDL^T pivots; a zero pivot is replaced by -pmin).
__device__ int sturm_count(const double *a, const double *b, int n, double x, double pmin) {
  int c = 0;
  double q = a[0] - x;
  if (fabs(q) < pmin) q = -pmin;
  c += q < 0.0;
  for (int i = 1; i < n; ++i) {
    q = a[i] - x - b[i - 1] * b[i - 1] / q;
    if (fabs(q) < pmin) q = -pmin;
    c += q < 0.0;
  }
  return c;
}

// Eigenvalue t (0-based, ascending) of the tridiagonal (a, b) in [lo, hi]
// by 32-point multisection over one warp.
__device__ double warp_tri_eig(const double *a, const double *b, int n, int t, double lo,
                               double hi, double pmin, int lane) {
  for (int it = 0; it < 24; ++it) {
    const double h = (hi - lo) / 33.0;
    const double x = lo + (lane + 1) * h;
    const bool above = sturm_count(a, b, n, x, pmin) > t;
    const unsigned mask = __ballot_sync(0xffffffffu, above);
    const int f = mask ? __ffs(mask) - 1 : 32;  // first point above the target
    const double xf = __shfl_sync(0xffffffffu, x, f < 32 ? f : 31);
    const double xb = __shfl_sync(0xffffffffu, x, f > 0 ? f - 1 : 0);
    const double nlo = f > 0 ? xb : lo, nhi = f < 32 ? xf : hi;
    lo = nlo;
    hi = nhi;
    if (hi - lo <= 4e-16 * fmax(fabs(lo), fabs(hi)) + pmin) break;
  }
  return 0.5 * (lo + hi);
}

__global__ void __launch_bounds__(LZ_THREADS) k_lanczos(LzArgs a) {
  __shared__ double red_s[LZ_THREADS / 32];
  __shared__ double ab_s[2][LZ_MAX_M + 1];
  __shared__ double zc_s[2][LZ_MAX_M];  // inverse iteration on the tridiagonal
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int G = gridDim.x, g = blockIdx.x;
  const int64_t R = a.R;
  const int64_t nwarps = (int64_t)G * (LZ_THREADS / 32), gw = (int64_t)g * (LZ_THREADS / 32) + warp;
  const int64_t GT = (int64_t)G * LZ_THREADS, gt = (int64_t)g * LZ_THREADS + tid;
  unsigned ep = 0;
  auto gsync = [&]() -> bool { ++ep; return cc_sync_ep(a.bar, a.status, ep * (unsigned)G); };
  auto bail = [&]() {
    if (g == 0 && tid == 0) a.out->status = *reinterpret_cast<volatile int32_t *>(a.status);
  };
  // sum over the grid of one value per thread: CTA partials in part[], then
  // every CTA adds them up in the same order
  auto grid_sum = [&](double v, bool &ok) -> double {
    v = warp_sum(v);
    if (lane == 0) red_s[warp] = v;
    __syncthreads();
    if (tid == 0) {
      double s = 0.0;
      for (int q = 0; q < LZ_THREADS / 32; ++q) s += red_s[q];
      a.part[g] = s;
    }
    ok = gsync();
    // one partial per thread (G <= LZ_THREADS), then a fixed-order tree: the
    // same sum in every CTA
    double s = tid < G ? __ldcg(a.part + tid) : 0.0;
    s = warp_sum(s);
    __syncthreads();  // red_s of the CTA partial has been read
    if (lane == 0) red_s[warp] = s;
    __syncthreads();
    s = 0.0;
#pragma unroll
    for (int q = 0; q < LZ_THREADS / 32; ++q) s += red_s[q];
    __syncthreads();  // red_s is free for the next call
    return s;
  };
  double *V = a.V;

  // (0) start vector: Philox uniforms of the seed, centred and normalised
  double nv = 0.0;
  for (int64_t i = gt; i < R; i += GT) {
    const double u = uniform53(a.seed, 0x5bd1e995ull, (uint32_t)i, (uint32_t)(i >> 32)) - 0.5;
    a.w[i] = u;
    nv += u * u;
  }
  bool ok = true;
  const double n0 = sqrt(grid_sum(nv, ok));
  if (!ok) { bail(); return; }
  for (int64_t i = gt; i < R; i += GT) V[i] = a.w[i] / n0;
  if (!gsync()) { bail(); return; }

  double tscale = 0.0;  // |alpha| + |beta| seen so far: the scale of T
  int mk = a.m;
  for (int j = 0; j < a.m; ++j) {
    const double *vj = V + (int64_t)j * R;
    // w = T v_j, one warp per row
    for (int64_t i = gw; i < R; i += nwarps) {
      const double *Ti = a.T + i * R;
      double s = 0.0;
#pragma unroll 8
      for (int64_t c = lane; c < R; c += 32) s = fma(Ti[c], __ldcg(vj + c), s);
      s = warp_sum(s);
      if (lane == 0) {
        a.w[i] = s;
        if (!isfinite(s)) atomicCAS(reinterpret_cast<int *>(a.status), 0, (int)NQS_ERR_NONFINITE);
      }
    }
    if (!gsync()) { bail(); return; }
    // two passes of classical Gram-Schmidt against v_0 .. v_j
    for (int pass = 0; pass < 2; ++pass) {
      double *h = pass == 0 ? a.h1 : a.h2;
      for (int64_t k = gw; k <= j; k += nwarps) {
        const double *vk = V + k * R;
        double s = 0.0;
#pragma unroll 8
        for (int64_t c = lane; c < R; c += 32) s = fma(__ldcg(vk + c), __ldcg(a.w + c), s);
        s = warp_sum(s);
        if (lane == 0) h[k] = s;
      }
      if (!gsync()) { bail(); return; }
      for (int k = tid; k <= j; k += LZ_THREADS) ab_s[0][k] = __ldcg(h + k);
      __syncthreads();
      double nw = 0.0;
      for (int64_t i = gt; i < R; i += GT) {
        // four partial sums, eight basis vectors' loads in flight at a time
        double x0 = 0.0, x1 = 0.0, x2 = 0.0, x3 = 0.0;
        int k = 0;
        for (; k + 8 <= j + 1; k += 8) {
          double v[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) v[q] = __ldcg(V + (int64_t)(k + q) * R + i);
          x0 = fma(ab_s[0][k + 0], v[0], x0); x1 = fma(ab_s[0][k + 1], v[1], x1);
          x2 = fma(ab_s[0][k + 2], v[2], x2); x3 = fma(ab_s[0][k + 3], v[3], x3);
          x0 = fma(ab_s[0][k + 4], v[4], x0); x1 = fma(ab_s[0][k + 5], v[5], x1);
          x2 = fma(ab_s[0][k + 6], v[6], x2); x3 = fma(ab_s[0][k + 7], v[7], x3);
        }
        for (; k <= j; ++k) x0 = fma(ab_s[0][k], __ldcg(V + (int64_t)k * R + i), x0);
        const double x = a.w[i] - ((x0 + x1) + (x2 + x3));
        a.w[i] = x;
        nw += x * x;
      }
      if (pass == 0) {
        if (!gsync()) { bail(); return; }
      } else {
        const double beta = sqrt(grid_sum(nw, ok));
        if (!ok) { bail(); return; }
        const double alpha = __ldcg(a.h1 + j) + __ldcg(a.h2 + j);
        if (g == 0 && tid == 0) { a.alpha[j] = alpha; a.beta[j] = beta; }
        tscale = fmax(tscale, fabs(alpha) + beta);
        if (j + 1 == a.m || beta <= 1e-14 * tscale) { mk = j + 1; break; }
        for (int64_t i = gt; i < R; i += GT) V[(int64_t)(j + 1) * R + i] = a.w[i] / beta;
        if (!gsync()) { bail(); return; }
      }
    }
    if (mk == j + 1) break;
  }
  if (!gsync()) { bail(); return; }

  // (2) extreme eigenvalues of the tridiagonal matrix, warp 0 of CTA 0
  if (g != 0 || warp != 0) return;
  for (int i = lane; i < mk; i += 32) { ab_s[0][i] = a.alpha[i]; ab_s[1][i] = a.beta[i]; }
  __syncwarp();
  const double *al = ab_s[0], *be = ab_s[1];
  double lo = 0.0, hi = 0.0, sc = 0.0;
  for (int i = 0; i < mk; ++i) {
    const double off = (i > 0 ? fabs(be[i - 1]) : 0.0) + (i + 1 < mk ? fabs(be[i]) : 0.0);
    lo = i == 0 ? al[i] - off : fmin(lo, al[i] - off);
    hi = i == 0 ? al[i] + off : fmax(hi, al[i] + off);
    sc = fmax(sc, fabs(al[i]) + off);
  }
  const double pmin = 1e-300 + 1e-30 * sc;
  const double lmax = warp_tri_eig(al, be, mk, mk - 1, lo, hi, pmin, lane);
  const double lmin = warp_tri_eig(al, be, mk, 0, lo, hi, pmin, lane);
  // Ritz residual of the top pair: beta_m |s_m| with s the tridiagonal's
  // eigenvector (three steps of inverse iteration, Thomas algorithm)
  double resid = 0.0;
  if (lane == 0) {
    double s_last = 1.0;
    if (mk > 1) {
      // solve (Tm - mu I) y = z three times, z the previous normalised y
      const double mu = lmax + 1e-12 * fmax(sc, 1e-300);
      double ynorm_last = 0.0;
      double *z = zc_s[0], *c = zc_s[1];
      for (int i = 0; i < mk; ++i) z[i] = 1.0;
      for (int itn = 0; itn < 3; ++itn) {
        // forward elimination with diagonal d_i and right-hand side z
        double d = al[0] - mu;
        if (fabs(d) < pmin) d = pmin;
        c[0] = be[0] / d;
        z[0] = z[0] / d;
        for (int i = 1; i < mk; ++i) {
          d = al[i] - mu - be[i - 1] * c[i - 1];
          if (fabs(d) < pmin) d = pmin;
          c[i] = i + 1 < mk ? be[i] / d : 0.0;
          z[i] = (z[i] - be[i - 1] * z[i - 1]) / d;
        }
        for (int i = mk - 2; i >= 0; --i) z[i] -= c[i] * z[i + 1];
        double nz = 0.0;
        for (int i = 0; i < mk; ++i) nz += z[i] * z[i];
        nz = sqrt(nz);
        for (int i = 0; i < mk; ++i) z[i] /= nz;
        ynorm_last = z[mk - 1];
      }
      s_last = ynorm_last;
    }
    resid = fabs(be[mk - 1] * s_last);
  }
  if (lane == 0) {
    nqs_spectrum_stats st;
    st.lambda_max = lmax;
    st.lambda_min_ritz = lmin;
    st.kappa = a.lam > 0.0 ? (lmax + a.lam) / a.lam : INFINITY;
    st.digits_fp32 = -log10(st.kappa * 1.1920928955078125e-07);
    st.digits_fp64 = -log10(st.kappa * 2.220446049250313e-16);
    st.residual = resid;
    st.iterations = mk;
    st.status = *reinterpret_cast<volatile int32_t *>(a.status);
    *a.out = st;
  }
}

}  // namespace

extern "C" size_t nqs_spectrum_workspace(int64_t R, int m) {
  if (R < 1 || m < 1 || m > LZ_MAX_M) return 0;
  return lz_layout(R, m).total;
}

extern "C" nqs_status nqs_spectrum(const double *T, int64_t R, double lambda, int m,
                                   uint64_t seed, void *work, size_t work_bytes,
                                   nqs_spectrum_stats *out, void *stream) {
  if (!T || !work || !out || R < 1 || m < 1 || m > LZ_MAX_M || !(lambda >= 0.0))
    return NQS_ERR_ARG;
  if ((reinterpret_cast<uintptr_t>(work) & 255) != 0) return NQS_ERR_ARG;
  if (m > R) m = (int)R;  // the Krylov space has at most R dimensions
  const LzLayout L = lz_layout(R, m);
  if (work_bytes < L.total) return NQS_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0, per = 0, coop = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return NQS_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess)
    return NQS_ERR_CUDA;
  if (!coop) return NQS_ERR_UNSUPPORTED;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_lanczos, LZ_THREADS, 0) != cudaSuccess)
    return NQS_ERR_CUDA;
  if (per < 1) return NQS_ERR_UNSUPPORTED;
  int G = sms < LZ_MAX_GRID ? sms : LZ_MAX_GRID;
  char *w = static_cast<char *>(work);
  LzArgs a;
  a.T = T; a.R = R; a.lam = lambda; a.m = m; a.seed = seed;
  a.bar = reinterpret_cast<unsigned *>(w + L.hdr);
  a.status = reinterpret_cast<int32_t *>(w + L.hdr + 4);
  a.alpha = reinterpret_cast<double *>(w + L.alpha);
  a.beta = reinterpret_cast<double *>(w + L.beta);
  a.h1 = reinterpret_cast<double *>(w + L.h1);
  a.h2 = reinterpret_cast<double *>(w + L.h2);
  a.part = reinterpret_cast<double *>(w + L.part);
  a.w = reinterpret_cast<double *>(w + L.w);
  a.V = reinterpret_cast<double *>(w + L.V);
  a.out = out;
  if (cudaMemsetAsync(w + L.hdr, 0, 8, st) != cudaSuccess) return NQS_ERR_CUDA;
  if (cudaMemsetAsync(out, 0, sizeof(nqs_spectrum_stats), st) != cudaSuccess) return NQS_ERR_CUDA;
  void *args[] = {&a};
  if (cudaLaunchCooperativeKernel((const void *)k_lanczos, dim3(G), dim3(LZ_THREADS), args, 0, st) !=
      cudaSuccess)
    return NQS_ERR_CUDA;
  return NQS_OK;
}
