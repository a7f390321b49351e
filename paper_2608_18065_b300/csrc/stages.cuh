// stages.cuh -- the non-recurrent stages of one minSR step (sm_103a):
// parameter packing, connected-configuration lists and local-energy
// reduction (Sec. II.C), FP64 energy statistics (Eq. energy, Eq. vscore),
// centring and real representation (Algorithm 1, log-derivative and Gram steps), the FP64
// blocked Cholesky solve (Eq. minsrR) and the update with momentum (App. B).
#pragma once
#include "common.cuh"
#include "pack.cuh"

namespace nqs {

// ----------------------------------------------- Hamiltonian op tables
// Off-diagonal operator o: kind 1 = flip f1 (and f2 >= 0) with element
// coeff * z(z1) * z(z2); kind 2 = exchange of f1, f2 if antiparallel with
// element coeff.  sign carries the Marshall factor (-1)^{#flips on A}.
struct OffOp {
  int kind, f1, f2, z1, z2, start, pad0, pad1;
  double coeff;
};
struct DiagOp {
  int z1, z2;
  double coeff;
};

__device__ __forceinline__ double zval(const uint8_t *sp, int k) {
  return k < 0 ? 1.0 : (sp[k] ? -1.0 : 1.0);
}

// One CTA per off-diagonal operator: list the samples it connects
// (compacted, ascending), their matrix elements, and zero its slots of the
// per-(operator, sample) contribution matrix.
__global__ void k_eloc_gen(const OffOp *__restrict__ ops, const uint8_t *__restrict__ spins,
                           int N, int64_t ns, int *item_s, double *item_e, int *item_cnt,
                           double *contrib) {
  const int o = blockIdx.x;
  const OffOp op = ops[o];
  __shared__ int warp_tot[32];
  __shared__ int running;
  if (threadIdx.x == 0) running = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int64_t s0 = 0; s0 < ns; s0 += blockDim.x) {
    const int64_t s = s0 + threadIdx.x;
    int conn = 0;
    double el = 0.0;
    if (s < ns) {
      const uint8_t *sp = spins + s * N;
      if (op.kind == 1) {
        conn = 1;
        el = op.coeff * zval(sp, op.z1) * zval(sp, op.z2);
      } else {
        conn = sp[op.f1] != sp[op.f2];
        el = op.coeff;
      }
      double *c = contrib + ((int64_t)o * ns + s) * 2;
      c[0] = 0.0; c[1] = 0.0;
    }
    const unsigned bal = __ballot_sync(0xffffffffu, conn);
    const int before = __popc(bal & ((1u << lane) - 1u));
    if (lane == 0) warp_tot[wid] = __popc(bal);
    __syncthreads();
    int off = 0, tot = 0;
    for (int w2 = 0; w2 < nw; ++w2) {
      if (w2 < wid) off += warp_tot[w2];
      tot += warp_tot[w2];
    }
    if (conn) {
      const int pos = running + off + before;
      item_s[(int64_t)o * ns + pos] = (int)s;
      item_e[(int64_t)o * ns + pos] = el;
    }
    __syncthreads();
    if (threadIdx.x == 0) running += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) item_cnt[o] = running;
}

// eps_s = sum of diagonal elements + sum over operators of the connected
// contributions (already H_ss' Psi(s')/Psi(s)).
// One warp per sample: the lanes take the diagonal terms and the operators'
// contributions in strides of 32, then a fixed-order shuffle tree.
__global__ void k_eloc_reduce(const DiagOp *__restrict__ dops, int n_diag, int n_off,
                              const uint8_t *__restrict__ spins, int N, int64_t ns,
                              const double *__restrict__ contrib, double *eloc) {
  const int lane = threadIdx.x & 31;
  const int64_t s = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (s >= ns) return;  // uniform over the warp
  const uint8_t *sp = spins + s * N;
  double re = 0.0, im = 0.0;
  for (int d = lane; d < n_diag; d += 32)
    re += dops[d].coeff * zval(sp, dops[d].z1) * zval(sp, dops[d].z2);
  for (int o = lane; o < n_off; o += 32) {
    const double *c = contrib + ((int64_t)o * ns + s) * 2;
    re += c[0];
    im += c[1];
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, off);
    im += __shfl_xor_sync(0xffffffffu, im, off);
  }
  if (lane == 0) {
    eloc[2 * s] = re;
    eloc[2 * s + 1] = im;
  }
}
// threads of k_eloc_reduce for ns samples
inline int64_t eloc_reduce_threads(int64_t ns) { return ns * 32; }

// ------------------------------------------------------ energy stats
// One CTA: E = mean eps, var = mean |eps - E|^2, V-score; then
// eps-bar' = 2 (Re, -Im)(eps - E)^* / sqrt(Ns) = 2 (Re(eps-E), Im(eps-E)) / sqrt(Ns).
__global__ void k_energy(const double *__restrict__ eloc, int64_t ns, int N, int cplx,
                         nqs_step_stats *st, double *eps) {
  __shared__ double sr[1024], si[1024];
  double r = 0.0, i = 0.0;
  for (int64_t s = threadIdx.x; s < ns; s += blockDim.x) { r += eloc[2 * s]; i += eloc[2 * s + 1]; }
  sr[threadIdx.x] = r; si[threadIdx.x] = i;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) { sr[threadIdx.x] += sr[threadIdx.x + o]; si[threadIdx.x] += si[threadIdx.x + o]; }
    __syncthreads();
  }
  const double Er = sr[0] / (double)ns, Ei = si[0] / (double)ns;
  __syncthreads();
  double v = 0.0;
  const double isq = 1.0 / sqrt((double)ns);
  for (int64_t s = threadIdx.x; s < ns; s += blockDim.x) {
    const double a = eloc[2 * s] - Er, b = eloc[2 * s + 1] - Ei;
    v += a * a + b * b;
    eps[s] = 2.0 * a * isq;
    if (cplx) eps[ns + s] = 2.0 * b * isq;
  }
  sr[threadIdx.x] = v;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sr[threadIdx.x] += sr[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double var = sr[0] / (double)ns;
    st->E_re = Er; st->E_im = Ei; st->var = var;
    st->vscore = (double)N * var / (Er * Er);
    int bad = !(isfinite(Er) && isfinite(Ei) && isfinite(var));
    st->status = bad ? NQS_ERR_NONFINITE : NQS_OK;
  }
}

// ---------------------------------------------------------- centring
// Column means over the Ns samples of each block (real rows, imaginary
// rows): partial sums over 64-row chunks (grid.y = block * chunks + chunk),
// then one pass that adds the chunks in FP64.  FP64 data is summed in FP64;
// FP32 data is summed in FP32 with Knuth's error-free TwoSum on every term
// (the rounding error of each addition is recovered exactly and carried in
// a second FP32 word), which keeps the chunk sum to about twice FP32's
// precision without the FP64 pipe (64 times slower than FP32 on this part).
constexpr int COL_ROWS = 64;
template <typename T>
__global__ void k_colsum_part(const T *__restrict__ O, int64_t ns, int64_t np, int chunks,
                              double *part) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= np) return;
  const int blk = blockIdx.y / chunks, ch = blockIdx.y % chunks;
  const int64_t r0 = (int64_t)ch * COL_ROWS, r1 = min64(ns, r0 + COL_ROWS);
  const T *B = O + (int64_t)blk * ns * np;
  if constexpr (sizeof(T) == 4) {
    float sum = 0.f, err = 0.f;
#pragma unroll 8
    for (int64_t s = r0; s < r1; ++s) {
      const float x = B[s * np + p];
      const float t = sum + x, z = t - sum;
      err += (sum - (t - z)) + (x - z);
      sum = t;
    }
    part[(int64_t)blockIdx.y * np + p] = (double)sum + (double)err;
  } else {
    double acc = 0.0;
    for (int64_t s = r0; s < r1; ++s) acc += (double)B[s * np + p];
    part[(int64_t)blockIdx.y * np + p] = acc;
  }
}

// pairs: store each mean as the FP32 pair (hi, lo) with hi + lo = mean to
// about 2^-48 relative (for the FP32 centring), else as an FP64 value.
__global__ void k_colmean_fin(const double *__restrict__ part, int64_t ns, int64_t np, int chunks,
                              double *mean, int pairs) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= np) return;
  const int blk = blockIdx.y;
  double acc = 0.0;
  for (int c = 0; c < chunks; ++c) acc += part[((int64_t)blk * chunks + c) * np + p];
  const double m = acc / (double)ns;
  if (pairs) {
    const float hi = (float)m;
    reinterpret_cast<float2 *>(mean)[(int64_t)blk * np + p] = make_float2(hi, (float)(m - (double)hi));
  } else {
    mean[(int64_t)blk * np + p] = m;
  }
}

// O' = (O - mean) / sqrt(Ns), in FP64 arithmetic, stored back in T.
template <typename T>
__global__ void k_center(T *__restrict__ O, int64_t ns, int64_t np, int64_t rows,
                         const double *__restrict__ mean) {
  const double isq = 1.0 / sqrt((double)ns);
  const int64_t tot = rows * np;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / np, p = e - r * np;
    const double m = mean[(r / ns) * np + p];
    O[e] = (T)(((double)O[e] - m) * isq);
  }
}

// ------------------------------------------------------------- Gram
// T = A A^T on CUDA cores, 64x64 output tiles of the upper triangle, K in
// chunks of 16 through shared memory; accumulation in TA (double for the
// FP64 path); both triangles written.
template <typename TI, typename TA>
__global__ void __launch_bounds__(256) k_gram_simt(const TI *__restrict__ A, int64_t R, int64_t np,
                                                   double *__restrict__ T) {
  const int bi = blockIdx.y, bj = blockIdx.x;
  if (bj < bi) return;
  __shared__ TA sa[16][64 + 1], sb[16][64 + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  TA acc[4][4] = {};
  const int64_t i0 = (int64_t)bi * 64, j0 = (int64_t)bj * 64;
  for (int64_t k0 = 0; k0 < np; k0 += 16) {
    for (int e = threadIdx.x; e < 16 * 64; e += 256) {
      const int r = e / 16, kk = e % 16;
      const int64_t k = k0 + kk;
      sa[kk][r] = (i0 + r < R && k < np) ? (TA)A[(i0 + r) * np + k] : TA(0);
      sb[kk][r] = (j0 + r < R && k < np) ? (TA)A[(j0 + r) * np + k] : TA(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      TA a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) { a[q] = sa[kk][ty + 16 * q]; b[q] = sb[kk][tx + 16 * q]; }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = fma(a[p], b[q], acc[p][q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t i = i0 + ty + 16 * p, j = j0 + tx + 16 * q;
      if (i < R && j < R && j >= i) {
        T[i * R + j] = (double)acc[p][q];
        T[j * R + i] = (double)acc[p][q];
      }
    }
}

// ||T||_F, lambda (constant or coeff*||T||^pow), and the diagonal shift.
__global__ void k_lambda(double *T, int64_t R, int mode, double lam_c, double coeff, double pw,
                         nqs_step_stats *st) {
  __shared__ double s[1024];
  double acc = 0.0;
  for (int64_t e = threadIdx.x; e < R * R; e += blockDim.x) acc += T[e] * T[e];
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  const double nT = sqrt(s[0]);
  const double lam = mode == 1 ? coeff * pow(nT, pw) : lam_c;
  for (int64_t i = threadIdx.x; i < R; i += blockDim.x) T[i * R + i] += lam;
  if (threadIdx.x == 0) { st->normT = nT; st->lambda = lam; }
}

// tau = eps - lambda x (App. F), ||tau||, eta_t = eta0/(1+t/decay_T) with
// the step t read from the device, and eta* = eta_t/||tau|| in trust-region
// mode.
__global__ void k_eta(const double *__restrict__ eps, const double *__restrict__ x, int64_t R,
                      double eta0, double decay_T, int trust, const int64_t *step_dev,
                      nqs_step_stats *st, const int32_t *solve_status, const int32_t *solve_fp64) {
  __shared__ double s[1024];
  const double lam = st->lambda;
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < R; i += blockDim.x) {
    const double t = eps[i] - lam * x[i];
    acc += t * t;
  }
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double tn = sqrt(s[0]);
    double eta_t = eta0;
    if (decay_T > 0.0 && isfinite(decay_T)) eta_t = eta0 / (1.0 + (double)*step_dev / decay_T);
    st->tau_norm = tn;
    st->eta_eff = trust ? eta_t / tn : eta_t;
    if (st->status == NQS_OK && *solve_status != 0) st->status = *solve_status;
    st->solve_fp64 = *solve_fp64;
  }
}

// Partial sums of O'x over row chunks: part[c][p] = sum_{r in chunk c} A[r][p] x[r].
template <typename T>
__global__ void k_gemv_part(const T *__restrict__ A, int64_t R, int64_t np,
                            const double *__restrict__ x, int rows_per, double *part) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= np) return;
  const int64_t r0 = (int64_t)blockIdx.y * rows_per;
  const int64_t r1 = min64(R, r0 + rows_per);
  double acc = 0.0;
  for (int64_t r = r0; r < r1; ++r) acc += (double)A[r * np + p] * x[r];
  part[(int64_t)blockIdx.y * np + p] = acc;
}

// delta theta = eta_eff * sum of the partials; flags non-finite values.
__global__ void k_dtheta(const double *__restrict__ part, int nparts, int64_t np,
                         nqs_step_stats *st, double *dth) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= np) return;
  double acc = 0.0;
  for (int c = 0; c < nparts; ++c) acc += part[(int64_t)c * np + p];
  const double d = st->eta_eff * acc;
  dth[p] = d;
  if (!isfinite(d)) atomicCAS(reinterpret_cast<int *>(&st->status), (int)NQS_OK, (int)NQS_ERR_NONFINITE);
}

// ------------------------------------------------- sample-sharded step
// Partial sums of a rank's samples: the chunk partials of k_colsum_part
// added up without dividing (per block, [blk][np]).
__global__ void k_colsum_fin(const double *__restrict__ part, int64_t np, int chunks,
                             double *sums) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= np) return;
  const int blk = blockIdx.y;
  double acc = 0.0;
  for (int c = 0; c < chunks; ++c) acc += part[((int64_t)blk * chunks + c) * np + p];
  sums[(int64_t)blk * np + p] = acc;
}

// sum Re eps, sum Im eps, sum |eps|^2 of a rank's local energies (one block)
__global__ void k_energy_sums(const double *__restrict__ eloc, int64_t n, double *out) {
  __shared__ double a[1024], b[1024], q[1024];
  double r = 0.0, i = 0.0, m = 0.0;
  for (int64_t s = threadIdx.x; s < n; s += blockDim.x) {
    const double x = eloc[2 * s], y = eloc[2 * s + 1];
    r += x; i += y; m += x * x + y * y;
  }
  a[threadIdx.x] = r; b[threadIdx.x] = i; q[threadIdx.x] = m;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      a[threadIdx.x] += a[threadIdx.x + o];
      b[threadIdx.x] += b[threadIdx.x + o];
      q[threadIdx.x] += q[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) { out[0] = a[0]; out[1] = b[0]; out[2] = q[0]; }
}

// E, Var (= sum |eps|^2 / Ns - |E|^2) and the V-score from the summed
// energies of all ranks, and this rank's rows of eps-bar' (as k_energy)
__global__ void k_shard_eps(const double *__restrict__ eloc, int64_t n, int N, int cplx,
                            const double *__restrict__ esum, int64_t ns, nqs_step_stats *st,
                            double *eps) {
  const double Er = esum[0] / (double)ns, Ei = esum[1] / (double)ns;
  const double isq = 1.0 / sqrt((double)ns);
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n;
       s += (int64_t)gridDim.x * blockDim.x) {
    eps[s] = 2.0 * (eloc[2 * s] - Er) * isq;
    if (cplx) eps[n + s] = 2.0 * (eloc[2 * s + 1] - Ei) * isq;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const double var = esum[2] / (double)ns - (Er * Er + Ei * Ei);
    st->E_re = Er; st->E_im = Ei; st->var = var;
    st->vscore = (double)N * var / (Er * Er);
    int bad = !(isfinite(Er) && isfinite(Ei) && isfinite(var));
    st->status = bad ? NQS_ERR_NONFINITE : NQS_OK;
  }
}

// A rank's rows of O' = (O - sum / Ns) / sqrt(Ns) into out (FP64
// arithmetic, rounded once to the working precision); sums per block.
template <typename T>
__global__ void k_shard_center(const T *__restrict__ O, int64_t n, int64_t np, int64_t rows,
                               const double *__restrict__ sums, int64_t ns, T *__restrict__ out) {
  const double isq = 1.0 / sqrt((double)ns), ins = 1.0 / (double)ns;
  const int64_t tot = rows * np;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / np, p = e - r * np;
    const double m = sums[(r / n) * np + p] * ins;
    out[e] = (T)(((double)O[e] - m) * isq);
  }
}

// partial products of columns p0 .. p0 + nc - 1 of a row-major A (row
// stride lda) with x over rows_per rows per grid.y block
template <typename T>
__global__ void k_gemv_cols(const T *__restrict__ A, int64_t R, int64_t lda, int64_t p0,
                            int64_t nc, const double *__restrict__ x, int rows_per, double *part) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= nc) return;
  const int64_t r0 = (int64_t)blockIdx.y * rows_per;
  const int64_t r1 = min64(R, r0 + rows_per);
  double acc = 0.0;
  for (int64_t r = r0; r < r1; ++r) acc += (double)A[r * lda + p0 + q] * x[r];
  part[(int64_t)blockIdx.y * nc + q] = acc;
}

// flags a non-finite delta theta (all shards gathered) in the step status
__global__ void k_check_finite(const double *__restrict__ v, int64_t n, nqs_step_stats *st) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    if (!isfinite(v[i]))
      atomicCAS(reinterpret_cast<int *>(&st->status), (int)NQS_OK, (int)NQS_ERR_NONFINITE);
}

// ------------------------------------------------------------- Adam
// g = sum of the partial products Obar'^T eps-bar' (the sampled energy
// gradient); a non-finite entry flags the step.
__global__ void k_grad_sum(const double *__restrict__ part, int nparts, int64_t np,
                           nqs_step_stats *st, double *g) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= np) return;
  double acc = 0.0;
  for (int c = 0; c < nparts; ++c) acc += part[(int64_t)c * np + p];
  g[p] = acc;
  if (!isfinite(acc)) atomicCAS(reinterpret_cast<int *>(&st->status), (int)NQS_OK, (int)NQS_ERR_NONFINITE);
}

// Adam (Kingma and Ba) with bias corrections of iteration t = step + 1 and
// eta_t = eta0 / (1 + step / T); only when the step's status is OK.
__global__ void k_adam(double *theta, double *m, double *v, const double *__restrict__ g,
                       int64_t np, double b1, double b2, double eps, double eta0, double decay_T,
                       int64_t step, nqs_step_stats *st) {
  if (st->status != NQS_OK) return;
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= np) return;
  const double t = (double)(step + 1);
  const double eta = (decay_T > 0.0 && isfinite(decay_T)) ? eta0 / (1.0 + (double)step / decay_T)
                                                           : eta0;
  const double gp = g[p];
  const double mp = b1 * m[p] + (1.0 - b1) * gp, vp = b2 * v[p] + (1.0 - b2) * gp * gp;
  m[p] = mp;
  v[p] = vp;
  const double mh = mp / (1.0 - pow(b1, t)), vh = vp / (1.0 - pow(b2, t));
  theta[p] -= eta * mh / (sqrt(vh) + eps);
  if (p == 0) st->eta_eff = eta;
}

// theta0 + x v1 + y v2 (a point of the loss landscape)
__global__ void k_axpy2(const double *__restrict__ t0, const double *__restrict__ v1,
                        const double *__restrict__ v2, double x, double y, int64_t n,
                        double *out) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p < n) out[p] = t0[p] + x * v1[p] + y * v2[p];
}

// E (re, im), Var and the status of a landscape point
__global__ void k_scan_store(const nqs_step_stats *st, double *out) {
  out[0] = st->E_re; out[1] = st->E_im; out[2] = st->var; out[3] = (double)st->status;
}

// m <- mu m + (1-mu) dtheta; theta <- theta - m (App. B), only when the
// step's status is OK.
__global__ void k_apply(double *theta, double *mom, const double *__restrict__ dth, int64_t np,
                        double mu, const nqs_step_stats *st) {
  if (st->status != NQS_OK) return;
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= np) return;
  const double m = mu * mom[p] + (1.0 - mu) * dth[p];
  mom[p] = m;
  theta[p] -= m;
}

}  // namespace nqs
