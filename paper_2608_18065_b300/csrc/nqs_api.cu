// nqs_api.cu -- the C-ABI of libnqs (include/nqs.h): context, workspace
// carving, Hamiltonian tables and the stream-ordered minSR step.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "chol_coop.cuh"
#include "chol_blk.cuh"
#include "chol_ir.cuh"
#include "eloc_tc.h"
#include "eloc2d_tc.h"
#include "jac_tc.h"
#include "gram_tc.h"
#include "launch.h"
#include "stages.cuh"

using namespace nqs;

namespace {

struct WsOff {
  size_t pack, spins, logpsi, hcache, lccache, eloc, item_s, item_e, item_cnt, contrib, colbuf,
      adj, adjcol, O, mean, T, eps, x, part, dth, frob, sstat, split, crhs, cy, cpart, cbar, gcache, L32, Li32, Tm32, wv32, dpart32, dg32, dstep, tth, tmo, tstats, hseg, carry, dlm, wimg, tctr, total;
};

}  // namespace

struct nqs_ctx {
  nqs_model_desc m;
  nqs_ham_desc h;
  int prec;  // nqs_precision
  int64_t max_ns;
  Layout L;
  PackOff P;
  RecDesc rd;
  int n_off = 0, n_diag = 0;
  std::vector<int> op_start;  // first changed site of each off-diagonal operator
  OffOp *d_off = nullptr;
  DiagOp *d_diag = nullptr;
  int *d_opf = nullptr;
  int eloc_grid = 0, eloc_R = 0;
  int adjw = 0;
  int gw = 0;  // gate-cache record width: 4 dh (+ dh in 2D)
  size_t es = 8;  // element size of the recurrence precision
  // hidden-state checkpoints (1D): stride ck (0 = every state cached), nck
  // checkpoint slots, nseg segments of the reverse sweep
  int ck = 0, nck = 0, nseg = 1;
  // Levenberg-Marquardt damping factor (0: off); the damping lives on the device
  double lm_omega = 0.0;
  // tests of failure detection (nqs_test_wait_timeout): wait limit of the
  // streamed local-energy engine and its dropped tile
  unsigned long long test_spin_limit = 0;
  int solve_form = -1;  // nqs_set_solve_form (-1: tuned or built-in)
  int sampler_form = -1;  // nqs_set_sampler (-1: built-in)
  int test_drop_tile = 0;
  WsOff off{};
  char *ws = nullptr;
  size_t ws_bytes = 0;
  int nsplit = 1;
  // instrumentation: (NQS_N_STAGES + 1) boundary events per timed step
  std::vector<cudaEvent_t> tev;
  int tmax = 0, tstep = 0;
  int64_t launches = 0;
  // CUDA graph of the step (optional)
  int graph_enabled = 0, graph_broken = 0;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t gexec = nullptr;
  struct Key {
    const void *theta, *mom, *stats;
    nqs_step_hparams hp;  // step_index ignored
  } gkey{};
  int64_t gnext = -1;
  // launch shapes chosen by nqs_autotune for tuned_ns samples (0 = built-in)
  int64_t tuned_ns = 0;
  int t_eloc_grid = 0, t_gram_splits = 0, t_solve_grid = 0, t_chol_var = -1, t_chol_subst = -1;
  double t_ms[3] = {0, 0, 0}, t_ms_default[3] = {0, 0, 0};
  int64_t cur_ns = 0;  // sample count of the step being issued
  // batched steps: order this context's cooperative solve after another's
  cudaEvent_t solve_wait = nullptr, solve_rec = nullptr;
  // batched steps by stage: issue only the part of the step up to the
  // local-energy engine (STEP_PRE_A), from there to the solve (STEP_PRE_B)
  // or from the solve on (STEP_POST); in_group: the FP32 factor runs in the
  // batch's grouped launch; in_eloc_group: so does the streamed local-energy
  // engine, with the arguments left in eloc_args
  int phase = 0, in_group = 0, in_eloc_group = 0;
  Eloc2dTcArgs eloc_args{};
  // batched steps: the local-energy engine takes this many eighths of its
  // grid (the rest of the SMs stays free for the other instances' kernels)
  int eloc_eighths = 8;
};

constexpr int STEP_ALL = 0, STEP_PRE_A = 1, STEP_PRE_B = 2, STEP_POST = 3;
constexpr int GROUP_SOLVE = 1, GROUP_ELOC = 2;

namespace {

inline size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

bool f32(const nqs_ctx *c) { return c->prec == NQS_PREC_MIXED; }

// Off-diagonal and diagonal operator tables of the Hamiltonian families
// (Sec. III), sites in path order.
void build_hamiltonian(const nqs_model_desc &m, const nqs_ham_desc &h, std::vector<OffOp> &off,
                       std::vector<DiagOp> &dg) {
  const int N = m.Lx * m.Ly;
  auto col = [&](int k) {
    int j = k / m.Lx, r = k % m.Lx;
    return (j % 2 == 0) ? r : m.Lx - 1 - r;
  };
  auto onA = [&](int k) { return ((col(k) + k / m.Lx) % 2) == 1; };
  auto flip_op = [&](int kind, int f1, int f2, int z1, int z2, double coeff) {
    OffOp o{};
    o.kind = kind; o.f1 = f1; o.f2 = f2; o.z1 = z1; o.z2 = z2;
    o.start = f2 >= 0 ? std::min(f1, f2) : f1;
    double s = 1.0;
    if (m.marshall) {
      if (onA(f1)) s = -s;
      if (f2 >= 0 && onA(f2)) s = -s;
    }
    o.coeff = coeff * s;
    off.push_back(o);
  };
  switch (h.family) {
    case NQS_HAM_TFIM:
      for (int i = 0; i + 1 < N; ++i) dg.push_back(DiagOp{i, i + 1, -h.J});
      for (int i = 0; i < N; ++i) flip_op(1, i, -1, -1, -1, -h.h);
      break;
    case NQS_HAM_CLUSTER_ZXZ:
      for (int i = 1; i + 1 < N; ++i) flip_op(1, i, -1, i - 1, i + 1, -1.0);
      break;
    case NQS_HAM_CLUSTER_PAPER:
      // 1-indexed k = 2..N-2: X_{k-1} Z_k X_{k+1} -> 0-indexed (k-2, k-1, k)
      for (int k = 2; k <= N - 2; ++k) flip_op(1, k - 2, k, k - 1, -1, -1.0);
      flip_op(1, 1, -1, 0, -1, -1.0);           // Z_1 X_2
      flip_op(1, N - 2, N - 1, -1, -1, -1.0);   // X_{N-1} X_N
      flip_op(1, N - 3, -1, N - 2, N - 1, -1.0);// X_{N-2} Z_{N-1} Z_N
      break;
    case NQS_HAM_J1J2: {
      std::vector<int> idx((size_t)m.Lx * m.Ly);
      for (int k = 0; k < N; ++k) idx[(size_t)(k / m.Lx) * m.Lx + col(k)] = k;
      auto at = [&](int i, int j) {
        return (i < 0 || i >= m.Lx || j < 0 || j >= m.Ly) ? -1 : idx[(size_t)j * m.Lx + i];
      };
      for (int j = 0; j < m.Ly; ++j)
        for (int i = 0; i < m.Lx; ++i) {
          const int k = at(i, j);
          const int nb[4] = {at(i + 1, j), at(i, j + 1), at(i + 1, j + 1), at(i + 1, j - 1)};
          const double J[4] = {h.J1, h.J1, h.J2, h.J2};
          for (int q = 0; q < 4; ++q) {
            if (nb[q] < 0 || J[q] == 0.0) continue;
            dg.push_back(DiagOp{k, nb[q], J[q] / 4.0});
            flip_op(2, k, nb[q], -1, -1, J[q] / 2.0);
          }
        }
      break;
    }
  }
  std::stable_sort(off.begin(), off.end(),
                   [](const OffOp &a, const OffOp &b) { return a.start < b.start; });
}

// the last CUDA error a call of this thread returned as NQS_ERR_CUDA
thread_local cudaError_t g_last_cuda = cudaSuccess;
nqs_status cu(cudaError_t e) {
  if (e == cudaSuccess) return NQS_OK;
  g_last_cuda = e;
  return NQS_ERR_CUDA;
}
#define CU(x) do { cudaError_t _e = (x); if (_e != cudaSuccess) { g_last_cuda = _e; return NQS_ERR_CUDA; } } while (0)
#define ST(x) do { nqs_status _s = (x); if (_s != NQS_OK) return _s; } while (0)

void carve(nqs_ctx *c) {
  const int64_t ns = c->max_ns, N = c->L.N, dh = c->L.dh, np = c->L.np;
  const int64_t R = c->L.cplx ? 2 * ns : ns;
  const size_t es = c->es;
  WsOff &o = c->off;
  size_t p = 0;
  auto take = [&](size_t bytes) { size_t at = p; p = al256(p + bytes); return at; };
  o.pack = take(c->P.total * es);
  o.spins = take(ns * N);
  o.logpsi = take(ns * 2 * 8);
  o.hcache = take(c->ck ? ns * std::max(c->nck, 1) * dh * es : ns * N * dh * es);
  o.lccache = take(ns * N * 2 * es);
  o.eloc = take(ns * 2 * 8);
  o.item_s = take((size_t)c->n_off * ns * 4);
  o.item_e = take((size_t)c->n_off * ns * 8);
  o.item_cnt = take((size_t)c->n_off * 4);
  o.contrib = take((size_t)c->n_off * ns * 16);
  // column buffers of the 2D local-energy engines: the SIMT / warp-MMA
  // engines' grid x 64 rows, the tensor-core engine's SM count x 128
  size_t cb_rows = (size_t)c->eloc_grid * c->eloc_R;
  if (c->L.dim == 2 && c->es == 4 &&
      (eloc2d_tc_supported(c->L.dim, (int)dh) || eloc2d_tcs_supported(c->L.dim, (int)dh)))
    cb_rows = std::max(cb_rows, (size_t)c->rd.sm_count * ELOC2D_TC_ROWS);
  // (a hidden size 32 lattice on the tensor-core engine runs padded to 64)
  const size_t cbw = (c->L.dim == 2 && c->es == 4 && eloc2d_tc_supported(c->L.dim, (int)dh))
                         ? std::max<int64_t>(dh, 64) : dh;
  o.colbuf = take(c->L.dim == 2 ? cb_rows * c->L.Lx * cbw * es : 0);
  o.adj = take(R * (c->ck ? c->ck : N) * c->adjw * es);
  o.adjcol = take(c->L.dim == 2 ? R * c->L.Lx * dh * es : 0);
  o.O = take(R * np * es);
  o.mean = take(2 * np * 8);
  o.T = take(R * R * 8);
  o.eps = take(R * 8);
  o.x = take(R * 8);
  c->nsplit = (int)((R + 63) / 64) + 2;  // also holds the column-sum chunks
  o.part = take((size_t)c->nsplit * np * 8);
  o.dth = take(np * 8);
  o.frob = take(1024 * 8);
  o.sstat = take(64);
  o.tctr = take(64);  // tile counter of the tensor-core local-energy engines
  o.split = take(gram_tc_split_bytes(R, np));
  o.crhs = take(R * 8);
  o.cy = take(R * 8);
  o.cpart = take((size_t)2 * c->rd.sm_count * CC_B * 8);
  o.cbar = take(64);
  o.gcache = take(ns * (c->ck ? c->ck : N) * c->gw * es);
  o.hseg = take(c->ck ? ns * (c->ck + 1) * dh * es : 0);
  o.carry = take(c->ck ? R * dh * es : 0);
  o.dlm = take(64);
  o.wimg = take(c->L.dim == 2 && c->es == 4 ? eloc2d_tcs_image_bytes((int)dh) : 0);
  o.L32 = take(c->prec == NQS_PREC_MIXED ? R * R * 4 : 0);
  o.Li32 = take(c->prec == NQS_PREC_MIXED ? R * R * 4 : 0);
  o.Tm32 = take(c->prec == NQS_PREC_MIXED ? R * R * 4 : 0);
  o.wv32 = take(R * 4);
  o.dpart32 = take(((R + 63) / 64) * R * 4);
  o.dg32 = take(c->prec == NQS_PREC_MIXED ? 2 * IR_DG * 4 : 0);
  o.dstep = take(64);
  o.tth = take(np * 8);
  o.tmo = take(np * 8);
  o.tstats = take(256);
  o.total = p;
}

template <typename T> T *W(nqs_ctx *c, size_t off) { return reinterpret_cast<T *>(c->ws + off); }

nqs_status need_ws(nqs_ctx *c) { return c->ws ? NQS_OK : NQS_ERR_WORKSPACE; }

// Tuned launch shapes apply to the sample count they were measured for.
bool tuned(const nqs_ctx *c) { return c->tuned_ns > 0 && c->tuned_ns == c->cur_ns; }
int eloc_grid_cap(const nqs_ctx *c, int dflt) {
  const int g = tuned(c) && c->t_eloc_grid > 0 ? std::min(c->t_eloc_grid, dflt) : dflt;
  return std::max(1, g * c->eloc_eighths / 8);
}
int gram_splits(const nqs_ctx *c) { return tuned(c) ? c->t_gram_splits : 0; }
// grid of the cooperative solve: the tuned value (at most two CTAs per SM,
// which the launch checks against the kernel's occupancy), else one per SM
int solve_grid(const nqs_ctx *c) {
  return tuned(c) && c->t_solve_grid > 0 ? std::min(c->t_solve_grid, 2 * c->rd.sm_count)
                                         : c->rd.sm_count;
}

// Record stage boundary i of the current step when a timing window is open.
void mark(nqs_ctx *c, int i, cudaStream_t st) {
  if (c->tstep < c->tmax) cudaEventRecord(c->tev[(size_t)c->tstep * (NQS_N_STAGES + 1) + i], st);
}

template <typename T> nqs_status pack_theta(nqs_ctx *c, const double *theta, cudaStream_t st) {
  const int64_t tot = c->P.total;
  const int blocks = (int)std::min<int64_t>((tot + 255) / 256, 4096);
  k_pack<T><<<blocks, 256, 0, st>>>(theta, W<T>(c, c->off.pack), c->L, c->P);
  c->launches += 1;
  return cu(cudaGetLastError());
}

template <typename T>
FwdArgs<T> fwd_args(nqs_ctx *c) {
  FwdArgs<T> a{};
  a.pack = W<T>(c, c->off.pack);
  a.N = c->L.N; a.Lx = c->L.Lx; a.cplx = c->L.cplx; a.marshall = c->L.marshall; a.zmask = c->L.zmask;
  a.hcache = W<T>(c, c->off.hcache);
  a.lccache = W<T>(c, c->off.lccache);
  a.ck = c->ck;
  a.nck = c->nck;
  return a;
}

// Alg. 1, sampling.  Mixed-precision 2D models of hidden size 96 or 128
// with every state cached draw on the streamed tensor-core engine (the same
// uniforms, the same FP32 decision, the same caches); the others on the
// recurrence kernels' sampler.
template <typename T>
nqs_status run_sample(nqs_ctx *c, const FwdArgs<T> &a, cudaStream_t st) {
  if constexpr (std::is_same<T, float>::value) {
    if (c->sampler_form != 0 && c->ck == 0 && gram_tc_available() &&
        eloc2d_tcs_sample_supported(c->L.dim, c->L.dh, c->L.Lx)) {
      Eloc2dTcArgs e{};
      e.pack = a.pack;
      e.oWgT = (int)c->P.WgT; e.oxw = (int)c->P.xw; e.obias = (int)c->P.bias;
      e.ohead = (int)c->P.head; e.ohc = (int)c->P.hc; e.oU12T = (int)c->P.U12T;
      e.N = c->L.N; e.Lx = c->L.Lx; e.cplx = c->L.cplx; e.zmask = c->L.zmask; e.ns = a.nrows;
      e.ntiles = (int)((a.nrows + ELOC2D_TC_ROWS - 1) / ELOC2D_TC_ROWS);
      e.colbuf = W<float>(c, c->off.colbuf);
      e.err = W<int>(c, c->off.sstat);
      e.tile_ctr = W<int>(c, c->off.tctr);
      e.wimg = reinterpret_cast<const unsigned char *>(c->ws + c->off.wimg);
      e.spin_limit = c->test_spin_limit;
      e.seed = a.seed; e.step = a.step; e.step_dev = a.step_dev; e.s0 = a.s0;
      e.marshall = c->L.marshall;
      e.spins_out = a.spins; e.logpsi = a.logpsi;
      e.hcache_out = a.hcache; e.lccache_out = a.lccache; e.gcache = a.gcache;
      c->launches += 2;
      CU(cudaMemsetAsync(e.tile_ctr, 0, sizeof(int), st));
      return cu(eloc2d_tcs_sample(e, c->L.dh, eloc_grid_cap(c, c->rd.sm_count), st));
    }
  }
  c->launches += 1;
  return cu(run_forward<T>(c->rd, MODE_SAMPLE, a, 0, st));
}

// with_gates: also store the gate activations the reverse sweep reads.
template <typename T>
nqs_status forward_T(nqs_ctx *c, int mode, int64_t n, uint64_t seed, uint64_t step, uint8_t *spins,
                     double *logpsi, cudaStream_t st, bool with_gates = false) {
  FwdArgs<T> a = fwd_args<T>(c);
  a.nrows = n; a.seed = seed; a.step = step; a.spins = spins; a.logpsi = logpsi;
  if (with_gates && c->ck == 0) {
    a.gcache = W<T>(c, c->off.gcache);
    a.gw = c->gw;
  }
  if (mode == MODE_SAMPLE) return run_sample<T>(c, a, st);
  c->launches += 1;
  return cu(run_forward<T>(c->rd, mode, a, 0, st));
}

nqs_status forward(nqs_ctx *c, int mode, int64_t n, uint64_t seed, uint64_t step, uint8_t *spins,
                   double *logpsi, cudaStream_t st, bool with_gates = false) {
  return f32(c) ? forward_T<float>(c, mode, n, seed, step, spins, logpsi, st, with_gates)
                : forward_T<double>(c, mode, n, seed, step, spins, logpsi, st, with_gates);
}

template <typename T> nqs_status pack(nqs_ctx *c, const double *theta, cudaStream_t st) {
  return pack_theta<T>(c, theta, st);
}
nqs_status pack_any(nqs_ctx *c, const double *theta, cudaStream_t st) {
  return f32(c) ? pack<float>(c, theta, st) : pack<double>(c, theta, st);
}

// Local energies of the ns configurations whose hidden states are cached.
template <typename T>
// part: 0 the whole stage; 1 up to the engine of the streamed local-energy
// engine, whose arguments go to c->eloc_args for a grouped launch; 2 the
// reduction after that launch.
nqs_status eloc_T(nqs_ctx *c, int64_t ns, const uint8_t *spins, double *eloc, cudaStream_t st,
                  int part = 0) {
  if (part == 2) {
    mark(c, 4, st);
    c->launches += 1;
    k_eloc_reduce<<<(unsigned)((eloc_reduce_threads(ns) + 255) / 256), 256, 0, st>>>(
        c->d_diag, c->n_diag, c->n_off, spins, c->L.N, ns, W<double>(c, c->off.contrib), eloc);
    return cu(cudaGetLastError());
  }
  mark(c, 2, st);
  if (c->n_off > 0) {
    c->launches += 2;
    k_eloc_gen<<<c->n_off, 256, 0, st>>>(c->d_off, spins, c->L.N, ns, W<int>(c, c->off.item_s),
                                         W<double>(c, c->off.item_e), W<int>(c, c->off.item_cnt),
                                         W<double>(c, c->off.contrib));
    CU(cudaGetLastError());
    FwdArgs<T> a = fwd_args<T>(c);
    a.nrows = ns;
    a.spins = const_cast<uint8_t *>(spins);
    a.tiles_per_op = (int)((ns + c->eloc_R - 1) / c->eloc_R);
    a.ntiles = a.tiles_per_op * c->n_off;
    a.op_f = c->d_opf;
    a.item_s = W<int>(c, c->off.item_s);
    a.item_e = W<double>(c, c->off.item_e);
    a.item_cnt = W<int>(c, c->off.item_cnt);
    a.contrib = W<double>(c, c->off.contrib);
    a.colbuf = W<T>(c, c->off.colbuf);
    mark(c, 3, st);
    if (f32(c) && gram_tc_available() && eloc_tc_supported(c->L.dim, c->L.dh)) {
      // tensor-core engine: 128-row tiles
      ElocTcArgs e{};
      e.pack = reinterpret_cast<const float *>(a.pack);
      e.oWgT = (int)c->P.WgT; e.oxw = (int)c->P.xw; e.obias = (int)c->P.bias;
      e.ohead = (int)c->P.head; e.ohc = (int)c->P.hc;
      e.spins = spins;
      e.hcache = reinterpret_cast<const float *>(a.hcache);
      e.lccache = reinterpret_cast<const float *>(a.lccache);
      e.N = c->L.N; e.cplx = c->L.cplx; e.zmask = c->L.zmask; e.ns = ns;
      e.tiles_per_op = (int)((ns + 127) / 128);
      e.ntiles = e.tiles_per_op * c->n_off;
      e.op_f = c->d_opf; e.item_s = a.item_s; e.item_e = a.item_e; e.item_cnt = a.item_cnt;
      e.contrib = a.contrib;
      e.err = W<int>(c, c->off.sstat);
      e.ck = c->ck;
      e.nck = c->nck;
      e.dhm = c->L.dh;
      e.tile_ctr = W<int>(c, c->off.tctr);
      CU(cudaMemsetAsync(e.tile_ctr, 0, sizeof(int), st));
      CU(eloc_tc_run(e, eloc_grid_cap(c, c->rd.sm_count), st));
    } else if (f32(c) && c->ck == 0 && gram_tc_available() &&
               eloc2d_tc_supported(c->L.dim, c->L.dh)) {
      // 2D tensor-core engine: 128-row tiles, one CTA per SM
      Eloc2dTcArgs e{};
      e.pack = reinterpret_cast<const float *>(a.pack);
      e.oWgT = (int)c->P.WgT; e.oxw = (int)c->P.xw; e.obias = (int)c->P.bias;
      e.ohead = (int)c->P.head; e.ohc = (int)c->P.hc; e.oU12T = (int)c->P.U12T;
      e.spins = spins;
      e.hcache = reinterpret_cast<const float *>(a.hcache);
      e.lccache = reinterpret_cast<const float *>(a.lccache);
      e.N = c->L.N; e.Lx = c->L.Lx; e.cplx = c->L.cplx; e.zmask = c->L.zmask; e.ns = ns;
      e.tiles_per_op = (int)((ns + ELOC2D_TC_ROWS - 1) / ELOC2D_TC_ROWS);
      e.ntiles = e.tiles_per_op * c->n_off;
      e.op_f = c->d_opf; e.item_s = a.item_s; e.item_e = a.item_e; e.item_cnt = a.item_cnt;
      e.contrib = a.contrib;
      e.colbuf = reinterpret_cast<float *>(a.colbuf);
      e.err = W<int>(c, c->off.sstat);
      e.tile_ctr = W<int>(c, c->off.tctr);
      CU(cudaMemsetAsync(e.tile_ctr, 0, sizeof(int), st));
      CU(eloc2d_tc_run(e, c->L.dh, eloc_grid_cap(c, c->rd.sm_count), st));
    } else if (f32(c) && c->ck == 0 && gram_tc_available() &&
               eloc2d_tcs_supported(c->L.dim, c->L.dh)) {
      // 2D tensor-core engine with the weights streamed from L2 (d_h 96, 128)
      Eloc2dTcArgs e{};
      e.pack = reinterpret_cast<const float *>(a.pack);
      e.oWgT = (int)c->P.WgT; e.oxw = (int)c->P.xw; e.obias = (int)c->P.bias;
      e.ohead = (int)c->P.head; e.ohc = (int)c->P.hc; e.oU12T = (int)c->P.U12T;
      e.spins = spins;
      e.hcache = reinterpret_cast<const float *>(a.hcache);
      e.lccache = reinterpret_cast<const float *>(a.lccache);
      e.N = c->L.N; e.Lx = c->L.Lx; e.cplx = c->L.cplx; e.zmask = c->L.zmask; e.ns = ns;
      e.tiles_per_op = (int)((ns + ELOC2D_TC_ROWS - 1) / ELOC2D_TC_ROWS);
      e.ntiles = e.tiles_per_op * c->n_off;
      e.op_f = c->d_opf; e.item_s = a.item_s; e.item_e = a.item_e; e.item_cnt = a.item_cnt;
      e.contrib = a.contrib;
      e.colbuf = reinterpret_cast<float *>(a.colbuf);
      e.err = W<int>(c, c->off.sstat);
      e.tile_ctr = W<int>(c, c->off.tctr);
      e.wimg = reinterpret_cast<const unsigned char *>(c->ws + c->off.wimg);
      e.spin_limit = c->test_spin_limit;
      e.test_drop_tile = c->test_drop_tile;
      c->launches += part == 1 ? 1 : 2;
      CU(cudaMemsetAsync(e.tile_ctr, 0, sizeof(int), st));
      if (part == 1) {  // the engine runs in the batch's grouped launch
        c->eloc_args = e;
        CU(eloc2d_tcs_image(e, c->L.dh, st));
        return NQS_OK;
      }
      CU(eloc2d_tcs_run(e, c->L.dh, eloc_grid_cap(c, c->rd.sm_count), st));
    } else {
      CU(run_forward<T>(c->rd, MODE_ELOC, a, eloc_grid_cap(c, c->eloc_grid), st));
    }
  } else {
    mark(c, 3, st);
  }
  mark(c, 4, st);
  c->launches += 1;
  k_eloc_reduce<<<(unsigned)((eloc_reduce_threads(ns) + 255) / 256), 256, 0, st>>>(
      c->d_diag, c->n_diag, c->n_off, spins, c->L.N, ns, W<double>(c, c->off.contrib), eloc);
  return cu(cudaGetLastError());
}

nqs_status eloc_any(nqs_ctx *c, int64_t ns, const uint8_t *spins, double *eloc, cudaStream_t st) {
  return f32(c) ? eloc_T<float>(c, ns, spins, eloc, st) : eloc_T<double>(c, ns, spins, eloc, st);
}

// Jacobian rows of the ns cached configurations into O (precision T).  With
// checkpoints, the reverse sweep runs segment by segment from the last: the
// segment's states and gates are recomputed from its checkpoint, the sweep
// carries the adjoint of the state into the previous segment, and the
// segment's contributions are added into O.
template <typename T>
nqs_status jac_T(nqs_ctx *c, int64_t ns, const uint8_t *spins, T *O, cudaStream_t st) {
  const int64_t R = c->L.cplx ? 2 * ns : ns;
  const int N = c->L.N;
  BwdArgs<T> b{};
  b.pack = W<T>(c, c->off.pack);
  b.N = N; b.Lx = c->L.Lx; b.cplx = c->L.cplx; b.zmask = c->L.zmask;
  b.ns = ns; b.nrows = R;
  b.spins = spins;
  b.gcache = W<T>(c, c->off.gcache);
  b.gw = c->gw;
  b.lccache = W<T>(c, c->off.lccache);
  b.adj = W<T>(c, c->off.adj);
  b.adjw = c->adjw;
  b.adjcol = W<T>(c, c->off.adjcol);
  GradArgs<T, T> g{};
  g.N = N; g.Lx = c->L.Lx; g.cplx = c->L.cplx; g.dim = c->L.dim;
  g.ns = ns; g.nrows = R; g.spins = spins; g.adj = b.adj; g.adjw = c->adjw;
  g.O = O; g.np = c->L.np;
  g.U1 = c->L.U1; g.U2 = c->L.U2; g.Wu = c->L.Wu; g.bu = c->L.bu; g.Wr = c->L.Wr; g.br = c->L.br;
  g.Wh = c->L.Wh; g.bh = c->L.bh; g.Win = c->L.Win; g.bin = c->L.bin; g.Uo = c->L.Uo;
  g.co = c->L.co; g.Up = c->L.Up; g.cp = c->L.cp;
  if (c->ck == 0) {
    b.hcache = W<T>(c, c->off.hcache);
    b.k_lo = 0; b.k_hi = N; b.hN = N; b.hoff = 0; b.gN = N; b.goff = 0; b.aN = N; b.aoff = 0;
    mark(c, 6, st);
    CU(run_bwd<T>(c->rd, b, st));
    mark(c, 7, st);
    c->launches += 2;
    g.hcache = b.hcache;
    g.k_lo = 0; g.k_hi = N; g.hN = N; g.hoff = 0; g.aN = N; g.aoff = 0; g.accumulate = 0;
    if constexpr (std::is_same<T, float>::value) {
      if (gram_tc_available() && jac_tc_supported(c->L.dim, c->L.dh)) {
        // mixed 1D chains: the rows of O as tensor-core products
        JacTcArgs j{};
        j.N = N; j.cplx = c->L.cplx; j.dh = c->L.dh;
        j.ns = ns; j.nrows = R; j.spins = spins;
        j.hcache = b.hcache; j.adj = b.adj; j.adjw = c->adjw;
        j.O = O; j.np = c->L.np;
        j.Wu = c->L.Wu; j.bu = c->L.bu; j.Wr = c->L.Wr; j.br = c->L.br; j.Wh = c->L.Wh;
        j.bh = c->L.bh; j.Win = c->L.Win; j.bin = c->L.bin; j.Uo = c->L.Uo; j.co = c->L.co;
        j.Up = c->L.Up; j.cp = c->L.cp;
        j.err = W<int>(c, c->off.sstat);
        return cu(jac_tc_run(j, c->rd.sm_count, st));
      }
      if (gram_tc_available() && jac2d_tc_supported(c->L.dim, c->L.dh)) {
        // mixed 2D lattices: the rows of O as tensor-core products
        Jac2dTcArgs j{};
        j.N = N; j.Lx = c->L.Lx; j.cplx = c->L.cplx; j.dh = c->L.dh;
        j.ns = ns; j.nrows = R; j.spins = spins;
        j.hcache = b.hcache; j.adj = b.adj; j.adjw = c->adjw;
        j.odz = 4 * c->L.dh; j.odhp = 4 * c->L.dh + 4; j.ohp = 5 * c->L.dh + 4;
        j.O = O; j.np = c->L.np;
        j.U1 = c->L.U1; j.U2 = c->L.U2; j.Wu = c->L.Wu; j.bu = c->L.bu; j.Wr = c->L.Wr;
        j.br = c->L.br; j.Wh = c->L.Wh; j.bh = c->L.bh; j.Win = c->L.Win; j.bin = c->L.bin;
        j.Uo = c->L.Uo; j.co = c->L.co; j.Up = c->L.Up; j.cp = c->L.cp;
        j.err = W<int>(c, c->off.sstat);
        return cu(jac2d_tc_run(j, c->rd.sm_count, st));
      }
    }
    return cu(run_grad<T>(c->rd, g, st));
  }
  const int ck = c->ck;
  T *hseg = W<T>(c, c->off.hseg);
  T *carry = W<T>(c, c->off.carry);
  mark(c, 6, st);
  CU(cudaMemsetAsync(carry, 0, (size_t)R * c->L.dh * sizeof(T), st));
  for (int m = c->nseg - 1; m >= 0; --m) {
    const int k_lo = m * ck, k_hi = std::min(N, k_lo + ck);
    FwdArgs<T> a = fwd_args<T>(c);
    a.nrows = ns;
    a.spins = const_cast<uint8_t *>(spins);
    a.gcache = W<T>(c, c->off.gcache);
    a.gw = c->gw;
    a.hseg = hseg;
    a.k_lo = k_lo; a.k_hi = k_hi;
    CU(run_forward<T>(c->rd, MODE_GIVEN, a, 0, st));
    b.hcache = hseg;
    b.k_lo = k_lo; b.k_hi = k_hi;
    b.hN = ck + 1; b.hoff = k_lo - 1;
    b.gN = ck; b.goff = k_lo;
    b.aN = ck; b.aoff = k_lo;
    b.carry = carry;
    CU(run_bwd<T>(c->rd, b, st));
    g.hcache = hseg;
    g.k_lo = k_lo; g.k_hi = k_hi;
    g.hN = ck + 1; g.hoff = k_lo - 1;
    g.aN = ck; g.aoff = k_lo;
    g.accumulate = m != c->nseg - 1;
    CU(run_grad<T>(c->rd, g, st));
    c->launches += 3;
  }
  mark(c, 7, st);
  return NQS_OK;
}

// T = A A^T in FP64 (see nqs_gram).
nqs_status gram_any(nqs_ctx *c, const void *A, int64_t R, int64_t np, double *T, cudaStream_t st) {
  c->launches += gram_tc_available() && f32(c) ? gram_tc_launches() : 1;
  if (f32(c)) {
    if (gram_tc_available())
      return cu(gram_tc_bf16x3(reinterpret_cast<const float *>(A), R, np, T,
                               c->ws + c->off.split, W<int>(c, c->off.sstat) + 1, st));
    dim3 g((unsigned)((R + 63) / 64), (unsigned)((R + 63) / 64));
    k_gram_simt<float, float><<<g, 256, 0, st>>>(reinterpret_cast<const float *>(A), R, np, T);
  } else {
    dim3 g((unsigned)((R + 63) / 64), (unsigned)((R + 63) / 64));
    k_gram_simt<double, double><<<g, 256, 0, st>>>(reinterpret_cast<const double *>(A), R, np, T);
  }
  return cu(cudaGetLastError());
}

__global__ void k_set_i32(int32_t *p, int32_t v) { *p = v; }

// After the FP64 Cholesky of the tensor-core T: a non-positive pivot arms the
// FP64-Gram retry (status cleared, need_fp64 = 2), anything else disarms it.
__global__ void k_retry_arm(int32_t *status, int32_t *retry, int32_t *need_fp64) {
  const bool arm = *status == (int32_t)NQS_ERR_NOT_SPD;
  *retry = arm ? 1 : 0;
  if (arm) {
    *status = 0;
    *need_fp64 = 2;
  }
}
__global__ void k_set_i64(int64_t *p, int64_t v) { *p = v; }
__global__ void k_inc_i64(int64_t *p) { *p += 1; }

// Cotangents (re, im) interleaved -> [re block; im block].
__global__ void k_split_cot(const double *__restrict__ g, int64_t ns, int cplx, double *v) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= ns) return;
  v[s] = g[2 * s];
  if (cplx) v[ns + s] = g[2 * s + 1];
}

__global__ void k_sum_parts(const double *__restrict__ part, int nparts, int64_t np, double *out) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= np) return;
  double acc = 0.0;
  for (int c = 0; c < nparts; ++c) acc += part[(int64_t)c * np + p];
  out[p] = acc;
}

__global__ void k_shift(double *T, int64_t R, double lam) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < R) T[i * R + i] += lam;
}

__global__ void k_frob_part(const double *__restrict__ T, int64_t n2, double *part,
                            const int32_t *gate = nullptr) {
  if (gate && *gate == 0) return;
  __shared__ double s[256];
  double acc = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n2;
       e += (int64_t)gridDim.x * blockDim.x)
    acc += T[e] * T[e];
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

// lam_dev (optional): the damping held on the device (Levenberg-Marquardt
// mode) instead of mode / lam_c.
__global__ void k_lambda_finish(double *T, int64_t R, const double *part, int nparts, int mode,
                                double lam_c, double coeff, double pw, nqs_step_stats *st,
                                const int32_t *gate = nullptr, const double *lam_dev = nullptr) {
  if (gate && *gate == 0) return;
  __shared__ double lam_s;
  if (threadIdx.x == 0) {
    double acc = 0.0;
    for (int i = 0; i < nparts; ++i) acc += part[i];
    const double nT = sqrt(acc);
    const double lam = lam_dev ? *lam_dev : (mode == 1 ? coeff * pow(nT, pw) : lam_c);
    st->normT = nT;
    st->lambda = lam;
    st->rho = 0.0;
    st->lambda_next = lam;
    lam_s = lam;
  }
  __syncthreads();
  for (int64_t i = threadIdx.x; i < R; i += blockDim.x) T[i * R + i] += lam_s;
}

// Philox key offset of the samples that estimate E(theta - delta theta) for
// the damping ratio (the step's key plus 2^64 / golden ratio).
constexpr uint64_t LM_KEY_OFFSET = 0x9E3779B97F4A7C15ull;

// The point of the damping ratio: theta - delta theta before momentum, i.e.
// theta' + m' - delta theta after an accepted update; theta if rejected.
__global__ void k_lm_point(const double *__restrict__ theta, const double *__restrict__ mom,
                           const double *__restrict__ dth, int64_t np, const nqs_step_stats *st,
                           double *out) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= np) return;
  out[k] = st->status == NQS_OK ? theta[k] + mom[k] - dth[k] : theta[k];
}

// Gain ratio and next damping (App. G): rho = (E - E2) / (eta eps'^T tau -
// 1/2 eta^2 ||tau||^2) with tau = eps' - lambda x; one block.
__global__ void k_lm_update(const double *__restrict__ eloc2, int64_t ns,
                            const double *__restrict__ eps, const double *__restrict__ x, int64_t R,
                            nqs_step_stats *st, double *lam_dev, double omega) {
  __shared__ double s1[1024], s2[1024];
  const double lam = st->lambda;
  double a = 0.0, b = 0.0;
  for (int64_t i = threadIdx.x; i < ns; i += blockDim.x) a += eloc2[2 * i];
  for (int64_t i = threadIdx.x; i < R; i += blockDim.x) b += eps[i] * (eps[i] - lam * x[i]);
  s1[threadIdx.x] = a;
  s2[threadIdx.x] = b;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      s1[threadIdx.x] += s1[threadIdx.x + o];
      s2[threadIdx.x] += s2[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double E2 = s1[0] / (double)ns;
    const double eta = st->eta_eff, tn = st->tau_norm;
    const double pred = eta * s2[0] - 0.5 * eta * eta * tn * tn;
    const double rho = (st->E_re - E2) / pred;
    double ln = lam;
    if (st->status != NQS_OK || !(rho >= 0.25)) ln = omega * lam;
    else if (rho > 0.75) ln = lam / omega;
    st->rho = rho;
    st->lambda_next = ln;
    *lam_dev = ln;
  }
}

// x = (T + lambda I)^{-1} b for the shifted T.  FP64 context: FP64 Cholesky
// and both substitutions in one cooperative launch (chol_coop.cuh).  Mixed
// context: FP32 factor and FP64 iterative refinement (chol_ir.cuh); the FP64
// kernel follows on the stream and runs only if the refinement reports that
// it must (non-positive FP32 pivot or no convergence).  *need_fp64 (device)
// ends as 0 (refined) or 1 (FP64 factorisation).
struct RetryInfo {
  const nqs_step_hparams *hp;  // lambda of the step
  nqs_step_stats *stats;
};

// Arguments of the blocked FP32 factor and refinement for this context.
CholBlkArgs blk_args(nqs_ctx *c, const double *T, int64_t R, const double *b, double *x,
                     int32_t *status) {
  unsigned *bar = W<unsigned>(c, c->off.cbar);
  CholBlkArgs bk;
  bk.A = T; bk.n = R; bk.b = b; bk.x = x;
  bk.L = W<float>(c, c->off.L32);
  bk.Dinv = W<float>(c, c->off.Tm32);
  bk.t = W<float>(c, c->off.dpart32);
  bk.w = W<float>(c, c->off.wv32);
  bk.r = W<double>(c, c->off.crhs);
  bk.part = W<double>(c, c->off.cpart);
  bk.bar = bar + 2;
  bk.status = status;
  bk.need_fp64 = reinterpret_cast<int32_t *>(bar + 4);
  bk.maxit = 12;
  return bk;
}

// Whether a batch may run this context's FP32 factor in its grouped launch.
bool group_solvable(const nqs_ctx *c, int64_t R) {
  return f32(c) && chol_blk_supported(R) && (c->solve_form < 0 || c->solve_form == 2);
}

// part: 0 the whole solve; 1 only the reset of the barrier counters and
// flags (the factor follows in a grouped launch); 2 what follows the FP32
// factor (the gated FP64 fallback and the FP64 Gram retry).
nqs_status chol_solve(nqs_ctx *c, double *T, int64_t R, const double *b, double *x,
                      int32_t *status, cudaStream_t st, const RetryInfo *retry = nullptr,
                      int part = 0) {
  unsigned *bar = W<unsigned>(c, c->off.cbar);
  int32_t *need = reinterpret_cast<int32_t *>(bar + 4);
  const int G = solve_grid(c);
  if (part != 2) CU(cudaMemsetAsync(bar, 0, 32, st));
  if (part == 1) return NQS_OK;
  // blocked FP32 factor (128-wide panels) where it applies and is chosen:
  // by the autotuner, else from R = 3072 on (measured: 0.49 against 1.2 ms
  // at R = 1024 for the 32-wide panels, 4.1 against 6.2 ms at R = 4096 for
  // the 128-wide ones)
  const int var = c->solve_form >= 0                  ? c->solve_form
                  : tuned(c) && c->t_chol_var >= 0 ? c->t_chol_var
                                                   : (R >= 3072 ? 2 : 0);
  if (part == 2) {
    // the grouped launch ran the FP32 factor and refinement
  } else if (f32(c) && var == 2 && chol_blk_supported(R)) {
    CholBlkArgs bk = blk_args(c, T, R, b, x, status);
    const size_t smem = chol_blk_smem();
    CU(cudaFuncSetAttribute((const void *)k_chol_blk, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)smem));
    // no more CTAs than the first panel has trailing tiles (plus the CTA
    // that factors the diagonal blocks): the rest of the SMs stay free for
    // the other instances of a batch
    const int64_t nr = (R + BKB - 1) / BKB - 1;
    const int Gb = (int)std::max<int64_t>(2, std::min<int64_t>(std::min(G, c->rd.sm_count),
                                                                 nr * (nr + 1) / 2 + 1));
    void *args[] = {&bk};
    c->launches += 1;
    CU(cudaLaunchCooperativeKernel((const void *)k_chol_blk, dim3(Gb), dim3(BKB_THREADS), args, smem,
                                   st));
  } else if (f32(c)) {
    CholIrArgs ir;
    ir.A = T; ir.n = R; ir.b = b; ir.x = x;
    ir.L = W<float>(c, c->off.L32);
    ir.Li = W<float>(c, c->off.Li32);
    ir.Tm = W<float>(c, c->off.Tm32);
    ir.wv = W<float>(c, c->off.wv32);
    ir.dpart = W<float>(c, c->off.dpart32);
    ir.r = W<double>(c, c->off.crhs);
    ir.part = W<double>(c, c->off.cpart);
    ir.bar = bar + 2;
    ir.status = status;
    ir.need_fp64 = need;
    ir.maxit = 12;
    // sweeps with the explicit inverse at every size (measured at n = 4096,
    // probe copy of the kernel: inversion levels 1.67 ms + 3 product sweeps
    // 0.47 ms, against 4.2 ms for 3 block-substitution sweeps)
    ir.subst = tuned(c) && c->t_chol_subst >= 0 ? c->t_chol_subst : 0;
    ir.dv = ir.dpart;
    ir.dg = W<float>(c, c->off.dg32);
    const size_t smem = chol_ir_smem(R);
    // CTA tiles in batches of four at every size (measured: factor 4.7 ms
    // against 6.6 ms with a tile per warp at n = 4096; 0.26 ms against 0.93
    // at n = 1024)
    const bool wt = var == 1;
    const void *kern = wt ? (const void *)k_chol_ir<true> : (const void *)k_chol_ir<false>;
    CU(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    // a grid above one CTA per SM only where the occupancy allows it: every
    // CTA of the cooperative launch must be resident at once
    int per = 0;
    CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, IR_THREADS, smem));
    const int Gi = std::min(G, std::max(per, 1) * c->rd.sm_count);
    void *args[] = {&ir};
    c->launches += 1;
    CU(cudaLaunchCooperativeKernel(kern, dim3(Gi), dim3(IR_THREADS), args, smem, st));
  } else {
    k_set_i32<<<1, 1, 0, st>>>(need, 1);
    c->launches += 1;
    CU(cudaGetLastError());
  }
  CholCoopArgs a;
  a.A = T; a.n = R; a.b = b; a.x = x;
  a.rhs = W<double>(c, c->off.crhs);
  a.y = W<double>(c, c->off.cy);
  a.part = W<double>(c, c->off.cpart);
  a.bar = bar;
  a.status = status;
  a.gate = need;
  const size_t smem = chol_coop_smem(R);
  CU(cudaFuncSetAttribute(k_chol_coop, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per = 0;
  CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_chol_coop, CC_THREADS, smem));
  if (per < 1) return NQS_ERR_UNSUPPORTED;
  // one CTA per SM at most: its partial sums are sized for that grid
  const int Gc = std::min(G, c->rd.sm_count);
  void *args[] = {&a};
  c->launches += 1;
  CU(cudaLaunchCooperativeKernel((void *)k_chol_coop, dim3(Gc), dim3(CC_THREADS), args, smem, st));
  if (retry && f32(c) && gram_tc_available()) {
    // T from the tensor cores can miss positive definiteness by its rounding
    // when lambda is tiny against ||T||: then rebuild T in FP64 from the same
    // split planes, recompute lambda and factor again in FP64 (all gated on
    // the device, so the sequence is graph-capturable)
    int32_t *rflag = need + 1;
    k_retry_arm<<<1, 1, 0, st>>>(status, rflag, need);
    const int64_t np = c->L.np;
    CU(gram_split_f64(c->ws + c->off.split, R, np, T, rflag, st));
    const int nparts = 256;
    k_frob_part<<<nparts, 256, 0, st>>>(T, R * R, W<double>(c, c->off.frob), rflag);
    k_lambda_finish<<<1, 1024, 0, st>>>(T, R, W<double>(c, c->off.frob), nparts,
                                        retry->hp->lambda_mode, retry->hp->lambda,
                                        retry->hp->lambda_coeff, retry->hp->lambda_pow,
                                        retry->stats, rflag,
                                        c->lm_omega > 1.0 ? W<double>(c, c->off.dlm) : nullptr);
    CU(cudaMemsetAsync(bar, 0, 4, st));
    a.gate = rflag;
    c->launches += 5;
    CU(cudaLaunchCooperativeKernel((void *)k_chol_coop, dim3(Gc), dim3(CC_THREADS), args, smem, st));
  }
  mark(c, 12, st);
  return NQS_OK;
}

template <typename T>
nqs_status step_T(nqs_ctx *c, double *theta, double *mom, const nqs_step_hparams *hp,
                  nqs_step_stats *stats, const nqs_step_outputs *out, cudaStream_t st) {
  const int64_t ns = hp->n_samples, N = c->L.N, np = c->L.np;
  const int64_t R = c->L.cplx ? 2 * ns : ns;
  uint8_t *spins = W<uint8_t>(c, c->off.spins);
  double *logpsi = W<double>(c, c->off.logpsi);
  double *eloc = W<double>(c, c->off.eloc);
  T *O = W<T>(c, c->off.O);
  double *Tm = W<double>(c, c->off.T);
  double *eps = W<double>(c, c->off.eps);
  double *x = W<double>(c, c->off.x);
  int32_t *sstat = W<int32_t>(c, c->off.sstat);
  c->cur_ns = ns;
  // tensor-core route of the mixed path: centring writes the BF16 hi/lo
  // planes that the Gram and O'x read; otherwise O is centred in place
  const bool tc = f32(c) && gram_tc_available();
  const RetryInfo rinfo{hp, stats};
  const int ph = c->phase;
  if (ph == STEP_ALL || ph == STEP_PRE_A) {
    mark(c, 0, st);
    CU(cudaMemsetAsync(sstat, 0, 64, st));
    // Alg. 1, sampling: sample (also fills the hidden-state caches)
    ST(pack_theta<T>(c, theta, st));
    mark(c, 1, st);
    {
      FwdArgs<T> a = fwd_args<T>(c);
      a.nrows = ns; a.seed = hp->seed; a.step = (uint64_t)hp->step_index;
      a.step_dev = W<int64_t>(c, c->off.dstep);
      a.spins = spins; a.logpsi = logpsi;
      if (c->ck == 0) {  // gates for the reverse sweep (recomputed per segment otherwise)
        a.gcache = W<T>(c, c->off.gcache);
        a.gw = c->gw;
      }
      ST(run_sample<T>(c, a, st));
    }
    // Alg. 1, energy: local energies, E, variance; eps-bar'
    ST(eloc_T<T>(c, ns, spins, eloc, st, ph == STEP_PRE_A && c->in_eloc_group ? 1 : 0));
    if (ph == STEP_PRE_A) return NQS_OK;
  }  // ph == STEP_ALL || ph == STEP_PRE_A
  if (ph == STEP_ALL || ph == STEP_PRE_B) {
    if (ph == STEP_PRE_B && c->in_eloc_group) ST(eloc_T<T>(c, ns, spins, eloc, st, 2));
    mark(c, 5, st);
    k_energy<<<1, 1024, 0, st>>>(eloc, ns, (int)N, c->L.cplx, stats, eps);
    c->launches += 1;
    CU(cudaGetLastError());
    // Alg. 1, log-derivatives: O, centred over samples per block, / sqrt(Ns)
    ST(jac_T<T>(c, ns, spins, O, st));
    mark(c, 8, st);
    {
      c->launches += 3;
      const int chunks = (int)((ns + COL_ROWS - 1) / COL_ROWS);
      const unsigned nblk = c->L.cplx ? 2u : 1u;
      dim3 g((unsigned)((np + 255) / 256), nblk * chunks);
      k_colsum_part<T><<<g, 256, 0, st>>>(O, ns, np, chunks, W<double>(c, c->off.part));
      k_colmean_fin<<<dim3((unsigned)((np + 255) / 256), nblk), 256, 0, st>>>(
          W<double>(c, c->off.part), ns, np, chunks, W<double>(c, c->off.mean), tc ? 1 : 0);
      CU(cudaGetLastError());
      if (tc) {
        CU(center_split(reinterpret_cast<const float *>(O), ns, np, R, W<float2>(c, c->off.mean),
                        c->ws + c->off.split, st));
      } else {
        const int64_t tot = R * np;
        const int blocks = (int)std::min<int64_t>((tot + 255) / 256, 148 * 16);
        k_center<T><<<blocks, 256, 0, st>>>(O, ns, np, R, W<double>(c, c->off.mean));
        CU(cudaGetLastError());
      }
    }
    // Alg. 1, Gram: T = O'^T O'
    mark(c, 9, st);
    if (tc) {
      c->launches += 2;
      CU(gram_from_center_split(c->ws + c->off.split, R, np, Tm, sstat, st, gram_splits(c)));
    } else {
      ST(gram_any(c, O, R, np, Tm, st));
    }
    mark(c, 10, st);
    if (out && out->T) CU(cudaMemcpyAsync(out->T, Tm, R * R * 8, cudaMemcpyDeviceToDevice, st));
    // lambda and shift
    {
      const int nparts = 256;
      c->launches += 2;
      k_frob_part<<<nparts, 256, 0, st>>>(Tm, R * R, W<double>(c, c->off.frob));
      k_lambda_finish<<<1, 1024, 0, st>>>(Tm, R, W<double>(c, c->off.frob), nparts, hp->lambda_mode,
                                          hp->lambda, hp->lambda_coeff, hp->lambda_pow, stats,
                                          nullptr,
                                          c->lm_omega > 1.0 ? W<double>(c, c->off.dlm) : nullptr);
      CU(cudaGetLastError());
    }
    mark(c, 11, st);
    if (ph == STEP_PRE_B)
      return c->in_group ? chol_solve(c, Tm, R, eps, x, sstat, st, &rinfo, 1) : NQS_OK;
  }  // ph == STEP_ALL || ph == STEP_PRE_B
  // Alg. 1, solve: x = (T + lambda I)^{-1} eps', eta, delta theta = eta O' x
  if (c->solve_wait) CU(cudaStreamWaitEvent(st, c->solve_wait, 0));
  ST(chol_solve(c, Tm, R, eps, x, sstat, st, &rinfo, ph == STEP_POST && c->in_group ? 2 : 0));
  if (c->solve_rec) CU(cudaEventRecord(c->solve_rec, st));
  mark(c, 13, st);
  k_eta<<<1, 1024, 0, st>>>(eps, x, R, hp->eta0, hp->decay_T, hp->trust_region,
                            W<int64_t>(c, c->off.dstep), stats, sstat,
                            reinterpret_cast<int32_t *>(W<unsigned>(c, c->off.cbar) + 4));
  CU(cudaGetLastError());
  {
    c->launches += 4;
    const int rows_per = 64;
    const int nparts = (int)((R + rows_per - 1) / rows_per);
    dim3 g((unsigned)((np + 255) / 256), (unsigned)nparts);
    if (tc)
      CU(gemv_split(c->ws + c->off.split, R, np, x, rows_per, W<double>(c, c->off.part), st));
    else
      k_gemv_part<T><<<g, 256, 0, st>>>(O, R, np, x, rows_per, W<double>(c, c->off.part));
    k_dtheta<<<(unsigned)((np + 255) / 256), 256, 0, st>>>(W<double>(c, c->off.part), nparts, np,
                                                          stats, W<double>(c, c->off.dth));
    // Alg. 1, momentum and update (skipped unless status is OK)
    k_apply<<<(unsigned)((np + 255) / 256), 256, 0, st>>>(theta, mom, W<double>(c, c->off.dth),
                                                         np, hp->mu, stats);
    CU(cudaGetLastError());
  }
  if (out) {
    if (out->spins) CU(cudaMemcpyAsync(out->spins, spins, ns * N, cudaMemcpyDeviceToDevice, st));
    if (out->logpsi) CU(cudaMemcpyAsync(out->logpsi, logpsi, ns * 16, cudaMemcpyDeviceToDevice, st));
    if (out->eloc) CU(cudaMemcpyAsync(out->eloc, eloc, ns * 16, cudaMemcpyDeviceToDevice, st));
    if (out->eps) CU(cudaMemcpyAsync(out->eps, eps, R * 8, cudaMemcpyDeviceToDevice, st));
    if (out->x) CU(cudaMemcpyAsync(out->x, x, R * 8, cudaMemcpyDeviceToDevice, st));
    if (out->dtheta)
      CU(cudaMemcpyAsync(out->dtheta, W<double>(c, c->off.dth), np * 8, cudaMemcpyDeviceToDevice, st));
  }
  if (c->lm_omega > 1.0) {
    // damping ratio (App. G): E at theta - delta theta from fresh samples;
    // the pass reuses the step's caches, so it runs after the outputs are
    // copied, and it records no stage events
    const int saved_tmax = c->tmax;
    c->tmax = c->tstep;
    double *tth = W<double>(c, c->off.tth);
    k_lm_point<<<(unsigned)((np + 255) / 256), 256, 0, st>>>(theta, mom, W<double>(c, c->off.dth),
                                                            np, stats, tth);
    CU(cudaGetLastError());
    ST(pack_theta<T>(c, tth, st));
    FwdArgs<T> a = fwd_args<T>(c);
    a.nrows = ns; a.seed = hp->seed + LM_KEY_OFFSET; a.step = (uint64_t)hp->step_index;
    a.step_dev = W<int64_t>(c, c->off.dstep);
    a.spins = spins; a.logpsi = logpsi;
    c->launches += 1;
    ST(run_sample<T>(c, a, st));
    ST(eloc_T<T>(c, ns, spins, eloc, st));
    k_lm_update<<<1, 1024, 0, st>>>(eloc, ns, eps, x, R, stats, W<double>(c, c->off.dlm),
                                    c->lm_omega);
    CU(cudaGetLastError());
    c->tmax = saved_tmax;
  }
  k_inc_i64<<<1, 1, 0, st>>>(W<int64_t>(c, c->off.dstep));  // next step's counter
  c->launches += 1;
  CU(cudaGetLastError());
  mark(c, 14, st);
  if (c->tstep < c->tmax) ++c->tstep;
  return NQS_OK;
}

}  // namespace

static void timing_free(nqs_ctx *c) {
  for (cudaEvent_t e : c->tev) cudaEventDestroy(e);
  c->tev.clear();
  c->tmax = c->tstep = 0;
}

namespace {
template <typename T>
nqs_status vjp_T(nqs_ctx *c, const uint8_t *spins, int64_t ns, const double *g, double *out,
                 cudaStream_t st) {
  const int64_t R = c->L.cplx ? 2 * ns : ns, np = c->L.np;
  T *O = W<T>(c, c->off.O);
  ST(jac_T<T>(c, ns, spins, O, st));
  double *v = W<double>(c, c->off.eps);
  k_split_cot<<<(unsigned)((ns + 255) / 256), 256, 0, st>>>(g, ns, c->L.cplx, v);
  const int rows_per = 64;
  const int nparts = (int)((R + rows_per - 1) / rows_per);
  dim3 gr((unsigned)((np + 255) / 256), (unsigned)nparts);
  k_gemv_part<T><<<gr, 256, 0, st>>>(O, R, np, v, rows_per, W<double>(c, c->off.part));
  k_sum_parts<<<(unsigned)((np + 255) / 256), 256, 0, st>>>(W<double>(c, c->off.part), nparts, np, out);
  c->launches += 3;
  return cu(cudaGetLastError());
}

}  // namespace

// ===================================================================== ABI
extern "C" {

nqs_status nqs_create(const nqs_model_desc *model, const nqs_ham_desc *ham, int precision,
                      int64_t max_samples, nqs_ctx **out) {
  return nqs_create_ex(model, ham, precision, max_samples, nullptr, out);
}

nqs_status nqs_create_ex(const nqs_model_desc *model, const nqs_ham_desc *ham, int precision,
                         int64_t max_samples, const nqs_options *opt, nqs_ctx **out) {
  if (!model || !ham || !out || max_samples <= 0) return NQS_ERR_ARG;
  *out = nullptr;
  const nqs_model_desc &m = *model;
  if (m.dim != 1 && m.dim != 2) return NQS_ERR_ARG;
  if (m.Lx <= 0 || m.Ly <= 0 || (m.dim == 1 && m.Ly != 1)) return NQS_ERR_ARG;
  const int N = m.Lx * m.Ly;
  if (N < 2 || N > 4096) return NQS_ERR_ARG;
  if (m.zmask && (N % 2)) return NQS_ERR_ARG;
  if (precision != NQS_PREC_FP64 && precision != NQS_PREC_MIXED) return NQS_ERR_ARG;
  if (ham->family < NQS_HAM_TFIM || ham->family > NQS_HAM_J1J2) return NQS_ERR_ARG;
  if ((ham->family == NQS_HAM_J1J2) != (m.dim == 2)) return NQS_ERR_ARG;
  if (ham->family == NQS_HAM_CLUSTER_PAPER && N < 4) return NQS_ERR_ARG;
  if (!dh_supported(m.dh)) return NQS_ERR_UNSUPPORTED;
  nqs_ctx *c = new (std::nothrow) nqs_ctx();
  if (!c) return NQS_ERR_ARG;
  c->m = m; c->h = *ham; c->prec = precision; c->max_ns = max_samples;
  if (opt && opt->checkpoint_stride != 0) {
    int ck = opt->checkpoint_stride;
    if (ck < -1) { delete c; return NQS_ERR_ARG; }
    if (m.dim != 1) { delete c; return NQS_ERR_UNSUPPORTED; }
    if (ck == -1) {
      ck = 1;
      while (ck * ck < N) ++ck;  // ceil(sqrt(N))
    }
    ck = std::min(ck, N);
    c->ck = ck;
    c->nseg = (N + ck - 1) / ck;
    c->nck = c->nseg - 1;
  }
  c->L = make_layout(m);
  c->P = pack_offsets(c->L);
  c->es = precision == NQS_PREC_MIXED ? 4 : 8;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    delete c;
    return NQS_ERR_CUDA;
  }
  c->rd = RecDesc{m.dim, m.dh, N, m.Lx, m.cplx, m.marshall, m.zmask, sms};
  c->adjw = 4 * m.dh + 4 + (m.dim == 2 ? 2 * m.dh : 0);
  c->gw = 4 * m.dh + (m.dim == 2 ? m.dh : 0);
  c->eloc_R = eloc_rows(c->rd, precision == NQS_PREC_MIXED);
  c->eloc_grid = precision == NQS_PREC_MIXED ? eloc_max_grid<float>(c->rd) : eloc_max_grid<double>(c->rd);
  if (c->eloc_grid <= 0) { delete c; return NQS_ERR_CUDA; }
  std::vector<OffOp> off;
  std::vector<DiagOp> dg;
  build_hamiltonian(m, *ham, off, dg);
  c->n_off = (int)off.size();
  c->n_diag = (int)dg.size();
  for (const OffOp &o : off) c->op_start.push_back(o.start);
  std::vector<int> opf(4 * std::max<size_t>(off.size(), 1));
  // field 3 of entry i: the operator of rank i by first changed site, so the
  // tensor-core engines hand out the longest suffixes first
  std::vector<int> rank(off.size());
  for (size_t i = 0; i < off.size(); ++i) rank[i] = (int)i;
  std::stable_sort(rank.begin(), rank.end(), [&](int x, int y) { return off[x].start < off[y].start; });
  for (size_t i = 0; i < off.size(); ++i) {
    opf[4 * i] = off[i].f1; opf[4 * i + 1] = off[i].f2; opf[4 * i + 2] = off[i].start;
    opf[4 * i + 3] = rank[i];
  }
  bool ok = cudaMalloc(&c->d_off, sizeof(OffOp) * std::max<size_t>(off.size(), 1)) == cudaSuccess &&
            cudaMalloc(&c->d_diag, sizeof(DiagOp) * std::max<size_t>(dg.size(), 1)) == cudaSuccess &&
            cudaMalloc(&c->d_opf, sizeof(int) * opf.size()) == cudaSuccess;
  if (ok && !off.empty())
    ok = cudaMemcpy(c->d_off, off.data(), sizeof(OffOp) * off.size(), cudaMemcpyHostToDevice) == cudaSuccess;
  if (ok && !dg.empty())
    ok = cudaMemcpy(c->d_diag, dg.data(), sizeof(DiagOp) * dg.size(), cudaMemcpyHostToDevice) == cudaSuccess;
  if (ok) ok = cudaMemcpy(c->d_opf, opf.data(), sizeof(int) * opf.size(), cudaMemcpyHostToDevice) == cudaSuccess;
  if (!ok) { nqs_destroy(c); return NQS_ERR_CUDA; }
  carve(c);
  *out = c;
  return NQS_OK;
}

nqs_status nqs_destroy(nqs_ctx *c) {
  if (!c) return NQS_ERR_ARG;
  cudaDeviceSynchronize();
  timing_free(c);
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->d_off) cudaFree(c->d_off);
  if (c->d_diag) cudaFree(c->d_diag);
  if (c->d_opf) cudaFree(c->d_opf);
  delete c;
  return NQS_OK;
}

nqs_status nqs_checkpoint_stride(const nqs_ctx *c, int *stride) {
  if (!c || !stride) return NQS_ERR_ARG;
  *stride = c->ck;
  return NQS_OK;
}

nqs_status nqs_param_count(const nqs_ctx *c, int64_t *n) {
  if (!c || !n) return NQS_ERR_ARG;
  *n = c->L.np;
  return NQS_OK;
}

nqs_status nqs_workspace_size(const nqs_ctx *c, size_t *bytes) {
  if (!c || !bytes) return NQS_ERR_ARG;
  *bytes = c->off.total;
  return NQS_OK;
}

nqs_status nqs_set_workspace(nqs_ctx *c, void *p, size_t bytes) {
  if (!c || !p) return NQS_ERR_ARG;
  if (bytes < c->off.total) return NQS_ERR_WORKSPACE;
  if (reinterpret_cast<uintptr_t>(p) % 256) return NQS_ERR_ARG;
  c->ws = static_cast<char *>(p);
  c->ws_bytes = bytes;
  return NQS_OK;
}

nqs_status nqs_sample(nqs_ctx *c, const double *theta, int64_t ns, uint64_t seed, uint64_t step,
                      uint8_t *spins, double *logpsi, void *stream) {
  if (!c || !theta || !spins || !logpsi || ns <= 0 || ns > c->max_ns) return NQS_ERR_ARG;
  ST(need_ws(c));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  ST(pack_any(c, theta, st));
  return forward(c, MODE_SAMPLE, ns, seed, step, spins, logpsi, st);
}

nqs_status nqs_logpsi(nqs_ctx *c, const double *theta, const uint8_t *spins, int64_t n,
                      double *logpsi, void *stream) {
  if (!c || !theta || !spins || !logpsi || n <= 0 || n > c->max_ns) return NQS_ERR_ARG;
  ST(need_ws(c));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  ST(pack_any(c, theta, st));
  return forward(c, MODE_GIVEN, n, 0, 0, const_cast<uint8_t *>(spins), logpsi, st);
}

nqs_status nqs_local_energy(nqs_ctx *c, const double *theta, const uint8_t *spins, int64_t ns,
                            double *eloc, void *stream) {
  if (!c || !theta || !spins || !eloc || ns <= 0 || ns > c->max_ns) return NQS_ERR_ARG;
  ST(need_ws(c));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  c->cur_ns = ns;
  ST(pack_any(c, theta, st));
  ST(forward(c, MODE_GIVEN, ns, 0, 0, const_cast<uint8_t *>(spins), W<double>(c, c->off.logpsi), st));
  return eloc_any(c, ns, spins, eloc, st);
}

nqs_status nqs_jacobian(nqs_ctx *c, const double *theta, const uint8_t *spins, int64_t ns, void *O,
                        void *stream) {
  if (!c || !theta || !spins || !O || ns <= 0 || ns > c->max_ns) return NQS_ERR_ARG;
  ST(need_ws(c));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  ST(pack_any(c, theta, st));
  ST(forward(c, MODE_GIVEN, ns, 0, 0, const_cast<uint8_t *>(spins), W<double>(c, c->off.logpsi), st,
             true));
  return f32(c) ? jac_T<float>(c, ns, spins, static_cast<float *>(O), st)
                : jac_T<double>(c, ns, spins, static_cast<double *>(O), st);
}

nqs_status nqs_logpsi_vjp(nqs_ctx *c, const double *theta, const uint8_t *spins, int64_t ns,
                          const double *grad_logpsi, double *grad_theta, void *stream) {
  if (!c || !theta || !spins || !grad_logpsi || !grad_theta || ns <= 0 || ns > c->max_ns)
    return NQS_ERR_ARG;
  ST(need_ws(c));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  ST(pack_any(c, theta, st));
  ST(forward(c, MODE_GIVEN, ns, 0, 0, const_cast<uint8_t *>(spins), W<double>(c, c->off.logpsi), st,
             true));
  return f32(c) ? vjp_T<float>(c, spins, ns, grad_logpsi, grad_theta, st)
                : vjp_T<double>(c, spins, ns, grad_logpsi, grad_theta, st);
}

nqs_status nqs_gram(nqs_ctx *c, const void *A, int64_t R, int64_t np, double *T, void *stream) {
  if (!c || !A || !T || R <= 0 || np <= 0) return NQS_ERR_ARG;
  const int64_t Rmax = c->L.cplx ? 2 * c->max_ns : c->max_ns;
  if (f32(c) && (R > Rmax || np > c->L.np)) return NQS_ERR_ARG;  // split buffer sized for these
  ST(need_ws(c));
  return gram_any(c, A, R, np, T, static_cast<cudaStream_t>(stream));
}

nqs_status nqs_regularized_solve(nqs_ctx *c, double *T, int64_t R, double lambda, const double *b,
                                 double *x, int32_t *dev_status, void *stream) {
  if (!c || !T || !b || !x || !dev_status || R <= 0 || !(lambda >= 0.0)) return NQS_ERR_ARG;
  if (R > (c->L.cplx ? 2 * c->max_ns : c->max_ns)) return NQS_ERR_ARG;
  ST(need_ws(c));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  c->cur_ns = c->L.cplx ? R / 2 : R;
  CU(cudaMemsetAsync(dev_status, 0, sizeof(int32_t), st));
  if (lambda != 0.0) {
    k_shift<<<(unsigned)((R + 255) / 256), 256, 0, st>>>(T, R, lambda);
    CU(cudaGetLastError());
  }
  return chol_solve(c, T, R, b, x, dev_status, st);
}

static nqs_status step_body(nqs_ctx *c, double *theta, double *mom, const nqs_step_hparams *hp,
                            nqs_step_stats *stats, const nqs_step_outputs *out, cudaStream_t st) {
  return f32(c) ? step_T<float>(c, theta, mom, hp, stats, out, st)
                : step_T<double>(c, theta, mom, hp, stats, out, st);
}

static bool same_key(const nqs_ctx::Key &k, const void *th, const void *mo, const void *sts,
                     const nqs_step_hparams *hp) {
  nqs_step_hparams a = k.hp, b = *hp;
  a.step_index = b.step_index = 0;
  return k.theta == th && k.mom == mo && k.stats == sts && std::memcmp(&a, &b, sizeof(a)) == 0;
}

nqs_status nqs_minsr_step_ex(nqs_ctx *c, double *theta, double *mom, const nqs_step_hparams *hp,
                             nqs_step_stats *stats, const nqs_step_outputs *out, void *stream) {
  if (!c || !theta || !mom || !hp || !stats) return NQS_ERR_ARG;
  if (hp->n_samples < 2 || hp->n_samples > c->max_ns) return NQS_ERR_ARG;
  if (hp->lambda_mode != 0 && hp->lambda_mode != 1) return NQS_ERR_ARG;
  ST(need_ws(c));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int64_t *dstep = W<int64_t>(c, c->off.dstep);
  const bool graph = c->graph_enabled && !c->graph_broken && !out && c->tstep >= c->tmax;
  if (graph) {
    if (!c->gexec || !same_key(c->gkey, theta, mom, stats, hp)) {
      if (c->gexec) { cudaGraphExecDestroy(c->gexec); c->gexec = nullptr; }
      if (!c->cap_stream && cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
        return NQS_ERR_CUDA;
      cudaGraph_t g = nullptr;
      bool ok = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
      nqs_status s = NQS_OK;
      if (ok) s = step_body(c, theta, mom, hp, stats, nullptr, c->cap_stream);
      const bool ended = cudaStreamEndCapture(c->cap_stream, &g) == cudaSuccess;
      ok = ok && ended && s == NQS_OK && g;
      if (ok) ok = cudaGraphInstantiate(&c->gexec, g, 0) == cudaSuccess;
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();  // clear a failed capture's sticky-free error
      if (!ok) {
        c->gexec = nullptr;
        c->graph_broken = 1;  // eager launches from now on
      } else {
        c->gkey = nqs_ctx::Key{theta, mom, stats, *hp};
        c->gnext = -1;
      }
    }
    if (c->gexec) {
      if (hp->step_index != c->gnext) {
        k_set_i64<<<1, 1, 0, st>>>(dstep, hp->step_index);
        c->launches += 1;
        CU(cudaGetLastError());
      }
      CU(cudaGraphLaunch(c->gexec, st));
      c->gnext = hp->step_index + 1;
      return NQS_OK;
    }
  }
  k_set_i64<<<1, 1, 0, st>>>(dstep, hp->step_index);
  c->launches += 1;
  CU(cudaGetLastError());
  c->gnext = -1;
  return step_body(c, theta, mom, hp, stats, out, st);
}

nqs_status nqs_set_graph(nqs_ctx *c, int enable) {
  if (!c) return NQS_ERR_ARG;
  c->graph_enabled = enable != 0;
  return NQS_OK;
}

nqs_status nqs_graph_active(const nqs_ctx *c, int *active) {
  if (!c || !active) return NQS_ERR_ARG;
  *active = c->gexec != nullptr && !c->graph_broken;
  return NQS_OK;
}

nqs_status nqs_minsr_step(nqs_ctx *c, double *theta, double *mom, const nqs_step_hparams *hp,
                          nqs_step_stats *stats, void *stream) {
  return nqs_minsr_step_ex(c, theta, mom, hp, stats, nullptr, stream);
}

// ------------------------------------------------------------- autotuner

}  // extern "C"

namespace {

struct Tuned {
  int eloc_grid, gram_splits, solve_grid, chol_var, chol_subst;
  double ms[3], ms_default[3];
};
std::mutex g_tune_mu;
std::map<std::string, Tuned> g_tune_cache;  // process-wide, keyed by problem shape

std::string tune_key(const nqs_ctx *c, int64_t ns) {
  char b[256];
  const int dev = [] { int d = 0; cudaGetDevice(&d); return d; }();
  std::snprintf(b, sizeof b, "%d|%d|%d|%d|%d|%d|%d|%d|%d|%d|%lld", dev, c->m.dim, c->m.Lx,
                c->m.Ly, c->m.dh, c->m.cplx, c->m.zmask, c->h.family, c->prec,
                c->n_off, (long long)ns);
  return b;
}

struct EvPair {
  cudaEvent_t a = nullptr, b = nullptr;
  bool ok() {
    return cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess;
  }
  ~EvPair() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};

// Best of `reps` timings of body(); pre() runs untimed before each.
template <class Pre, class Body>
nqs_status best_ms(cudaStream_t st, int reps, Pre pre, Body body, double *out) {
  EvPair ev;
  if (!ev.ok()) return NQS_ERR_CUDA;
  double best = 1e300;
  for (int r = 0; r < reps; ++r) {
    ST(pre());
    CU(cudaEventRecord(ev.a, st));
    ST(body());
    CU(cudaEventRecord(ev.b, st));
    CU(cudaEventSynchronize(ev.b));
    float ms = 0.f;
    CU(cudaEventElapsedTime(&ms, ev.a, ev.b));
    best = std::min(best, (double)ms);
  }
  *out = best;
  return NQS_OK;
}

// T from the current centred O (untimed part of the solve measurement).
template <typename T>
nqs_status regram(nqs_ctx *c, int64_t ns, const nqs_step_hparams &h, nqs_step_stats *stats,
                  cudaStream_t st) {
  const int64_t R = c->L.cplx ? 2 * ns : ns, np = c->L.np;
  double *Tm = W<double>(c, c->off.T);
  if (f32(c) && gram_tc_available())
    CU(gram_from_center_split(c->ws + c->off.split, R, np, Tm, W<int>(c, c->off.sstat), st, 0));
  else
    ST(gram_any(c, W<T>(c, c->off.O), R, np, Tm, st));
  k_frob_part<<<256, 256, 0, st>>>(Tm, R * R, W<double>(c, c->off.frob));
  k_lambda_finish<<<1, 1024, 0, st>>>(Tm, R, W<double>(c, c->off.frob), 256, h.lambda_mode,
                                      h.lambda, h.lambda_coeff, h.lambda_pow, stats);
  return cu(cudaGetLastError());
}

void uniq_push(std::vector<int> &v, int x) {
  if (x >= 1 && std::find(v.begin(), v.end(), x) == v.end()) v.push_back(x);
}

template <typename T>
nqs_status autotune_T(nqs_ctx *c, const double *theta, const nqs_step_hparams *hp, cudaStream_t st) {
  const int64_t ns = hp->n_samples, np = c->L.np;
  const int64_t R = c->L.cplx ? 2 * ns : ns;
  double *tth = W<double>(c, c->off.tth), *tmo = W<double>(c, c->off.tmo);
  nqs_step_stats *tstats = W<nqs_step_stats>(c, c->off.tstats);
  // one eager step on scratch copies fills the caches, O, the split planes and T
  c->tuned_ns = 0;
  CU(cudaMemcpyAsync(tth, theta, np * 8, cudaMemcpyDeviceToDevice, st));
  CU(cudaMemsetAsync(tmo, 0, np * 8, st));
  k_set_i64<<<1, 1, 0, st>>>(W<int64_t>(c, c->off.dstep), hp->step_index);
  ST(step_T<T>(c, tth, tmo, hp, tstats, nullptr, st));
  CU(cudaStreamSynchronize(st));
  c->tuned_ns = ns;
  c->t_eloc_grid = c->t_gram_splits = c->t_solve_grid = 0;
  c->t_chol_var = c->t_chol_subst = -1;
  const int reps = 2;
  auto none = [] { return NQS_OK; };
  uint8_t *spins = W<uint8_t>(c, c->off.spins);
  double *eloc = W<double>(c, c->off.eloc);
  // (1) grid of the connected-configuration engine
  {
    const bool tce = f32(c) && gram_tc_available() &&
                     (eloc_tc_supported(c->L.dim, c->L.dh) ||
                      (c->ck == 0 && (eloc2d_tc_supported(c->L.dim, c->L.dh) ||
                                      eloc2d_tcs_supported(c->L.dim, c->L.dh))));
    const int emax = tce ? c->rd.sm_count : c->eloc_grid;
    std::vector<int> cand;
    for (int d : {1, 2, 4}) uniq_push(cand, emax / d);
    uniq_push(cand, emax * 3 / 4);
    double best = 1e300;
    int pick = emax;
    for (int g : cand) {
      c->t_eloc_grid = g;
      double ms = 0;
      ST(best_ms(st, reps, none, [&] { return eloc_T<T>(c, ns, spins, eloc, st); }, &ms));
      if (g == emax) c->t_ms_default[0] = ms;
      if (ms < best) { best = ms; pick = g; }
    }
    c->t_eloc_grid = pick;
    c->t_ms[0] = best;
  }
  // (2) K-split of the tensor-core Gram
  if (f32(c) && gram_tc_available()) {
    const int smax = gram_tc_max_splits(R, np), sdef = gram_tc_default_splits(R, np);
    std::vector<int> cand;
    uniq_push(cand, sdef);
    for (int q : {1, 2, 3, 4, 6, 8, 12, 16, 24, 32})
      if (q <= smax) uniq_push(cand, q);
    double best = 1e300;
    int pick = sdef;
    double *Tm = W<double>(c, c->off.T);
    for (int q : cand) {
      double ms = 0;
      ST(best_ms(st, reps, none, [&] {
        return cu(gram_from_center_split(c->ws + c->off.split, R, np, Tm,
                                         W<int>(c, c->off.sstat), st, q));
      }, &ms));
      if (q == sdef) c->t_ms_default[1] = ms;
      if (ms < best) { best = ms; pick = q; }
    }
    c->t_gram_splits = pick;
    c->t_ms[1] = best;
  }
  // (3) tile mapping, sweep form and grid of the cooperative solve (T
  //     rebuilt before every timed solve)
  {
    const int G0 = c->rd.sm_count;
    double *Tm = W<double>(c, c->off.T);
    auto time_solve = [&](double *ms) {
      return best_ms(st, reps, [&] { return regram<T>(c, ns, *hp, tstats, st); },
                     [&] {
                       return chol_solve(c, Tm, R, W<double>(c, c->off.eps),
                                         W<double>(c, c->off.x), W<int32_t>(c, c->off.sstat), st);
                     }, ms);
    };
    const bool blk_ok = f32(c) && chol_blk_supported(R);
    const int var0 = blk_ok && R >= 3072 ? 2 : (R >= 2048 ? 1 : 0), sub0 = R >= 2048 ? 1 : 0;
    double best = 1e300;
    int pvar = var0, psub = sub0, pick = G0;
    c->t_solve_grid = G0;
    for (int var : {0, 1, 2})
      for (int sub : {0, 1}) {
        if (!f32(c) && (var != var0 || sub != sub0)) continue;  // FP64 path: one form
        if (var == 2 && (!blk_ok || sub != sub0)) continue;     // blocked: no sweep variants
        c->t_chol_var = var;
        c->t_chol_subst = sub;
        double ms = 0;
        ST(time_solve(&ms));
        if (var == var0 && sub == sub0) c->t_ms_default[2] = ms;
        if (ms < best) { best = ms; pvar = var; psub = sub; }
      }
    c->t_chol_var = pvar;
    c->t_chol_subst = psub;
    for (int g : {2 * G0, G0 / 2, G0 / 4, G0 / 8}) {
      if (g < 1) continue;
      c->t_solve_grid = g;
      double ms = 0;
      ST(time_solve(&ms));
      if (ms < best) { best = ms; pick = g; }
    }
    c->t_solve_grid = pick;
    c->t_ms[2] = best;
  }
  return NQS_OK;
}

void drop_graph(nqs_ctx *c) {
  if (c->gexec) { cudaGraphExecDestroy(c->gexec); c->gexec = nullptr; }
}

}  // namespace

extern "C" {

nqs_status nqs_autotune(nqs_ctx *c, const double *theta, const nqs_step_hparams *hp, int flags,
                        void *stream) {
  if (!c || !theta || !hp) return NQS_ERR_ARG;
  if (hp->n_samples < 2 || hp->n_samples > c->max_ns) return NQS_ERR_ARG;
  if (hp->lambda_mode != 0 && hp->lambda_mode != 1) return NQS_ERR_ARG;
  if (flags & ~NQS_TUNE_FORCE) return NQS_ERR_ARG;
  ST(need_ws(c));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const std::string key = tune_key(c, hp->n_samples);
  drop_graph(c);
  if (!(flags & NQS_TUNE_FORCE)) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      const Tuned &t = it->second;
      c->tuned_ns = hp->n_samples;
      c->t_eloc_grid = t.eloc_grid; c->t_gram_splits = t.gram_splits; c->t_solve_grid = t.solve_grid;
      c->t_chol_var = t.chol_var;
      c->t_chol_subst = t.chol_subst;
      std::memcpy(c->t_ms, t.ms, sizeof t.ms);
      std::memcpy(c->t_ms_default, t.ms_default, sizeof t.ms_default);
      return NQS_OK;
    }
  }
  const int64_t saved_tmax = c->tmax;
  c->tmax = c->tstep;  // no timing marks while tuning
  nqs_status s = f32(c) ? autotune_T<float>(c, theta, hp, st) : autotune_T<double>(c, theta, hp, st);
  c->tmax = (int)saved_tmax;
  if (s != NQS_OK) {
    c->tuned_ns = 0;
    return s;
  }
  Tuned t{c->t_eloc_grid, c->t_gram_splits, c->t_solve_grid, c->t_chol_var, c->t_chol_subst,
          {}, {}};
  std::memcpy(t.ms, c->t_ms, sizeof t.ms);
  std::memcpy(t.ms_default, c->t_ms_default, sizeof t.ms_default);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache[key] = t;
  return NQS_OK;
}

nqs_status nqs_get_tuning(const nqs_ctx *c, nqs_tuning *out) {
  if (!c || !out) return NQS_ERR_ARG;
  out->n_samples = c->tuned_ns;
  out->eloc_grid = c->t_eloc_grid;
  out->gram_splits = c->t_gram_splits;
  out->solve_grid = c->t_solve_grid;
  out->solve_form = c->t_chol_var;
  out->solve_substitution = c->t_chol_subst;
  for (int i = 0; i < 3; ++i) { out->ms[i] = c->t_ms[i]; out->ms_default[i] = c->t_ms_default[i]; }
  return NQS_OK;
}

nqs_status nqs_clear_tuning(nqs_ctx *c) {
  if (!c) return NQS_ERR_ARG;
  drop_graph(c);
  c->tuned_ns = 0;
  c->t_eloc_grid = c->t_gram_splits = c->t_solve_grid = 0;
  c->t_chol_var = c->t_chol_subst = -1;
  return NQS_OK;
}

nqs_status nqs_set_sampler(nqs_ctx *c, int form) {
  if (!c || form < -1 || form > 1) return NQS_ERR_ARG;
  drop_graph(c);
  c->sampler_form = form;
  return NQS_OK;
}

nqs_status nqs_set_solve_form(nqs_ctx *c, int form) {
  if (!c || form < -1 || form > 2) return NQS_ERR_ARG;
  drop_graph(c);
  c->solve_form = form;
  return NQS_OK;
}

nqs_status nqs_test_wait_timeout(nqs_ctx *c, uint64_t spin_limit, int drop_tile) {
  if (!c) return NQS_ERR_ARG;
  c->test_spin_limit = spin_limit;
  c->test_drop_tile = drop_tile ? 1 : 0;
  drop_graph(c);
  return NQS_OK;
}

nqs_status nqs_set_damping(nqs_ctx *c, double omega, double lambda0) {
  if (!c || !(omega == omega) || !(lambda0 == lambda0)) return NQS_ERR_ARG;
  if (omega > 1.0) {
    if (!(lambda0 > 0.0) || !std::isfinite(omega) || !std::isfinite(lambda0)) return NQS_ERR_ARG;
    ST(need_ws(c));
    // a step still running on any stream may read or rewrite the device-held
    // damping; the device is drained first so the new value is not raced
    CU(cudaDeviceSynchronize());
    CU(cudaMemcpy(c->ws + c->off.dlm, &lambda0, sizeof(double), cudaMemcpyHostToDevice));
    c->lm_omega = omega;
  } else {
    c->lm_omega = 0.0;
  }
  drop_graph(c);
  return NQS_OK;
}

// ------------------------------------------------------------ batched step

}  // extern "C"

// ---------------------------------------------------- sample-sharded step
// The steps of Algorithm 1 with the Ns samples split over G ranks: each rank
// samples, evaluates and differentiates its own range of samples; the
// centring sums are added over the ranks, the centred rows gathered, and the
// Gram, the solve and (by parameter ranges) delta theta formed from them.
namespace {

template <typename T>
nqs_status shard_forward_T(nqs_ctx *c, const double *theta, const nqs_step_hparams *hp,
                           int64_t s0, int64_t n, double *sums, cudaStream_t st) {
  const int64_t np = c->L.np;
  uint8_t *spins = W<uint8_t>(c, c->off.spins);
  double *eloc = W<double>(c, c->off.eloc);
  T *O = W<T>(c, c->off.O);
  c->cur_ns = n;
  CU(cudaMemsetAsync(W<int32_t>(c, c->off.sstat), 0, 64, st));
  k_set_i64<<<1, 1, 0, st>>>(W<int64_t>(c, c->off.dstep), hp->step_index);
  c->launches += 1;
  ST(pack_theta<T>(c, theta, st));
  {
    FwdArgs<T> a = fwd_args<T>(c);
    a.nrows = n; a.seed = hp->seed; a.step = (uint64_t)hp->step_index; a.s0 = s0;
    a.step_dev = W<int64_t>(c, c->off.dstep);
    a.spins = spins; a.logpsi = W<double>(c, c->off.logpsi);
    if (c->ck == 0) {
      a.gcache = W<T>(c, c->off.gcache);
      a.gw = c->gw;
    }
    ST(run_sample<T>(c, a, st));
  }
  ST(eloc_T<T>(c, n, spins, eloc, st));
  const unsigned nblk = c->L.cplx ? 2u : 1u;
  k_energy_sums<<<1, 1024, 0, st>>>(eloc, n, sums + nblk * np);
  ST(jac_T<T>(c, n, spins, O, st));
  const int chunks = (int)((n + COL_ROWS - 1) / COL_ROWS);
  dim3 g((unsigned)((np + 255) / 256), nblk * chunks);
  k_colsum_part<T><<<g, 256, 0, st>>>(O, n, np, chunks, W<double>(c, c->off.part));
  k_colsum_fin<<<dim3((unsigned)((np + 255) / 256), nblk), 256, 0, st>>>(
      W<double>(c, c->off.part), np, chunks, sums);
  c->launches += 3;
  return cu(cudaGetLastError());
}

template <typename T>
nqs_status shard_center_T(nqs_ctx *c, const double *sums, int64_t ns, int64_t n, void *rows,
                          double *eps, nqs_step_stats *stats, cudaStream_t st) {
  const int64_t np = c->L.np, nblk = c->L.cplx ? 2 : 1;
  k_shard_eps<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
      W<double>(c, c->off.eloc), n, c->L.N, c->L.cplx, sums + nblk * np, ns, stats, eps);
  const int64_t tot = nblk * n * np;
  const int blocks = (int)std::min<int64_t>((tot + 255) / 256, 148 * 16);
  k_shard_center<T><<<blocks, 256, 0, st>>>(W<T>(c, c->off.O), n, np, nblk * n, sums, ns,
                                            static_cast<T *>(rows));
  c->launches += 2;
  return cu(cudaGetLastError());
}

template <typename T>
nqs_status shard_solve_T(nqs_ctx *c, const void *A, int64_t R, const double *eps,
                         const nqs_step_hparams *hp, int64_t p0, int64_t p1, double *dtheta,
                         nqs_step_stats *stats, cudaStream_t st) {
  const int64_t np = c->L.np;
  double *Tm = W<double>(c, c->off.T);
  double *x = W<double>(c, c->off.x);
  int32_t *sstat = W<int32_t>(c, c->off.sstat);
  ST(gram_any(c, A, R, np, Tm, st));
  {
    const int nparts = 256;
    c->launches += 2;
    k_frob_part<<<nparts, 256, 0, st>>>(Tm, R * R, W<double>(c, c->off.frob));
    k_lambda_finish<<<1, 1024, 0, st>>>(Tm, R, W<double>(c, c->off.frob), nparts,
                                        hp->lambda_mode, hp->lambda, hp->lambda_coeff,
                                        hp->lambda_pow, stats, nullptr, nullptr);
    CU(cudaGetLastError());
  }
  const RetryInfo rinfo{hp, stats};
  ST(chol_solve(c, Tm, R, eps, x, sstat, st, f32(c) && gram_tc_available() ? &rinfo : nullptr));
  k_eta<<<1, 1024, 0, st>>>(eps, x, R, hp->eta0, hp->decay_T, hp->trust_region,
                            W<int64_t>(c, c->off.dstep), stats, sstat,
                            reinterpret_cast<int32_t *>(W<unsigned>(c, c->off.cbar) + 4));
  const int64_t nc = p1 - p0;
  if (nc > 0) {
    const int rows_per = 64;
    const int nparts = (int)((R + rows_per - 1) / rows_per);
    dim3 g((unsigned)((nc + 255) / 256), (unsigned)nparts);
    k_gemv_cols<T><<<g, 256, 0, st>>>(static_cast<const T *>(A), R, np, p0, nc, x, rows_per,
                                      W<double>(c, c->off.part));
    k_dtheta<<<(unsigned)((nc + 255) / 256), 256, 0, st>>>(W<double>(c, c->off.part), nparts,
                                                          nc, stats, dtheta);
    c->launches += 2;
  }
  c->launches += 1;
  return cu(cudaGetLastError());
}

// ------------------------------------------------------------ Adam, scan
// Sampling, local energies, E, Var and eps-bar' of theta (into the step's
// workspace regions); the first stages of Algorithm 1.
template <typename T>
nqs_status forward_energy_T(nqs_ctx *c, const double *theta, int64_t ns, uint64_t seed,
                            int64_t step, nqs_step_stats *stats, bool want_gates, cudaStream_t st) {
  uint8_t *spins = W<uint8_t>(c, c->off.spins);
  double *eloc = W<double>(c, c->off.eloc);
  c->cur_ns = ns;
  k_set_i64<<<1, 1, 0, st>>>(W<int64_t>(c, c->off.dstep), step);
  c->launches += 1;
  ST(pack_theta<T>(c, theta, st));
  {
    FwdArgs<T> a = fwd_args<T>(c);
    a.nrows = ns; a.seed = seed; a.step = (uint64_t)step;
    a.step_dev = W<int64_t>(c, c->off.dstep);
    a.spins = spins; a.logpsi = W<double>(c, c->off.logpsi);
    if (want_gates && c->ck == 0) {
      a.gcache = W<T>(c, c->off.gcache);
      a.gw = c->gw;
    }
    ST(run_sample<T>(c, a, st));
  }
  ST(eloc_T<T>(c, ns, spins, eloc, st));
  k_energy<<<1, 1024, 0, st>>>(eloc, ns, c->L.N, c->L.cplx, stats, W<double>(c, c->off.eps));
  c->launches += 1;
  return cu(cudaGetLastError());
}

template <typename T>
nqs_status adam_T(nqs_ctx *c, double *theta, double *m1, double *m2, const nqs_adam_hparams *ap,
                  nqs_step_stats *stats, double *grad_out, cudaStream_t st) {
  const int64_t ns = ap->n_samples, np = c->L.np;
  const int64_t R = c->L.cplx ? 2 * ns : ns;
  T *O = W<T>(c, c->off.O);
  double *eps = W<double>(c, c->off.eps);
  double *g = W<double>(c, c->off.dth);
  CU(cudaMemsetAsync(W<int32_t>(c, c->off.sstat), 0, 64, st));
  ST(forward_energy_T<T>(c, theta, ns, ap->seed, ap->step_index, stats, true, st));
  ST(jac_T<T>(c, ns, W<uint8_t>(c, c->off.spins), O, st));
  // centring as in the step: FP64 means, O' = (O - mean) / sqrt(Ns); the
  // tensor-core route of the mixed path keeps O' as the split planes
  const bool tc = f32(c) && gram_tc_available();
  {
    c->launches += 3;
    const int chunks = (int)((ns + COL_ROWS - 1) / COL_ROWS);
    const unsigned nblk = c->L.cplx ? 2u : 1u;
    dim3 gg((unsigned)((np + 255) / 256), nblk * chunks);
    k_colsum_part<T><<<gg, 256, 0, st>>>(O, ns, np, chunks, W<double>(c, c->off.part));
    k_colmean_fin<<<dim3((unsigned)((np + 255) / 256), nblk), 256, 0, st>>>(
        W<double>(c, c->off.part), ns, np, chunks, W<double>(c, c->off.mean), tc ? 1 : 0);
    CU(cudaGetLastError());
    if (tc) {
      CU(center_split(reinterpret_cast<const float *>(O), ns, np, R, W<float2>(c, c->off.mean),
                      c->ws + c->off.split, st));
    } else {
      const int64_t tot = R * np;
      const int blocks = (int)std::min<int64_t>((tot + 255) / 256, 148 * 16);
      k_center<T><<<blocks, 256, 0, st>>>(O, ns, np, R, W<double>(c, c->off.mean));
      CU(cudaGetLastError());
    }
  }
  // g = Obar'^T eps-bar', then the Adam update
  {
    const int rows_per = 64;
    const int nparts = (int)((R + rows_per - 1) / rows_per);
    dim3 gg((unsigned)((np + 255) / 256), (unsigned)nparts);
    if (tc)
      CU(gemv_split(c->ws + c->off.split, R, np, eps, rows_per, W<double>(c, c->off.part), st));
    else
      k_gemv_part<T><<<gg, 256, 0, st>>>(O, R, np, eps, rows_per, W<double>(c, c->off.part));
    k_grad_sum<<<(unsigned)((np + 255) / 256), 256, 0, st>>>(W<double>(c, c->off.part), nparts,
                                                            np, stats, g);
    k_adam<<<(unsigned)((np + 255) / 256), 256, 0, st>>>(theta, m1, m2, g, np, ap->beta1,
                                                        ap->beta2, ap->epsilon, ap->eta0,
                                                        ap->decay_T, ap->step_index, stats);
    c->launches += 3;
    CU(cudaGetLastError());
  }
  if (grad_out) CU(cudaMemcpyAsync(grad_out, g, np * 8, cudaMemcpyDeviceToDevice, st));
  return NQS_OK;
}

template <typename T>
nqs_status scan_T(nqs_ctx *c, const double *theta0, const double *v1, const double *v2,
                  const double *xy, int64_t npts, int64_t ns, uint64_t seed, double *out,
                  cudaStream_t st) {
  const int64_t np = c->L.np;
  double *th = W<double>(c, c->off.tth);
  nqs_step_stats *sst = reinterpret_cast<nqs_step_stats *>(W<double>(c, c->off.tstats));
  for (int64_t i = 0; i < npts; ++i) {
    k_axpy2<<<(unsigned)((np + 255) / 256), 256, 0, st>>>(theta0, v1, v2, xy[2 * i], xy[2 * i + 1],
                                                          np, th);
    ST(forward_energy_T<T>(c, th, ns, seed, 0, sst, false, st));
    k_scan_store<<<1, 1, 0, st>>>(sst, out + 4 * i);
    c->launches += 2;
  }
  return cu(cudaGetLastError());
}

}  // namespace

extern "C" {

nqs_status nqs_shard_forward(nqs_ctx *c, const double *theta, const nqs_step_hparams *hp,
                             int64_t s0, int64_t n, double *sums, void *stream) {
  if (!c || !theta || !hp || !sums || n < 1 || n > c->max_ns || s0 < 0 ||
      s0 + n > ((int64_t)1 << 32))
    return NQS_ERR_ARG;
  ST(need_ws(c));
  c->gnext = -1;  // the device step counter changes: a replayed step must set it again
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return f32(c) ? shard_forward_T<float>(c, theta, hp, s0, n, sums, st)
                : shard_forward_T<double>(c, theta, hp, s0, n, sums, st);
}

nqs_status nqs_shard_center(nqs_ctx *c, const double *sums, int64_t ns, int64_t n, void *rows,
                            double *eps, nqs_step_stats *dev_stats, void *stream) {
  if (!c || !sums || !rows || !eps || !dev_stats || n < 1 || n > c->max_ns || ns < n ||
      n != c->cur_ns)
    return NQS_ERR_ARG;
  ST(need_ws(c));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return f32(c) ? shard_center_T<float>(c, sums, ns, n, rows, eps, dev_stats, st)
                : shard_center_T<double>(c, sums, ns, n, rows, eps, dev_stats, st);
}

nqs_status nqs_shard_solve(nqs_ctx *c, const void *rows, int64_t R, const double *eps,
                           const nqs_step_hparams *hp, int64_t p0, int64_t p1, double *dtheta,
                           nqs_step_stats *dev_stats, void *stream) {
  const int64_t rmax = c ? (c->L.cplx ? 2 * c->max_ns : c->max_ns) : 0;
  if (!c || !rows || !eps || !hp || !dev_stats || R < 2 || R > rmax ||
      (c->L.cplx && R % 2) || p0 < 0 || p1 < p0 || p1 > c->L.np || (p1 > p0 && !dtheta) ||
      (hp->lambda_mode != 0 && hp->lambda_mode != 1))
    return NQS_ERR_ARG;
  ST(need_ws(c));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return f32(c) ? shard_solve_T<float>(c, rows, R, eps, hp, p0, p1, dtheta, dev_stats, st)
                : shard_solve_T<double>(c, rows, R, eps, hp, p0, p1, dtheta, dev_stats, st);
}

nqs_status nqs_shard_apply(nqs_ctx *c, double *theta, double *mom, const double *dtheta,
                           const nqs_step_hparams *hp, nqs_step_stats *dev_stats, void *stream) {
  if (!c || !theta || !mom || !dtheta || !hp || !dev_stats) return NQS_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t np = c->L.np;
  const unsigned blocks = (unsigned)((np + 255) / 256);
  k_check_finite<<<blocks, 256, 0, st>>>(dtheta, np, dev_stats);
  k_apply<<<blocks, 256, 0, st>>>(theta, mom, dtheta, np, hp->mu, dev_stats);
  c->launches += 2;
  return cu(cudaGetLastError());
}

nqs_status nqs_adam_step(nqs_ctx *c, double *theta, double *m1, double *m2,
                         const nqs_adam_hparams *ap, nqs_step_stats *dev_stats, double *grad,
                         void *stream) {
  if (!c || !theta || !m1 || !m2 || !ap || !dev_stats) return NQS_ERR_ARG;
  if (ap->n_samples < 2 || ap->n_samples > c->max_ns || ap->step_index < 0) return NQS_ERR_ARG;
  if (!(ap->beta1 >= 0.0 && ap->beta1 < 1.0 && ap->beta2 >= 0.0 && ap->beta2 < 1.0 &&
        ap->epsilon > 0.0))
    return NQS_ERR_ARG;
  ST(need_ws(c));
  c->gnext = -1;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return f32(c) ? adam_T<float>(c, theta, m1, m2, ap, dev_stats, grad, st)
                : adam_T<double>(c, theta, m1, m2, ap, dev_stats, grad, st);
}

nqs_status nqs_energy_scan(nqs_ctx *c, const double *theta0, const double *v1, const double *v2,
                           const double *xy, int64_t npts, int64_t ns, uint64_t seed,
                           double *out, void *stream) {
  if (!c || !theta0 || !v1 || !v2 || !xy || !out || npts < 0 || ns < 1 || ns > c->max_ns)
    return NQS_ERR_ARG;
  ST(need_ws(c));
  c->gnext = -1;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return f32(c) ? scan_T<float>(c, theta0, v1, v2, xy, npts, ns, seed, out, st)
                : scan_T<double>(c, theta0, v1, v2, xy, npts, ns, seed, out, st);
}

}  // extern "C"

struct nqs_batch {
  std::vector<nqs_ctx *> ctx;
  int conc = 0;  // instance streams in use (0: one per instance)
  std::vector<cudaStream_t> st;
  std::vector<cudaEvent_t> done, solved;
  cudaEvent_t fork = nullptr;
  cudaStream_t cap = nullptr;
  // by stage: an instance's part issued (part), the grouped launches' stream
  // and their completion (grp)
  std::vector<cudaEvent_t> part;
  cudaStream_t gst = nullptr;
  cudaEvent_t grp = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int graph_enabled = 0, graph_broken = 0;
  // by stage: GROUP_SOLVE, the FP32 solves of all instances in one launch;
  // GROUP_ELOC, the streamed local-energy engines in one launch per hidden size
  int grouped = 0;
  int eloc_eighths = 8;  // the local-energy engines' share of their grids
  struct Key {
    std::vector<const void *> ptr;  // theta, momentum, stats of every instance
    std::vector<nqs_step_hparams> hp;
    int conc, grouped, eloc_eighths;
  } key;
  std::vector<int64_t> gnext;
};

namespace {

void batch_free(nqs_batch *b) {
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  for (cudaStream_t s : b->st) if (s) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->done) if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : b->solved) if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : b->part) if (e) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->grp) cudaEventDestroy(b->grp);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->gst) cudaStreamDestroy(b->gst);
  delete b;
}

int batch_conc(const nqs_batch *b) {
  const int n = (int)b->ctx.size();
  return b->conc > 0 && b->conc < n ? b->conc : n;
}

// Predicted duration (us) of the blocked solve of order n on G CTAs: per
// panel one tile product per row block for the panel rows, then the
// trailing tiles on G - 1 CTAs while CTA 0 factors the next diagonal block,
// at least the panel's dependent chain (panel solve, diagonal tile, factor
// and inverse, publish: about 80 us, measured at n = 8192); three
// refinement sweeps of 2 nb block steps.  A tile product takes about 22 us
// (8.6 ms for the n = 8192 factor on 148 CTAs).
double blk_solve_us(int64_t n, int G) {
  const double tile = 22.0, chain = 80.0, step = 8.0;
  const int64_t nb = (n + BKB - 1) / BKB;
  double t = 0.0;
  for (int64_t p = 0; p + 1 < nb; ++p) {
    const int64_t nr = nb - 1 - p, tiles = nr * (nr + 1) / 2;
    t += (double)((nr + G - 1) / G) * tile;
    const int64_t Gr = std::max(G - 1, 1);
    t += std::max((double)((tiles - 1 + Gr - 1) / Gr) * tile, chain);
  }
  return t + 3.0 * 2.0 * (double)nb * step;
}

// CTAs per instance of a grouped solve on S SMs (two at least): each spare
// CTA goes to the instance predicted to finish last, up to the CTAs its
// first panel can use.  Empty if S cannot give every instance two.
std::vector<int> blk_split(const std::vector<int64_t> &n, int S) {
  const int k = (int)n.size();
  if (2 * k > S) return {};
  std::vector<int> G(k, 2);
  std::vector<double> t(k);
  for (int i = 0; i < k; ++i) t[i] = blk_solve_us(n[i], 2);
  for (int used = 2 * k; used < S; ++used) {
    int w = -1;
    for (int i = 0; i < k; ++i) {
      const int64_t nr = (n[i] + BKB - 1) / BKB - 1;
      if (G[i] < nr * (nr + 1) / 2 + 1 && (w < 0 || t[i] > t[w])) w = i;
    }
    if (w < 0) break;
    t[w] = blk_solve_us(n[w], ++G[w]);
  }
  return G;
}

// One cooperative launch of the FP32 factors and refinements of the
// instances in `idx` (batches of BLK_GROUP_MAX, each on the whole GPU).
nqs_status batch_group_solve(nqs_batch *b, const std::vector<int> &idx,
                             const nqs_step_hparams *hps, cudaStream_t st) {
  if (idx.empty()) return NQS_OK;
  const size_t smem = chol_blk_smem();
  CU(cudaFuncSetAttribute((const void *)k_chol_blk_group,
                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per = 0;
  CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_chol_blk_group, BKB_THREADS, smem));
  if (per < 1) return NQS_ERR_UNSUPPORTED;
  // one CTA per SM at most: an instance's partial norms are sized for that
  const int S = b->ctx[idx[0]]->rd.sm_count;
  const int chunk = std::min<int>(BLK_GROUP_MAX, S / 2);
  for (size_t i0 = 0; i0 < idx.size(); i0 += chunk) {
    const int k = (int)std::min<size_t>(chunk, idx.size() - i0);
    std::vector<int64_t> R(k);
    for (int j = 0; j < k; ++j) {
      const nqs_ctx *c = b->ctx[idx[i0 + j]];
      R[j] = c->L.cplx ? 2 * hps[idx[i0 + j]].n_samples : hps[idx[i0 + j]].n_samples;
    }
    const std::vector<int> G = blk_split(R, S);
    if ((int)G.size() != k) return NQS_ERR_UNSUPPORTED;
    CholBlkGroup gr{};
    gr.n = k;
    gr.cta0[0] = 0;
    for (int j = 0; j < k; ++j) {
      nqs_ctx *c = b->ctx[idx[i0 + j]];
      gr.inst[j] = blk_args(c, W<double>(c, c->off.T), R[j], W<double>(c, c->off.eps),
                            W<double>(c, c->off.x), W<int32_t>(c, c->off.sstat));
      gr.cta0[j + 1] = gr.cta0[j] + G[j];
      if (j == 0) c->launches += 1;  // the grouped launch, counted once
    }
    void *args[] = {&gr};
    CU(cudaLaunchCooperativeKernel((const void *)k_chol_blk_group, dim3(gr.cta0[k]),
                                   dim3(BKB_THREADS), args, smem, st));
  }
  return NQS_OK;
}

// Whether a batch may run this context's local-energy engine in its grouped
// launch (the streamed tensor-core engine, hidden sizes 96 and 128).
bool eloc_groupable(const nqs_ctx *c) {
  return f32(c) && c->ck == 0 && c->n_off > 0 && gram_tc_available() &&
         eloc2d_tcs_supported(c->L.dim, c->L.dh) && !eloc2d_tc_supported(c->L.dim, c->L.dh);
}

// CTAs per instance of a grouped engine launch on S SMs: one each, then each
// spare CTA to the instance with the most work per CTA, up to its tile count.
std::vector<int> eloc_split(const std::vector<double> &work, const std::vector<int> &cap, int S) {
  const int k = (int)work.size();
  std::vector<int> G(k, 1);
  for (int used = k; used < S; ++used) {
    int w = -1;
    for (int i = 0; i < k; ++i)
      if (G[i] < cap[i] && (w < 0 || work[i] / G[i] > work[w] / G[w])) w = i;
    if (w < 0) break;
    ++G[w];
  }
  return G;
}

// One launch of the streamed local-energy engine per hidden size over the
// instances whose step left its arguments (in_eloc_group).  An instance's
// share of the SMs follows its engine time measured by the autotuner (times
// the CTAs it was measured on), else its tiles times its sites.
nqs_status batch_group_eloc(nqs_batch *b, cudaStream_t st) {
  for (int dh : {128, 96}) {
    std::vector<int> idx;
    for (int i = 0; i < (int)b->ctx.size(); ++i)
      if (b->ctx[i]->in_eloc_group && b->ctx[i]->L.dh == dh) idx.push_back(i);
    if (idx.empty()) continue;
    const int S = b->ctx[idx[0]]->rd.sm_count;
    bool measured = true;
    for (int i : idx) measured = measured && tuned(b->ctx[i]) && b->ctx[i]->t_ms[0] > 0;
    const int chunk = std::min(ELOC2D_GROUP_MAX, S);
    for (size_t i0 = 0; i0 < idx.size(); i0 += chunk) {
      const int k = (int)std::min<size_t>(chunk, idx.size() - i0);
      std::vector<double> work(k);
      std::vector<int> cap(k);
      for (int j = 0; j < k; ++j) {
        const nqs_ctx *c = b->ctx[idx[i0 + j]];
        cap[j] = c->eloc_args.ntiles;
        work[j] = measured ? c->t_ms[0] * eloc_grid_cap(c, S)
                           : (double)c->eloc_args.ntiles * (double)c->L.N;
      }
      const std::vector<int> G = eloc_split(work, cap, S);
      Eloc2dTcGroup g{};
      g.n = k;
      g.cta0[0] = 0;
      for (int j = 0; j < k; ++j) {
        g.inst[j] = b->ctx[idx[i0 + j]]->eloc_args;
        g.cta0[j + 1] = g.cta0[j] + G[j];
      }
      b->ctx[idx[i0]]->launches += 1;  // the grouped launch, counted once
      CU(eloc2d_tcs_group_run(g, dh, st));
    }
  }
  return NQS_OK;
}

// The batched step by stage.  Every instance's step runs on its instance
// stream in three parts; only the members of a grouped launch wait for it:
// the streamed local-energy engine of the members of that group runs as one
// launch per hidden size on the batch's group stream once their first parts
// are done, and their second parts wait for it; the FP32 solves of the solve
// group run as one cooperative launch once those members' second parts are
// done.  The cooperative work after it (the members' gated FP64 fallbacks,
// the other instances' own solves) stays chained in instance order behind
// the grouped solve, so that no two cooperative kernels are resident at once.
nqs_status batch_issue_grouped(nqs_batch *b, double *const *th, double *const *mo,
                               const nqs_step_hparams *hps, nqs_step_stats *const *stats,
                               bool set_steps, cudaStream_t origin) {
  const int n = (int)b->ctx.size(), q = batch_conc(b);
  std::vector<int> idx;
  bool any_eloc = false;
  for (int i = 0; i < n; ++i) {
    nqs_ctx *c = b->ctx[i];
    const int64_t R = c->L.cplx ? 2 * hps[i].n_samples : hps[i].n_samples;
    c->in_group = (b->grouped & GROUP_SOLVE) && group_solvable(c, R) ? 1 : 0;
    c->in_eloc_group = (b->grouped & GROUP_ELOC) && eloc_groupable(c) ? 1 : 0;
    if (c->in_group) idx.push_back(i);
    any_eloc = any_eloc || c->in_eloc_group;
  }
  CU(cudaEventRecord(b->fork, origin));
  for (int j = 0; j < q; ++j) CU(cudaStreamWaitEvent(b->st[j], b->fork, 0));
  CU(cudaStreamWaitEvent(b->gst, b->fork, 0));
  nqs_status s = NQS_OK;
  auto issue = [&](int i, int ph) {
    nqs_ctx *c = b->ctx[i];
    c->phase = ph;
    c->eloc_eighths = b->eloc_eighths;
    const nqs_status r = step_body(c, th[i], mo[i], &hps[i], stats[i], nullptr, b->st[i % q]);
    c->eloc_eighths = 8;
    c->phase = STEP_ALL;
    return r;
  };
  // first parts; the engine group waits for its members'
  for (int i = 0; i < n && s == NQS_OK; ++i) {
    nqs_ctx *c = b->ctx[i];
    if (set_steps) {
      k_set_i64<<<1, 1, 0, b->st[i % q]>>>(W<int64_t>(c, c->off.dstep), hps[i].step_index);
      c->launches += 1;
    }
    s = issue(i, STEP_PRE_A);
    if (s == NQS_OK && c->in_eloc_group) {
      CU(cudaEventRecord(b->part[i], b->st[i % q]));
      CU(cudaStreamWaitEvent(b->gst, b->part[i], 0));
    }
  }
  if (s == NQS_OK && any_eloc) {
    s = batch_group_eloc(b, b->gst);
    if (s == NQS_OK) CU(cudaEventRecord(b->grp, b->gst));
  }
  // second parts; the solve group waits for its members'
  for (int i = 0; i < n && s == NQS_OK; ++i) {
    nqs_ctx *c = b->ctx[i];
    if (c->in_eloc_group) CU(cudaStreamWaitEvent(b->st[i % q], b->grp, 0));
    s = issue(i, STEP_PRE_B);
    if (s == NQS_OK && c->in_group) {
      CU(cudaEventRecord(b->part[i], b->st[i % q]));
      CU(cudaStreamWaitEvent(b->gst, b->part[i], 0));
    }
  }
  bool solve_grouped = false;
  if (s == NQS_OK && !idx.empty()) {
    s = batch_group_solve(b, idx, hps, b->gst);
    if (s == NQS_OK) CU(cudaEventRecord(b->grp, b->gst));
    solve_grouped = s == NQS_OK;
  }
  // the rest: cooperative work chained in instance order behind the group
  for (int i = 0; i < n && s == NQS_OK; ++i) {
    nqs_ctx *c = b->ctx[i];
    c->solve_wait = i > 0 ? b->solved[i - 1] : (solve_grouped ? b->grp : nullptr);
    c->solve_rec = b->solved[i];
    s = issue(i, STEP_POST);
    c->solve_wait = c->solve_rec = nullptr;
  }
  for (int j = 0; j < q; ++j) {
    CU(cudaEventRecord(b->done[j], b->st[j]));
    CU(cudaStreamWaitEvent(origin, b->done[j], 0));
  }
  CU(cudaEventRecord(b->grp, b->gst));
  CU(cudaStreamWaitEvent(origin, b->grp, 0));
  for (nqs_ctx *c : b->ctx) c->in_group = c->in_eloc_group = 0;
  return s;
}

// Fork the instances' steps from `origin` onto the instance streams and join
// them back; cooperative solves run one after another (instance order).
nqs_status batch_issue(nqs_batch *b, double *const *th, double *const *mo,
                       const nqs_step_hparams *hps, nqs_step_stats *const *stats, bool set_steps,
                       cudaStream_t origin) {
  if (b->grouped) return batch_issue_grouped(b, th, mo, hps, stats, set_steps, origin);
  const int n = (int)b->ctx.size(), q = batch_conc(b);
  CU(cudaEventRecord(b->fork, origin));
  for (int j = 0; j < q; ++j) CU(cudaStreamWaitEvent(b->st[j], b->fork, 0));
  nqs_status s = NQS_OK;
  for (int i = 0; i < n && s == NQS_OK; ++i) {
    nqs_ctx *c = b->ctx[i];
    cudaStream_t st = b->st[i % q];
    if (set_steps) {
      k_set_i64<<<1, 1, 0, st>>>(W<int64_t>(c, c->off.dstep), hps[i].step_index);
      c->launches += 1;
    }
    c->solve_wait = i > 0 ? b->solved[i - 1] : nullptr;
    c->solve_rec = b->solved[i];
    c->eloc_eighths = b->eloc_eighths;
    s = step_body(c, th[i], mo[i], &hps[i], stats[i], nullptr, st);
    c->eloc_eighths = 8;
    c->solve_wait = c->solve_rec = nullptr;
  }
  for (int j = 0; j < q; ++j) {
    CU(cudaEventRecord(b->done[j], b->st[j]));
    CU(cudaStreamWaitEvent(origin, b->done[j], 0));
  }
  return s;
}

nqs_status batch_check(nqs_batch *b, double *const *th, double *const *mo,
                       const nqs_step_hparams *hps) {
  for (size_t i = 0; i < b->ctx.size(); ++i) {
    nqs_ctx *c = b->ctx[i];
    if (!th[i] || !mo[i]) return NQS_ERR_ARG;
    if (hps[i].n_samples < 2 || hps[i].n_samples > c->max_ns) return NQS_ERR_ARG;
    if (hps[i].lambda_mode != 0 && hps[i].lambda_mode != 1) return NQS_ERR_ARG;
    ST(need_ws(c));
  }
  return NQS_OK;
}

nqs_status batch_step(nqs_batch *b, double *const *th, double *const *mo,
                      const nqs_step_hparams *hps, nqs_step_stats *const *stats, cudaStream_t st) {
  const int n = (int)b->ctx.size();
  bool timing = false;
  for (nqs_ctx *c : b->ctx) timing |= c->tstep < c->tmax;
  if (b->graph_enabled && !b->graph_broken && !timing) {
    nqs_batch::Key k;
    for (int i = 0; i < n; ++i) {
      k.ptr.push_back(th[i]); k.ptr.push_back(mo[i]); k.ptr.push_back(stats[i]);
      nqs_step_hparams h = hps[i];
      h.step_index = 0;
      k.hp.push_back(h);
    }
    k.conc = batch_conc(b);
    k.grouped = b->grouped;
    k.eloc_eighths = b->eloc_eighths;
    bool same = b->gexec && k.ptr == b->key.ptr && k.conc == b->key.conc &&
                k.grouped == b->key.grouped && k.eloc_eighths == b->key.eloc_eighths;
    for (int i = 0; same && i < n; ++i)
      same = std::memcmp(&k.hp[i], &b->key.hp[i], sizeof(nqs_step_hparams)) == 0;
    if (!same) {
      if (b->gexec) { cudaGraphExecDestroy(b->gexec); b->gexec = nullptr; }
      cudaGraph_t g = nullptr;
      bool ok = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
      nqs_status s = NQS_OK;
      if (ok) s = batch_issue(b, th, mo, hps, stats, false, b->cap);
      const bool ended = cudaStreamEndCapture(b->cap, &g) == cudaSuccess;
      ok = ok && ended && s == NQS_OK && g;
      if (ok) ok = cudaGraphInstantiate(&b->gexec, g, 0) == cudaSuccess;
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      if (!ok) {
        b->gexec = nullptr;
        b->graph_broken = 1;
      } else {
        b->key = k;
        b->gnext.assign(n, -1);
      }
    }
    if (b->gexec) {
      for (int i = 0; i < n; ++i)
        if (hps[i].step_index != b->gnext[i]) {
          nqs_ctx *c = b->ctx[i];
          k_set_i64<<<1, 1, 0, st>>>(W<int64_t>(c, c->off.dstep), hps[i].step_index);
          c->launches += 1;
          CU(cudaGetLastError());
        }
      CU(cudaGraphLaunch(b->gexec, st));
      for (int i = 0; i < n; ++i) b->gnext[i] = hps[i].step_index + 1;
      return NQS_OK;
    }
  }
  b->gnext.assign(n, -1);
  return batch_issue(b, th, mo, hps, stats, true, st);
}

}  // namespace

extern "C" {

nqs_status nqs_batch_create(int n, nqs_ctx *const *ctxs, nqs_batch **out) {
  if (!out || n <= 0 || n > 4096 || !ctxs) return NQS_ERR_ARG;
  *out = nullptr;
  for (int i = 0; i < n; ++i) {
    if (!ctxs[i]) return NQS_ERR_ARG;
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i]) return NQS_ERR_ARG;  // one workspace per instance
  }
  nqs_batch *b = new (std::nothrow) nqs_batch();
  if (!b) return NQS_ERR_ARG;
  b->ctx.assign(ctxs, ctxs + n);
  b->st.assign(n, nullptr);
  b->done.assign(n, nullptr);
  b->solved.assign(n, nullptr);
  b->part.assign(n, nullptr);
  bool ok = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&b->grp, cudaEventDisableTiming) == cudaSuccess &&
            cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) == cudaSuccess &&
            cudaStreamCreateWithFlags(&b->gst, cudaStreamNonBlocking) == cudaSuccess;
  for (int i = 0; ok && i < n; ++i)
    ok = cudaStreamCreateWithFlags(&b->st[i], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&b->done[i], cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&b->solved[i], cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&b->part[i], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) { batch_free(b); return NQS_ERR_CUDA; }
  *out = b;
  return NQS_OK;
}

nqs_status nqs_batch_destroy(nqs_batch *b) {
  if (!b) return NQS_ERR_ARG;
  cudaDeviceSynchronize();
  batch_free(b);
  return NQS_OK;
}

nqs_status nqs_batch_set_graph(nqs_batch *b, int enable) {
  if (!b) return NQS_ERR_ARG;
  b->graph_enabled = enable != 0;
  return NQS_OK;
}

nqs_status nqs_batch_graph_active(const nqs_batch *b, int *active) {
  if (!b || !active) return NQS_ERR_ARG;
  *active = b->gexec != nullptr && !b->graph_broken;
  return NQS_OK;
}

nqs_status nqs_batch_set_concurrency(nqs_batch *b, int streams) {
  if (!b || streams < 0) return NQS_ERR_ARG;
  b->conc = streams;
  return NQS_OK;
}

nqs_status nqs_batch_get_concurrency(const nqs_batch *b, int *streams) {
  if (!b || !streams) return NQS_ERR_ARG;
  *streams = batch_conc(b);
  return NQS_OK;
}

nqs_status nqs_batch_set_grouped(nqs_batch *b, int stages) {
  if (!b || stages < 0 || stages > 3) return NQS_ERR_ARG;
  b->grouped = stages;
  return NQS_OK;
}

nqs_status nqs_batch_set_eloc_share(nqs_batch *b, int eighths) {
  if (!b || eighths < 1 || eighths > 8) return NQS_ERR_ARG;
  b->eloc_eighths = eighths;
  return NQS_OK;
}

nqs_status nqs_batch_get_eloc_share(const nqs_batch *b, int *eighths) {
  if (!b || !eighths) return NQS_ERR_ARG;
  *eighths = b->eloc_eighths;
  return NQS_OK;
}

nqs_status nqs_batch_get_grouped(const nqs_batch *b, int *stages) {
  if (!b || !stages) return NQS_ERR_ARG;
  *stages = b->grouped;
  return NQS_OK;
}

nqs_status nqs_minsr_step_batched(nqs_batch *b, double *const *thetas, double *const *moms,
                                  const nqs_step_hparams *hps, nqs_step_stats *dev_stats,
                                  void *stream) {
  if (!b || !thetas || !moms || !hps || !dev_stats) return NQS_ERR_ARG;
  ST(batch_check(b, thetas, moms, hps));
  std::vector<nqs_step_stats *> sp(b->ctx.size());
  for (size_t i = 0; i < sp.size(); ++i) sp[i] = dev_stats + i;
  return batch_step(b, thetas, moms, hps, sp.data(), static_cast<cudaStream_t>(stream));
}

nqs_status nqs_batch_autotune(nqs_batch *b, double *const *thetas, const nqs_step_hparams *hps,
                              int flags, double *step_ms, void *stream) {
  if (!b || !thetas || !hps) return NQS_ERR_ARG;
  const int n = (int)b->ctx.size();
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // (1) every instance alone
  for (int i = 0; i < n; ++i) ST(nqs_autotune(b->ctx[i], thetas[i], &hps[i], flags, stream));
  // (2) instance streams: whole batched steps on scratch copies of theta
  std::vector<double *> th(n), mo(n);
  std::vector<nqs_step_stats *> sp(n);
  for (int i = 0; i < n; ++i) {
    nqs_ctx *c = b->ctx[i];
    th[i] = W<double>(c, c->off.tth);
    mo[i] = W<double>(c, c->off.tmo);
    sp[i] = W<nqs_step_stats>(c, c->off.tstats);
  }
  std::vector<int> cand;
  for (int q : {1, 2, 4, 8, 16}) if (q < n) uniq_push(cand, q);
  uniq_push(cand, n);
  const int saved_graph = b->graph_enabled;
  b->graph_enabled = 0;
  double best = 1e300;
  int pick = n;
  nqs_status s = NQS_OK;
  for (int q : cand) {
    b->conc = q;
    double ms = 0;
    s = best_ms(st, 2, [&] {
      for (int i = 0; i < n; ++i) {
        const int64_t np = b->ctx[i]->L.np;
        CU(cudaMemcpyAsync(th[i], thetas[i], np * 8, cudaMemcpyDeviceToDevice, st));
        CU(cudaMemsetAsync(mo[i], 0, np * 8, st));
      }
      return NQS_OK;
    }, [&] { return batch_step(b, th.data(), mo.data(), hps, sp.data(), st); }, &ms);
    if (s != NQS_OK) break;
    if (ms < best) { best = ms; pick = q; }
  }
  b->conc = pick;
  // (3) grids of the instances' cooperative solves: each takes the whole
  // GPU alone, so one other instance's kernels wait for it; a fraction of
  // the SMs per solve lets them run beside it
  std::vector<int> g0(n);
  for (int i = 0; i < n; ++i) g0[i] = b->ctx[i]->t_solve_grid;
  int pdiv = 1;
  for (int div : {2, 4}) {
    if (s != NQS_OK) break;
    for (int i = 0; i < n; ++i) {
      const int g = g0[i] > 0 ? g0[i] : b->ctx[i]->rd.sm_count;
      b->ctx[i]->t_solve_grid = std::max(1, g / div);
    }
    double ms = 0;
    s = best_ms(st, 2, [&] {
      for (int i = 0; i < n; ++i) {
        const int64_t np = b->ctx[i]->L.np;
        CU(cudaMemcpyAsync(th[i], thetas[i], np * 8, cudaMemcpyDeviceToDevice, st));
        CU(cudaMemsetAsync(mo[i], 0, np * 8, st));
      }
      return NQS_OK;
    }, [&] { return batch_step(b, th.data(), mo.data(), hps, sp.data(), st); }, &ms);
    if (s == NQS_OK && ms < best) { best = ms; pdiv = div; }
  }
  for (int i = 0; i < n; ++i) {
    const int g = g0[i] > 0 ? g0[i] : b->ctx[i]->rd.sm_count;
    b->ctx[i]->t_solve_grid = pdiv == 1 ? g0[i] : std::max(1, g / pdiv);
  }
  if (pdiv != 1) {  // the process-wide choices follow, so a context tuned later matches
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (int i = 0; i < n; ++i) {
      auto it = g_tune_cache.find(tune_key(b->ctx[i], b->ctx[i]->tuned_ns));
      if (it != g_tune_cache.end()) it->second.solve_grid = b->ctx[i]->t_solve_grid;
    }
  }
  // (4) by stage (the FP32 solves, and the streamed local-energy engines,
  // of all instances in grouped launches) or whole steps per stream: the
  // candidates in turn, five rounds, the median of each (consecutive
  // batched steps of one setting vary by several per cent with the clocks
  // and the power cap, so a best-of-two favours the noisier setting)
  auto reset = [&] {
    for (int i = 0; i < n; ++i) {
      const int64_t np = b->ctx[i]->L.np;
      CU(cudaMemcpyAsync(th[i], thetas[i], np * 8, cudaMemcpyDeviceToDevice, st));
      CU(cudaMemsetAsync(mo[i], 0, np * 8, st));
    }
    return NQS_OK;
  };
  auto step = [&] { return batch_step(b, th.data(), mo.data(), hps, sp.data(), st); };
  auto median3 = [](std::vector<double> v) {
    std::sort(v.begin(), v.end());
    return v[v.size() / 2];
  };
  if (s == NQS_OK) {
    const int cands[3] = {0, GROUP_SOLVE, GROUP_SOLVE | GROUP_ELOC};
    std::vector<double> t[3];
    for (int r = 0; r < 5 && s == NQS_OK; ++r)
      for (int j = 0; j < 3 && s == NQS_OK; ++j) {
        b->grouped = cands[j];
        double ms = 0;
        s = best_ms(st, 1, reset, step, &ms);
        t[j].push_back(ms);
      }
    if (s == NQS_OK) {
      // the fewest grouped stages within 2 % of the fastest: the grouped
      // local-energy launch trades overlap for fewer launches, and over
      // longer runs it measured a few per cent slower than the grouped solve
      // alone although short rounds sometimes favour it
      double m[3], mbest = 1e300;
      for (int j = 0; j < 3; ++j) mbest = std::min(mbest, m[j] = median3(t[j]));
      int pj = 0;
      while (m[pj] > 1.02 * mbest) ++pj;
      b->grouped = cands[pj];
      best = m[pj];
    }
  }
  // (5) one graph replay per step, or the launches themselves, whichever is
  // faster for this batch (a captured step can order the instances' kernels
  // less favourably than the eager issue)
  b->graph_enabled = saved_graph;
  if (saved_graph && s == NQS_OK) {
    if (b->gexec) { cudaGraphExecDestroy(b->gexec); b->gexec = nullptr; }
    // graph and eager steps in turn after one capture, medians of three
    std::vector<double> tg, te;
    double ms = 0;
    s = best_ms(st, 1, reset, step, &ms);  // the capture
    for (int r = 0; r < 3 && s == NQS_OK; ++r) {
      b->graph_enabled = saved_graph;
      s = best_ms(st, 1, reset, step, &ms);
      tg.push_back(ms);
      if (s != NQS_OK) break;
      b->graph_enabled = 0;
      s = best_ms(st, 1, reset, step, &ms);
      te.push_back(ms);
    }
    if (s == NQS_OK) {
      const bool g = median3(tg) <= median3(te);
      b->graph_enabled = g ? saved_graph : 0;
      best = g ? median3(tg) : median3(te);
    }
  }
  if (b->gexec) { cudaGraphExecDestroy(b->gexec); b->gexec = nullptr; }
  if (step_ms) *step_ms = best;
  return s;
}

nqs_status nqs_eloc_work(const nqs_ctx *c, int64_t *configs, int64_t *sites) {
  if (!c || !configs || !sites) return NQS_ERR_ARG;
  if (!c->ws) return NQS_ERR_WORKSPACE;
  std::vector<int> cnt(std::max(c->n_off, 1));
  if (c->n_off > 0 &&
      cudaMemcpy(cnt.data(), c->ws + c->off.item_cnt, sizeof(int) * c->n_off,
                 cudaMemcpyDeviceToHost) != cudaSuccess)
    return NQS_ERR_CUDA;
  int64_t nc = 0, ns = 0;
  for (int i = 0; i < c->n_off; ++i) {
    nc += cnt[i];
    ns += (int64_t)cnt[i] * (c->L.N - c->op_start[i]);
  }
  *configs = nc;
  *sites = ns;
  return NQS_OK;
}

const char *nqs_stage_name(int i) {
  static const char *names[NQS_N_STAGES] = {"pack", "sample", "eloc_gen", "eloc_suffix",
                                            "eloc_reduce", "energy", "jac_bwd", "jac_grad",
                                            "center", "gram", "lambda", "cholesky", "solve",
                                            "update"};
  return (i >= 0 && i < NQS_N_STAGES) ? names[i] : nullptr;
}

nqs_status nqs_timing_begin(nqs_ctx *c, int max_steps) {
  if (!c || max_steps <= 0 || max_steps > 100000) return NQS_ERR_ARG;
  timing_free(c);
  c->tev.resize((size_t)max_steps * (NQS_N_STAGES + 1));
  for (auto &e : c->tev)
    if (cudaEventCreate(&e) != cudaSuccess) { e = nullptr; timing_free(c); return NQS_ERR_CUDA; }
  c->tmax = max_steps;
  c->tstep = 0;
  return NQS_OK;
}

nqs_status nqs_timing_end(nqs_ctx *c, double *stage_ms, int *n_steps) {
  if (!c || !stage_ms || !n_steps) return NQS_ERR_ARG;
  for (int i = 0; i < NQS_N_STAGES; ++i) stage_ms[i] = 0.0;
  *n_steps = c->tstep;
  for (int t = 0; t < c->tstep; ++t) {
    cudaEvent_t *e = &c->tev[(size_t)t * (NQS_N_STAGES + 1)];
    if (cudaEventSynchronize(e[NQS_N_STAGES]) != cudaSuccess) { timing_free(c); return NQS_ERR_CUDA; }
    for (int i = 0; i < NQS_N_STAGES; ++i) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, e[i], e[i + 1]) != cudaSuccess) { timing_free(c); return NQS_ERR_CUDA; }
      stage_ms[i] += ms;
    }
  }
  timing_free(c);
  return NQS_OK;
}

nqs_status nqs_launch_count(const nqs_ctx *c, int64_t *n) {
  if (!c || !n) return NQS_ERR_ARG;
  *n = c->launches;
  return NQS_OK;
}

const char *nqs_last_cuda_error(void) {
  return g_last_cuda == cudaSuccess ? "no CUDA error" : cudaGetErrorString(g_last_cuda);
}

const char *nqs_status_string(int s) {
  switch (s) {
    case NQS_OK: return "ok";
    case NQS_ERR_ARG: return "invalid argument";
    case NQS_ERR_CUDA: return "CUDA runtime error";
    case NQS_ERR_UNSUPPORTED: return "hidden size not built into this library";
    case NQS_ERR_NONFINITE: return "non-finite energy or update";
    case NQS_ERR_NOT_SPD: return "T + lambda I not positive definite";
    case NQS_ERR_TIMEOUT: return "bounded device wait ran out";
    case NQS_ERR_WORKSPACE: return "workspace missing or too small";
  }
  return "unknown status";
}

}  // extern "C"

namespace nqs {
bool dh_supported(int dh) {
  return dh == 8 || dh == 16 || dh == 32 || dh == 64 || dh == 96 || dh == 128 || dh == 200 ||
         dh == 256;
}
}  // namespace nqs
