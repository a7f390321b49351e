/*
 * nqs.h -- C-ABI of the B300 (sm_103a) regularized-minSR step for
 * autoregressive GRU wave functions (arXiv 2608.18065).
 *
 * One call of nqs_minsr_step performs one iteration of the paper's
 * Algorithm 1 on one GPU: exact autoregressive sampling, local energies over
 * every connected configuration, the per-sample log-derivative matrix O,
 * centring, the real representation, T = O'^T O', the Tikhonov-regularized
 * FP64 solve, delta theta = eta O' (T + lambda I)^{-1} eps', momentum and the
 * parameter update.  The other entry points expose the stages one by one.
 *
 * Conventions shared by every call
 *  - Pointers named "device" must point to CUDA device memory of the current
 *    device; the caller owns all of them.  The library owns only its context
 *    (host memory) and the small device tables it builds in nqs_create.
 *  - Every call that takes a stream is asynchronous on that stream
 *    (cudaStream_t passed as void*; NULL = legacy default stream).
 *    Argument errors are detected on the host and returned at once; errors
 *    found on the device (non-finite values, a non-positive Cholesky pivot)
 *    are written to the status field of the device-side nqs_step_stats.
 *  - Spins: sigma in {0,1} is the one-hot index, s^z = 1 - 2 sigma.  A
 *    configuration is N = Lx*Ly bytes in the order of the zig-zag path
 *    pi(k) of Sec. II.B (for 1D chains the site order).
 *  - log Psi is stored as (re, im) doubles: re = 1/2 log P (Sec. II.A),
 *    im = sum_k phi_k (softsign head, Sec. II.A) + pi (sigma_A mod 2) with the
 *    Marshall sign of Sec. III.C on sublattice A = {(i,j): i+j odd}.
 *  - theta is the FP64 master copy, flat, row-major blocks in this order
 *    (App. A; hidden-state columns first, then one-hot input columns):
 *      2D only:  U1[dh x dh], U2[dh x dh]
 *      Wu[dh x (dh+din)], bu[dh], Wr[dh x (dh+din)], br[dh],
 *      Wh[dh x dh], bh[dh], Win[dh x din], bin[dh], U[2 x dh], c[2],
 *      complex head only: Uphi[2 x dh], cphi[2]
 *    with din = 2 (1D) or 4 (2D: one-hots of the horizontal then vertical
 *    neighbour).  The GRU is App. A literally: u, r = sigmoid(W[h';x] + b),
 *    c = tanh(r * (Wh h' + bh) + Win x + bin), h = (1-u) h' + u c, with
 *    h' = h_{k-1} (1D) or U1 h_hor + U2 h_ver (2D).
 *  - Random numbers: u(s,k) = Philox4x32-10 (Salmon et al., SC'11) with
 *    key = (lo32 seed, hi32 seed) and counter = (k, s, lo32 step, hi32 step);
 *    u = ((out1 << 32 | out0) >> 11) * 2^-53; sigma_k = 0 iff u < p_k(0).
 */
#ifndef NQS_H
#define NQS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  NQS_OK = 0,
  NQS_ERR_ARG = 1,          /* invalid argument (host-side check) */
  NQS_ERR_CUDA = 2,         /* a CUDA runtime call failed */
  NQS_ERR_UNSUPPORTED = 3,  /* model size not compiled into this library */
  NQS_ERR_NONFINITE = 4,    /* device: non-finite E, eps or delta theta */
  NQS_ERR_NOT_SPD = 5,      /* device: Cholesky pivot of T + lambda I <= 0 */
  NQS_ERR_TIMEOUT = 6,      /* device: a bounded wait ran out */
  NQS_ERR_WORKSPACE = 7     /* no workspace, or smaller than required */
} nqs_status;

typedef enum { NQS_PREC_FP64 = 0, NQS_PREC_MIXED = 1 } nqs_precision;

typedef enum {
  NQS_HAM_TFIM = 0,          /* -J sum Z_i Z_{i+1} - h sum X_i, open chain (Sec. III.A) */
  NQS_HAM_CLUSTER_ZXZ = 1,   /* -sum_{i=2}^{N-1} Z_{i-1} X_i Z_{i+1}, open chain */
  NQS_HAM_CLUSTER_PAPER = 2, /* Sec. III.B: XZX bulk + 3 boundary terms, E_0 = -N */
  NQS_HAM_J1J2 = 3           /* Sec. III.C: J1/4 sum_<ij> s.s + J2/4 sum_<<ij>> s.s, open */
} nqs_ham_family;

typedef struct {
  int dim;      /* 1 or 2 */
  int Lx, Ly;   /* N = Lx*Ly; Ly = 1 for dim 1 */
  int dh;       /* hidden size: 8, 16, 32, 64, 96 or 128 in this build */
  int cplx;     /* 1: softsign phase head (cRNN), 0: positive (pRNN) */
  int marshall; /* 1: Marshall sign (-1)^{sigma_A} (Sec. III.C) */
  int zmask;    /* 1: zero-magnetisation mask during sampling (N even) */
} nqs_model_desc;

typedef struct {
  int family;   /* nqs_ham_family */
  double J, h;  /* TFIM couplings */
  double J1, J2;/* J1-J2 couplings */
} nqs_ham_desc;

typedef struct {
  double eta0;         /* base learning rate */
  double decay_T;      /* eta_t = eta0 / (1 + t/decay_T); <= 0: no decay (Tab. I) */
  double mu;           /* momentum (App. B) */
  double lambda;       /* constant Tikhonov shift (lambda_mode 0) */
  double lambda_coeff; /* lambda_mode 1: lambda = coeff * ||T||_F^pow (Sec. III.C) */
  double lambda_pow;
  int32_t lambda_mode; /* 0 constant, 1 norm power */
  int32_t trust_region;/* 1: eta* = eta_t / ||tau||, tau = (I - lambda (T+lambda I)^-1) eps' (App. F) */
  int64_t step_index;  /* t: Philox step counter and lr decay */
  uint64_t seed;       /* Philox key */
  int64_t n_samples;   /* Ns, <= the ctx's max_samples */
} nqs_step_hparams;

typedef struct {
  double E_re, E_im;   /* E = mean eps (Eq. energy) */
  double var;          /* mean |eps - E|^2 */
  double vscore;       /* N var / E_re^2 (Eq. vscore, E_inf = 0) */
  double lambda;       /* shift used */
  double normT;        /* ||T||_F before the shift */
  double eta_eff;      /* eta_t or eta* */
  double tau_norm;     /* ||tau|| */
  int32_t status;      /* nqs_status of the device-side checks */
  int32_t solve_fp64;  /* 1: x came from the FP64 Cholesky factorisation (FP64
                          context, or fallback of the mixed context); 0: from
                          FP64 iterative refinement on an FP32 factor; 2: T
                          rebuilt in FP64 and factored in FP64 (mixed context,
                          lambda below the tensor-core T's rounding) */
  double rho;          /* Levenberg-Marquardt gain ratio (0 when damping is off) */
  double lambda_next;  /* damping of the next step (= lambda when off) */
} nqs_step_stats;

/* Optional device outputs of nqs_minsr_step_ex (any pointer may be NULL). */
typedef struct {
  uint8_t *spins;   /* [Ns*N] */
  double *logpsi;   /* [Ns*2] */
  double *eloc;     /* [Ns*2] (re, im) */
  double *T;        /* [R*R] FP64, before the shift; R = Ns (pRNN) or 2Ns */
  double *eps;      /* [R] eps-bar' */
  double *x;        /* [R] (T + lambda I)^{-1} eps-bar' */
  double *dtheta;   /* [Np] delta theta (eta_eff included) */
} nqs_step_outputs;

typedef struct nqs_ctx nqs_ctx;

/* Create a context for one model, Hamiltonian and precision on the current
 * device.  precision: NQS_PREC_FP64 runs every stage in FP64 (the plain GPU
 * path); NQS_PREC_MIXED runs the recurrences and O in FP32, T and O'x as
 * split BF16x3 tensor-core products with FP32 accumulation, and the
 * centring, reductions and the regularized solve in FP64.  In the mixed
 * context the per-site products of hidden size 64 (32 for 1D local
 * energies, with zero-padded units) are also split BF16x3 products with
 * FP32 accumulation:
 *  - the local-energy recomputations (1D and 2D) and the rows of O (1D) on
 *    tcgen05;
 *  - the gate products of the 1D sampler and of the reverse sweep (1D and
 *    2D) on warp-level MMAs.
 * Nonlinearities and state updates stay in FP32.  max_samples
 * bounds Ns of every later call.  *out receives the context; release it with
 * nqs_destroy.  Errors: NQS_ERR_ARG for an invalid description,
 * NQS_ERR_UNSUPPORTED for a hidden size not built. */
nqs_status nqs_create(const nqs_model_desc *model, const nqs_ham_desc *ham,
                      int precision, int64_t max_samples, nqs_ctx **out);

/* Options of nqs_create_ex. */
typedef struct {
  /* Hidden-state checkpoints for the per-sample Jacobian (1D chains only):
   * 0 caches every h_k (the default of nqs_create); c > 0 keeps h_k only for
   * k = c-1, 2c-1, ... and the reverse sweep recomputes each segment of c
   * sites from its checkpoint (and the local energies restart from the
   * last checkpoint before their first changed site); -1 takes
   * c = ceil(sqrt(N)).  Memory of the hidden-state, gate and adjoint caches
   * drops from O(Ns N dh) to O(Ns (N/c + c) dh) for about one extra forward
   * pass.  NQS_ERR_UNSUPPORTED for 2D lattices (the zig-zag vertical
   * neighbour reaches a full row back). */
  int checkpoint_stride;
} nqs_options;

/* nqs_create with options (opt may be NULL: all defaults). */
nqs_status nqs_create_ex(const nqs_model_desc *model, const nqs_ham_desc *ham,
                         int precision, int64_t max_samples,
                         const nqs_options *opt, nqs_ctx **out);

/* The checkpoint stride in use (0: every state cached). */
nqs_status nqs_checkpoint_stride(const nqs_ctx *ctx, int *stride);

/* Release the context (host memory and its device tables).  Synchronises
 * the device first. */
nqs_status nqs_destroy(nqs_ctx *ctx);

/* Number of parameters Np of the model (layout above). */
nqs_status nqs_param_count(const nqs_ctx *ctx, int64_t *n_params);

/* Bytes of device workspace the context needs for up to max_samples. */
nqs_status nqs_workspace_size(const nqs_ctx *ctx, size_t *bytes);

/* Attach caller-owned device workspace (>= nqs_workspace_size bytes,
 * 256-byte aligned).  The workspace must stay valid while calls that use it
 * are in flight; calls on one context must not overlap on the device. */
nqs_status nqs_set_workspace(nqs_ctx *ctx, void *dev_ptr, size_t bytes);

/* Exact autoregressive sampling (Sec. II.A, Algorithm 1, sampling step).
 * theta: device [Np] FP64.  Writes spins (device [ns*N] uint8) and logpsi
 * (device [ns*2] FP64) using u(seed, step, s, k).  Also fills the context's
 * hidden-state cache used by later stages of a step. */
nqs_status nqs_sample(nqs_ctx *ctx, const double *theta, int64_t ns,
                      uint64_t seed, uint64_t step, uint8_t *spins,
                      double *logpsi, void *stream);

/* log Psi of n given configurations (device spins [n*N]) -> device logpsi
 * [n*2].  n <= max_samples. */
nqs_status nqs_logpsi(nqs_ctx *ctx, const double *theta, const uint8_t *spins,
                      int64_t n, double *logpsi, void *stream);

/* Local energies eps(sigma) = sum_s' H_ss' Psi(s')/Psi(s) (Sec. II.C) of ns
 * given configurations: device spins [ns*N] -> device eloc [ns*2] (re, im).
 * Every connected s' is re-evaluated from the first site it differs at,
 * starting from the cached hidden state of sigma. */
nqs_status nqs_local_energy(nqs_ctx *ctx, const double *theta,
                            const uint8_t *spins, int64_t ns, double *eloc,
                            void *stream);

/* Per-sample log-derivatives O[r][k] = d log Psi(sigma_s)/d theta_k
 * (Sec. II.C), rows r = s for the real part and r = ns + s for the
 * imaginary part (complex head only), without the 1/sqrt(Ns) factor.
 * O: device [R*Np], FP64 for NQS_PREC_FP64, FP32 for NQS_PREC_MIXED. */
nqs_status nqs_jacobian(nqs_ctx *ctx, const double *theta, const uint8_t *spins,
                        int64_t ns, void *O, void *stream);

/* Vector-Jacobian product of log Psi (the backward of log Psi as a
 * differentiable function of theta): grad_theta[k] = sum_s ( g_s^re
 * d Re log Psi(sigma_s)/d theta_k + g_s^im d Im log Psi(sigma_s)/d theta_k ),
 * with the log-derivatives of nqs_jacobian.  grad_logpsi: device [ns*2]
 * FP64 (re, im) cotangents; grad_theta: device [Np] FP64 (overwritten). */
nqs_status nqs_logpsi_vjp(nqs_ctx *ctx, const double *theta, const uint8_t *spins,
                          int64_t ns, const double *grad_logpsi, double *grad_theta,
                          void *stream);

/* T = A A^T (Algorithm 1, Gram step) for a row-major A [R x np] of centred,
 * scaled log-derivatives (rows = samples): FP64 A -> FP64 T on CUDA cores
 * for the FP64 context; FP32 A -> FP64 T via BF16x3 tcgen05 products with
 * FP32 accumulation for the mixed context.  T: device [R*R], both
 * triangles written. */
nqs_status nqs_gram(nqs_ctx *ctx, const void *A, int64_t R, int64_t np,
                    double *T, void *stream);

/* Solve (T + lambda I) x = b (Eq. minsrR) to FP64 accuracy.  FP64 context:
 * FP64 Cholesky and substitutions.  Mixed context: FP32 Cholesky factor and
 * FP64 iterative refinement until ||r||_inf <= sqrt(R) u64 ||A||_inf
 * ||x||_inf, falling back to the FP64 Cholesky if the FP32 factorisation
 * breaks down or the refinement does not converge in 12 sweeps.  T device
 * [R*R] FP64 (both triangles) may be overwritten; b, x device [R].
 * *dev_status (device int32) receives 0, NQS_ERR_NOT_SPD or
 * NQS_ERR_TIMEOUT.  R <= the context's largest R. */
nqs_status nqs_regularized_solve(nqs_ctx *ctx, double *T, int64_t R,
                                 double lambda, const double *b, double *x,
                                 int32_t *dev_status, void *stream);

/* One minSR step (Algorithm 1, all steps).  theta, momentum: device [Np]
 * FP64, updated in place unless the device-side checks fail, in which case
 * both are left unchanged.  dev_stats: device nqs_step_stats. */
nqs_status nqs_minsr_step(nqs_ctx *ctx, double *theta, double *momentum,
                          const nqs_step_hparams *hp, nqs_step_stats *dev_stats,
                          void *stream);

/* As nqs_minsr_step, also copying the step's intermediates to the non-NULL
 * device pointers of out. */
nqs_status nqs_minsr_step_ex(nqs_ctx *ctx, double *theta, double *momentum,
                             const nqs_step_hparams *hp,
                             nqs_step_stats *dev_stats,
                             const nqs_step_outputs *out, void *stream);

/* ------------------------------------------------ adaptive damping (LM) */

/* Levenberg-Marquardt damping (App. G).  omega > 1 switches it on with
 * lambda0 as the damping of the next step; omega <= 1 switches it off (the
 * steps use nqs_step_hparams' lambda again).  While on, every step:
 *  - uses the damping held on the device (hp->lambda and lambda_mode are
 *    ignored) and reports it in stats.lambda;
 *  - after the update, estimates E at theta - delta theta (the SR step
 *    itself, without momentum) from n_samples fresh samples drawn with the
 *    Philox key seed + 0x9E3779B97F4A7C15 and the step's counter;
 *  - forms rho = (E - E(theta - delta theta)) / (eta eps'^T tau -
 *    1/2 eta^2 ||tau||^2), the decrease predicted by the quadratic model
 *    with metric S (App. G; eta* eps'^T tau - 1/2 eta_t^2 in the trust-region
 *    mode), and multiplies the damping by omega if rho < 1/4 (or the step
 *    was rejected), divides it by omega if rho > 3/4 (stats.rho,
 *    stats.lambda_next).
 * The extra sampling and local-energy pass roughly doubles the forward
 * work of a step.  Synchronous: waits for all work on the device (so a
 * step in flight on any stream finishes before the damping it reads or
 * writes is replaced), then copies lambda0 to the device; call it outside
 * stream capture.  Invalidates the context's captured graph. */
nqs_status nqs_set_damping(nqs_ctx *ctx, double omega, double lambda0);

/* ------------------------------------------------------------ autotuner */

/* Launch shapes the autotuner chose for one context (0 = built-in choice). */
typedef struct {
  int64_t n_samples;  /* sample count they were measured for (0: not tuned) */
  int eloc_grid;      /* CTAs of the connected-configuration engine */
  int gram_splits;    /* K-slices per 128x128 tile of the tensor-core Gram */
  int solve_grid;     /* CTAs of the cooperative Cholesky / refinement */
  int solve_form;           /* mixed solve: 0 32-wide panels, tiles per CTA; 1 the
                               same, tiles per warp; 2 128-wide panels; -1 built-in */
  int solve_substitution;   /* refinement sweeps: 1 block substitution, 0 explicit inverse, -1 built-in */
  int reserved;
  double ms[3];         /* time of the chosen shape: eloc, gram, solve */
  double ms_default[3]; /* time of the built-in shape */
} nqs_tuning;

/* Re-measure even if the process-wide cache holds this problem shape. */
#define NQS_TUNE_FORCE 1

/* Choose the launch shapes of the step's three largest stages for
 * hp->n_samples samples by timing candidates on the device: the grid of the
 * connected-configuration engine (local energies, Sec. II.C), the K-split
 * of the Gram T (Eq. minsrT) and the grid of the regularized solve.  Runs
 * one eager step on copies of theta kept in the workspace (theta itself is
 * not modified), then times every candidate (best of two) with CUDA events;
 * synchronises `stream`; must not be called during stream capture.  The
 * choice is kept in the context (used by every later step with the same
 * sample count, and it invalidates the context's captured graph) and in a
 * process-wide cache keyed by device, model, Hamiltonian family, precision
 * and sample count; a later call on a matching context takes the cached
 * shapes without measuring unless flags has NQS_TUNE_FORCE.  A shape changes
 * only how the work is spread over CTAs; where that regroups a sum (the
 * K-slices of T, the row partials of the substitutions) results differ from
 * the built-in shapes by rounding only, and two contexts with the same
 * shapes give bit-identical results. */
nqs_status nqs_autotune(nqs_ctx *ctx, const double *theta,
                        const nqs_step_hparams *hp, int flags, void *stream);
nqs_status nqs_get_tuning(const nqs_ctx *ctx, nqs_tuning *out);
/* Back to the built-in shapes. */
nqs_status nqs_clear_tuning(nqs_ctx *ctx);
/* Fix the form of the mixed context's regularized solve (Eq. minsrR; the
 * values of nqs_tuning.solve_form; -1: the built-in choice, 128-wide panels
 * from R = 3072 on where R % 4 == 0, otherwise 32-wide) for every later
 * solve, over any tuning.  The 128-wide form needs R % 4 == 0 and R >= 256
 * and takes the 32-wide one otherwise.  Every form ends at FP64 backward
 * error or in the FP64 Cholesky.  NQS_ERR_ARG for another value. */
nqs_status nqs_set_solve_form(nqs_ctx *ctx, int form);
/* Sampler of a mixed 2D context of hidden size 96 or 128 with every state
 * cached (Sec. II.A): 1 (or -1, the built-in choice) the streamed
 * tensor-core engine, 0 the recurrence kernels.  Both draw with the same
 * Philox uniforms and decide in FP32; their conditionals differ by the
 * rounding of their products.  Other contexts always take the recurrence
 * kernels.  NQS_ERR_ARG for another value. */
nqs_status nqs_set_sampler(nqs_ctx *ctx, int form);

/* ------------------------------------------------------ batched instances */

/* A batch steps n independent contexts (different lattices, hidden sizes,
 * couplings and sample counts) together.  The paper runs one instance per
 * GPU; a batch fills one B300 with many.  The batch owns one stream per
 * instance, the events that fork them from and join them to the caller's
 * stream, and optionally one CUDA graph of the whole batched step.  The
 * contexts stay owned by the caller, must outlive the batch, must each have
 * their own workspace and must not be stepped elsewhere while a batched step
 * is in flight. */
typedef struct nqs_batch nqs_batch;

/* ctxs: host array of n distinct contexts (1 <= n <= 4096). */
nqs_status nqs_batch_create(int n, nqs_ctx *const *ctxs, nqs_batch **out);
/* Synchronises the device, then frees the batch (not the contexts). */
nqs_status nqs_batch_destroy(nqs_batch *b);

/* One minSR step of every instance (Algorithm 1, all steps each, exactly as
 * nqs_minsr_step of that context would compute it: the results are
 * bit-identical).  thetas, moms: host arrays of n device pointers [Np_i]
 * FP64, updated in place; hps: host array of n hyper-parameter sets;
 * dev_stats: device array of n nqs_step_stats.  The instances run
 * concurrently on the batch's streams, ordered after the work already on
 * `stream`, and `stream` waits for all of them; the cooperative solves of
 * the instances run one after another in instance order, since each of them
 * spreads over every SM.  Device-side failures of one instance leave only
 * that instance's theta and momentum unchanged. */
nqs_status nqs_minsr_step_batched(nqs_batch *b, double *const *thetas,
                                  double *const *moms,
                                  const nqs_step_hparams *hps,
                                  nqs_step_stats *dev_stats, void *stream);

/* Replay the batched step as one CUDA graph (captured on the first call and
 * again when a pointer, a hyper-parameter other than step_index or the
 * concurrency changes).  As for nqs_set_graph, failed capture falls back
 * to eager launches. */
nqs_status nqs_batch_set_graph(nqs_batch *b, int enable);
nqs_status nqs_batch_graph_active(const nqs_batch *b, int *active);

/* Number of instance streams (0 or >= n: one per instance; 1: the
 * instances run back to back). */
nqs_status nqs_batch_set_concurrency(nqs_batch *b, int streams);
nqs_status nqs_batch_get_concurrency(const nqs_batch *b, int *streams);

/* Batched step by stage.  stages = 0 (default): whole steps per instance
 * stream.  Bit 1: every instance's step up to its solve on the instance
 * streams; then one cooperative launch of the FP32 factors and refinements
 * (128-wide panels, Eq. minsrR) of all mixed instances with R % 4 == 0 and
 * R >= 256 (unless nqs_set_solve_form picked another form), each instance on
 * its own range of CTAs sized by a model of its panel chain; then the rest
 * of every step.  x stays FP64-accurate (the same refinement test and FP64
 * fallback) and is bit-identical to the instance's own step with solve form
 * 2.  Bit 2: the local-energy engines of the mixed 2D instances of hidden
 * size 96 or 128 (Sec. II.C) run as one launch per hidden size, each instance
 * on its own range of CTAs (shares from the autotuner's engine times) with
 * its own tile counter; the local energies are bit-identical to the
 * instance's own step. */
nqs_status nqs_batch_set_grouped(nqs_batch *b, int stages);
nqs_status nqs_batch_get_grouped(const nqs_batch *b, int *stages);

/* Share of its grid (eighths, 1..8; default 8) that each instance's
 * local-energy engine takes inside a batched step (whole steps per stream;
 * the grouped engine launch splits all SMs itself): an engine CTA fills its
 * SM's shared and tensor memory, so the SMs it leaves free serve the other
 * instances' kernels.  Steps of a context outside the batch use the whole
 * grid.  Results do not depend on the grid.  (Measured on the headline
 * batch: 7/8 and 3/4 were no faster than the whole grid, so the batch
 * autotuner leaves it at 8.) */
nqs_status nqs_batch_set_eloc_share(nqs_batch *b, int eighths);
nqs_status nqs_batch_get_eloc_share(const nqs_batch *b, int *eighths);

/* nqs_autotune for every instance, then, by timing whole batched steps on
 * the workspace copies of theta (best of two for the concurrency and the
 * solve SMs; candidates in turn and the median of five or three rounds for
 * the grouped stages and the graph): the concurrency, the fraction of the
 * SMs each instance's cooperative solve takes, which stages run grouped
 * (nqs_batch_set_grouped: none, the solves, the solves and the
 * local-energy engines; the fewest within 2 % of the fastest), and, if
 * graphs are enabled (nqs_batch_set_graph),
 * whether a graph replay or the eager launches are faster (graphs stay off
 * when they are not).  The fastest batched step time goes to *step_ms (may
 * be NULL).  Synchronous; the callers' thetas are not modified. */
nqs_status nqs_batch_autotune(nqs_batch *b, double *const *thetas,
                              const nqs_step_hparams *hps, int flags,
                              double *step_ms, void *stream);

/* ------------------------------------- Adam comparator, loss landscape */

typedef struct {
  double eta0, decay_T;  /* eta_t = eta0 / (1 + t / decay_T); decay_T <= 0 or inf: constant */
  double beta1, beta2;   /* moment decays (Kingma and Ba: 0.9, 0.999) */
  double epsilon;        /* denominator guard (1e-8) */
  int64_t step_index;    /* t = 0, 1, ...: Philox step counter, bias corrections use t + 1 */
  uint64_t seed;         /* Philox key */
  int64_t n_samples;     /* Ns <= the ctx's max_samples */
} nqs_adam_hparams;

/* One Adam iteration, the first-order baseline the paper compares minSR
 * with (Sec. II.C, Tab. I's Adam column): samples, local energies, E, O,
 * centring as in nqs_minsr_step, the sampled energy gradient
 * g = Obar'^T eps-bar' (= 2 Re mean (O - <O>)^* (E_loc - E), Eq.
 * real-valued), then m1 <- b1 m1 + (1 - b1) g, m2 <- b2 m2 + (1 - b2) g^2,
 * theta <- theta - eta_t (m1 / (1 - b1^(t+1))) / (sqrt(m2 / (1 - b2^(t+1)))
 * + epsilon).  theta, m1, m2: device FP64 [Np], updated in place unless a
 * device-side check fails (dev_stats.status; E, Var in dev_stats, eta_t in
 * eta_eff).  grad: optional device FP64 [Np] copy of g. */
nqs_status nqs_adam_step(nqs_ctx *ctx, double *theta, double *m1, double *m2,
                         const nqs_adam_hparams *hp, nqs_step_stats *dev_stats, double *grad,
                         void *stream);

/* Energies of the loss landscape (Sec. IV): for every point i of xy (host
 * FP64 [npts][2] = (x, y)), E(theta0 + x v1 + y v2) from ns samples drawn at
 * Philox step 0 with key seed (every point shares the random numbers).
 * theta0, v1, v2: device FP64 [Np].  out: device FP64 [npts][4] = (Re E,
 * Im E, Var, status).  Launches 8-9 kernels per point. */
nqs_status nqs_energy_scan(nqs_ctx *ctx, const double *theta0, const double *v1,
                           const double *v2, const double *xy, int64_t npts, int64_t ns,
                           uint64_t seed, double *out, void *stream);

/* Test of the failure detection of the bounded waits (no counterpart in
 * the paper).  For 2D lattices of hidden size 96 / 128 in the mixed
 * context, whose local energies run on the streamed tensor-core engine:
 * spin_limit > 0 sets the polls of every bounded wait of that engine (0:
 * the default, about half a second); drop_tile != 0 makes its tile
 * producer never publish the first tile, so that every other role's wait
 * for it runs out: the engine then ends its loops, drains its MMAs, frees
 * its tensor memory and returns, and the step reports NQS_ERR_TIMEOUT in
 * dev_stats.status and leaves theta and momentum unchanged.  Drops the
 * context's captured graph; (0, 0) restores normal operation. */
nqs_status nqs_test_wait_timeout(nqs_ctx *ctx, uint64_t spin_limit, int drop_tile);

/* ------------------------------------------------ sample-sharded step */

/* One minSR step (Algorithm 1) with the Ns samples split over G ranks, one
 * context per rank (each created with max_samples >= Ns: T and the gathered
 * rows are Ns-sized).  The paper runs one instance per GPU; the split below
 * follows from the samples being independent (exact autoregressive
 * sampling, Sec. II.A): rank r draws samples s0 .. s0 + n - 1 of the draw
 * with their own Philox counters, so the ranks together draw exactly the
 * single-rank step's samples.  Per step, on every rank, in order:
 *   nqs_shard_forward   sampling, local energies and O of the rank's
 *                       samples; partial sums
 *   (caller)            sum of the partial sums over the ranks (allreduce)
 *   nqs_shard_center    the rank's centred rows O' and eps-bar'; E, Var
 *   (caller)            gather of every rank's rows and eps-bar' in rank order
 *   nqs_shard_solve     T of the gathered rows, lambda, x, eta; the entries
 *                       [p0, p1) of delta theta
 *   (caller)            gather of the delta theta ranges (allgather)
 *   nqs_shard_apply     momentum and update of theta
 * Rows gathered in rank order are a permutation of the single-rank rows;
 * T, x and eps-bar' permute alike and delta theta = eta O'^T x does not
 * change (up to rounding).  The Levenberg-Marquardt damping is not applied
 * on this path.  All calls are asynchronous on `stream`; host-side argument
 * errors return at once, device-side ones go to dev_stats.status. */

/* Sampling (Sec. II.A), local energies (Sec. II.C) and O (Sec. II.D) of
 * samples s0 .. s0 + n - 1 (s0 + n <= 2^32, n <= max_samples), kept in the
 * context.  sums: device FP64 [nblk*Np + 3], nblk = 2 for the complex head
 * else 1: the column sums of O per block (real rows, imaginary rows), then
 * sum Re E_loc, sum Im E_loc, sum |E_loc|^2 over the n samples. */
nqs_status nqs_shard_forward(nqs_ctx *ctx, const double *theta, const nqs_step_hparams *hp,
                             int64_t s0, int64_t n, double *sums, void *stream);

/* From the sums of all ranks (device, layout of nqs_shard_forward) and the
 * total Ns: E, Var = sum|E_loc|^2/Ns - |E|^2 and the V-score into dev_stats
 * (status reset); rows: device [nblk*n][Np], working precision (FP64
 * context: double, mixed: float), the rank's rows of O' = (O - mean) /
 * sqrt(Ns) (Eq. real-valued; real block then imaginary block); eps: device
 * FP64 [nblk*n], the rank's rows of eps-bar'.  n: the last forward's n. */
nqs_status nqs_shard_center(nqs_ctx *ctx, const double *sums, int64_t ns, int64_t n,
                            void *rows, double *eps, nqs_step_stats *dev_stats, void *stream);

/* On the gathered rows (device [R][Np], working precision, R = nblk*Ns) and
 * eps-bar' (device FP64 [R]): T = O'O'^T (Algorithm 1, Gram step), lambda
 * (Tab. I modes), the solve and eta (Eq. minsrR, App. F; as
 * nqs_minsr_step), and delta theta entries p0 .. p1 - 1 into dtheta (device
 * FP64 [p1 - p0]; eta_eff included).  0 <= p0 <= p1 <= Np. */
nqs_status nqs_shard_solve(nqs_ctx *ctx, const void *rows, int64_t R, const double *eps,
                           const nqs_step_hparams *hp, int64_t p0, int64_t p1, double *dtheta,
                           nqs_step_stats *dev_stats, void *stream);

/* Momentum and update (App. B) with the gathered delta theta (device FP64
 * [Np]); a non-finite entry sets NQS_ERR_NONFINITE and, as any device-side
 * error, leaves theta and momentum unchanged. */
nqs_status nqs_shard_apply(nqs_ctx *ctx, double *theta, double *momentum, const double *dtheta,
                           const nqs_step_hparams *hp, nqs_step_stats *dev_stats, void *stream);

/* ------------------------------------------------- allocation-free log Psi */

/* Size of the static device scratch array behind nqs_logpsi_noalloc. */
#define NQS_NOALLOC_SCRATCH_BYTES (16u << 20)

/* log Psi of n given configurations in FP64 without allocating any device
 * memory and without a context -- the paper has no counterpart to this
 * call; it exists for callers that cannot call cudaMalloc where they
 * evaluate the wave function (a host framework whose pool owns the device,
 * a plug-in limited to the memory it is handed, a loop where allocation and
 * its implicit synchronisation are not allowed).
 * model: as for nqs_create; theta: device [Np] FP64; spins: device [n*N]
 * uint8; logpsi: device [n*2] FP64 (re, im), same values as nqs_logpsi of an
 * NQS_PREC_FP64 context.  Scratch (the packed theta and, for 2D lattices,
 * the hidden-state cache of 8*(n*N*dh) bytes that the vertical neighbours
 * read back; a 1D chain needs the packed weights only) comes from one
 * file-scope device array of NQS_NOALLOC_SCRATCH_BYTES that every GPU
 * loading the library reserves until the process exits; a 2D batch whose
 * cache does not fit, or n > 2^31 - 1, returns NQS_ERR_WORKSPACE without
 * launching anything (split the batch).  The first
 * call on each device looks up the array's address (cudaGetSymbolAddress)
 * with that device current; make that first call before any stream capture.
 * All calls share the one array and leave their data in it: calls that
 * overlap on the GPU (different streams, or graphs replayed concurrently)
 * race on it and must be serialised by the caller. */
nqs_status nqs_logpsi_noalloc(const nqs_model_desc *model, const double *theta,
                              const uint8_t *spins, int64_t n, double *logpsi,
                              void *stream);

/* ------------------------------------------------ spectrum diagnostics */

/* Conditioning of the damped minSR system (App. E): T + lambda I has
 * kappa_2 = (lambda_max(T) + lambda) / (lambda_min(T) + lambda), and
 * d = -log10(kappa_2 eps) decimal digits survive a solve in a precision of
 * machine epsilon eps (2^-23 FP32, 2^-52 FP64).  T, centred over the
 * samples, has the all-ones vector of each real block in its null space, so
 * lambda_min(T) = 0 and kappa_2 = 1 + lambda_max / lambda. */
typedef struct {
  double lambda_max;       /* largest eigenvalue of T (Lanczos Ritz value) */
  double lambda_min_ritz;  /* smallest Ritz value: an upper bound on lambda_min(T) */
  double kappa;            /* (lambda_max + lambda) / lambda: lambda_min(T) = 0 */
  double digits_fp32;      /* -log10(kappa * 2^-23) */
  double digits_fp64;      /* -log10(kappa * 2^-52) */
  double residual;         /* |T y - lambda_max y| for the top Ritz pair */
  int32_t iterations;      /* Lanczos steps taken (fewer than m when the
                              Krylov space became invariant) */
  int32_t status;          /* nqs_status of the device-side checks */
} nqs_spectrum_stats;

/* Bytes of device scratch that nqs_spectrum needs for an R x R matrix and at
 * most m Lanczos steps. */
size_t nqs_spectrum_workspace(int64_t R, int m);

/* Extreme eigenvalues of the symmetric R x R FP64 matrix T (device,
 * row-major, both triangles, e.g. the Gram matrix of nqs_gram or of a step's
 * outputs; not modified) by m steps of Lanczos with full
 * reorthogonalisation in FP64 (classical Gram-Schmidt applied twice), from
 * a start vector of Philox uniforms of `seed`, then bisection on the
 * tridiagonal matrix; one cooperative launch, deterministic.  lambda >= 0
 * is the Tikhonov damping of the step.  work: device scratch of at least
 * nqs_spectrum_workspace(R, m) bytes, 256-byte aligned, owned by the caller;
 * out: device nqs_spectrum_stats written by the kernel.  Errors:
 * NQS_ERR_ARG for R < 1, m < 1, m > 512, lambda < 0 or a NULL pointer,
 * NQS_ERR_WORKSPACE if work_bytes is too small; out->status is
 * NQS_ERR_NONFINITE if T holds non-finite values and NQS_ERR_TIMEOUT if a
 * grid barrier timed out. */
nqs_status nqs_spectrum(const double *T, int64_t R, double lambda, int m, uint64_t seed,
                        void *work, size_t work_bytes, nqs_spectrum_stats *out,
                        void *stream);

/* ------------------------------------------------------- instrumentation */

/* Stages timed by the step instrumentation, in step order. */
#define NQS_N_STAGES 14
/* Name of stage i (static storage), NULL if out of range:
 * pack, sample, eloc_gen, eloc_suffix, eloc_reduce, energy, jac_bwd,
 * jac_grad, center, gram, lambda, cholesky (factorisation and both
 * substitutions), solve (empty since they were fused), update. */
const char *nqs_stage_name(int i);

/* Start per-stage CUDA-event timing of the next max_steps calls of
 * nqs_minsr_step[_ex] on this context (events are recorded on the step's
 * stream, no host synchronisation is added).  Replaces an earlier timing
 * window. */
nqs_status nqs_timing_begin(nqs_ctx *ctx, int max_steps);

/* End the timing window: synchronises the recorded events and writes the
 * summed milliseconds of each stage to stage_ms[0..NQS_N_STAGES-1] and the
 * number of timed steps to *n_steps. */
nqs_status nqs_timing_end(nqs_ctx *ctx, double *stage_ms, int *n_steps);

/* Work of the connected-configuration engine in the last local-energy pass
 * (nqs_local_energy or a step) of this context: *configs = number of
 * connected configurations sigma' with H_{sigma sigma'} != 0 off the
 * diagonal, *sites = sites recomputed for them (sum of N - j over sigma',
 * j its first changed site).  Synchronous: waits for the device copy of the
 * per-operator counts, so call it after that pass has completed. */
nqs_status nqs_eloc_work(const nqs_ctx *ctx, int64_t *configs, int64_t *sites);

/* Number of kernels this context has launched since it was created. */
nqs_status nqs_launch_count(const nqs_ctx *ctx, int64_t *n);

/* --------------------------------------------------------- CUDA graphs */

/* Enable (1) or disable (0) replay of nqs_minsr_step as a CUDA graph.  When
 * enabled, the first call captures the whole step (on a stream private to
 * the context) and later calls replay it on the caller's stream; the step
 * counter lives on the device and advances with every step, so consecutive
 * step_index values cost one graph launch, any other value one extra tiny
 * kernel.  A different theta/momentum/stats pointer or any other
 * hyper-parameter re-captures the graph; nqs_minsr_step_ex with outputs and
 * steps inside a timing window always launch eagerly.  If capture fails the
 * context silently keeps launching eagerly (nqs_graph_active reports it). */
nqs_status nqs_set_graph(nqs_ctx *ctx, int enable);
nqs_status nqs_graph_active(const nqs_ctx *ctx, int *active);

/* Short text for a status code (static storage). */
const char *nqs_status_string(int status);

/* Text of the CUDA error behind the last NQS_ERR_CUDA that a call made on
 * the calling host thread returned (static storage; "no CUDA error" if
 * none).  Not cleared by later successful calls. */
const char *nqs_last_cuda_error(void);

#ifdef __cplusplus
}
#endif
#endif /* NQS_H */
