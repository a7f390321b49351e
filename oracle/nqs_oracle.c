/*
 * nqs_oracle.c -- plain, slow, FP64 CPU restatement of one regularized minSR
 * step for autoregressive GRU wave functions (arXiv 2608.18065).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call
 * this file; only the tests, the package's smoke check and the benchmark's
 * CPU-baseline leg do.  It shares no code, header, table or helper with the
 * CUDA library: every formula here is written out again from the paper.
 *
 * What each function follows (sections and equations of the paper):
 *   philox / uniform ........ Philox4x32-10 (Salmon et al., SC'11), the
 *                             counter-based generator both sides implement.
 *   forward / logpsi ........ Sec. II.A (Psi = sqrt(P) e^{i phi}, softmax and
 *                             softsign heads), Sec. II.B (zig-zag path pi(k),
 *                             2D neighbours), App. A (1D and 2D GRU cells),
 *                             Sec. III.C (Marshall sign (-1)^{sigma_A}).
 *   sample .................. Sec. II.A chain rule: exact site-by-site sampling
 *                             by inverse CDF on a shared uniform.
 *   local_energy ............ Sec. II.C, eps(s) = sum_s' H_ss' Psi(s')/Psi(s),
 *                             evaluated term by term with a full re-evaluation
 *                             of log Psi(s') for every connected s'.
 *   jacobian ................ O_ks = d log Psi(s) / d theta_k (Sec. II.C), by a
 *                             hand-derived reverse pass through App. A.
 *   minsr_step .............. Algorithm 1: centring, real representation
 *                             (Eq. real-valued), T = O'^T O', Tikhonov solve,
 *                             Eq. minsrR, momentum (App. B), lr decay (Tab. I),
 *                             lambda = c ||T||^p (Sec. III.C), trust-region
 *                             eta* = eta/||tau|| (App. F, Eq. trust-region-lr).
 *
 * Conventions (readings where the paper is silent):
 *   spin sigma in {0,1} is the one-hot index, s^z = 1 - 2 sigma (0 = up);
 *   spins of a configuration are stored in path order (sigma_k at pi(k));
 *   h_0 = 0 and the first input is the zero vector (Sec. II.A);
 *   2D boundary spins and hidden states are zero vectors (Sec. II.B);
 *   Marshall sublattice A = {(i,j): i+j odd}, sigma_A = #{sigma=1 on A};
 *   zero-magnetisation mask: once N/2 ups (or downs) are placed, the other
 *   value has conditional probability 1 (log 1 = 0, no gradient); the phase
 *   head is not masked;
 *   Im log Psi = sum_k phi_k + pi (sigma_A mod 2).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846

/* ------------------------------------------------------------------ types */

typedef struct {
  int dim;      /* 1 or 2 */
  int Lx, Ly;   /* N = Lx*Ly, Ly = 1 in 1D */
  int dh;       /* hidden size */
  int cplx;     /* 1: softsign phase head (cRNN) */
  int marshall; /* 1: Marshall sign */
  int zmask;    /* 1: zero-magnetisation masking */
} or_model;

/* A Hamiltonian is a real linear combination of Pauli strings.
 * Term t acts with op[t][q] in {'X','Y','Z'} on path-ordered site site[t][q]
 * for q < nops[t] (at most 4 factors). */
typedef struct {
  int n_terms;
  const double *coeff;
  const int *nops;   /* [n_terms] */
  const int *site;   /* [n_terms*4] */
  const char *op;    /* [n_terms*4] */
} or_ham;

typedef struct {
  double eta0, decay_T, mu;
  double lambda;              /* constant Tikhonov shift (lambda_mode 0) */
  double lambda_coeff, lambda_pow; /* lambda = coeff*||T||_F^pow (mode 1) */
  int lambda_mode;
  int trust_region;           /* 1: eta* = eta_t / ||tau|| */
  int64_t step_index;         /* t, for eta_t = eta0/(1+t/decay_T) */
  uint64_t seed;              /* Philox key */
  int64_t ns;                 /* number of samples */
  double lm_omega;            /* > 1: Levenberg-Marquardt damping (App. G) */
} or_hparams;

typedef struct {
  double E_re, E_im, var, vscore, lambda, normT, eta_eff, tau_norm;
  int status; /* 0 ok, 4 non-finite, 5 not SPD */
  double rho;          /* Levenberg-Marquardt gain ratio (0 when off) */
  double lambda_next;  /* damping for the next step (lambda when off) */
} or_stats;

/* Philox key of the samples that estimate E(theta + delta theta) for the
 * damping ratio: the step's key plus this odd constant (2^64 / golden
 * ratio), same counter layout, so they are independent of the step's own
 * samples. */
#define OR_LM_KEY_OFFSET 0x9E3779B97F4A7C15ULL

/* ------------------------------------------------------- Philox4x32-10 */

/* One Philox4x32-10 block: Salmon, Moraes, Dror, Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11.  Ten rounds of the S-box
 * (hi,lo) = M*x on lanes 0 and 2, with a Weyl key schedule. */
void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                      uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += W0; k1 += W1; }
    uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform u in [0,1) for (seed, step, sample s, site k):
 * key = (lo32 seed, hi32 seed), counter = (k, s, lo32 step, hi32 step);
 * u = ((out1 << 32 | out0) >> 11) * 2^-53. */
double or_uniform(uint64_t seed, uint64_t step, uint64_t s, uint64_t k) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t ctr[4] = {(uint32_t)k, (uint32_t)s, (uint32_t)step,
                     (uint32_t)(step >> 32)};
  uint32_t o[4];
  or_philox4x32_10(ctr, key, o);
  uint64_t bits = ((uint64_t)o[1] << 32) | (uint64_t)o[0];
  return (double)(bits >> 11) * (1.0 / 9007199254740992.0);
}

/* --------------------------------------------------- parameter layout */

typedef struct {
  int N, dh, din;
  int64_t U1, U2;          /* 2D only */
  int64_t Wu, bu, Wr, br, Wh, bh, Win, bin, Uo, co, Up, cp;
  int64_t np;
} or_layout;

/* Flat theta, row-major blocks, h-columns before one-hot columns:
 * [U1 U2 (2D)] Wu bu Wr br Wh bh Win bin U c [Uphi cphi (cRNN)]. */
static or_layout or_make_layout(const or_model *m) {
  or_layout L;
  int dh = m->dh;
  L.N = m->Lx * m->Ly;
  L.dh = dh;
  L.din = (m->dim == 2) ? 4 : 2;
  int64_t o = 0;
  L.U1 = L.U2 = -1;
  if (m->dim == 2) {
    L.U1 = o; o += (int64_t)dh * dh;
    L.U2 = o; o += (int64_t)dh * dh;
  }
  L.Wu = o; o += (int64_t)dh * (dh + L.din);
  L.bu = o; o += dh;
  L.Wr = o; o += (int64_t)dh * (dh + L.din);
  L.br = o; o += dh;
  L.Wh = o; o += (int64_t)dh * dh;
  L.bh = o; o += dh;
  L.Win = o; o += (int64_t)dh * L.din;
  L.bin = o; o += dh;
  L.Uo = o; o += 2 * dh;
  L.co = o; o += 2;
  L.Up = L.cp = -1;
  if (m->cplx) {
    L.Up = o; o += 2 * dh;
    L.cp = o; o += 2;
  }
  L.np = o;
  return L;
}

int64_t or_param_count(const or_model *m) { return or_make_layout(m).np; }

/* ------------------------------------------------------ zig-zag path */

/* pi(k) = (i_k, j_k): j = floor(k/Lx); i = k mod Lx on even rows and
 * Lx-1-(k mod Lx) on odd rows (Sec. II.B). */
static void or_path(const or_model *m, int k, int *i, int *j) {
  int Lx = m->Lx;
  *j = k / Lx;
  *i = ((*j) % 2 == 0) ? (k % Lx) : (Lx - 1 - (k % Lx));
}

/* inverse of pi: (i,j) -> k, or -1 outside the lattice */
static int or_path_index(const or_model *m, int i, int j) {
  if (i < 0 || i >= m->Lx || j < 0 || j >= m->Ly) return -1;
  return (j % 2 == 0) ? (j * m->Lx + i) : (j * m->Lx + (m->Lx - 1 - i));
}

/* The two inputs of site k in 2D: horizontal (i - (-1)^j, j) and vertical
 * (i, j-1) (App. A); -1 marks a zero boundary.  In 1D only "hor" = k-1. */
static void or_neighbours(const or_model *m, int k, int *hor, int *ver) {
  if (m->dim == 1) {
    *hor = k - 1;
    *ver = -1;
    return;
  }
  int i, j;
  or_path(m, k, &i, &j);
  int sgn = (j % 2 == 0) ? 1 : -1; /* (-1)^j */
  *hor = or_path_index(m, i - sgn, j);
  *ver = or_path_index(m, i, j - 1);
}

static int or_on_sublattice_A(const or_model *m, int k) {
  int i, j;
  or_path(m, k, &i, &j);
  return ((i + j) % 2) == 1;
}

/* ------------------------------------------------------ GRU forward */

static double or_sigmoid(double x) { return 1.0 / (1.0 + exp(-x)); }

/* Per-site record of the forward pass, kept for the reverse pass. */
typedef struct {
  double *hp;  /* h' (2D) or h_{k-1} (1D): [dh] */
  double *x;   /* one-hot inputs [din] */
  double *u, *r, *g, *c, *h; /* gates, W_h h'+b_h, candidate, new state */
  double lp[2];  /* log conditional probabilities (after masking) */
  double p[2];   /* unmasked softmax probabilities */
  int forced;    /* 1 if the mask fixed this site */
  double y[2];   /* phase head pre-activations */
} or_site;

/* Workspace for one configuration: N site records. */
typedef struct {
  int N, dh, din;
  double *buf;
  or_site *site;
} or_fwd;

static int or_fwd_alloc(or_fwd *F, const or_layout *L) {
  F->N = L->N; F->dh = L->dh; F->din = L->din;
  size_t per = (size_t)6 * L->dh + L->din;
  F->buf = (double *)calloc((size_t)L->N * per, sizeof(double));
  F->site = (or_site *)calloc((size_t)L->N, sizeof(or_site));
  if (!F->buf || !F->site) return -1;
  for (int k = 0; k < L->N; ++k) {
    double *b = F->buf + (size_t)k * per;
    or_site *S = &F->site[k];
    S->hp = b; b += L->dh;
    S->x = b; b += L->din;
    S->u = b; b += L->dh;
    S->r = b; b += L->dh;
    S->g = b; b += L->dh;
    S->c = b; b += L->dh;
    S->h = b; b += L->dh;
  }
  return 0;
}

static void or_fwd_free(or_fwd *F) {
  free(F->buf);
  free(F->site);
}

/* One site of the GRU (App. A) given h' and x, filling S->u..S->h. */
static void or_gru_cell(const or_layout *L, const double *th, or_site *S) {
  int dh = L->dh, din = L->din, w = dh + din;
  for (int a = 0; a < dh; ++a) {
    double au = th[L->bu + a], ar = th[L->br + a];
    double g = th[L->bh + a], ai = th[L->bin + a];
    for (int b = 0; b < dh; ++b) {
      au += th[L->Wu + (int64_t)a * w + b] * S->hp[b];
      ar += th[L->Wr + (int64_t)a * w + b] * S->hp[b];
      g += th[L->Wh + (int64_t)a * dh + b] * S->hp[b];
    }
    for (int b = 0; b < din; ++b) {
      au += th[L->Wu + (int64_t)a * w + dh + b] * S->x[b];
      ar += th[L->Wr + (int64_t)a * w + dh + b] * S->x[b];
      ai += th[L->Win + (int64_t)a * din + b] * S->x[b];
    }
    S->u[a] = or_sigmoid(au);
    S->r[a] = or_sigmoid(ar);
    S->g[a] = g;
    S->c[a] = tanh(S->r[a] * g + ai);
    S->h[a] = (1.0 - S->u[a]) * S->hp[a] + S->u[a] * S->c[a];
  }
}

/* Softmax head of site k (Sec. II.A): logits z = U h + c, log-softmax,
 * then the zero-magnetisation mask given the ups/downs placed so far. */
static void or_head(const or_model *m, const or_layout *L, const double *th,
                    or_site *S, int n_up, int n_dn) {
  int dh = L->dh;
  double z[2];
  for (int o = 0; o < 2; ++o) {
    z[o] = th[L->co + o];
    for (int b = 0; b < dh; ++b) z[o] += th[L->Uo + o * dh + b] * S->h[b];
  }
  double mx = z[0] > z[1] ? z[0] : z[1];
  double lse = mx + log(exp(z[0] - mx) + exp(z[1] - mx));
  S->p[0] = exp(z[0] - lse);
  S->p[1] = exp(z[1] - lse);
  S->lp[0] = z[0] - lse;
  S->lp[1] = z[1] - lse;
  S->forced = 0;
  if (m->zmask) {
    int half = L->N / 2;
    if (n_up >= half) { S->lp[0] = -INFINITY; S->lp[1] = 0.0; S->forced = 1; }
    else if (n_dn >= half) { S->lp[0] = 0.0; S->lp[1] = -INFINITY; S->forced = 1; }
  }
  if (m->cplx) {
    for (int o = 0; o < 2; ++o) {
      S->y[o] = th[L->cp + o];
      for (int b = 0; b < dh; ++b) S->y[o] += th[L->Up + o * dh + b] * S->h[b];
    }
  }
}

/* Inputs of site k: h' and x from the already computed earlier sites. */
static void or_site_inputs(const or_model *m, const or_layout *L,
                           const double *th, or_fwd *F, const uint8_t *spins,
                           int k) {
  int dh = L->dh;
  int hor, ver;
  or_neighbours(m, k, &hor, &ver);
  or_site *S = &F->site[k];
  for (int b = 0; b < L->din; ++b) S->x[b] = 0.0;
  if (m->dim == 1) {
    for (int b = 0; b < dh; ++b) S->hp[b] = (hor >= 0) ? F->site[hor].h[b] : 0.0;
    if (hor >= 0) S->x[spins[hor]] = 1.0;
  } else {
    for (int a = 0; a < dh; ++a) {
      double v = 0.0;
      for (int b = 0; b < dh; ++b) {
        if (hor >= 0) v += th[L->U1 + (int64_t)a * dh + b] * F->site[hor].h[b];
        if (ver >= 0) v += th[L->U2 + (int64_t)a * dh + b] * F->site[ver].h[b];
      }
      S->hp[a] = v;
    }
    if (hor >= 0) S->x[spins[hor]] = 1.0;
    if (ver >= 0) S->x[2 + spins[ver]] = 1.0;
  }
}

/* Full forward pass over one configuration; returns log Psi. If sample_u is
 * non-NULL the spins are drawn (sigma_k = 0 iff u_k < p_k(0)) and written. */
static void or_forward(const or_model *m, const or_layout *L, const double *th,
                       or_fwd *F, uint8_t *spins, const double *sample_u,
                       double *lre, double *lim) {
  int n_up = 0, n_dn = 0, nA = 0;
  double logP = 0.0, phi = 0.0;
  for (int k = 0; k < L->N; ++k) {
    or_site_inputs(m, L, th, F, spins, k);
    or_site *S = &F->site[k];
    or_gru_cell(L, th, S);
    or_head(m, L, th, S, n_up, n_dn);
    if (sample_u) {
      double p0 = exp(S->lp[0]);
      spins[k] = (sample_u[k] < p0) ? 0 : 1;
    }
    int s = spins[k];
    logP += S->lp[s];
    if (m->cplx) {
      double y = S->y[s];
      phi += OR_PI * y / (1.0 + fabs(y));
    }
    if (s == 0) ++n_up; else ++n_dn;
    if (m->marshall && s == 1 && or_on_sublattice_A(m, k)) ++nA;
  }
  *lre = 0.5 * logP;
  *lim = phi + (m->marshall ? OR_PI * (double)(nA % 2) : 0.0);
}

/* ------------------------------------------------------------ log psi */

int or_logpsi(const or_model *m, const double *theta, const uint8_t *spins,
              int64_t n, double *logpsi) {
  or_layout L = or_make_layout(m);
  int err = 0;
#pragma omp parallel
  {
    or_fwd F;
    if (or_fwd_alloc(&F, &L)) {
#pragma omp atomic write
      err = -1;
    } else {
      uint8_t *sp = (uint8_t *)malloc((size_t)L.N);
#pragma omp for schedule(dynamic, 1)
      for (int64_t s = 0; s < n; ++s) {
        memcpy(sp, spins + s * L.N, (size_t)L.N);
        or_forward(m, &L, theta, &F, sp, NULL, &logpsi[2 * s], &logpsi[2 * s + 1]);
      }
      free(sp);
    }
    or_fwd_free(&F);
  }
  return err;
}

/* Conditional probabilities p_k(0) along a given configuration (after the
 * mask), for tests of the sampler's decisions. */
int or_conditionals(const or_model *m, const double *theta, const uint8_t *spins,
                    double *p0) {
  or_layout L = or_make_layout(m);
  or_fwd F;
  if (or_fwd_alloc(&F, &L)) return -1;
  uint8_t *sp = (uint8_t *)malloc((size_t)L.N);
  memcpy(sp, spins, (size_t)L.N);
  double a, b;
  or_forward(m, &L, theta, &F, sp, NULL, &a, &b);
  for (int k = 0; k < L.N; ++k) p0[k] = exp(F.site[k].lp[0]);
  free(sp);
  or_fwd_free(&F);
  return 0;
}

/* ------------------------------------------------------------ sampler */

/* Samples s0 .. s0 + n - 1 of a draw: sample s uses the Philox uniforms of
 * counter (k, s, step) at every site k, so disjoint ranges of one draw are
 * drawn independently (a rank of a sharded step draws its own range). */
int or_sample_range(const or_model *m, const double *theta, int64_t s0, int64_t n,
                    uint64_t seed, uint64_t step, uint8_t *spins, double *logpsi) {
  or_layout L = or_make_layout(m);
  int err = 0;
#pragma omp parallel
  {
    or_fwd F;
    double *u = (double *)malloc(sizeof(double) * (size_t)L.N);
    if (or_fwd_alloc(&F, &L) || !u) {
#pragma omp atomic write
      err = -1;
    } else {
#pragma omp for schedule(dynamic, 1)
      for (int64_t s = 0; s < n; ++s) {
        for (int k = 0; k < L.N; ++k)
          u[k] = or_uniform(seed, step, (uint64_t)(s0 + s), (uint64_t)k);
        or_forward(m, &L, theta, &F, spins + s * L.N, u, &logpsi[2 * s],
                   &logpsi[2 * s + 1]);
      }
    }
    free(u);
    or_fwd_free(&F);
  }
  return err;
}

int or_sample(const or_model *m, const double *theta, int64_t ns, uint64_t seed,
              uint64_t step, uint8_t *spins, double *logpsi) {
  return or_sample_range(m, theta, 0, ns, seed, step, spins, logpsi);
}

/* ------------------------------------------------------- local energy */

/* <sigma| P |sigma'> for the Pauli string t with sigma' = sigma flipped on
 * the X/Y sites: coeff * prod_Z z_k(sigma) * prod_Y (-i z_k(sigma)), where
 * z = 1 - 2 sigma; Y = [[0,-i],[i,0]] gives <s|Y|1-s> = -i z(s). */
static void or_term_element(const or_ham *H, int t, const uint8_t *sp,
                            double *re, double *im, int *flips, int *nflip) {
  double er = H->coeff[t], ei = 0.0;
  *nflip = 0;
  for (int q = 0; q < H->nops[t]; ++q) {
    int k = H->site[4 * t + q];
    char o = H->op[4 * t + q];
    double z = 1.0 - 2.0 * (double)sp[k];
    if (o == 'Z') {
      er *= z; ei *= z;
    } else if (o == 'X') {
      flips[(*nflip)++] = k;
    } else { /* 'Y': multiply by -i z */
      double nr = ei * z, ni = -er * z;
      er = nr; ei = ni;
      flips[(*nflip)++] = k;
    }
  }
  *re = er; *im = ei;
}

int or_local_energy(const or_model *m, const or_ham *H, const double *theta,
                    const uint8_t *spins, int64_t ns, double *eloc) {
  or_layout L = or_make_layout(m);
  int err = 0;
#pragma omp parallel
  {
    or_fwd F;
    uint8_t *sp = (uint8_t *)malloc((size_t)L.N);
    if (or_fwd_alloc(&F, &L) || !sp) {
#pragma omp atomic write
      err = -1;
    } else {
#pragma omp for schedule(dynamic, 1)
      for (int64_t s = 0; s < ns; ++s) {
        const uint8_t *sg = spins + s * L.N;
        double l0r, l0i;
        memcpy(sp, sg, (size_t)L.N);
        or_forward(m, &L, theta, &F, sp, NULL, &l0r, &l0i);
        double er = 0.0, ei = 0.0;
        for (int t = 0; t < H->n_terms; ++t) {
          int flips[4], nf;
          double hr, hi;
          or_term_element(H, t, sg, &hr, &hi, flips, &nf);
          if (nf == 0) { er += hr; ei += hi; continue; }
          memcpy(sp, sg, (size_t)L.N);
          for (int q = 0; q < nf; ++q) sp[flips[q]] ^= 1;
          double l1r, l1i;
          or_forward(m, &L, theta, &F, sp, NULL, &l1r, &l1i);
          if (isinf(l1r) && l1r < 0) continue; /* Psi(sigma') = 0 */
          double a = exp(l1r - l0r), ph = l1i - l0i;
          double rr = a * cos(ph), ri = a * sin(ph);
          er += hr * rr - hi * ri;
          ei += hr * ri + hi * rr;
        }
        eloc[2 * s] = er;
        eloc[2 * s + 1] = ei;
      }
    }
    free(sp);
    or_fwd_free(&F);
  }
  return err;
}

/* ------------------------------------------------------------ Jacobian */

/* Reverse pass for one configuration with the forward records in F.
 * which = 0: d(Re log Psi) = d(1/2 log P);  which = 1: d(Im log Psi) = d phi.
 * grad (length np) is overwritten.  dhs is scratch [N*dh]. */
static void or_backward(const or_model *m, const or_layout *L, const double *th,
                        const or_fwd *F, const uint8_t *sp, int which,
                        double *grad, double *dhs) {
  int N = L->N, dh = L->dh, din = L->din, w = dh + din;
  memset(grad, 0, sizeof(double) * (size_t)L->np);
  memset(dhs, 0, sizeof(double) * (size_t)N * dh);
  double *dhp = (double *)malloc(sizeof(double) * (size_t)dh);
  for (int k = N - 1; k >= 0; --k) {
    const or_site *S = &F->site[k];
    double *dh_k = dhs + (size_t)k * dh;
    int s = sp[k];
    /* output heads of site k */
    if (which == 0) {
      if (!S->forced) {
        double dz[2];
        for (int o = 0; o < 2; ++o) dz[o] = 0.5 * ((o == s ? 1.0 : 0.0) - S->p[o]);
        for (int o = 0; o < 2; ++o) {
          grad[L->co + o] += dz[o];
          for (int b = 0; b < dh; ++b) {
            grad[L->Uo + o * dh + b] += dz[o] * S->h[b];
            dh_k[b] += th[L->Uo + o * dh + b] * dz[o];
          }
        }
      }
    } else {
      double y = S->y[s];
      double d = OR_PI / ((1.0 + fabs(y)) * (1.0 + fabs(y)));
      grad[L->cp + s] += d;
      for (int b = 0; b < dh; ++b) {
        grad[L->Up + s * dh + b] += d * S->h[b];
        dh_k[b] += th[L->Up + s * dh + b] * d;
      }
    }
    /* GRU cell of site k */
    for (int b = 0; b < dh; ++b) dhp[b] = 0.0;
    for (int a = 0; a < dh; ++a) {
      double dhv = dh_k[a];
      double dc = dhv * S->u[a];
      double du = dhv * (S->c[a] - S->hp[a]);
      dhp[a] += dhv * (1.0 - S->u[a]);
      double dac = dc * (1.0 - S->c[a] * S->c[a]);
      double dr = dac * S->g[a];
      double dg = dac * S->r[a];
      double dar = dr * S->r[a] * (1.0 - S->r[a]);
      double dau = du * S->u[a] * (1.0 - S->u[a]);
      grad[L->bin + a] += dac;
      grad[L->bh + a] += dg;
      grad[L->br + a] += dar;
      grad[L->bu + a] += dau;
      for (int b = 0; b < din; ++b) {
        grad[L->Win + (int64_t)a * din + b] += dac * S->x[b];
        grad[L->Wr + (int64_t)a * w + dh + b] += dar * S->x[b];
        grad[L->Wu + (int64_t)a * w + dh + b] += dau * S->x[b];
      }
      for (int b = 0; b < dh; ++b) {
        grad[L->Wh + (int64_t)a * dh + b] += dg * S->hp[b];
        grad[L->Wr + (int64_t)a * w + b] += dar * S->hp[b];
        grad[L->Wu + (int64_t)a * w + b] += dau * S->hp[b];
        dhp[b] += th[L->Wh + (int64_t)a * dh + b] * dg
                + th[L->Wr + (int64_t)a * w + b] * dar
                + th[L->Wu + (int64_t)a * w + b] * dau;
      }
    }
    /* route d h' to the earlier sites */
    int hor, ver;
    or_neighbours(m, k, &hor, &ver);
    if (m->dim == 1) {
      if (hor >= 0)
        for (int b = 0; b < dh; ++b) dhs[(size_t)hor * dh + b] += dhp[b];
    } else {
      for (int a = 0; a < dh; ++a) {
        for (int b = 0; b < dh; ++b) {
          if (hor >= 0) {
            grad[L->U1 + (int64_t)a * dh + b] += dhp[a] * F->site[hor].h[b];
            dhs[(size_t)hor * dh + b] += th[L->U1 + (int64_t)a * dh + b] * dhp[a];
          }
          if (ver >= 0) {
            grad[L->U2 + (int64_t)a * dh + b] += dhp[a] * F->site[ver].h[b];
            dhs[(size_t)ver * dh + b] += th[L->U2 + (int64_t)a * dh + b] * dhp[a];
          }
        }
      }
    }
  }
  free(dhp);
}

/* Raw log-derivatives d log Psi(sigma_s)/d theta, sample-major:
 * rows 0..ns-1 hold the real parts, rows ns..2ns-1 the imaginary parts
 * (cRNN only).  No 1/sqrt(Ns) factor. */
int or_jacobian(const or_model *m, const double *theta, const uint8_t *spins,
                int64_t ns, double *O) {
  or_layout L = or_make_layout(m);
  int err = 0;
#pragma omp parallel
  {
    or_fwd F;
    uint8_t *sp = (uint8_t *)malloc((size_t)L.N);
    double *dhs = (double *)malloc(sizeof(double) * (size_t)L.N * L.dh);
    if (or_fwd_alloc(&F, &L) || !sp || !dhs) {
#pragma omp atomic write
      err = -1;
    } else {
#pragma omp for schedule(dynamic, 1)
      for (int64_t s = 0; s < ns; ++s) {
        double a, b;
        memcpy(sp, spins + s * L.N, (size_t)L.N);
        or_forward(m, &L, theta, &F, sp, NULL, &a, &b);
        or_backward(m, &L, theta, &F, sp, 0, O + (size_t)s * L.np, dhs);
        if (m->cplx)
          or_backward(m, &L, theta, &F, sp, 1, O + (size_t)(ns + s) * L.np, dhs);
      }
    }
    free(sp);
    free(dhs);
    or_fwd_free(&F);
  }
  return err;
}

/* ------------------------------------------------------- dense algebra */

/* T = A A^T for A [R x np] row-major (rows are samples). */
static void or_gram(const double *A, int64_t R, int64_t np, double *T) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t i = 0; i < R; ++i)
    for (int64_t j = 0; j <= i; ++j) {
      double acc = 0.0;
      for (int64_t k = 0; k < np; ++k) acc += A[i * np + k] * A[j * np + k];
      T[i * R + j] = acc;
      T[j * R + i] = acc;
    }
}

/* Cholesky A = L L^T (lower, in place in a copy), then solve A x = b.
 * Returns 0, or -1 if a pivot is not positive. */
int or_cholesky_solve(const double *A, int64_t n, const double *b, double *x) {
  double *Lm = (double *)malloc(sizeof(double) * (size_t)(n * n));
  if (!Lm) return -2;
  memcpy(Lm, A, sizeof(double) * (size_t)(n * n));
  for (int64_t j = 0; j < n; ++j) {
    double d = Lm[j * n + j];
    for (int64_t k = 0; k < j; ++k) d -= Lm[j * n + k] * Lm[j * n + k];
    if (!(d > 0.0)) { free(Lm); return -1; }
    d = sqrt(d);
    Lm[j * n + j] = d;
#pragma omp parallel for
    for (int64_t i = j + 1; i < n; ++i) {
      double v = Lm[i * n + j];
      for (int64_t k = 0; k < j; ++k) v -= Lm[i * n + k] * Lm[j * n + k];
      Lm[i * n + j] = v / d;
    }
  }
  /* L y = b */
  for (int64_t i = 0; i < n; ++i) {
    double v = b[i];
    for (int64_t k = 0; k < i; ++k) v -= Lm[i * n + k] * x[k];
    x[i] = v / Lm[i * n + i];
  }
  /* L^T x = y */
  for (int64_t i = n - 1; i >= 0; --i) {
    double v = x[i];
    for (int64_t k = i + 1; k < n; ++k) v -= Lm[k * n + i] * x[k];
    x[i] = v / Lm[i * n + i];
  }
  free(Lm);
  return 0;
}

/* ----------------------------------------------------- minSR step */

/* Optional intermediate outputs (any pointer may be NULL). */
typedef struct {
  uint8_t *spins;  /* [ns*N] */
  double *logpsi;  /* [ns*2] */
  double *eloc;    /* [ns*2] */
  double *T;       /* [R*R], before the shift */
  double *eps;     /* [R]    eps-bar' */
  double *x;       /* [R]    (T + lambda I)^{-1} eps-bar' */
  double *dtheta;  /* [np]   delta theta (with eta_eff) */
} or_step_out;

/* One iteration of Algorithm 1.  theta and mom are updated in place unless
 * the step is rejected (status != 0). */
int or_minsr_step(const or_model *m, const or_ham *H, double *theta, double *mom,
                  const or_hparams *hp, or_stats *st, const or_step_out *out) {
  or_layout L = or_make_layout(m);
  int64_t ns = hp->ns, N = L.N, np = L.np;
  int64_t R = m->cplx ? 2 * ns : ns;
  memset(st, 0, sizeof(*st));

  uint8_t *spins = (uint8_t *)malloc((size_t)(ns * N));
  double *lp = (double *)malloc(sizeof(double) * (size_t)(2 * ns));
  double *el = (double *)malloc(sizeof(double) * (size_t)(2 * ns));
  double *O = (double *)malloc(sizeof(double) * (size_t)(R * np));
  double *T = (double *)malloc(sizeof(double) * (size_t)(R * R));
  double *eps = (double *)malloc(sizeof(double) * (size_t)R);
  double *x = (double *)malloc(sizeof(double) * (size_t)R);
  double *dth = (double *)malloc(sizeof(double) * (size_t)np);
  if (!spins || !lp || !el || !O || !T || !eps || !x || !dth) return -2;

  /* Alg. 1, sampling: draw Ns configurations */
  or_sample(m, theta, ns, hp->seed, (uint64_t)hp->step_index, spins, lp);
  /* Alg. 1, energy: local energies and E */
  or_local_energy(m, H, theta, spins, ns, el);
  double Er = 0.0, Ei = 0.0;
  for (int64_t s = 0; s < ns; ++s) { Er += el[2 * s]; Ei += el[2 * s + 1]; }
  Er /= (double)ns; Ei /= (double)ns;
  double var = 0.0;
  for (int64_t s = 0; s < ns; ++s) {
    double a = el[2 * s] - Er, b = el[2 * s + 1] - Ei;
    var += a * a + b * b;
  }
  var /= (double)ns;
  st->E_re = Er; st->E_im = Ei; st->var = var;
  st->vscore = (double)N * var / (Er * Er);

  /* Alg. 1, log-derivatives: O_ks = d log Psi / d theta_k / sqrt(Ns), centred over samples,
   * separately for the real and the imaginary rows */
  or_jacobian(m, theta, spins, ns, O);
  double isq = 1.0 / sqrt((double)ns);
  int nblk = m->cplx ? 2 : 1;
  for (int blk = 0; blk < nblk; ++blk) {
    double *B = O + (size_t)(blk * ns) * np;
#pragma omp parallel for
    for (int64_t k = 0; k < np; ++k) {
      double mean = 0.0;
      for (int64_t s = 0; s < ns; ++s) mean += B[s * np + k];
      mean /= (double)ns;
      for (int64_t s = 0; s < ns; ++s) B[s * np + k] = (B[s * np + k] - mean) * isq;
    }
  }
  /* eps-bar_i = (eps_i - E)^* / sqrt(Ns); eps-bar' = 2 (Re; -Im) */
  for (int64_t s = 0; s < ns; ++s) {
    eps[s] = 2.0 * (el[2 * s] - Er) * isq;
    if (m->cplx) eps[ns + s] = 2.0 * (el[2 * s + 1] - Ei) * isq;
  }
  /* Alg. 1, Gram: T = O'^T O' */
  or_gram(O, R, np, T);
  double nT = 0.0;
  for (int64_t i = 0; i < R * R; ++i) nT += T[i] * T[i];
  nT = sqrt(nT);
  double lam = (hp->lambda_mode == 1) ? hp->lambda_coeff * pow(nT, hp->lambda_pow)
                                      : hp->lambda;
  st->normT = nT;
  st->lambda = lam;
  if (out && out->T) memcpy(out->T, T, sizeof(double) * (size_t)(R * R));
  /* Alg. 1, solve: x = (T + lambda I)^{-1} eps-bar' */
  for (int64_t i = 0; i < R; ++i) T[i * R + i] += lam;
  int ok = or_cholesky_solve(T, R, eps, x);
  int status = 0;
  if (ok != 0) status = 5;
  /* tau = T (T + lambda I)^{-1} eps' = eps' - lambda x (App. F) */
  double tn = 0.0;
  for (int64_t i = 0; i < R; ++i) {
    double t = eps[i] - lam * x[i];
    tn += t * t;
  }
  tn = sqrt(tn);
  st->tau_norm = tn;
  double eta = hp->eta0;
  if (hp->decay_T > 0.0 && isfinite(hp->decay_T))
    eta = hp->eta0 / (1.0 + (double)hp->step_index / hp->decay_T);
  if (hp->trust_region) eta = eta / tn;
  st->eta_eff = eta;
  /* delta theta = eta O' x */
#pragma omp parallel for
  for (int64_t k = 0; k < np; ++k) {
    double acc = 0.0;
    for (int64_t r = 0; r < R; ++r) acc += O[r * np + k] * x[r];
    dth[k] = eta * acc;
  }
  int finite = isfinite(Er) && isfinite(Ei);
  for (int64_t k = 0; k < np && finite; ++k) finite = isfinite(dth[k]);
  if (status == 0 && !finite) status = 4;
  st->status = status;
  /* Levenberg-Marquardt damping (App. G): gain ratio of the step against
   * its quadratic model.  The model's predicted decrease for the step
   * delta theta (theta -> theta - delta theta) is
   *   g^T dtheta - 1/2 dtheta^T S dtheta,  g = O'^T eps', S = O'^T O',
   * and with dtheta = eta O'^T x, T x = tau this is
   *   eta eps'^T tau - 1/2 eta^2 ||tau||^2
   * (= eta* eps'^T tau - 1/2 eta_t^2 in the trust-region mode, App. G).
   * The actual decrease uses E at theta - delta theta, estimated from Ns
   * fresh samples (key seed + OR_LM_KEY_OFFSET, counter step t). */
  st->rho = 0.0;
  st->lambda_next = lam;
  if (hp->lm_omega > 1.0) {
    double et = 0.0;
    for (int64_t i = 0; i < R; ++i) et += eps[i] * (eps[i] - lam * x[i]);
    const double pred = eta * et - 0.5 * eta * eta * tn * tn;
    double *th2 = (double *)malloc(sizeof(double) * (size_t)np);
    uint8_t *sp2 = (uint8_t *)malloc((size_t)(ns * N));
    double *lp2 = (double *)malloc(sizeof(double) * (size_t)(2 * ns));
    double *el2 = (double *)malloc(sizeof(double) * (size_t)(2 * ns));
    if (!th2 || !sp2 || !lp2 || !el2) return -2;
    for (int64_t k = 0; k < np; ++k) th2[k] = status == 0 ? theta[k] - dth[k] : theta[k];
    or_sample(m, th2, ns, hp->seed + OR_LM_KEY_OFFSET, (uint64_t)hp->step_index, sp2, lp2);
    or_local_energy(m, H, th2, sp2, ns, el2);
    double E2 = 0.0;
    for (int64_t s = 0; s < ns; ++s) E2 += el2[2 * s];
    E2 /= (double)ns;
    const double rho = (Er - E2) / pred;
    st->rho = rho;
    /* a rejected step or an undefined ratio counts as a poor step */
    if (status != 0 || !(rho >= 0.25)) st->lambda_next = hp->lm_omega * lam;
    else if (rho > 0.75) st->lambda_next = lam / hp->lm_omega;
    free(th2); free(sp2); free(lp2); free(el2);
  }
  /* Alg. 1, momentum and update, only for an accepted step */
  if (status == 0) {
    for (int64_t k = 0; k < np; ++k) {
      mom[k] = hp->mu * mom[k] + (1.0 - hp->mu) * dth[k];
      theta[k] -= mom[k];
    }
  }
  if (out) {
    if (out->spins) memcpy(out->spins, spins, (size_t)(ns * N));
    if (out->logpsi) memcpy(out->logpsi, lp, sizeof(double) * (size_t)(2 * ns));
    if (out->eloc) memcpy(out->eloc, el, sizeof(double) * (size_t)(2 * ns));
    if (out->eps) memcpy(out->eps, eps, sizeof(double) * (size_t)R);
    if (out->x) memcpy(out->x, x, sizeof(double) * (size_t)R);
    if (out->dtheta) memcpy(out->dtheta, dth, sizeof(double) * (size_t)np);
  }
  free(spins); free(lp); free(el); free(O); free(T); free(eps); free(x); free(dth);
  return 0;
}

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void or_set_num_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}
