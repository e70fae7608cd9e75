/*
 * qt_oracle.c -- plain, slow, FP64 CPU oracle for the two solvers of
 * Johansson, Nation & Nori, "QuTiP: An open-source Python framework for the
 * dynamics of open quantum systems" (QuTiP 1.1.3):
 *
 *   - the Lindblad master equation, paper section 3.1, Eq. (master_equation),
 *     integrated in time (the paper's odesolve, section 3.1);
 *   - the Monte-Carlo wave-function method, paper section 3.2, Eq. (heff),
 *     Eq. (project), Eq. (pcn) and the four-step algorithm I-IV with
 *     Eq. (mc3).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent reference the CUDA
 * library is checked against.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark load it.  It shares no code, header,
 * constant table or helper with the CUDA library, and the library never calls
 * it: there is no CPU fallback.
 *
 * Everything here is written for a reader checking it against the paper by
 * eye: sparse CSR loops, no blocking, no fusion, FP64 throughout.
 *
 * Readings of the paper that this file fixes (the paper names no integrator
 * and leaves several details open; each reading is listed with its reason in
 * the design notes of the repository):
 *   R1  The time integrator is the Dormand-Prince 5(4) pair (Dormand & Prince
 *       1980), propagating the 5th-order solution, with the Hairer-Norsett-
 *       Wanner starting-step rule and the step controller in dp45_control().
 *   R2  Error norm: root-mean-square over all real components of
 *       E_i / (atol + rtol * max(|y_i|, |ynew_i|)); a step is accepted when
 *       the norm is <= 1.
 *   R3  Steps are clipped so that every output time t_k is hit exactly; the
 *       clipped length never shrinks the step proposal carried forward.
 *   R4  Step II of the MC algorithm compares the squared norm <psi|psi> with
 *       r.  The crossing time is located by bisection: each trial state is one
 *       Dormand-Prince step of length (tau - t) from the last accepted (t, psi).
 *   R5  Step III uses a second, independent uniform r2 for the channel
 *       choice (Eq. (mc3) as printed reuses r and sums P_n; the standard
 *       Dalibard / Dum / Molmer method it cites draws a fresh number).
 *   R6  Random numbers: Philox4x32-10 (Salmon et al., SC'11), key = seed,
 *       counter = (trajectory, jump index, stream, 0); stream 0 is the jump
 *       threshold r, stream 1 the channel draw r2.
 *   R7  Eq. (heff) sums over i but indexes C_n: read as a sum over n.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Status codes: the same numeric meaning as the library's public codes, so a
 * test can compare them; the values are restated here, not shared. */
enum {
  OR_OK = 0,
  OR_EINVAL = -1,
  OR_ENORM = -3,
  OR_ENOMEM = -4,
  OR_ESTEP = -6,
  OR_ENUMERIC = -9,
  OR_ECAP = -10
};

typedef struct { double re, im; } cx;

typedef struct {
  int32_t d;
  const int64_t *indptr;  /* d+1 row pointers            */
  const int32_t *indices; /* column of each stored entry */
  const cx *values;       /* value of each stored entry  */
} csr;

typedef struct {
  int64_t traj;
  int64_t k;        /* jump index within the trajectory (0, 1, ...)  */
  int64_t channel;  /* collapse operator chosen, 0-based             */
  double tau;       /* jump time                                     */
  int64_t degenerate; /* bit 0: channel draw within 1e-5 of a cumulative
                         boundary; bit 1: tau within 1e-5 of an output time */
} or_jump;

typedef struct {
  int64_t accepted;
  int64_t rejected;
  int64_t rhs_evals;
  int64_t bisect_iters;
  int64_t jumps;
} or_stats;

/* ---------------------------------------------------------------- complex */

static inline cx c_mul(cx a, cx b) {
  cx r = {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
  return r;
}
static inline cx c_conj(cx a) { cx r = {a.re, -a.im}; return r; }
static inline cx c_add(cx a, cx b) { cx r = {a.re + b.re, a.im + b.im}; return r; }
static inline cx c_scale(cx a, double s) { cx r = {a.re * s, a.im * s}; return r; }

/* ------------------------------------------------- Philox4x32-10, R6 */
/*
 * Philox4x32 (Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as easy
 * as 1, 2, 3", SC'11): each round multiplies words 0 and 2 of the counter by
 * two fixed odd constants, and the output is (hi(w2*M1) ^ w1 ^ k0,
 * lo(w2*M1), hi(w0*M0) ^ w3 ^ k1, lo(w0*M0)).  Between rounds the key words
 * are bumped by the Weyl constants (golden ratio and sqrt(3) - 1 in 32-bit
 * fixed point).  Ten rounds.
 */
void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                      uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t w[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) { k0 += W0; k1 += W1; }
    uint64_t p0 = (uint64_t)M0 * (uint64_t)w[0];
    uint64_t p1 = (uint64_t)M1 * (uint64_t)w[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ w[1] ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ w[3] ^ k1;
    uint32_t n3 = lo0;
    w[0] = n0; w[1] = n1; w[2] = n2; w[3] = n3;
  }
  out[0] = w[0]; out[1] = w[1]; out[2] = w[2]; out[3] = w[3];
}

/* Uniform in the open interval (0, 1) from 52 random bits (R6):
 * m = (x0 >> 6) * 2^26 + (x1 >> 6), U = (m + 1/2) * 2^-52.  m + 1/2 needs 53
 * significant bits, so U is exact and lies in [2^-53, 1 - 2^-53]. */
double or_uniform(uint64_t seed, uint64_t traj, uint64_t k, uint32_t stream) {
  uint32_t ctr[4] = {(uint32_t)traj, (uint32_t)k, stream, 0u};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t x[4];
  or_philox4x32_10(ctr, key, x);
  double m = (double)(x[0] >> 6) * 67108864.0 + (double)(x[1] >> 6);
  return (m + 0.5) * (1.0 / 4503599627370496.0);
}

/* ------------------------------------------------------ sparse products */

/* y = A x for a CSR operator A and a vector x. */
static void csr_matvec(const csr *A, const cx *x, cx *y) {
  for (int i = 0; i < A->d; ++i) {
    cx acc = {0.0, 0.0};
    for (int64_t p = A->indptr[i]; p < A->indptr[i + 1]; ++p)
      acc = c_add(acc, c_mul(A->values[p], x[A->indices[p]]));
    y[i] = acc;
  }
}

/* y = A^dagger x:  (A^dag x)_i = sum_k conj(A_ki) x_k. */
static void csr_matvec_dag(const csr *A, const cx *x, cx *y) {
  for (int i = 0; i < A->d; ++i) { y[i].re = 0.0; y[i].im = 0.0; }
  for (int k = 0; k < A->d; ++k)
    for (int64_t p = A->indptr[k]; p < A->indptr[k + 1]; ++p) {
      int i = A->indices[p];
      y[i] = c_add(y[i], c_mul(c_conj(A->values[p]), x[k]));
    }
}

/* Y = A X  (X, Y dense d x d, row-major). */
static void csr_left(const csr *A, const cx *X, cx *Y) {
  int d = A->d;
  memset(Y, 0, sizeof(cx) * (size_t)d * d);
  for (int i = 0; i < d; ++i)
    for (int64_t p = A->indptr[i]; p < A->indptr[i + 1]; ++p) {
      int k = A->indices[p];
      cx v = A->values[p];
      for (int j = 0; j < d; ++j)
        Y[(size_t)i * d + j] = c_add(Y[(size_t)i * d + j], c_mul(v, X[(size_t)k * d + j]));
    }
}

/* Y = A^dag X:  (A^dag X)_ij = sum_k conj(A_ki) X_kj. */
static void csr_left_dag(const csr *A, const cx *X, cx *Y) {
  int d = A->d;
  memset(Y, 0, sizeof(cx) * (size_t)d * d);
  for (int k = 0; k < d; ++k)
    for (int64_t p = A->indptr[k]; p < A->indptr[k + 1]; ++p) {
      int i = A->indices[p];
      cx v = c_conj(A->values[p]);
      for (int j = 0; j < d; ++j)
        Y[(size_t)i * d + j] = c_add(Y[(size_t)i * d + j], c_mul(v, X[(size_t)k * d + j]));
    }
}

/* Y = X A:  (X A)_ij = sum_k X_ik A_kj. */
static void csr_right(const cx *X, const csr *A, cx *Y) {
  int d = A->d;
  memset(Y, 0, sizeof(cx) * (size_t)d * d);
  for (int k = 0; k < d; ++k)
    for (int64_t p = A->indptr[k]; p < A->indptr[k + 1]; ++p) {
      int j = A->indices[p];
      cx v = A->values[p];
      for (int i = 0; i < d; ++i)
        Y[(size_t)i * d + j] = c_add(Y[(size_t)i * d + j], c_mul(X[(size_t)i * d + k], v));
    }
}

/* Y = X A^dag:  (X A^dag)_ij = sum_k X_ik conj(A_jk). */
static void csr_right_dag(const cx *X, const csr *A, cx *Y) {
  int d = A->d;
  memset(Y, 0, sizeof(cx) * (size_t)d * d);
  for (int j = 0; j < d; ++j)
    for (int64_t p = A->indptr[j]; p < A->indptr[j + 1]; ++p) {
      int k = A->indices[p];
      cx v = c_conj(A->values[p]);
      for (int i = 0; i < d; ++i)
        Y[(size_t)i * d + j] = c_add(Y[(size_t)i * d + j], c_mul(X[(size_t)i * d + k], v));
    }
}

/* ------------------------------------------- Lindblad right-hand side */

typedef struct {
  int d;
  const csr *H;
  const csr *c;
  int nc;
  cx *t1, *t2, *t3; /* d*d scratch each */
} me_ctx;

/*
 * Eq. (master_equation), hbar = 1, in its literal form:
 *   drho = -i [H, rho] + sum_n ( C rho C^dag - 1/2 rho C^dag C - 1/2 C^dag C rho )
 * Every product is evaluated as written (C^dag C rho = C^dag (C rho),
 * rho C^dag C = (rho C^dag) C); no effective Hamiltonian is formed.
 */
void or_lindblad_rhs(int d, const csr *H, const csr *c, int nc, const cx *rho,
                     cx *drho, cx *t1, cx *t2, cx *t3) {
  size_t n = (size_t)d * d;
  /* -i (H rho - rho H) */
  csr_left(H, rho, t1);
  csr_right(rho, H, t2);
  for (size_t q = 0; q < n; ++q) {
    cx comm = {t1[q].re - t2[q].re, t1[q].im - t2[q].im};
    drho[q].re = comm.im;   /* -i * (a + ib) = b - ia */
    drho[q].im = -comm.re;
  }
  for (int m = 0; m < nc; ++m) {
    const csr *C = &c[m];
    csr_left(C, rho, t1);       /* t1 = C rho             */
    csr_right_dag(t1, C, t2);   /* t2 = C rho C^dag       */
    for (size_t q = 0; q < n; ++q) drho[q] = c_add(drho[q], t2[q]);
    csr_left_dag(C, t1, t2);    /* t2 = C^dag C rho       */
    for (size_t q = 0; q < n; ++q) drho[q] = c_add(drho[q], c_scale(t2[q], -0.5));
    csr_right_dag(rho, C, t1);  /* t1 = rho C^dag         */
    csr_right(t1, C, t3);       /* t3 = rho C^dag C       */
    for (size_t q = 0; q < n; ++q) drho[q] = c_add(drho[q], c_scale(t3[q], -0.5));
  }
}

static void me_rhs(void *vctx, double t, const double *y, double *dy) {
  (void)t;
  me_ctx *m = (me_ctx *)vctx;
  or_lindblad_rhs(m->d, m->H, m->c, m->nc, (const cx *)y, (cx *)dy, m->t1, m->t2, m->t3);
}

/* --------------------------------------- non-Hermitian Schrodinger RHS */

typedef struct {
  int d;
  const csr *H;
  const csr *c;
  int nc;
  cx *t1, *t2; /* d scratch each */
} mc_ctx;

/*
 * d psi/dt = -i H_eff psi with Eq. (heff), hbar = 1:
 *   H_eff = H - (i/2) sum_n C_n^dag C_n,
 * so -i H_eff psi = -i H psi - 1/2 sum_n C_n^dag (C_n psi).
 */
static void mc_rhs(void *vctx, double t, const double *y, double *dy) {
  (void)t;
  mc_ctx *m = (mc_ctx *)vctx;
  const cx *psi = (const cx *)y;
  cx *out = (cx *)dy;
  csr_matvec(m->H, psi, m->t1);
  for (int i = 0; i < m->d; ++i) { out[i].re = m->t1[i].im; out[i].im = -m->t1[i].re; }
  for (int n = 0; n < m->nc; ++n) {
    csr_matvec(&m->c[n], psi, m->t1);
    csr_matvec_dag(&m->c[n], m->t1, m->t2);
    for (int i = 0; i < m->d; ++i) out[i] = c_add(out[i], c_scale(m->t2[i], -0.5));
  }
}

/* ------------------------------------------------ Dormand-Prince 5(4), R1 */

typedef void (*rhs_fn)(void *ctx, double t, const double *y, double *dy);

/* Butcher tableau of Dormand & Prince (1980), "A family of embedded
 * Runge-Kutta formulae", J. Comput. Appl. Math. 6, 19-26. */
static const double DP_C[7] = {0.0, 1.0 / 5.0, 3.0 / 10.0, 4.0 / 5.0, 8.0 / 9.0, 1.0, 1.0};
static const double DP_A[7][6] = {
    {0, 0, 0, 0, 0, 0},
    {1.0 / 5.0, 0, 0, 0, 0, 0},
    {3.0 / 40.0, 9.0 / 40.0, 0, 0, 0, 0},
    {44.0 / 45.0, -56.0 / 15.0, 32.0 / 9.0, 0, 0, 0},
    {19372.0 / 6561.0, -25360.0 / 2187.0, 64448.0 / 6561.0, -212.0 / 729.0, 0, 0},
    {9017.0 / 3168.0, -355.0 / 33.0, 46732.0 / 5247.0, 49.0 / 176.0, -5103.0 / 18656.0, 0},
    {35.0 / 384.0, 0.0, 500.0 / 1113.0, 125.0 / 192.0, -2187.0 / 6784.0, 11.0 / 84.0}};
/* 5th-order weights (equal to the last row of A: first-same-as-last). */
static const double DP_B5[7] = {35.0 / 384.0, 0.0, 500.0 / 1113.0, 125.0 / 192.0,
                                -2187.0 / 6784.0, 11.0 / 84.0, 0.0};
/* 4th-order embedded weights. */
static const double DP_B4[7] = {5179.0 / 57600.0, 0.0, 7571.0 / 16695.0, 393.0 / 640.0,
                                -92097.0 / 339200.0, 187.0 / 2100.0, 1.0 / 40.0};

/* Exported so that the tests can check the order conditions of the table. */
void or_dp45_tableau(double *c, double *a, double *b5, double *b4) {
  for (int i = 0; i < 7; ++i) {
    c[i] = DP_C[i]; b5[i] = DP_B5[i]; b4[i] = DP_B4[i];
    for (int j = 0; j < 6; ++j) a[i * 6 + j] = DP_A[i][j];
  }
}

typedef struct {
  rhs_fn f;
  void *ctx;
  int64_t n;       /* number of real components */
  double rtol, atol;
  double *k[7];    /* stage derivatives */
  double *ytmp;
  int64_t rhs_evals;
} dp45;

static int dp45_init(dp45 *s, rhs_fn f, void *ctx, int64_t n, double rtol, double atol) {
  s->f = f; s->ctx = ctx; s->n = n; s->rtol = rtol; s->atol = atol; s->rhs_evals = 0;
  for (int i = 0; i < 7; ++i) {
    s->k[i] = (double *)calloc((size_t)n, sizeof(double));
    if (!s->k[i]) return OR_ENOMEM;
  }
  s->ytmp = (double *)calloc((size_t)n, sizeof(double));
  return s->ytmp ? OR_OK : OR_ENOMEM;
}

static void dp45_free(dp45 *s) {
  for (int i = 0; i < 7; ++i) free(s->k[i]);
  free(s->ytmp);
}

static void dp45_eval(dp45 *s, double t, const double *y, double *dy) {
  s->f(s->ctx, t, y, dy);
  s->rhs_evals++;
}

/*
 * One Dormand-Prince step of length h from (t, y) with s->k[0] = f(t, y)
 * already in place.  Writes the 5th-order solution to ynew.  With
 * want_err != 0 it also evaluates k7 = f(t + h, ynew) and returns the scaled
 * RMS error of R2; otherwise it stops after ynew and returns 0.
 */
static double dp45_step(dp45 *s, double t, double h, const double *y, double *ynew,
                        int want_err) {
  int64_t n = s->n;
  for (int st = 1; st < 6; ++st) {
    for (int64_t i = 0; i < n; ++i) {
      double acc = 0.0;
      for (int j = 0; j < st; ++j) acc += DP_A[st][j] * s->k[j][i];
      s->ytmp[i] = y[i] + h * acc;
    }
    dp45_eval(s, t + DP_C[st] * h, s->ytmp, s->k[st]);
  }
  for (int64_t i = 0; i < n; ++i) {
    double acc = 0.0;
    for (int j = 0; j < 6; ++j) acc += DP_B5[j] * s->k[j][i];
    ynew[i] = y[i] + h * acc;
  }
  if (!want_err) return 0.0;
  dp45_eval(s, t + h, ynew, s->k[6]);
  double sum = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double e = 0.0;
    for (int j = 0; j < 7; ++j) e += (DP_B5[j] - DP_B4[j]) * s->k[j][i];
    e *= h;
    double sc = s->atol + s->rtol * fmax(fabs(y[i]), fabs(ynew[i]));
    double q = e / sc;
    sum += q * q;
  }
  return sqrt(sum / (double)n);
}

/* Scaled RMS of v with weights sc_i = atol + rtol |y0_i|. */
static double scaled_rms(const dp45 *s, const double *y0, const double *v) {
  double sum = 0.0;
  for (int64_t i = 0; i < s->n; ++i) {
    double q = v[i] / (s->atol + s->rtol * fabs(y0[i]));
    sum += q * q;
  }
  return sqrt(sum / (double)s->n);
}

/*
 * Starting step (Hairer, Norsett & Wanner, Solving ODEs I, section II.4),
 * for a method of order 5.  s->k[0] must hold f(t0, y0).  Uses s->k[1] and
 * s->ytmp as scratch.
 */
static double dp45_initial_step(dp45 *s, double t0, const double *y0) {
  double d0 = scaled_rms(s, y0, y0);
  double d1 = scaled_rms(s, y0, s->k[0]);
  double h0 = (d0 < 1e-5 || d1 < 1e-5) ? 1e-6 : 0.01 * d0 / d1;
  for (int64_t i = 0; i < s->n; ++i) s->ytmp[i] = y0[i] + h0 * s->k[0][i];
  dp45_eval(s, t0 + h0, s->ytmp, s->k[1]);
  for (int64_t i = 0; i < s->n; ++i) s->ytmp[i] = s->k[1][i] - s->k[0][i];
  double d2 = scaled_rms(s, y0, s->ytmp) / h0;
  double dm = fmax(d1, d2);
  double h1 = (dm <= 1e-15) ? fmax(1e-6, h0 * 1e-3) : pow(0.01 / dm, 1.0 / 5.0);
  return fmin(100.0 * h0, h1);
}

/*
 * Step-size controller (R1): after an accepted step the factor is
 * min(facmax, max(0.2, 0.9 err^(-1/5))), with facmax = 5, or 1 right after a
 * rejection; after a rejected step it is max(0.2, 0.9 err^(-1/5)).  When the
 * step had been clipped to an output time, the proposal carried forward is
 * never smaller than the unclipped proposal it replaced (R3).
 */
static double dp45_control(double h, double err, int accepted, int after_reject,
                           int clipped, double hprop) {
  if (accepted) {
    double facmax = after_reject ? 1.0 : 5.0;
    double fac = (err == 0.0) ? facmax : fmin(facmax, fmax(0.2, 0.9 * pow(err, -0.2)));
    double hn = h * fac;
    if (clipped && hn < hprop) hn = hprop;
    return hn;
  }
  return h * fmax(0.2, 0.9 * pow(err, -0.2));
}

/* An unclipped step below this length is a step-size underflow. */
static double dp45_hmin(double t, double tnext) {
  return 16.0 * 2.220446049250313e-16 * fmax(fabs(t), fabs(tnext));
}

/* ------------------------------------------------------------ expectation */

/* <psi|O|psi> (not normalised). */
static cx ket_expect(const csr *O, const cx *psi, cx *tmp) {
  csr_matvec(O, psi, tmp);
  cx acc = {0.0, 0.0};
  for (int i = 0; i < O->d; ++i) acc = c_add(acc, c_mul(c_conj(psi[i]), tmp[i]));
  return acc;
}

/* Tr(O rho) = sum_i sum_k O_ik rho_ki. */
static cx dm_expect(const csr *O, const cx *rho) {
  int d = O->d;
  cx acc = {0.0, 0.0};
  for (int i = 0; i < d; ++i)
    for (int64_t p = O->indptr[i]; p < O->indptr[i + 1]; ++p)
      acc = c_add(acc, c_mul(O->values[p], rho[(size_t)O->indices[p] * d + i]));
  return acc;
}

/* Exported: expectation of O over a batch of kets (<psi|O|psi>) or density
 * matrices (Tr(O rho)), the paper's expect() (section 2). */
int or_expect(const csr *O, const cx *states, int is_ket, int64_t batch, cx *out) {
  int d = O->d;
  cx *tmp = (cx *)calloc((size_t)d, sizeof(cx));
  if (!tmp) return OR_ENOMEM;
  for (int64_t b = 0; b < batch; ++b) {
    if (is_ket) out[b] = ket_expect(O, states + (size_t)b * d, tmp);
    else out[b] = dm_expect(O, states + (size_t)b * d * d);
  }
  free(tmp);
  return OR_OK;
}

/* ----------------------------------------------------- master equation */

/*
 * Integrate Eq. (master_equation) from rho0 over tlist (the paper's odesolve,
 * section 3.1).  Outputs Tr(O_m rho(t_k)) into expect_out[k * ne + m] and,
 * when states_out is non-null, rho(t_k) into states_out[k * d * d ...].
 */
int or_mesolve(int d, const csr *H, const csr *c, int nc, const csr *e, int ne,
               const cx *rho0, const double *tlist, int nt, double rtol, double atol,
               double h0, int64_t max_steps, cx *expect_out, cx *states_out,
               or_stats *stats) {
  if (d <= 0 || nt <= 0) return OR_EINVAL;
  size_t nn = (size_t)d * d;
  me_ctx m = {d, H, c, nc, NULL, NULL, NULL};
  m.t1 = (cx *)calloc(nn, sizeof(cx));
  m.t2 = (cx *)calloc(nn, sizeof(cx));
  m.t3 = (cx *)calloc(nn, sizeof(cx));
  double *y = (double *)calloc(2 * nn, sizeof(double));
  double *ynew = (double *)calloc(2 * nn, sizeof(double));
  dp45 s;
  int rc = dp45_init(&s, me_rhs, &m, (int64_t)(2 * nn), rtol, atol);
  if (!m.t1 || !m.t2 || !m.t3 || !y || !ynew || rc != OR_OK) { rc = OR_ENOMEM; goto done; }
  memcpy(y, rho0, sizeof(cx) * nn);

  double t = tlist[0];
  for (int q = 0; q < ne; ++q) expect_out[q] = dm_expect(&e[q], (const cx *)y);
  if (states_out) memcpy(states_out, y, sizeof(cx) * nn);
  if (nt == 1) { rc = OR_OK; goto done; }

  dp45_eval(&s, t, y, s.k[0]);
  double hprop = (h0 > 0.0) ? h0 : dp45_initial_step(&s, t, y);
  int after_reject = 0;
  int64_t acc = 0, rej = 0;
  for (int kk = 1; kk < nt; ++kk) {
    double tk = tlist[kk];
    int64_t attempts = 0;
    while (t < tk) {
      if (attempts++ >= max_steps) { rc = OR_ESTEP; goto done; }
      int clipped = hprop >= tk - t;
      double h = clipped ? tk - t : hprop;
      if (!clipped && h < dp45_hmin(t, tk)) { rc = OR_ESTEP; goto done; }
      double err = dp45_step(&s, t, h, y, ynew, 1);
      if (!isfinite(err)) { rc = OR_ENUMERIC; goto done; }
      if (err <= 1.0) {
        hprop = dp45_control(h, err, 1, after_reject, clipped, hprop);
        after_reject = 0;
        t = clipped ? tk : t + h;
        memcpy(y, ynew, sizeof(double) * 2 * nn);
        double *sw = s.k[0]; s.k[0] = s.k[6]; s.k[6] = sw; /* first-same-as-last */
        acc++;
      } else {
        hprop = dp45_control(h, err, 0, after_reject, clipped, hprop);
        after_reject = 1;
        rej++;
      }
    }
    for (int q = 0; q < ne; ++q) expect_out[(size_t)kk * ne + q] = dm_expect(&e[q], (const cx *)y);
    if (states_out) memcpy(states_out + (size_t)kk * nn, y, sizeof(cx) * nn);
  }
  rc = OR_OK;
  if (stats) {
    stats->accepted = acc; stats->rejected = rej; stats->rhs_evals = s.rhs_evals;
    stats->bisect_iters = 0; stats->jumps = 0;
  }
done:
  dp45_free(&s);
  free(m.t1); free(m.t2); free(m.t3); free(y); free(ynew);
  return rc;
}

/* --------------------------------------------- Monte-Carlo wave function */

typedef struct {
  or_jump *rec;
  int64_t n, cap;
} jump_list;

static int jl_push(jump_list *l, or_jump j) {
  if (l->n == l->cap) {
    int64_t nc = l->cap ? 2 * l->cap : 16;
    or_jump *p = (or_jump *)realloc(l->rec, sizeof(or_jump) * (size_t)nc);
    if (!p) return OR_ENOMEM;
    l->rec = p; l->cap = nc;
  }
  l->rec[l->n++] = j;
  return OR_OK;
}

static double sq_norm(const double *y, int64_t n) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s += y[i] * y[i];
  return s;
}

/*
 * One trajectory of the MC algorithm (section 3.2, steps I-IV):
 *   I   draw r;
 *   II  integrate d psi/dt = -i H_eff psi until <psi|psi> = r (R4);
 *   III pick the smallest n with sum_{i<=n} P_i >= r2 (Eq. (pcn), (mc3), R5)
 *       and apply Eq. (project);
 *   IV  draw a new r and continue from the jump time.
 * traj_expect receives the normalised expectation values
 * <psi|O_m|psi>/<psi|psi> at each output time, [k * ne + m].
 */
static int mc_trajectory(int d, const csr *H, const csr *c, int nc, const csr *e, int ne,
                         const cx *psi0, const double *tlist, int nt, int64_t j,
                         uint64_t seed, double rtol, double atol, double h0,
                         int64_t max_steps, double bisect_tol, cx *traj_expect,
                         jump_list *jl, or_stats *st) {
  int64_t n = 2 * (int64_t)d;
  mc_ctx m = {d, H, c, nc, NULL, NULL};
  m.t1 = (cx *)calloc((size_t)d, sizeof(cx));
  m.t2 = (cx *)calloc((size_t)d, sizeof(cx));
  double *y = (double *)calloc((size_t)n, sizeof(double));
  double *ynew = (double *)calloc((size_t)n, sizeof(double));
  double *ytry = (double *)calloc((size_t)n, sizeof(double));
  double *p = (double *)calloc((size_t)(nc > 0 ? nc : 1), sizeof(double));
  dp45 s;
  int rc = dp45_init(&s, mc_rhs, &m, n, rtol, atol);
  if (!m.t1 || !m.t2 || !y || !ynew || !ytry || !p || rc != OR_OK) { rc = OR_ENOMEM; goto done; }

  /* psi(0), normalised (Qobj.unit()). */
  double nrm0 = 0.0;
  for (int i = 0; i < d; ++i) nrm0 += psi0[i].re * psi0[i].re + psi0[i].im * psi0[i].im;
  if (!(nrm0 > 0.0)) { rc = OR_ENORM; goto done; }
  nrm0 = sqrt(nrm0);
  for (int i = 0; i < d; ++i) { y[2 * i] = psi0[i].re / nrm0; y[2 * i + 1] = psi0[i].im / nrm0; }

  int64_t jk = 0;                           /* jumps so far       */
  double r = or_uniform(seed, (uint64_t)j, 0, 0); /* step I          */
  double t = tlist[0];
  {
    double nn = sq_norm(y, n);
    for (int q = 0; q < ne; ++q)
      traj_expect[q] = c_scale(ket_expect(&e[q], (const cx *)y, m.t1), 1.0 / nn);
  }
  if (nt == 1) { rc = OR_OK; goto done; }

  dp45_eval(&s, t, y, s.k[0]);
  double hprop = (h0 > 0.0) ? h0 : dp45_initial_step(&s, t, y);
  int after_reject = 0;
  for (int kk = 1; kk < nt; ++kk) {
    double tk = tlist[kk];
    int64_t attempts = 0;
    while (t < tk) {
      if (attempts++ >= max_steps) { rc = OR_ESTEP; goto done; }
      int clipped = hprop >= tk - t;
      double h = clipped ? tk - t : hprop;
      if (!clipped && h < dp45_hmin(t, tk)) { rc = OR_ESTEP; goto done; }
      double err = dp45_step(&s, t, h, y, ynew, 1);
      if (!isfinite(err)) { rc = OR_ENUMERIC; goto done; }
      if (err > 1.0) {
        hprop = dp45_control(h, err, 0, after_reject, clipped, hprop);
        after_reject = 1;
        st->rejected++;
        continue;
      }
      hprop = dp45_control(h, err, 1, after_reject, clipped, hprop);
      after_reject = 0;
      st->accepted++;
      double tnew = clipped ? tk : t + h;
      double nn = sq_norm(ynew, n);
      if (!isfinite(nn)) { rc = OR_ENUMERIC; goto done; }
      if (nn > r) {  /* no jump in (t, tnew] */
        memcpy(y, ynew, sizeof(double) * (size_t)n);
        double *sw = s.k[0]; s.k[0] = s.k[6]; s.k[6] = sw;
        t = tnew;
        continue;
      }
      /* Step II: bisection for <psi(tau)|psi(tau)> = r on (t, tnew] (R4).
       * k[0] still holds f(t, y) for the accepted state (t, y). */
      double lo = t, hi = tnew;
      memcpy(ytry, ynew, sizeof(double) * (size_t)n); /* psi(hi) */
      double tol = bisect_tol * fmax(1.0, fabs(t));
      for (int it = 0; it < 64 && hi - lo > tol; ++it) {
        double mid = lo + 0.5 * (hi - lo);
        dp45_step(&s, t, mid - t, y, ynew, 0);
        st->bisect_iters++;
        if (sq_norm(ynew, n) <= r) { hi = mid; memcpy(ytry, ynew, sizeof(double) * (size_t)n); }
        else lo = mid;
      }
      double tau = hi;
      /* Step III: channel probabilities P_i proportional to <psi|C_i^dag C_i|psi>
       * = ||C_i psi||^2 (Eq. (pcn)), with a fresh uniform r2 (R5). */
      double psum = 0.0;
      for (int q = 0; q < nc; ++q) {
        csr_matvec(&c[q], (const cx *)ytry, m.t1);
        double pq = 0.0;
        for (int i = 0; i < d; ++i) pq += m.t1[i].re * m.t1[i].re + m.t1[i].im * m.t1[i].im;
        p[q] = pq;
        psum += pq;
      }
      if (!(psum > 0.0) || !isfinite(psum)) { rc = OR_ENUMERIC; goto done; }
      double r2 = or_uniform(seed, (uint64_t)j, (uint64_t)jk, 1);
      double target = r2 * psum;
      int chosen = -1;
      int degenerate = 0;
      double cum = 0.0;
      for (int q = 0; q < nc; ++q) {
        cum += p[q];
        if (fabs(cum - target) < 1e-5 * psum) degenerate = 1;
        if (chosen < 0 && cum >= target) chosen = q;
      }
      if (chosen < 0) { /* round-off left the last partial sum below target */
        for (int q = nc - 1; q >= 0; --q) if (p[q] > 0.0) { chosen = q; break; }
      }
      /* a jump this close to an output time may fall on the other side of it
       * in another precision (flag only) */
      double tscale = 1e-5 * fmax(1.0, fabs(tau));
      if (fabs(tau - tlist[kk - 1]) < tscale || fabs(tau - tk) < tscale) degenerate |= 2;
      /* Eq. (project): psi <- C_n psi / ||C_n psi||. */
      csr_matvec(&c[chosen], (const cx *)ytry, m.t1);
      double inv = 1.0 / sqrt(p[chosen]);
      for (int i = 0; i < d; ++i) { y[2 * i] = m.t1[i].re * inv; y[2 * i + 1] = m.t1[i].im * inv; }
      or_jump rec = {j, jk, chosen, tau, degenerate};
      if (jl_push(jl, rec) != OR_OK) { rc = OR_ENOMEM; goto done; }
      st->jumps++;
      /* Step IV: new threshold, restart from (tau, psi). */
      jk++;
      r = or_uniform(seed, (uint64_t)j, (uint64_t)jk, 0);
      t = tau;
      dp45_eval(&s, t, y, s.k[0]);
    }
    double nn = sq_norm(y, n);
    for (int q = 0; q < ne; ++q)
      traj_expect[(size_t)kk * ne + q] = c_scale(ket_expect(&e[q], (const cx *)y, m.t1), 1.0 / nn);
  }
  rc = OR_OK;
done:
  st->rhs_evals += s.rhs_evals;
  dp45_free(&s);
  free(m.t1); free(m.t2); free(y); free(ynew); free(ytry); free(p);
  return rc;
}

/*
 * Trajectories traj_begin .. traj_end-1 (global indices; the random stream
 * depends only on the global index, so any split of the range gives the same
 * records).  traj_expect: [(j - traj_begin) * nt * ne + k * ne + m].
 * Jump records are returned in (trajectory, jump index) order; *n_jumps is
 * the total count even when it exceeds jump_cap (then OR_ECAP).
 * nthreads > 1 runs trajectories on OpenMP threads (timing only; the result
 * does not depend on it).
 */
int or_mcsolve(int d, const csr *H, const csr *c, int nc, const csr *e, int ne,
               const cx *psi0, const double *tlist, int nt, int64_t traj_begin,
               int64_t traj_end, uint64_t seed, double rtol, double atol, double h0,
               int64_t max_steps, double bisect_tol, cx *traj_expect, or_jump *jumps,
               int64_t jump_cap, int64_t *n_jumps, or_stats *stats, int nthreads) {
  if (d <= 0 || nt <= 0 || traj_end < traj_begin) return OR_EINVAL;
  int64_t ntr = traj_end - traj_begin;
  jump_list *lists = (jump_list *)calloc((size_t)(ntr > 0 ? ntr : 1), sizeof(jump_list));
  or_stats *sts = (or_stats *)calloc((size_t)(ntr > 0 ? ntr : 1), sizeof(or_stats));
  int *rcs = (int *)calloc((size_t)(ntr > 0 ? ntr : 1), sizeof(int));
  if (!lists || !sts || !rcs) { free(lists); free(sts); free(rcs); return OR_ENOMEM; }
#ifdef _OPENMP
  if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#else
  (void)nthreads;
#endif
  for (int64_t q = 0; q < ntr; ++q) {
    rcs[q] = mc_trajectory(d, H, c, nc, e, ne, psi0, tlist, nt, traj_begin + q, seed, rtol,
                           atol, h0, max_steps, bisect_tol,
                           traj_expect + (size_t)q * nt * ne, &lists[q], &sts[q]);
  }
  int rc = OR_OK;
  int64_t total = 0;
  or_stats agg = {0, 0, 0, 0, 0};
  for (int64_t q = 0; q < ntr; ++q) {
    if (rcs[q] != OR_OK && rc == OR_OK) rc = rcs[q];
    for (int64_t i = 0; i < lists[q].n; ++i) {
      if (total < jump_cap && jumps) jumps[total] = lists[q].rec[i];
      total++;
    }
    agg.accepted += sts[q].accepted; agg.rejected += sts[q].rejected;
    agg.rhs_evals += sts[q].rhs_evals; agg.bisect_iters += sts[q].bisect_iters;
    agg.jumps += sts[q].jumps;
    free(lists[q].rec);
  }
  if (n_jumps) *n_jumps = total;
  if (stats) *stats = agg;
  if (rc == OR_OK && total > jump_cap) rc = OR_ECAP;
  free(lists); free(sts); free(rcs);
  return rc;
}

/* ------------------------------------------------ pieces for the tests */

/* One Dormand-Prince step of the linear ODE dy/dt = -i H_eff y, exposed so a
 * test can check the method's order against the exact exponential. */
int or_mc_dp45_step(int d, const csr *H, const csr *c, int nc, const cx *psi, double h,
                    cx *out) {
  mc_ctx m = {d, H, c, nc, NULL, NULL};
  m.t1 = (cx *)calloc((size_t)d, sizeof(cx));
  m.t2 = (cx *)calloc((size_t)d, sizeof(cx));
  dp45 s;
  int rc = dp45_init(&s, mc_rhs, &m, 2 * (int64_t)d, 1e-6, 1e-8);
  if (rc == OR_OK && m.t1 && m.t2) {
    dp45_eval(&s, 0.0, (const double *)psi, s.k[0]);
    dp45_step(&s, 0.0, h, (const double *)psi, (double *)out, 0);
  } else {
    rc = OR_ENOMEM;
  }
  dp45_free(&s);
  free(m.t1); free(m.t2);
  return rc;
}

/* d psi/dt for the MC equation of motion (Eq. (heff)), for the tests. */
void or_mc_rhs(int d, const csr *H, const csr *c, int nc, const cx *psi, cx *out) {
  cx *t1 = (cx *)calloc((size_t)d, sizeof(cx));
  cx *t2 = (cx *)calloc((size_t)d, sizeof(cx));
  mc_ctx m = {d, H, c, nc, t1, t2};
  mc_rhs(&m, 0.0, (const double *)psi, (double *)out);
  free(t1); free(t2);
}

/* drho/dt of Eq. (master_equation), allocating its own scratch. */
void or_me_rhs(int d, const csr *H, const csr *c, int nc, const cx *rho, cx *out) {
  size_t nn = (size_t)d * d;
  cx *t1 = (cx *)calloc(nn, sizeof(cx));
  cx *t2 = (cx *)calloc(nn, sizeof(cx));
  cx *t3 = (cx *)calloc(nn, sizeof(cx));
  or_lindblad_rhs(d, H, c, nc, rho, out, t1, t2, t3);
  free(t1); free(t2); free(t3);
}

int or_has_openmp(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 0;
#endif
}
