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
 *   R8  A time-dependent Hamiltonian (section 4.3 passes H(t) as a callback)
 *       is given as H(t) = H + sum_k f_k(t) H_k with real coefficients f_k
 *       that are piecewise linear between knots (t_ki, v_ki) and constant
 *       before the first and after the last knot; every stage of a step sees
 *       H at its own stage time.  The collapse operators do not depend on t.
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

/* ---------------------------------- time-dependent Hamiltonian terms, R8 */

typedef struct {
  int n;              /* number of terms H_k                          */
  const csr *H;       /* the operators H_k                            */
  const int64_t *off; /* knots of term k: off[k] .. off[k+1] - 1      */
  const double *t;    /* knot times, strictly increasing within a term */
  const double *v;    /* knot values                                  */
} or_td;

/* f_k(t): linear between neighbouring knots, the end value outside. */
double or_td_coef(const or_td *td, int k, double t) {
  int64_t a = td->off[k], b = td->off[k + 1] - 1;
  if (t <= td->t[a]) return td->v[a];
  if (t >= td->t[b]) return td->v[b];
  int64_t i = a;
  while (td->t[i + 1] < t) ++i;
  double w = (t - td->t[i]) / (td->t[i + 1] - td->t[i]);
  return td->v[i] + w * (td->v[i + 1] - td->v[i]);
}

/* ------------------------------------------- Lindblad right-hand side */

typedef struct {
  int d;
  const csr *H;
  const csr *c;
  int nc;
  cx *t1, *t2, *t3; /* d*d scratch each */
  const or_td *td;  /* time-dependent terms (NULL: none) */
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

/* The terms -i f_k(t) [H_k, rho] of H(t) (R8), added to drho. */
static void td_commutators(int d, const or_td *td, double t, const cx *rho, cx *drho,
                           cx *t1, cx *t2) {
  size_t n = (size_t)d * d;
  for (int k = 0; td && k < td->n; ++k) {
    double f = or_td_coef(td, k, t);
    csr_left(&td->H[k], rho, t1);
    csr_right(rho, &td->H[k], t2);
    for (size_t q = 0; q < n; ++q) {
      cx comm = {t1[q].re - t2[q].re, t1[q].im - t2[q].im};
      drho[q].re += f * comm.im;
      drho[q].im -= f * comm.re;
    }
  }
}

static void me_rhs(void *vctx, double t, const double *y, double *dy) {
  me_ctx *m = (me_ctx *)vctx;
  or_lindblad_rhs(m->d, m->H, m->c, m->nc, (const cx *)y, (cx *)dy, m->t1, m->t2, m->t3);
  td_commutators(m->d, m->td, t, (const cx *)y, (cx *)dy, m->t1, m->t2);
}

/* --------------------------------------- non-Hermitian Schrodinger RHS */

typedef struct {
  int d;
  const csr *H;
  const csr *c;
  int nc;
  cx *t1, *t2; /* d scratch each */
  const or_td *td; /* time-dependent terms (NULL: none) */
} mc_ctx;

/*
 * d psi/dt = -i H_eff psi with Eq. (heff), hbar = 1:
 *   H_eff = H - (i/2) sum_n C_n^dag C_n,
 * so -i H_eff psi = -i H psi - 1/2 sum_n C_n^dag (C_n psi).
 */
static void mc_rhs(void *vctx, double t, const double *y, double *dy) {
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
  /* -i f_k(t) H_k psi for the time-dependent terms (R8) */
  for (int k = 0; m->td && k < m->td->n; ++k) {
    double f = or_td_coef(m->td, k, t);
    csr_matvec(&m->td->H[k], psi, m->t1);
    for (int i = 0; i < m->d; ++i) {
      out[i].re += f * m->t1[i].im;
      out[i].im -= f * m->t1[i].re;
    }
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
               or_stats *stats, const or_td *td) {
  if (d <= 0 || nt <= 0) return OR_EINVAL;
  size_t nn = (size_t)d * d;
  me_ctx m = {d, H, c, nc, NULL, NULL, NULL, td};
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
                         jump_list *jl, or_stats *st, const or_td *td) {
  int64_t n = 2 * (int64_t)d;
  mc_ctx m = {d, H, c, nc, NULL, NULL, td};
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
      double tscale = 4e-6 * fmax(1.0, fabs(tau));
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
               int64_t jump_cap, int64_t *n_jumps, or_stats *stats, int nthreads,
               const or_td *td) {
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
                           traj_expect + (size_t)q * nt * ne, &lists[q], &sts[q], td);
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
  mc_ctx m = {d, H, c, nc, NULL, NULL, NULL};
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
  mc_ctx m = {d, H, c, nc, t1, t2, NULL};
  mc_rhs(&m, 0.0, (const double *)psi, (double *)out);
  free(t1); free(t2);
}

/* -i H_eff(t) psi with the time-dependent terms td at time t (R8). */
void or_mc_rhs_td(int d, const csr *H, const csr *c, int nc, const or_td *td, double t,
                  const cx *psi, cx *out) {
  cx *t1 = (cx *)calloc((size_t)d, sizeof(cx));
  cx *t2 = (cx *)calloc((size_t)d, sizeof(cx));
  mc_ctx m = {d, H, c, nc, t1, t2, td};
  mc_rhs(&m, t, (const double *)psi, (double *)out);
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

/* Eq. (master_equation) with H(t) = H + sum_k f_k(t) H_k at time t (R8). */
void or_me_rhs_td(int d, const csr *H, const csr *c, int nc, const or_td *td, double t,
                  const cx *rho, cx *out) {
  size_t nn = (size_t)d * d;
  cx *t1 = (cx *)calloc(nn, sizeof(cx));
  cx *t2 = (cx *)calloc(nn, sizeof(cx));
  cx *t3 = (cx *)calloc(nn, sizeof(cx));
  me_ctx m = {d, H, c, nc, t1, t2, t3, td};
  me_rhs(&m, t, (const double *)rho, (double *)out);
  free(t1); free(t2); free(t3);
}

int or_has_openmp(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 0;
#endif
}

/* ------------------------------------------- adjoint of the master equation */
/*
 * Differentiable master equation (an extension beyond the paper: gradients of
 * a loss of the solution of Eq. (master_equation) with respect to drive
 * amplitudes and decay rates).  The generator is
 *   F(rho) = -i [H0 + Omega_s Hd, rho]
 *            + sum_k gamma_k (A_k rho A_k^dag - 1/2 {A_k^dag A_k, rho}),
 * with Omega_s constant on segment s = [s T_seg, (s+1) T_seg).  The loss is
 *   L = Re Tr(P1 rho(T)) + Re q(T),   dq/dt = Tr(P2 rho),
 * q integrated by the same Runge-Kutta stages as rho.  On a frozen step grid
 * the solution is a smooth function of the parameters; the gradient is the
 * exact derivative of that discrete map (discrete adjoint): for a step with
 * stage inputs Y_l, weights b_l and coefficients a_lj,
 *   nu_i  = h b_i lambda_{n+1} + sum_{l>i} h a_li mu_l,
 *   mu_l  = F^dag(nu_l) + h b_l P2,
 *   lambda_n = lambda_{n+1} + sum_l mu_l,   lambda_N = P1,
 *   dL/dtheta += sum_l Re <nu_l, (dF/dtheta)(Y_l)>,   <X, Y> = Tr(X^dag Y),
 * with F^dag(X) = i [H, X] + sum_k gamma_k (A^dag X A - 1/2 {A^dag A, X}).
 */

typedef struct {
  int d;
  const csr *H0, *Hd, *A, *P1, *P2;
  int nk;
  cx *t1, *t2, *t3, *n;  /* d*d scratch */
} adj_sys;

/* out = -i s [H, M] + out   (s = +1 for F, -1 for F^dag) */
static void adj_comm_acc(adj_sys *S, const csr *H, double scale, double sign, const cx *M, cx *out) {
  size_t nn = (size_t)S->d * S->d;
  csr_left(H, M, S->t1);
  csr_right(M, H, S->t2);
  for (size_t q = 0; q < nn; ++q) {
    cx c = {S->t1[q].re - S->t2[q].re, S->t1[q].im - S->t2[q].im};
    /* -i sign scale c */
    out[q].re += sign * scale * c.im;
    out[q].im += -sign * scale * c.re;
  }
}

/* out += g (A M A^dag - 1/2 A^dag A M - 1/2 M A^dag A)  (dagger = 0), or
 * out += g (A^dag M A - 1/2 A^dag A M - 1/2 M A^dag A)  (dagger = 1). */
static void adj_diss_acc(adj_sys *S, const csr *A, double g, int dagger, const cx *M, cx *out) {
  size_t nn = (size_t)S->d * S->d;
  if (!dagger) {
    csr_left(A, M, S->t1);          /* A M          */
    csr_right_dag(S->t1, A, S->t2); /* A M A^dag    */
  } else {
    csr_left_dag(A, M, S->t1);      /* A^dag M      */
    csr_right(S->t1, A, S->t2);     /* A^dag M A    */
  }
  for (size_t q = 0; q < nn; ++q) { out[q].re += g * S->t2[q].re; out[q].im += g * S->t2[q].im; }
  csr_left(A, M, S->t1);            /* A M          */
  csr_left_dag(A, S->t1, S->t2);    /* A^dag A M    */
  csr_right_dag(M, A, S->t1);       /* M A^dag      */
  csr_right(S->t1, A, S->t3);       /* M A^dag A    */
  for (size_t q = 0; q < nn; ++q) {
    out[q].re -= 0.5 * g * (S->t2[q].re + S->t3[q].re);
    out[q].im -= 0.5 * g * (S->t2[q].im + S->t3[q].im);
  }
}

static void adj_F(adj_sys *S, double omega, const double *gam, int dagger, const cx *M, cx *out) {
  memset(out, 0, sizeof(cx) * (size_t)S->d * S->d);
  double sign = dagger ? -1.0 : 1.0;
  adj_comm_acc(S, S->H0, 1.0, sign, M, out);
  adj_comm_acc(S, S->Hd, omega, sign, M, out);
  for (int k = 0; k < S->nk; ++k) adj_diss_acc(S, &S->A[k], gam[k], dagger, M, out);
}

static cx adj_trace(const csr *P, const cx *M) {
  int d = P->d;
  cx acc = {0.0, 0.0};
  for (int i = 0; i < d; ++i)
    for (int64_t p = P->indptr[i]; p < P->indptr[i + 1]; ++p)
      acc = c_add(acc, c_mul(P->values[p], M[(size_t)P->indices[p] * d + i]));
  return acc;
}

/* Re <X, Y> = Re sum conj(X) Y */
static double adj_inner(const cx *X, const cx *Y, size_t nn) {
  double s = 0.0;
  for (size_t q = 0; q < nn; ++q) s += X[q].re * Y[q].re + X[q].im * Y[q].im;
  return s;
}

/* One Dormand-Prince step of the pair (rho, q) from rho with k[0] = F(rho)
 * given; fills Y[0..5] (stage inputs; Y[0] = rho), k[1..5] (and k[6] =
 * F(rho_new) with the error norm when want_err), rho_new and the increment of
 * q.  Returns the error norm (0 when !want_err). */
static double adj_step(adj_sys *S, double omega, const double *gam, double h, const cx *rho,
                       cx **k, cx **Y, cx *rho_new, cx *dq, int want_err, double rtol, double atol) {
  size_t nn = (size_t)S->d * S->d;
  memcpy(Y[0], rho, sizeof(cx) * nn);
  for (int st = 1; st < 6; ++st) {
    for (size_t q = 0; q < nn; ++q) {
      double ar = 0.0, ai = 0.0;
      for (int j = 0; j < st; ++j) { ar += DP_A[st][j] * k[j][q].re; ai += DP_A[st][j] * k[j][q].im; }
      Y[st][q].re = rho[q].re + h * ar;
      Y[st][q].im = rho[q].im + h * ai;
    }
    adj_F(S, omega, gam, 0, Y[st], k[st]);
  }
  for (size_t q = 0; q < nn; ++q) {
    double ar = 0.0, ai = 0.0;
    for (int j = 0; j < 6; ++j) { ar += DP_B5[j] * k[j][q].re; ai += DP_B5[j] * k[j][q].im; }
    rho_new[q].re = rho[q].re + h * ar;
    rho_new[q].im = rho[q].im + h * ai;
  }
  cx acc = {0.0, 0.0};
  for (int j = 0; j < 6; ++j) acc = c_add(acc, c_scale(adj_trace(S->P2, Y[j]), DP_B5[j]));
  *dq = c_scale(acc, h);
  if (!want_err) return 0.0;
  adj_F(S, omega, gam, 0, rho_new, k[6]);
  double sum = 0.0;
  const double *y0 = (const double *)rho, *y1 = (const double *)rho_new;
  for (size_t q = 0; q < 2 * nn; ++q) {
    double e = 0.0;
    for (int j = 0; j < 7; ++j) e += (DP_B5[j] - DP_B4[j]) * ((const double *)k[j])[q];
    e *= h;
    double sc = atol + rtol * fmax(fabs(y0[q]), fabs(y1[q]));
    sum += (e / sc) * (e / sc);
  }
  return sqrt(sum / (double)(2 * nn));
}

typedef struct {
  cx *k[7], *Y[6], *rho, *rho_new;
} adj_work;

static int adj_work_alloc(adj_work *w, int d) {
  size_t nn = (size_t)d * d;
  for (int i = 0; i < 7; ++i) if (!(w->k[i] = (cx *)calloc(nn, sizeof(cx)))) return OR_ENOMEM;
  for (int i = 0; i < 6; ++i) if (!(w->Y[i] = (cx *)calloc(nn, sizeof(cx)))) return OR_ENOMEM;
  if (!(w->rho = (cx *)calloc(nn, sizeof(cx))) || !(w->rho_new = (cx *)calloc(nn, sizeof(cx))))
    return OR_ENOMEM;
  return OR_OK;
}
static void adj_work_free(adj_work *w) {
  for (int i = 0; i < 7; ++i) free(w->k[i]);
  for (int i = 0; i < 6; ++i) free(w->Y[i]);
  free(w->rho); free(w->rho_new);
}

static int adj_sys_init(adj_sys *S, int d, const csr *H0, const csr *Hd, const csr *A, int nk,
                        const csr *P1, const csr *P2) {
  size_t nn = (size_t)d * d;
  S->d = d; S->H0 = H0; S->Hd = Hd; S->A = A; S->nk = nk; S->P1 = P1; S->P2 = P2;
  S->t1 = (cx *)calloc(nn, sizeof(cx)); S->t2 = (cx *)calloc(nn, sizeof(cx));
  S->t3 = (cx *)calloc(nn, sizeof(cx)); S->n = (cx *)calloc(nn, sizeof(cx));
  return (S->t1 && S->t2 && S->t3 && S->n) ? OR_OK : OR_ENOMEM;
}
static void adj_sys_free(adj_sys *S) { free(S->t1); free(S->t2); free(S->t3); free(S->n); }

/*
 * Adaptive forward solve from rho0 over n_seg segments of length t_seg with
 * the controller of the solvers above (segment ends are output times).
 * Records the accepted step lengths: nsteps[s] steps of segment s in
 * hgrid[s * max_per_seg ...].  Returns the loss in *loss.
 */
int or_adjoint_forward(int d, const csr *H0, const csr *Hd, const csr *A, int nk, const csr *P1,
                       const csr *P2, const cx *rho0, int n_seg, double t_seg,
                       const double *omega, const double *gam, double rtol, double atol,
                       int max_per_seg, int *nsteps, double *hgrid, double *loss) {
  adj_sys S;
  adj_work w;
  int rc = adj_sys_init(&S, d, H0, Hd, A, nk, P1, P2);
  if (rc == OR_OK) rc = adj_work_alloc(&w, d);
  if (rc != OR_OK) { adj_sys_free(&S); return rc; }
  size_t nn = (size_t)d * d;
  memcpy(w.rho, rho0, sizeof(cx) * nn);
  cx q = {0.0, 0.0};
  double hprop = 0.0;
  int after_reject = 0;
  for (int s = 0; s < n_seg && rc == OR_OK; ++s) {
    double t = 0.0;  /* time within the segment */
    nsteps[s] = 0;
    adj_F(&S, omega[s], gam, 0, w.rho, w.k[0]);
    if (s == 0) {
      /* starting step: Hairer-Norsett-Wanner with the generator of segment 0 */
      double s0 = 0.0, s1 = 0.0, s2 = 0.0;
      const double *y = (const double *)w.rho, *f = (const double *)w.k[0];
      for (size_t i = 0; i < 2 * nn; ++i) {
        double sc = atol + rtol * fabs(y[i]);
        s0 += (y[i] / sc) * (y[i] / sc);
        s1 += (f[i] / sc) * (f[i] / sc);
      }
      double d0 = sqrt(s0 / (2.0 * nn)), d1 = sqrt(s1 / (2.0 * nn));
      double h0 = (d0 < 1e-5 || d1 < 1e-5) ? 1e-6 : 0.01 * d0 / d1;
      for (size_t i = 0; i < nn; ++i) {
        w.rho_new[i].re = w.rho[i].re + h0 * w.k[0][i].re;
        w.rho_new[i].im = w.rho[i].im + h0 * w.k[0][i].im;
      }
      adj_F(&S, omega[s], gam, 0, w.rho_new, w.k[1]);
      const double *f1 = (const double *)w.k[1];
      for (size_t i = 0; i < 2 * nn; ++i) {
        double sc = atol + rtol * fabs(y[i]);
        double e = (f1[i] - f[i]) / sc;
        s2 += e * e;
      }
      double d2 = sqrt(s2 / (2.0 * nn)) / h0;
      double dm = fmax(d1, d2);
      double h1 = (dm <= 1e-15) ? fmax(1e-6, h0 * 1e-3) : pow(0.01 / dm, 0.2);
      hprop = fmin(100.0 * h0, h1);
    }
    int64_t attempts = 0;
    while (t < t_seg) {
      if (attempts++ >= 1000000) { rc = OR_ESTEP; break; }
      int clipped = hprop >= t_seg - t;
      double h = clipped ? t_seg - t : hprop;
      cx dq;
      double err = adj_step(&S, omega[s], gam, h, w.rho, w.k, w.Y, w.rho_new, &dq, 1, rtol, atol);
      if (!isfinite(err)) { rc = OR_ENUMERIC; break; }
      if (err <= 1.0) {
        hprop = dp45_control(h, err, 1, after_reject, clipped, hprop);
        after_reject = 0;
        if (nsteps[s] >= max_per_seg) { rc = OR_ESTEP; break; }
        hgrid[(size_t)s * max_per_seg + nsteps[s]++] = h;
        t = clipped ? t_seg : t + h;
        memcpy(w.rho, w.rho_new, sizeof(cx) * nn);
        q = c_add(q, dq);
        cx *sw = w.k[0]; w.k[0] = w.k[6]; w.k[6] = sw;
      } else {
        hprop = dp45_control(h, err, 0, after_reject, clipped, hprop);
        after_reject = 1;
      }
    }
  }
  if (rc == OR_OK) *loss = adj_trace(P1, w.rho).re + q.re;
  adj_work_free(&w);
  adj_sys_free(&S);
  return rc;
}

/* Loss on a fixed step grid (for finite differences). */
int or_adjoint_loss_fixed(int d, const csr *H0, const csr *Hd, const csr *A, int nk,
                          const csr *P1, const csr *P2, const cx *rho0, int n_seg,
                          const double *omega, const double *gam, int max_per_seg,
                          const int *nsteps, const double *hgrid, double *loss) {
  adj_sys S;
  adj_work w;
  int rc = adj_sys_init(&S, d, H0, Hd, A, nk, P1, P2);
  if (rc == OR_OK) rc = adj_work_alloc(&w, d);
  if (rc != OR_OK) { adj_sys_free(&S); return rc; }
  size_t nn = (size_t)d * d;
  memcpy(w.rho, rho0, sizeof(cx) * nn);
  cx q = {0.0, 0.0};
  for (int s = 0; s < n_seg; ++s) {
    for (int n = 0; n < nsteps[s]; ++n) {
      cx dq;
      adj_F(&S, omega[s], gam, 0, w.rho, w.k[0]);
      adj_step(&S, omega[s], gam, hgrid[(size_t)s * max_per_seg + n], w.rho, w.k, w.Y, w.rho_new,
               &dq, 0, 0.0, 0.0);
      memcpy(w.rho, w.rho_new, sizeof(cx) * nn);
      q = c_add(q, dq);
    }
  }
  *loss = adj_trace(P1, w.rho).re + q.re;
  adj_work_free(&w);
  adj_sys_free(&S);
  return OR_OK;
}

/* Gradient of the fixed-grid loss with respect to omega[n_seg] and gam[nk]
 * by the discrete adjoint (all states of the forward pass kept). */
int or_adjoint_grad(int d, const csr *H0, const csr *Hd, const csr *A, int nk, const csr *P1,
                    const csr *P2, const cx *rho0, int n_seg, const double *omega,
                    const double *gam, int max_per_seg, const int *nsteps, const double *hgrid,
                    double *loss, double *g_omega, double *g_gam) {
  adj_sys S;
  adj_work w;
  int rc = adj_sys_init(&S, d, H0, Hd, A, nk, P1, P2);
  if (rc == OR_OK) rc = adj_work_alloc(&w, d);
  if (rc != OR_OK) { adj_sys_free(&S); return rc; }
  size_t nn = (size_t)d * d;
  int64_t total = 0;
  for (int s = 0; s < n_seg; ++s) total += nsteps[s];
  cx *states = (cx *)calloc((size_t)(total + 1) * nn, sizeof(cx));
  cx *lam = (cx *)calloc(nn, sizeof(cx));
  cx *nu[6], *mu[6], *tmp = (cx *)calloc(nn, sizeof(cx));
  for (int i = 0; i < 6; ++i) { nu[i] = (cx *)calloc(nn, sizeof(cx)); mu[i] = (cx *)calloc(nn, sizeof(cx)); }
  if (!states || !lam || !tmp) { rc = OR_ENOMEM; goto out; }
  /* forward, keeping every state */
  memcpy(states, rho0, sizeof(cx) * nn);
  cx q = {0.0, 0.0};
  int64_t idx = 0;
  for (int s = 0; s < n_seg; ++s)
    for (int n = 0; n < nsteps[s]; ++n, ++idx) {
      cx dq;
      adj_F(&S, omega[s], gam, 0, states + idx * nn, w.k[0]);
      adj_step(&S, omega[s], gam, hgrid[(size_t)s * max_per_seg + n], states + idx * nn, w.k, w.Y,
               states + (idx + 1) * nn, &dq, 0, 0.0, 0.0);
      q = c_add(q, dq);
    }
  *loss = adj_trace(P1, states + total * nn).re + q.re;
  /* lambda_N = P1 (dense) */
  memset(lam, 0, sizeof(cx) * nn);
  for (int i = 0; i < d; ++i)
    for (int64_t p = P1->indptr[i]; p < P1->indptr[i + 1]; ++p)
      lam[(size_t)i * d + P1->indices[p]] = P1->values[p];
  for (int s = 0; s < n_seg; ++s) g_omega[s] = 0.0;
  for (int k = 0; k < nk; ++k) g_gam[k] = 0.0;
  idx = total;
  for (int s = n_seg - 1; s >= 0; --s)
    for (int n = nsteps[s] - 1; n >= 0; --n) {
      --idx;
      double h = hgrid[(size_t)s * max_per_seg + n];
      cx dq;
      /* recompute the stage inputs of this step */
      adj_F(&S, omega[s], gam, 0, states + idx * nn, w.k[0]);
      adj_step(&S, omega[s], gam, h, states + idx * nn, w.k, w.Y, w.rho_new, &dq, 0, 0.0, 0.0);
      /* stages backward */
      for (int i = 5; i >= 0; --i) {
        for (size_t qq = 0; qq < nn; ++qq) {
          double ar = h * DP_B5[i] * lam[qq].re, ai = h * DP_B5[i] * lam[qq].im;
          for (int l = i + 1; l < 6; ++l) {
            ar += h * DP_A[l][i] * mu[l][qq].re;
            ai += h * DP_A[l][i] * mu[l][qq].im;
          }
          nu[i][qq].re = ar;
          nu[i][qq].im = ai;
        }
        adj_F(&S, omega[s], gam, 1, nu[i], mu[i]);
        /* + h b_i P2 */
        for (int r = 0; r < d; ++r)
          for (int64_t p = P2->indptr[r]; p < P2->indptr[r + 1]; ++p) {
            size_t qq = (size_t)r * d + P2->indices[p];
            mu[i][qq].re += h * DP_B5[i] * P2->values[p].re;
            mu[i][qq].im += h * DP_B5[i] * P2->values[p].im;
          }
        /* parameter derivatives at Y_i */
        memset(tmp, 0, sizeof(cx) * nn);
        adj_comm_acc(&S, S.Hd, 1.0, 1.0, w.Y[i], tmp);
        g_omega[s] += adj_inner(nu[i], tmp, nn);
        for (int k = 0; k < nk; ++k) {
          memset(tmp, 0, sizeof(cx) * nn);
          adj_diss_acc(&S, &A[k], 1.0, 0, w.Y[i], tmp);
          g_gam[k] += adj_inner(nu[i], tmp, nn);
        }
      }
      for (size_t qq = 0; qq < nn; ++qq)
        for (int l = 0; l < 6; ++l) { lam[qq].re += mu[l][qq].re; lam[qq].im += mu[l][qq].im; }
    }
out:
  for (int i = 0; i < 6; ++i) { free(nu[i]); free(mu[i]); }
  free(states); free(lam); free(tmp);
  adj_work_free(&w);
  adj_sys_free(&S);
  return rc;
}
