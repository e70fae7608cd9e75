/*
 * qt.h -- C ABI of libqt, a CUDA (sm_103a) library for the two open-system
 * solvers of Johansson, Nation & Nori, "QuTiP: An open-source Python
 * framework for the dynamics of open quantum systems" (QuTiP 1.1.3):
 *
 *   qt_mesolve  the Lindblad master equation, paper section 3.1,
 *               Eq. (master_equation), integrated in time (the paper's
 *               odesolve);
 *   qt_mcsolve  the Monte-Carlo wave-function method, paper section 3.2:
 *               Eq. (heff), Eq. (jump), Eq. (project), Eq. (pcn) and the
 *               four-step algorithm I-IV with Eq. (mc3);
 *   qt_expect   expectation values <psi|O|psi> or Tr(O rho), the paper's
 *               expect() (section 2 and Appendix A).
 *
 * Conventions for every call:
 *   * hbar = 1.  Complex numbers are interleaved (re, im) pairs of doubles
 *     (qt_c128).  Matrices are row-major.
 *   * Calls without a _dev suffix take HOST pointers only.  They copy their
 *     inputs to the GPU, run, copy results back, synchronise, and keep no
 *     pointer after they return.  The caller owns every buffer.
 *   * _dev calls take DEVICE pointers for states, time lists and outputs,
 *     and a CUDA stream (a cudaStream_t passed as void*; NULL = the legacy
 *     default stream).  They only enqueue work and return; results, the
 *     solver statistics and the device-side status word are valid once the
 *     stream has been synchronised.
 *   * Every call returns QT_OK (0) or a negative QT_E* code; the text of the
 *     last error on the calling thread is available from qt_last_error().
 *     Outputs are undefined when a call fails.
 *   * All arithmetic runs in the library's CUDA kernels; there is no CPU
 *     fallback.  Without a usable CUDA device a call returns QT_ENODEV.
 *
 * The integrator is the Dormand-Prince 5(4) pair with the 5th-order solution
 * propagated, the Hairer-Norsett-Wanner starting step, the error norm
 *   err = sqrt(mean_i (E_i / (atol + rtol * max(|y_i|, |ynew_i|)))^2)
 * over all real components, acceptance at err <= 1, step factor
 * min(5, max(0.2, 0.9 err^(-1/5))) (capped at 1 right after a rejection),
 * and steps clipped to land exactly on every output time.  The paper names
 * no integrator (section 3.1); this is the library's reading.
 */
#ifndef QT_H
#define QT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status codes */
#define QT_OK 0
#define QT_EINVAL (-1)    /* null pointer, bad size, shape or index          */
#define QT_ENONHERM (-2)  /* reserved: non-Hermitian operator where required */
#define QT_ENORM (-3)     /* zero-norm initial ket or zero-trace rho0        */
#define QT_ENOMEM (-4)    /* device or host allocation failed                */
#define QT_ECUDA (-5)     /* a CUDA runtime call failed                      */
#define QT_ESTEP (-6)     /* max_steps attempts in one output interval, or
                             the step size fell below 16 eps |t|             */
#define QT_EBISECT (-7)   /* reserved: jump-time search did not converge     */
#define QT_ETIMEOUT (-8)  /* a bounded device wait ran out                   */
#define QT_ENUMERIC (-9)  /* NaN/Inf in the state or error norm, or all
                             collapse weights zero at a detected jump        */
#define QT_ECAP (-10)     /* jump buffer (jump_cap > 0) full: *n_jumps still
                             holds the total count, the first jump_cap are
                             stored; never returned when jump_cap == 0      */
#define QT_ENOTIMPL (-11) /* option combination not built                    */
#define QT_ENODEV (-12)   /* no CUDA device usable by the library            */

/* ------------------------------------------------------------------ types */
typedef struct {
  double re, im;
} qt_c128;

#define QT_DENSE 0 /* values: dim*dim row-major; indptr/indices unused */
#define QT_CSR 1   /* compressed sparse rows                           */

/* A square operator on a Hilbert space of dimension dim (paper section 2:
 * the data of a Qobj).  For QT_CSR: indptr[dim+1] (int64, indptr[0] = 0,
 * non-decreasing, indptr[dim] = nnz), indices[nnz] (int32 column, 0 <= c <
 * dim; duplicates are summed), values[nnz].  Host memory. */
typedef struct {
  int32_t dim;
  int32_t fmt;
  int64_t nnz;
  const int64_t *indptr;
  const int32_t *indices;
  const qt_c128 *values;
} qt_op;

#define QT_FP64 0  /* every vector and scalar in FP64                      */
#define QT_MIXED 1 /* state vectors and stages in complex FP32; FP64 for t,
                      h, the norm-decay comparison, the jump-time search,
                      the collapse weights, renormalisation and expectation
                      accumulation                                          */

/* Integrator and solver options (the paper's Odeoptions, Appendix A).
 * Fill with qt_opts_default() and override fields. */
typedef struct {
  double rtol;       /* relative tolerance (default 1e-8)                  */
  double atol;       /* absolute tolerance (default 1e-10)                 */
  double h0;         /* first step; <= 0 selects it automatically          */
  int64_t max_steps; /* attempted steps allowed per output interval (1e6)  */
  double bisect_tol; /* jump-time search stops when the bracket is below
                        bisect_tol * max(1, |t|) (default 1e-13)           */
  int32_t precision; /* QT_FP64 or QT_MIXED (default QT_FP64)              */
  int32_t traj_block;/* MC: threads per trajectory, 0 = chosen by the
                        library's tuning table (8, 16, 32, ...)            */
  int32_t me_method; /* ME: QT_ME_AUTO (= sparse), QT_ME_SPARSE or
                        QT_ME_DENSE_TC                                     */
  int32_t reserved;
} qt_opts;

/* Master-equation right-hand side (paper Eq. (master_equation) in the
 * effective-Hamiltonian form -i(H_eff rho - rho H_eff^dag) + sum C rho C^dag):
 *   QT_ME_SPARSE    every entry from the ELL rows of H_eff and C_n, in the
 *                   precision of o->precision;
 *   QT_ME_DENSE_TC  H_eff rho as a dense product on the tensor cores (BF16
 *                   hi/lo split operands, FP32 accumulation; relative error
 *                   of the product O(2^-16) of sum |H_eff||rho|), rho H_eff^dag
 *                   as its conjugate transpose (rho is Hermitian), the
 *                   collapse terms from the ELL rows in FP32.  Requires
 *                   precision QT_MIXED (else QT_EINVAL); the first call on a
 *                   system allocates its dense operands (about 16 dp^2 bytes,
 *                   dp = dim rounded up to 128). */
#define QT_ME_AUTO 0
#define QT_ME_SPARSE 1
#define QT_ME_DENSE_TC 2

/* One quantum jump of trajectory traj: the k-th jump (k = 0, 1, ...) at time
 * tau through collapse operator `channel` (0-based index into c_ops).
 * degenerate: bit 0 set when the channel draw lay within 1e-5 * sum_n p_n of
 * a cumulative boundary of Eq. (mc3); bit 1 set when tau lay within
 * 4e-6 * max(1, |tau|) of an output time.  Such events may legitimately
 * resolve differently in another precision. */
typedef struct {
  int64_t traj;
  int64_t k;
  int64_t channel;
  double tau;
  int64_t degenerate;
} qt_jump;

/* Solver statistics (all counts summed over trajectories for MC). */
typedef struct {
  int64_t accepted;     /* accepted Dormand-Prince steps                    */
  int64_t rejected;     /* rejected steps                                    */
  int64_t rhs_evals;    /* right-hand-side evaluations, all causes           */
  int64_t bisect_iters; /* trial steps of the jump-time search               */
  int64_t jumps;        /* quantum jumps                                     */
  int64_t near_miss;    /* MC: trajectories whose final <psi|psi> lay within
                           1e-5 r of their pending threshold r               */
  int32_t status;       /* QT_OK or the first device-side error code        */
  int32_t reserved;
} qt_stats;

/* --------------------------------------------------------------- general */
void qt_opts_default(qt_opts *o);
const char *qt_last_error(void); /* thread-local; "" when none */
const char *qt_version(void);

/* ----------------------------------------------------- host-memory calls */

/*
 * Master equation, paper section 3.1 Eq. (master_equation):
 *   d rho/dt = -i [H, rho] + sum_n (C_n rho C_n^dag - 1/2 {C_n^dag C_n, rho}).
 * state0: a ket (dim) when state_is_ket != 0 -- then rho0 = |psi><psi| /
 * <psi|psi> (paper section 4.1 passes a ket) -- else a density matrix
 * (dim*dim, used as given).  tlist[n_t]: increasing output times; the
 * integration starts at tlist[0].  expect_out[n_t * n_e] (nullable when
 * n_e == 0): Tr(O_m rho(t_k)) at [k * n_e + m].  states_out (nullable):
 * rho(t_k) at [k * dim * dim ...].  stats nullable.
 */
int qt_mesolve(const qt_op *H, const qt_op *c_ops, int n_c, const qt_op *e_ops, int n_e,
               const qt_c128 *state0, int state_is_ket, const double *tlist, int n_t,
               const qt_opts *o, qt_c128 *expect_out, qt_c128 *states_out, qt_stats *stats);

/*
 * Monte-Carlo wave function, paper section 3.2.  Trajectory j (0 <= j <
 * ntraj) starts from psi0 / ||psi0|| and integrates d psi/dt = -i H_eff psi
 * with H_eff = H - (i/2) sum_n C_n^dag C_n (Eq. (heff)).  After every
 * accepted step it compares <psi|psi> with its uniform r (step II); at a
 * crossing it locates the jump time tau by bisection on trial steps from the
 * last accepted state, picks the smallest channel n with
 * sum_{i<=n} p_i >= r2 sum_i p_i, p_i = ||C_i psi(tau)||^2 (Eq. (pcn),
 * (mc3)), applies psi <- C_n psi / sqrt(p_n) (Eq. (project)) and draws new
 * numbers (step IV).  Random numbers: Philox4x32-10 with key = seed and
 * counter = (j, jump index, stream, 0), 52-bit uniforms in (0, 1); stream 0
 * gives r, stream 1 gives r2.  With n_c == 0 a single trajectory is run.
 *
 * expect_out[n_t * n_e]: trajectory mean of <psi|O_m|psi>/<psi|psi>.
 * traj_expect_out (nullable): per trajectory, [(j * n_t + k) * n_e + m].
 * jumps (nullable when jump_cap == 0): records in no particular order;
 * *n_jumps (nullable) receives the total count.
 */
int qt_mcsolve(const qt_op *H, const qt_op *c_ops, int n_c, const qt_op *e_ops, int n_e,
               const qt_c128 *psi0, const double *tlist, int n_t, int64_t ntraj, uint64_t seed,
               const qt_opts *o, qt_c128 *expect_out, qt_c128 *traj_expect_out, qt_jump *jumps,
               int64_t jump_cap, int64_t *n_jumps, qt_stats *stats);

/*
 * Time-dependent Hamiltonians (paper section 4.3, where H(t) is a callback
 * such as H0 + t H1).  A callback cannot run inside GPU kernels, so the time
 * dependence is given as terms: H(t) = H + sum_k f_k(t) H_k with real
 * coefficients f_k that are piecewise linear between knots (times, values)
 * and constant before the first and after the last knot (a two-knot table
 * is an exact linear ramp, e.g. the Landau-Zener sweep of section 4.3).
 * Every Runge-Kutta stage sees H at its own stage time; the collapse
 * operators do not depend on time.  At most 8 terms.  Host memory, copied:
 *   H[n_terms]        the operators H_k (Hermitian)
 *   n_knots[n_terms]  knots of term k (>= 1)
 *   times, values     all terms' knots concatenated, times strictly
 *                     increasing within each term
 */
typedef struct {
  int32_t n_terms;
  const qt_op *H;
  const int64_t *n_knots;
  const double *times;
  const double *values;
} qt_td;

/* qt_mesolve / qt_mcsolve with the time-dependent terms td (nullable: none).
 * Not built with me_method QT_ME_DENSE_TC (QT_ENOTIMPL), nor for Monte-Carlo
 * trajectories of dimension above 1024. */
int qt_mesolve_td(const qt_op *H, const qt_td *td, const qt_op *c_ops, int n_c,
                  const qt_op *e_ops, int n_e, const qt_c128 *state0, int state_is_ket,
                  const double *tlist, int n_t, const qt_opts *o, qt_c128 *expect_out,
                  qt_c128 *states_out, qt_stats *stats);
int qt_mcsolve_td(const qt_op *H, const qt_td *td, const qt_op *c_ops, int n_c,
                  const qt_op *e_ops, int n_e, const qt_c128 *psi0, const double *tlist,
                  int n_t, int64_t ntraj, uint64_t seed, const qt_opts *o, qt_c128 *expect_out,
                  qt_c128 *traj_expect_out, qt_jump *jumps, int64_t jump_cap, int64_t *n_jumps,
                  qt_stats *stats);

/*
 * Two-time correlation function by the ODE solver (the paper's
 * correlation_ode, section 5 function list), through the quantum regression
 * theorem:  C(t_k, tau_j) = <A(t_k + tau_j) B(t_k)>
 *                         = Tr[ A V(t_k + tau_j, t_k) [B rho(t_k)] ],
 * where rho(t_k) solves the master equation from state0 (as in qt_mesolve)
 * over tlist and V(t', t) is the master-equation propagator, applied to the
 * (generally non-Hermitian) matrix X_k = B rho(t_k) from time t_k.
 * tlist[n_t]: increasing; taulist[n_tau]: increasing with taulist[0] == 0
 * (QT_EINVAL otherwise).  corr_out[n_t * n_tau] (host): C(t_k, tau_j) at
 * [k * n_tau + j].  td nullable (time-dependent terms as in qt_mesolve_td;
 * the tau evolution of X_k then sees H(t_k + tau)).  The first solve uses
 * o->me_method; the tau evolutions run the general solver (QT_ME_DENSE_TC is
 * taken as QT_ME_AUTO there).  stats (nullable) sums both stages.
 */
int qt_correlation_2op_2t(const qt_op *H, const qt_td *td, const qt_op *c_ops, int n_c,
                          const qt_op *A, const qt_op *B, const qt_c128 *state0, int state_is_ket,
                          const double *tlist, int n_t, const double *taulist, int n_tau,
                          const qt_opts *o, qt_c128 *corr_out, qt_stats *stats);

/*
 * Steady state of the master equation (the paper's steadystate, section 5
 * function list): rho_out[dim*dim] (host, row-major) receives the density
 * matrix with L(rho) = 0 and Tr rho = 1, where L is the right-hand side of
 * Eq. (master_equation) for H and c_ops.  Solved on the GPU in FP64 as the
 * linear system  L(x) + w Tr(x) I = w I  (invertible exactly when the
 * stationary state is unique; w is the mean magnitude of L's diagonal) by
 * restarted GMRES with krylov_dim basis vectors (<= 0: 600) and a diagonal
 * preconditioner, until ||w I - L(x) - w Tr(x) I||_F <= tol ||w I||_F; then
 * rho = (x + x^dag) / 2 / Tr.  Device memory: (krylov_dim + 4) dim^2 complex
 * FP64 values.  max_iter bounds the Arnoldi steps over all restarts:
 * QT_ESTEP when reached (rho_out holds the last iterate, info_out its
 * residual); Krylov methods can stall where the Hamiltonian dominates the
 * dissipation (use qt_propagator_steadystate there).  QT_ENOTIMPL when a
 * CTA's share of the dim^2 entries and the basis bookkeeping exceed 200 KB of
 * shared memory (about dim > 1400).  info_out[3] (nullable): final relative
 * residual, w, Arnoldi steps.  stats (nullable): accepted = Arnoldi steps,
 * rhs_evals = applications of L.  A non-unique stationary state (e.g. no
 * collapse operators) makes the system singular but consistent: the result
 * is then one stationary state, the one the iteration reaches from I/dim.
 */
int qt_steadystate(const qt_op *H, const qt_op *c_ops, int n_c, double tol, int64_t max_iter,
                   int krylov_dim, qt_c128 *rho_out, double *info_out, qt_stats *stats);

/*
 * Propagator steady state (the paper's propagator_steadystate, section 5
 * function list): the fixed point of rho -> V(T) rho, V(T) the master-equation
 * propagator over one period T, by repeated solves over [0, T] from rho0
 * (host dim*dim density matrix; nullable: I/dim) with the solver options o
 * (precision, method, tolerances), until ||rho_{k+1} - rho_k||_F <= tol.  The
 * distance to the steady state is about that change / (1 - exp(-g T)), g the
 * slowest decay rate; every period restarts the step-size selection.  Robust
 * where qt_steadystate's Krylov iteration stalls (strongly driven systems),
 * at the cost of integrating to t ~ log(1/tol) / g.  rho_out[dim*dim] (host);
 * info_out[2] (nullable): last change, periods; stats (nullable) sums the
 * periods.  QT_ESTEP when max_periods is reached, or when 50 periods pass
 * without a new smallest change (the change cannot fall below the solver's
 * integration error over one period, about rtol: choose tol above it);
 * rho_out then holds the last state.
 */
int qt_propagator_steadystate(const qt_op *H, const qt_op *c_ops, int n_c, const qt_c128 *rho0,
                              double period, double tol, int64_t max_periods, const qt_opts *o,
                              qt_c128 *rho_out, double *info_out, qt_stats *stats);

/*
 * Master-equation propagator (the paper's propagator, section 5 function
 * list): U_out[n_t][dim^2][dim^2] (host) receives U(t_k), the matrix that
 * maps row-major vec(rho(tlist[0])) to vec(rho(tlist[k])) for Eq.
 * (master_equation) with H (plus the time-dependent terms td, nullable) and
 * c_ops; U(t_0) = I.  Column a dim + b is the solution from the matrix unit
 * E_ab, computed on the GPU one CTA per unit with the general solver and the
 * options o (precision, tolerances; QT_ME_DENSE_TC is taken as QT_ME_AUTO).
 * Built for dim <= 64 (QT_ENOTIMPL above); stats sums the dim^2 solves.
 */
int qt_propagator(const qt_op *H, const qt_td *td, const qt_op *c_ops, int n_c,
                  const double *tlist, int n_t, const qt_opts *o, qt_c128 *U_out,
                  qt_stats *stats);

/*
 * Steady-state two-time correlation (the steady-state forms among the
 * paper's correlation functions): C(tau_j) = <A(tau_j) B(0)> with the system
 * in its steady state, i.e. qt_steadystate (FP64 GMRES to relative residual
 * tol) followed by qt_correlation_2op_2t from rho_ss at the single time 0.
 * taulist[n_tau]: increasing from 0; corr_out[n_tau] (host); o: options of
 * the tau evolution; stats (nullable): those of the tau evolution.
 * QT_ESTEP when the steady-state solve does not converge.
 */
int qt_correlation_ss(const qt_op *H, const qt_op *c_ops, int n_c, const qt_op *A,
                      const qt_op *B, const double *taulist, int n_tau, double tol,
                      const qt_opts *o, qt_c128 *corr_out, qt_stats *stats);

/*
 * Expectation values (paper section 2, expect()): for is_ket != 0,
 * out[b] = <psi_b|O|psi_b> (not normalised) for states[b * dim ...];
 * otherwise out[b] = Tr(O rho_b) for states[b * dim * dim ...].
 */
int qt_expect(const qt_op *O, const qt_c128 *states, int is_ket, int64_t batch, qt_c128 *out);

/* ---------------------------------------------- device-resident systems */

/* A system: H, collapse and observable operators packed for the GPU (the
 * effective Hamiltonian of Eq. (heff) formed in FP64 on the host, every
 * operator converted to ELLPACK and uploaded in the requested precision).
 * The handle owns its device memory and a workspace that grows on demand;
 * it must be used from one host thread at a time.  Operators are copied;
 * the caller's arrays may be freed after qt_system_create returns. */
typedef struct qt_system_s *qt_system;

int qt_system_create(const qt_op *H, const qt_op *c_ops, int n_c, const qt_op *e_ops, int n_e,
                     qt_system *out);
/* A system whose Hamiltonian has the time-dependent terms td (see qt_td;
 * nullable: the same as qt_system_create). */
int qt_system_create_td(const qt_op *H, const qt_td *td, const qt_op *c_ops, int n_c,
                        const qt_op *e_ops, int n_e, qt_system *out);
int qt_system_destroy(qt_system s);
int qt_system_dim(qt_system s);

/*
 * Asynchronous qt_mcsolve on trajectories traj_begin .. traj_begin+ntraj-1
 * (global indices: the random streams depend only on the global index, so
 * any split of a range gives the same trajectories).  Device pointers:
 * psi0_dev[dim] (normalised by the call), tlist_dev[n_t],
 * expect_sum_dev[n_t * n_e]: the SUM over this call's trajectories of
 * <psi|O_m|psi>/<psi|psi> (overwritten), traj_expect_dev (nullable),
 * jumps_dev[jump_cap] (nullable when jump_cap == 0), n_jumps_dev (int64,
 * nullable), stats_dev (qt_stats, nullable; its status field carries the
 * first device-side error).  o->precision selects the kernel.
 */
int qt_mcsolve_dev(qt_system s, const qt_c128 *psi0_dev, const double *tlist_dev, int n_t,
                   int64_t traj_begin, int64_t ntraj, uint64_t seed, const qt_opts *o,
                   qt_c128 *expect_sum_dev, qt_c128 *traj_expect_dev, qt_jump *jumps_dev,
                   int64_t jump_cap, int64_t *n_jumps_dev, qt_stats *stats_dev, void *stream);

/*
 * Asynchronous qt_mesolve.  Device pointers: state0_dev (ket or density
 * matrix as in qt_mesolve), tlist_dev[n_t], expect_dev[n_t * n_e]
 * (nullable when n_e == 0), states_dev (nullable), stats_dev (nullable).
 */
int qt_mesolve_dev(qt_system s, const qt_c128 *state0_dev, int state_is_ket,
                   const double *tlist_dev, int n_t, const qt_opts *o, qt_c128 *expect_dev,
                   qt_c128 *states_dev, qt_stats *stats_dev, void *stream);

/*
 * One evaluation of the master-equation right-hand side d rho/dt of paper
 * Eq. (master_equation) for system s at time t (which matters only for a
 * system with time-dependent terms), asynchronous: rho_dev[dim*dim]
 * (row-major complex FP64, device; rounded to FP32 first when
 * o->precision == QT_MIXED) -> out_dev[dim*dim] (FP64, device, overwritten).
 * o->me_method selects the method as for qt_mesolve_dev; QT_ME_DENSE_TC
 * assumes rho is Hermitian.  stats_dev (nullable) receives the device
 * status (QT_ETIMEOUT if a bounded tensor-core wait ran out).  Uses the
 * system's solver workspace: do not overlap with a solve on the same system.
 */
int qt_me_rhs_dev(qt_system s, double t, const qt_c128 *rho_dev, qt_c128 *out_dev,
                  const qt_opts *o, qt_stats *stats_dev, void *stream);

/*
 * Asynchronous qt_correlation_2op_2t for every observable of s at once:
 * corr_dev[n_t * n_tau * n_e] (device) receives
 *   <O_m(t_k + tau_j) B(t_k)> at [(k * n_tau + j) * n_e + m],
 * with B = observable b_index of s.  Device pointers: state0_dev, tlist_dev,
 * taulist_dev (taulist_dev[0] must be 0; not checked on the device).  The
 * call allocates (grow-only, owned by s) n_t + 1 FP64 density matrices and
 * a solver slab per CTA, so it synchronises the device when that store
 * grows.  Systems of dim <= 64 evolve all X_k in one launch, one CTA each;
 * larger ones one cooperative launch per t_k.  Do not overlap with another
 * solve on the same system.
 */
int qt_correlation_2op_2t_dev(qt_system s, const qt_c128 *state0_dev, int state_is_ket,
                              const double *tlist_dev, int n_t, const double *taulist_dev,
                              int n_tau, int b_index, const qt_opts *o, qt_c128 *corr_dev,
                              qt_stats *stats_dev, void *stream);

/*
 * Asynchronous qt_steadystate on system s (its observables are unused):
 * rho_dev[dim*dim] (device, overwritten), info_dev[3] (device doubles,
 * nullable), stats_dev (nullable; status QT_ESTEP when max_iter was
 * reached).  QT_ENOTIMPL for a system with time-dependent terms.  Uses the
 * system's solver workspace and store (grow-only; allocation synchronises
 * the device): do not overlap with a solve on the same system.
 */
int qt_steadystate_dev(qt_system s, double tol, int64_t max_iter, int krylov_dim,
                       qt_c128 *rho_dev, double *info_dev, qt_stats *stats_dev, void *stream);

/*
 * qt_propagator_steadystate on system s: rho0_dev (device, nullable: I/dim),
 * rho_dev (device, overwritten), info (HOST doubles [2], nullable), stats_dev
 * (device, nullable).  Synchronises with the stream after every period to
 * test the change, so it returns when the solve is done.  Uses the system's
 * store and solver workspace: do not overlap with a solve on the same system.
 */
int qt_propagator_steadystate_dev(qt_system s, const qt_c128 *rho0_dev, double period,
                                  double tol, int64_t max_periods, const qt_opts *o,
                                  qt_c128 *rho_dev, double *info, qt_stats *stats_dev,
                                  void *stream);

/*
 * Asynchronous qt_propagator on system s (its observables are unused):
 * tlist_dev[n_t], U_dev[n_t * dim^4] (device, overwritten), stats_dev
 * (nullable).  Uses the system's store (grow-only; allocation synchronises
 * the device): do not overlap with a solve on the same system.
 */
int qt_propagator_dev(qt_system s, const double *tlist_dev, int n_t, const qt_opts *o,
                      qt_c128 *U_dev, qt_stats *stats_dev, void *stream);

/*
 * qt_mesolve_dev without allocation.  The paper has no counterpart: this is
 * an entry point for callers that cannot allocate device memory -- a process
 * that has handed all free memory to another allocator, or a solve path
 * that must not enter cudaMalloc/cudaFree (they may synchronise the device).
 * Same arguments and semantics as qt_mesolve_dev, but the solver workspace
 * comes from a 16 MiB array in device memory that the library commits on a
 * device when the first system is created there with that device current
 * (qt_system_create, qt_system_create_td) and holds until the process exits;
 * the call itself allocates nothing.  It always runs the general sparse
 * solver (no Hermitian or single-CTA specialisation, no tensor cores:
 * QT_ME_DENSE_TC returns QT_ENOTIMPL), so its results match qt_mesolve_dev's
 * within the solvers' tolerance, not bit for bit.  Limit, on any device:
 * dim <= 307 in QT_FP64 and dim <= 431 in QT_MIXED; larger systems return
 * QT_EINVAL with the byte counts in qt_last_error().  A system created on
 * another device than the current one leaves the first call on the current
 * device to look up the array (cudaGetSymbolAddress, which may commit the
 * 16 MiB there), so make that first call before any stream capture.  A
 * device reset (cudaDeviceReset) after the look-up is not supported.  Every
 * call shares the one array: calls whose work overlaps on the GPU (two
 * streams, two host threads) race and corrupt each other's results; order
 * them on one stream.
 */
int qt_mesolve_dev_noalloc(qt_system s, const qt_c128 *state0_dev, int state_is_ket,
                           const double *tlist_dev, int n_t, const qt_opts *o,
                           qt_c128 *expect_dev, qt_c128 *states_dev, qt_stats *stats_dev,
                           void *stream);

/*
 * Asynchronous expectation values of observable e_index of system s over a
 * batch of device-resident states (layout as in qt_expect), FP64.
 */
int qt_expect_dev(qt_system s, int e_index, const qt_c128 *states_dev, int is_ket,
                  int64_t batch, qt_c128 *out_dev, void *stream);

/* ------------------------------------------------------- batched solves */

#define QT_KIND_ME 0 /* master equation (paper section 3.1)          */
#define QT_KIND_MC 1 /* Monte-Carlo wave function (paper section 3.2) */

/* One problem of a batch: its own operators (any dimension up to 64), kind,
 * initial state and, for QT_KIND_MC, trajectory count and seed.  All host
 * memory; copied by qt_batch_create. */
typedef struct {
  int32_t kind;         /* QT_KIND_ME or QT_KIND_MC                          */
  int32_t state_is_ket; /* ME: state0 is a ket (1) or a density matrix (0);
                           MC: must be 1                                     */
  const qt_op *H;
  const qt_op *c_ops;
  int32_t n_c;
  int32_t n_e;
  const qt_op *e_ops;
  const qt_c128 *state0;
  int64_t ntraj;        /* MC: trajectories (global indices 0..ntraj-1)     */
  uint64_t seed;        /* MC: Philox key                                    */
} qt_problem;

typedef struct qt_batch_s *qt_batch;

/*
 * Packs many independent problems of uneven dimension (the parameter sweeps
 * of the paper's examples) for one persistent launch: each master-equation
 * problem is one work item solved by one CTA; each Monte-Carlo problem is
 * split into blocks of trajectories that the warps of a CTA share; items are
 * ordered by estimated cost (largest first).  Every dimension must be
 * <= 64.  The handle owns its device memory and workspace.
 */
int qt_batch_create(const qt_problem *problems, int n_problems, qt_batch *out);
int qt_batch_destroy(qt_batch b);

/* Offset (in qt_c128 elements) of problem p's outputs in the expect buffer of
 * qt_batch_solve_dev: problem p writes n_t * n_e_p values at
 * [offset + k * n_e_p + m]; total size via p == n_problems. */
int64_t qt_batch_expect_offset(qt_batch b, int p, int n_t);

/*
 * Tunes the persistent launch on this batch by measurement (each candidate
 * solved twice on `stream`, the second solve timed with CUDA events,
 * synchronously) and keeps the fastest configuration for later solves:
 * first how the trajectories of small Monte-Carlo problems map onto warps
 * (every problem on whole warps -- one row per lane up to dimension 32, two
 * above --, or half-warp groups of 16 lanes, two trajectories per warp, for
 * dimensions up to 16 or up to 32), then the Monte-Carlo work-item size (32,
 * 64, 128 or 256 trajectories).  qt_batch_config reports the choice.
 * Optional; the default is whole warps and blocks of 64.  Not for use during
 * stream capture.
 */
int qt_batch_tune(qt_batch b, const double *tlist_dev, int n_t, const qt_opts *o,
                  qt_c128 *expect_dev, void *stream);

/*
 * Solves every problem of the batch in one persistent launch on `stream`
 * (asynchronous; allocates nothing, so it can be captured in a CUDA graph).
 * All problems share tlist_dev[n_t] and the options o.  expect_dev receives,
 * per problem (layout from qt_batch_expect_offset), Tr(O_m rho(t_k)) for
 * master-equation problems and the trajectory mean of
 * <psi|O_m|psi>/<psi|psi> for Monte-Carlo problems.  stats_dev (nullable)
 * receives the summed statistics and the first device-side error.
 */
int qt_batch_solve_dev(qt_batch b, const double *tlist_dev, int n_t, const qt_opts *o,
                       qt_c128 *expect_dev, qt_stats *stats_dev, void *stream);

/*
 * The batch's launch configuration (host outputs, each nullable): the
 * Monte-Carlo work-item size in trajectories, the largest dimension whose
 * Monte-Carlo problems run on half-warp groups (0: none), and the time of
 * the tuned configuration in ms (0 before qt_batch_tune).
 */
int qt_batch_config(qt_batch b, int *traj_block, int *small_group_dim, double *tuned_ms);

/*
 * Sets the launch configuration that qt_batch_tune would choose by
 * measurement: the Monte-Carlo work-item size (1 .. 2^20 trajectories) and
 * small_group_dim (0, 16 or 32; see qt_batch_tune).  Rebuilds the work items
 * on the host and uploads them, reallocating the item arrays when the size
 * needs more items than the batch holds (synchronous; not during a solve or
 * a stream capture).  QT_EINVAL for other values.
 */
int qt_batch_set_config(qt_batch b, int traj_block, int small_group_dim);

/*
 * Host copy of the statistics of every problem of the last qt_batch_solve_dev
 * (accepted steps, rejected steps, right-hand sides, jump-search trials and
 * jumps; summed over a problem's trajectories): stats[n_problems], host
 * memory.  Synchronous (copies from the device); status fields are 0, the
 * batch's status is in the stats of qt_batch_solve_dev.
 */
int qt_batch_problem_stats(qt_batch b, qt_stats *stats);

/* ------------------------------------------------- gradients (adjoint) */

/*
 * Gradients of a master-equation loss (an extension beyond the paper; the
 * forward problem is Eq. (master_equation), section 3.1).  The generator of
 * segment s (length t_seg, n_seg segments) is
 *   F_s(rho) = -i [H0 + Omega_s Hd, rho]
 *              + sum_k gamma_k (A_k rho A_k^dag - 1/2 {A_k^dag A_k, rho});
 * the loss is L = Re Tr(P1 rho(T)) + Re int_0^T Tr(P2 rho) dt, the integral
 * carried by the same Runge-Kutta stages as rho.  H0, Hd, P1, P2 must be
 * Hermitian; dimension <= 64; n_k <= 8.  A handle holds batch parameter
 * vectors (Omega[n_seg], gamma[n_k]), solved one per CTA in FP64.
 * state0: ket (rho0 = |psi><psi|/<psi|psi>) or density matrix.
 * max_per_seg bounds the accepted steps per segment (QT_ESTEP beyond).
 */
typedef struct qt_adjoint_s *qt_adjoint;

int qt_adjoint_create(const qt_op *H0, const qt_op *Hd, const qt_op *A, int n_k, const qt_op *P1,
                      const qt_op *P2, const qt_c128 *state0, int state_is_ket, int n_seg,
                      double t_seg, int batch, int max_per_seg, qt_adjoint *out);
int qt_adjoint_destroy(qt_adjoint a);

/* Adaptive forward solve of every vector (controller of qt.h, segment ends
 * as output times); keeps each vector's accepted step lengths (the frozen
 * grid), rho at the segment ends and a copy of the parameters for the
 * backward pass.  omega_dev[batch * n_seg], gamma_dev[batch * n_k],
 * loss_dev[batch]: device pointers.  Asynchronous on stream. */
int qt_adjoint_forward_dev(qt_adjoint a, const double *omega_dev, const double *gamma_dev,
                           const qt_opts *o, double *loss_dev, qt_stats *stats_dev,
                           void *stream);

/* The loss at other parameters on the grids of the last forward pass
 * (finite differences on a frozen grid).  Does not touch the stored state. */
int qt_adjoint_loss_fixed_dev(qt_adjoint a, const double *omega_dev, const double *gamma_dev,
                              double *loss_dev, void *stream);

/* Discrete adjoint on the grids of the last forward pass: the gradients of
 * sum_b dloss[b] L_b with respect to omega (grad_omega_dev[batch * n_seg])
 * and gamma (grad_gamma_dev[batch * n_k]).  dloss_dev nullable (all ones). */
int qt_adjoint_backward_dev(qt_adjoint a, const double *dloss_dev, double *grad_omega_dev,
                            double *grad_gamma_dev, void *stream);

/* Host copy of vector b's recorded grid: nsteps[n_seg], h[n_seg * max_per_seg]
 * (synchronous). */
int qt_adjoint_grid(qt_adjoint a, int b, int32_t *nsteps, double *h);

/* ------------------------------------------------------ measurement */

#define QT_PEAK_FP32 0   /* scalar FP32 fused multiply-add                */
#define QT_PEAK_FP32X2 1 /* packed two-lane FP32 multiply-add (f32x2)     */
#define QT_PEAK_FP64 2   /* FP64 fused multiply-add                       */

/*
 * Measures the multiply-add throughput of the current device: the paper has
 * no counterpart; this is the arithmetic roof against which the solvers'
 * ALU-bound kernels are reported.  Runs one warm-up launch and `reps` timed
 * launches (CUDA events on `stream`, synchronous) of a kernel whose threads
 * each carry independent multiply-add chains for iters x 128 steps, with the
 * grid filled to the occupancy limit on every SM.  Writes the rate in flop/s
 * (one multiply-add = 2 flop) to *flop_per_s, and, when non-null, the flops
 * and milliseconds of one launch.  Errors: QT_EINVAL (iters outside
 * [1, 2^30], reps outside [1, 10000], null flop_per_s, unknown kind),
 * QT_ENODEV, QT_ECUDA.  Changes no clock or other device setting.
 */
int qt_fma_peak(int kind, int64_t iters, int reps, double *flop_per_s, double *flop_per_launch,
                double *ms_per_launch, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* QT_H */
