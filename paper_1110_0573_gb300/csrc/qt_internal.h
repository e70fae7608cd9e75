// qt_internal.h -- declarations shared by the host side of libqt
// (qt_host.cpp) and its CUDA translation units.  Not part of the public ABI.
#pragma once

#include <cuda.h>  // CUtensorMap (type only; the encoder is fetched at run time)
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/qt.h"

namespace qt {

// Operators on the device are stored in ELLPACK form, slot-major: the s-th
// stored entry of row i sits at off + s * d + i (consecutive rows of one slot
// are contiguous, so threads that own consecutive rows load coalesced).
// Rows shorter than the width w are padded with value 0 and column = row.
// Operator 0 of a system is H_eff (Eq. (heff)), operators 1..n_c the
// collapse operators C_n, operators 1+n_c .. n_c+n_e the observables.
struct OpTable {
  int d;
  int n_ops;
  const int *w;          // [n_ops] ELL width of each operator
  const int64_t *off;    // [n_ops] slot offset of each operator
  const int *col;        // [total slots]
  const double2 *val64;  // [total slots] FP64 values
  const float2 *val32;   // [total slots] FP32 copy of the same values
  const float2 *val32lo; // [total slots] FP32 remainder: val64 = val32 + val32lo
                         // to ~2^-48 (null where no FP32 copy exists)
};

// Time-dependent Hamiltonian terms (paper section 4.3): H(t) = H +
// sum_k f_k(t) H_k, f_k piecewise linear between knots (td_t, td_v)[td_off[k]
// .. td_off[k+1]-1] and constant outside them; H_k is operator td_op0 + k of
// the table.  At most kTdMax terms.
constexpr int kTdMax = 8;

// Kernel arguments of the Monte-Carlo trajectory kernel.
struct McArgs {
  OpTable ops;
  int heff_w;  // host copy of ops.w[0], used to pick the kernel instance
  int stage_aux;      // set by the launcher: operators 1.. staged in shared memory
  int64_t aux_begin;  // first slot of operators 1.. (collapse, observables)
  int64_t aux_slots;  // number of slots of operators 1..
  int n_c, n_e, n_t;
  const double2 *psi0;  // [d], normalised
  const double *tlist;  // [n_t]
  int64_t traj_begin, ntraj;
  uint64_t seed;
  double rtol, atol, h0, bisect_tol;
  int64_t max_steps;
  double2 *expect_sum;           // [n_t * n_e] sum over trajectories
  double2 *traj_expect;          // nullable [ntraj * n_t * n_e]
  qt_jump *jumps;                // nullable
  int64_t jump_cap;
  unsigned long long *n_jumps;   // device counter (always valid)
  unsigned long long *counters;  // [6]: accepted, rejected, rhs, bisect, jumps, near_miss
  int *status;                   // first error code, 0 = ok
  unsigned long long *work;      // next trajectory to hand out
  int n_td, td_op0;              // time-dependent terms (0: none)
  const int64_t *td_off;
  const double *td_t, *td_v;
  void *stage_ws;                // dimensions above 2048: stage slabs, one per CTA
  int stage_ctas;                //   (stage_ctas slabs of mc_stage_slab_bytes each)
  // H_eff as a dictionary (null when the system has none): the diagonal,
  // and per row dict_w off-diagonal codes col | (value index << 16),
  // slot-major (code of slot s of row i at s * d + i; padding: col = i,
  // index 0), into a table of the dict_nv distinct off-diagonal values
  // (entry 0 is zero).  FP32 hi values followed by their FP32 remainders.
  const uint32_t *dict_code;     // [dict_w][d]
  const float2 *dict_diag;       // [2][d]
  const float2 *dict_tab;        // [2][dict_nv]
  int dict_w, dict_nv;
  // grouped dictionary (dict_groups > 0): codes are plain columns (d marks
  // padding), the entries of table value g + 1 in slots dict_gend[g - 1] ..
  // dict_gend[g] - 1 of every row (dict_gend[-1] = 0)
  int dict_groups;
  int dict_gend[16];
  // Mixed kernel without time-dependent terms: the output intervals, the
  // same for every trajectory, formed once per solve by launch_normalise
  // (null: each group forms them as it goes).  Interval m (1 <= m < n_t)
  // starts at ivl_tb[m] and has FP32 length ivl_len[m]; ivl_tb[1] =
  // tlist[0], ivl_len[m] = fl32(tlist[m] - ivl_tb[m]) and ivl_tb[m + 1] =
  // ivl_tb[m] + ivl_len[m], so an interval starts where the previous one
  // ended and the FP32 rounding of the lengths does not accumulate.
  const double *ivl_tb;
  const float *ivl_len;
};

// Largest value table of a dictionary H_eff (the Monte-Carlo kernels stage
// the dictionary in shared memory), and the most values of a grouped one.
constexpr int kDictMaxValues = 1024;
constexpr int kDictMaxGroups = 16;

// Kernel arguments of the master-equation solver.
struct MeArgs {
  OpTable ops;
  int n_c, n_e, n_t;
  int grid;  // CTAs of the cooperative launch
  const double *tlist;
  double rtol, atol, h0;
  int64_t max_steps;
  double2 *expect;               // nullable [n_t * n_e]
  double2 *states;               // nullable [n_t * d * d]
  unsigned long long *counters;  // [6] as in McArgs
  int *status;
  const double2 *state0;         // initial ket [d] or density matrix [d*d]
  int state_is_ket;
  void *work;                    // 11 * d * d elements of the kernel's complex
                                 // type: rho, ynew, two stage inputs, k1..k7
  double *partial;               // per-CTA reduction slots [grid * kMePartial]
  const double2 *rhs_in;         // non-null: evaluate drho/dt of this d*d state once
  double2 *rhs_out;              //   into this d*d array instead of solving
  double rhs_t;                  //   at this time
  // collapse operators in slot form for the Hermitian combine phase: slot q
  // is stored entry s of collapse operator c (row i at cslot_off[q] + i);
  // term k multiplies slot cterms[k].x of row i with slot cterms[k].y of
  // row j (all pairs s, t of each operator).  n_cslots = 0: not staged.
  const int *cslot_off;
  const int2 *cterms;
  int n_cslots, n_cterms;
  int n_td, td_op0;              // time-dependent terms (0: none), as in McArgs
  const int64_t *td_off;
  const double *td_t, *td_v;
  int single_cta;                // 1: one CTA solves (small systems; no grid barriers)
  int herm;                      // 0: general solver (no symmetry assumed);
                                 // 1: Hermitian solver (state0 is a ket or Hermitian);
                                 // 2: test the initial matrix on the device, then choose
};

// Hermitian-state test of the device: an initial matrix counts as Hermitian
// when sum |rho_ij - conj(rho_ji)|^2 <= kHermTol2 * sum |rho_ij|^2.
constexpr double kHermTol2 = 1e-20;

// Largest slot and term counts of the collapse operators staged in shared
// memory by the Hermitian combine phase (larger sets are read from global
// memory entry by entry).
constexpr int kCSlotsMax = 32;
constexpr int kCTermsMax = 512;

constexpr int kMeBlock = 256;
constexpr int kMeSmallDim = 64;  // systems up to this dimension are solved by one CTA

// Steady state (qt_ss.cu): GMRES(m) on A(x) = L(x) + w Tr(x) I.
constexpr int kGmBlock = 512;
struct GmArgs {
  double tol;          // stop at ||w I - A x||_F <= tol ||w I||_F
  int64_t max_iter;    // Arnoldi steps over all restarts
  int m;               // basis vectors per restart
  int chunk;           // entries of the d*d vectors owned by each CTA
  double2 *V;          // (m + 1) * d*d basis
  double2 *x, *zu, *minv;  // d*d each: iterate, preconditioned vector, 1 / diag
  double2 *pd;         // grid * (m + 1) per-CTA inner products
  double2 *hcol;       // m + 1 reduced inner products
  double2 *R;          // (m + 1) * m (column-major, leading dimension m + 1) Hessenberg matrix
  double *ctl;         // [2]: first converged column (-1: none), residual estimate
  double2 *y;          // m least-squares coefficients
  double2 *rho_out;    // d*d
  double *info;        // nullable: [final relative residual, w, iterations]
};

// Propagator (qt_corr.cu): one CTA per matrix unit; per-CTA slab of the
// solver workspace, the start matrix and the n_t output states.
struct PropArgs {
  double2 *U;            // [n_t][d*d][d*d]
  size_t ws_stride;      // bytes of one CTA's slab
  size_t x_off, st_off;  // offsets of the start matrix and of the states in a slab
};

// Two-time correlation functions (qt_corr.cu): the k-th tau evolution starts
// from X_k = B rho(t_k) at time t_k and outputs at t_k + tau_j.
struct CorrArgs {
  const double2 *rho_t;   // [n_t][d][d] FP64 states rho(t_k)
  const double *tlist;    // [n_t]
  const double *taulist;  // [n_tau], taulist[0] = 0
  int n_t, n_tau;
  int b_op;               // operator-table index of B
  size_t ws_stride;       // bytes of one CTA's slab (batched small-system path)
  size_t x_off, times_off;  // offsets of X_k (double2 [d*d]) and the times in a slab
};

// Dense operands of the tensor-core master-equation path (qt_me_tc.cu).
// With dp = d rounded up to 128, the product Y = H_eff y of a Hermitian
// state y is one real GEMM  Y(dp x 2dp, FP32) = A(dp x 2dp) * B(2dp x 2dp)^T:
//   A[m][2k], A[m][2k+1]     = Re, Im of H_eff[m][k]
//   B[2n][2k], B[2n][2k+1]   = Re, Im of y[n][k]
//   B[2n+1][2k], B[2n+1][2k+1] = -Im, Re of y[n][k]          (row n of i*y)
// so that Y, read as complex FP32 [dp][dp], is H_eff y (y^T = conj(y)).
// A and B are each held as a BF16 pair hi + lo (x = hi + lo + O(2^-17 |x|)).
//
// Dense collapse operators (nc > 0): sum_n C_n y C_n^dag as two more GEMMs of
// the same form (a GEMM of A planes of P and B planes of X gives P X^dag):
//   T = [C_1; ...; C_nc] y         A = the stacked C planes [nc dp][2dp], B = y;
//   W = [T_1 ... T_nc] [C_1 ... C_nc]^dag = sum_n T_n C_n^dag
//                                  A = the T planes [dp][2 nc dp] (written by
//                                  the first GEMM's epilogue), B = the planes
//                                  of [C_1 ... C_nc] [2dp][2 nc dp] (constant).
struct TcArgs {
  CUtensorMap a_hi, a_lo, b_hi, b_lo;  // 2-D BF16 maps, box 64 x 128, 128-byte swizzle
  uint16_t *b_hi_ptr, *b_lo_ptr;       // B planes (BF16 bit patterns), [2dp][2dp]
  float2 *Y;                           // [dp][dp] complex FP32
  int dp;
  int nc;                              // dense collapse operators (0: sparse collapse terms)
  CUtensorMap c_hi, c_lo;              // stacked C planes
  CUtensorMap t_hi, t_lo;              // T planes
  CUtensorMap cc_hi, cc_lo;            // planes of [C_1 ... C_nc] as B
  uint16_t *t_hi_ptr, *t_lo_ptr;       // T planes (BF16 bit patterns), [dp][2 nc dp]
  float2 *W;                           // [dp][dp] complex FP32: sum_n C_n y C_n^dag
};

// Collapse operators at least this wide (stored entries per row) make the
// tensor-core solver form all collapse terms as dense products.
constexpr int kTcDenseCWidth = 32;
constexpr int kMePartialMax = 64;  // reduction slots per CTA (2 per observable + 4)

// One problem of a batch on the device.
struct BatchProblem {
  OpTable ops;            // this problem's operators (H_eff, C_n, O_m)
  const int *opoff32;     // slot offset of each operator as int
  int kind;               // QT_KIND_ME / QT_KIND_MC
  int n_c, n_e;
  int state_is_ket;
  int64_t ntraj;
  uint64_t seed;
  const double2 *state0;  // ME: ket or rho0; MC: normalised ket
  int64_t expect_off;     // offset of the outputs (per unit n_t: off = base * n_t)
};

// A work item: a master-equation problem, or a block of trajectories.
struct BatchItem {
  int problem;
  int pad;
  int64_t traj_begin;
  int64_t ntraj;
};

struct BatchArgs {
  const BatchProblem *probs;
  const BatchItem *items;
  int n_items;
  int n_problems;
  const double *tlist;
  int n_t;
  double rtol, atol, h0, bisect_tol;
  int64_t max_steps;
  double2 *expect;
  unsigned long long *item_work;  // [n_items] trajectory hand-out per item
  unsigned long long *next_item;  // item hand-out
  unsigned long long *counters;   // [6]
  unsigned long long *prob_counters;  // [n_problems][6], summed into counters at the end
  unsigned long long *n_jumps;
  int *status;
  void *ws;                       // master-equation workspace, ws_stride bytes per CTA
  size_t ws_stride;
  int small_group_dim;            // MC items up to this dimension: half-warp groups
};

constexpr int kBatchBlock = 256;

cudaError_t launch_batch(const BatchArgs &a, int precision, int grid, cudaStream_t s);
int batch_grid(int precision);
size_t batch_ws_stride(int dmax, int precision);
cudaError_t launch_batch_finalize(const BatchArgs &a, cudaStream_t s);

// Arguments of the master-equation adjoint kernels (one CTA per parameter
// vector).  Operator table: 0 H0, 1 Hd, 2.. A_k, then A_k^dag, then
// A_k^dag A_k, then P1, P2.
struct AdjArgs {
  OpTable ops;
  int nk, n_seg, batch, maxs;
  double t_seg;
  const double *omega;   // [batch][n_seg]
  const double *gamma;   // [batch][nk]
  const double2 *rho0;   // d*d
  double rtol, atol;
  int64_t max_steps;
  int fixed;             // 1: integrate on the recorded grid, loss only
  int *nsteps;           // [batch][n_seg]
  double *hgrid;         // [batch][n_seg][maxs]
  double2 *ckpt;         // [batch][n_seg + 1][d*d]
  double2 *work;         // [batch][slots][d*d]
  int64_t slots;
  double *loss;          // [batch]
  const double *dloss;   // [batch] upstream gradient (backward)
  double *g_omega;       // [batch][n_seg]
  double *g_gamma;       // [batch][nk]
  unsigned long long *counters;
  int *status;
};

size_t adjoint_slots(int maxs);
cudaError_t launch_adjoint_forward(const AdjArgs &a, cudaStream_t s);
cudaError_t launch_adjoint_backward(const AdjArgs &a, cudaStream_t s);

// Launchers (return cudaError_t of the launch).
cudaError_t launch_mc(const McArgs &a, int precision, int group, cudaStream_t s);
cudaError_t launch_mc_f64(const McArgs &a, cudaStream_t s);
cudaError_t launch_mc_f32(const McArgs &a, cudaStream_t s);
// the time-dependent and CTA-wide instances, compiled in their own units
cudaError_t launch_mc_f32_td(const McArgs &a, int R, int W, cudaStream_t s);
cudaError_t launch_mc_f64_td(const McArgs &a, int R, int W, cudaStream_t s);
cudaError_t launch_mc_f32_wide(const McArgs &a, cudaStream_t s);
cudaError_t launch_mc_f32_dict(const McArgs &a, cudaStream_t s);
cudaError_t launch_mc_f64_wide(const McArgs &a, cudaStream_t s);
int mc_supported(int d, int w_heff, int precision, int group);
// Dimensions above 2048: bytes of one CTA's stage slab, and the CTAs the
// launch will run (the host provides stage_ctas slabs).
size_t mc_stage_slab_bytes(int precision);
int mc_stage_ctas();
cudaError_t launch_me(const MeArgs &a, int precision, cudaStream_t s);
int me_herm_grid(int d, int precision, int n_cslots, int n_cterms);  // CTAs of the Hermitian-path launch
int me_tc_grid();  // CTAs of the tensor-core master-equation launch (<= 0 on error)
cudaError_t launch_me_tc(const MeArgs &a, const TcArgs &t, cudaStream_t s);
size_t gmres_smem_bytes(int chunk, int m);  // dynamic shared memory of the GMRES launch
int gmres_grid(size_t smem);                // resident CTAs of the GMRES kernel (<= 0 on error)
cudaError_t launch_gmres(const MeArgs &a, const GmArgs &g, int grid, size_t smem,
                         cudaStream_t s);
cudaError_t launch_identity_state(double2 *rho, int d, cudaStream_t s);
cudaError_t launch_set_status(int *status, int code, cudaStream_t s);  // first error wins
cudaError_t launch_diff_norm(const double2 *a, const double2 *b, int64_t n, double *out,
                             cudaStream_t s);
int prop_block_grid(int64_t units, int precision);  // CTAs of the propagator launch
cudaError_t launch_prop_block(const MeArgs &a, const PropArgs &p, int grid, int precision,
                              cudaStream_t s);
int corr_block_grid(int n_t, int precision);  // CTAs of the batched small-system launch
cudaError_t launch_corr_block(const MeArgs &a, const CorrArgs &c, int grid, int precision,
                              cudaStream_t s);
cudaError_t launch_corr_prepare(const OpTable &ops, const CorrArgs &c, int k, double2 *X,
                                double *times, cudaStream_t s);
cudaError_t launch_expect(const OpTable &ops, int op_index, const double2 *states, int is_ket,
                          int64_t batch, double2 *out, cudaStream_t s);
cudaError_t launch_finalize_stats(const unsigned long long *counters, const int *status,
                                  const unsigned long long *n_jumps, qt_stats *stats,
                                  cudaStream_t s);
// psi0 / |psi0| into out; with ivl_len also the output intervals of the
// mixed Monte-Carlo kernel (McArgs::ivl_tb, ivl_len) for tlist[0 .. n_t).
cudaError_t launch_normalise(const double2 *in, double2 *out, int d, int *status,
                             cudaStream_t s, const double *tlist = nullptr, int n_t = 0,
                             double *ivl_tb = nullptr, float *ivl_len = nullptr);
size_t me_workspace_bytes(int d, int precision, int grid);

// Records msg as the calling thread's last error and returns code.
int set_error(int code, const char *msg);

// The master-equation solve of qt_mesolve_dev on a caller-provided
// workspace of ws_bytes bytes (no allocation); rejects a workspace that is
// too small with QT_EINVAL.
int mesolve_dev_ws(qt_system s, const qt_c128 *state0_dev, int state_is_ket,
                   const double *tlist_dev, int n_t, const qt_opts *o, qt_c128 *expect_dev,
                   qt_c128 *states_dev, qt_stats *stats_dev, void *stream, void *ws,
                   size_t ws_bytes);
int me_grid(int d, int precision);  // CTAs of the cooperative launch (<= 0 on error)
// Loads the preallocated workspace of qt_mesolve_dev_noalloc on the current
// device (called when a system is created).
void noalloc_prepare();

}  // namespace qt
