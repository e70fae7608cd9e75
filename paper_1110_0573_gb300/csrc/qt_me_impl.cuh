// qt_me_impl.cuh -- master-equation solver (paper section 3.1,
// Eq. (master_equation)), written for a team of threads: the whole grid of a
// cooperative launch (qt_me.cu) or one CTA of the batched kernel (qt_batch.cu).
//
// The right-hand side is evaluated in its effective-Hamiltonian form,
//   d rho/dt = -i (H_eff rho - rho H_eff^dag) + sum_n C_n rho C_n^dag,
// H_eff = H - (i/2) sum_n C_n^dag C_n, which expands to the Lindblad form term
// by term (the anticommutator {C^dag C, rho} is carried by H_eff).  Each entry
// (i, j) is formed from ELLPACK rows of the operators:
//   (H_eff rho)_ij      = sum_s H_eff[i, c_s] rho[c_s, j]
//   (rho H_eff^dag)_ij  = sum_s rho[i, c_s] conj(H_eff[j, c_s])
//   (C rho C^dag)_ij    = sum_s sum_t C[i, a_s] rho[a_s, b_t] conj(C[j, b_t])
// with no assumption on the symmetry of rho.
//
// The whole Dormand-Prince integration runs inside one launch on a team of
// threads.  Every thread executes the same control flow: the stage
// combinations are element-wise and fused into the phase that produced the
// last stage, one team barrier separates the stages, and the error norm and
// the expectation values are reduced so that every thread obtains the same
// totals in the same order and all take identical decisions.
#pragma once

#include <cooperative_groups.h>

#include "qt_device.cuh"
#include "qt_internal.h"

namespace cg = cooperative_groups;

namespace qt {

namespace {

template <typename V> __device__ __forceinline__ V cconj(V v) {
  v.y = -v.y;
  return v;
}

// Stage times c_s of the Dormand-Prince stages 1..6 (k[s] at t + c_s h).
__device__ constexpr double kDpC[7] = {0.0, DP::c2, DP::c3, DP::c4, DP::c5, 1.0, 1.0};

// f_k(t) of time-dependent term k (paper section 4.3).
__device__ __forceinline__ double td_coef_at(const MeArgs &a, int k, double t) {
  return td_piecewise(a.td_t, a.td_v, a.td_off[k], a.td_off[k + 1] - 1, t);
}

template <typename T>
struct Me {
  using V = typename CT<T>::V;
  const MeArgs &a;
  const int d;
  const int64_t n;  // d * d
  const V *val;
  const double *tdcoef = nullptr;  // f_k at the current stage time (shared memory)

  __device__ Me(const MeArgs &a_, const V *val_)
      : a(a_), d(a_.ops.d), n((int64_t)a_.ops.d * a_.ops.d), val(val_) {}

  // f_k(t) of the time-dependent terms into tdcoef (threads 0..n_td-1 of each
  // CTA; the caller synchronises the CTA before the values are read).
  __device__ __forceinline__ void td_eval(double t, double *coef) const {
    if ((int)threadIdx.x < a.n_td) coef[threadIdx.x] = td_coef_at(a, (int)threadIdx.x, t);
  }

  // sum_n (C_n y C_n^dag)_ij added to out, from the ELL rows i and j of C_n.
  // The FP32 solver adds the products with the FP32 remainders of C_n's
  // entries to first order (C = hi + lo): the jump terms then use the same C
  // as the anticommutator carried by H_eff (whose remainders rhs() adds), so
  // the trace is conserved to FP32 rounding instead of drifting with the
  // mismatch of two separately rounded copies of C.
  __device__ __forceinline__ void collapse(const V *__restrict__ y, int i, int j, V &out) const {
    const V *vlo = sizeof(T) == 4 ? reinterpret_cast<const V *>(a.ops.val32lo) : nullptr;
    V outl = cmake<V>(0.0, 0.0);
    for (int c = 1; c <= a.n_c; ++c) {
      const int wc = a.ops.w[c];
      const int64_t offc = a.ops.off[c];
      for (int s = 0; s < wc; ++s) {
        const int64_t ps = offc + (int64_t)s * d + i;
        const V u = val[ps];
        const V *yrow = y + (int64_t)__ldg(a.ops.col + ps) * d;
        V inner = cmake<V>(0.0, 0.0), innerl = cmake<V>(0.0, 0.0);
        for (int t = 0; t < wc; ++t) {
          const int64_t pt = offc + (int64_t)t * d + j;
          const V yv = yrow[__ldg(a.ops.col + pt)];
          cmac(inner, yv, cconj(val[pt]));
          if constexpr (sizeof(T) == 4) cmac(innerl, yv, cconj(__ldg(vlo + pt)));
        }
        cmac(out, u, inner);
        if constexpr (sizeof(T) == 4) {
          cmac(outl, __ldg(vlo + ps), inner);
          cmac(outl, u, innerl);
        }
      }
    }
    if constexpr (sizeof(T) == 4) {
      out.x += outl.x;
      out.y += outl.y;
    }
  }

  // drho/dt at entry (i, j) of the state y.  The FP32 solver adds the
  // products with the FP32 remainders of H_eff's entries (H_eff = hi + lo to
  // ~2^-48), so that its Hamiltonian carries no systematic rounding.
  __device__ __forceinline__ V rhs(const V *__restrict__ y, int i, int j) const {
    const int w0 = a.ops.w[0];
    const int64_t off0 = a.ops.off[0];
    V Y = cmake<V>(0.0, 0.0), Z = cmake<V>(0.0, 0.0);
    V Yl = cmake<V>(0.0, 0.0), Zl = cmake<V>(0.0, 0.0);
    const V *vlo = sizeof(T) == 4 ? reinterpret_cast<const V *>(a.ops.val32lo) : nullptr;
    for (int s = 0; s < w0; ++s) {
      const int64_t pi = off0 + (int64_t)s * d + i;
      const V yi = y[(int64_t)__ldg(a.ops.col + pi) * d + j];
      cmac(Y, val[pi], yi);
      const int64_t pj = off0 + (int64_t)s * d + j;
      const V yj = y[(int64_t)i * d + __ldg(a.ops.col + pj)];
      cmac(Z, yj, cconj(val[pj]));
      if constexpr (sizeof(T) == 4) {
        cmac(Yl, __ldg(vlo + pi), yi);
        cmac(Zl, yj, cconj(__ldg(vlo + pj)));
      }
    }
    if constexpr (sizeof(T) == 4) {
      Y.x += Yl.x;
      Y.y += Yl.y;
      Z.x += Zl.x;
      Z.y += Zl.y;
    }
    for (int k = 0; k < a.n_td; ++k) {  // f_k(t) (H_k y - y H_k)
      const T f = (T)tdcoef[k];
      const int op = a.td_op0 + k;
      const int wk = a.ops.w[op];
      const int64_t offk = a.ops.off[op];
      V Yk = cmake<V>(0.0, 0.0), Zk = cmake<V>(0.0, 0.0);
      for (int s = 0; s < wk; ++s) {
        const int64_t pi = offk + (int64_t)s * d + i;
        cmac(Yk, val[pi], y[(int64_t)__ldg(a.ops.col + pi) * d + j]);
        const int64_t pj = offk + (int64_t)s * d + j;
        cmac(Zk, y[(int64_t)i * d + __ldg(a.ops.col + pj)], cconj(val[pj]));
      }
      Y.x = tfma(f, Yk.x, Y.x);
      Y.y = tfma(f, Yk.y, Y.y);
      Z.x = tfma(f, Zk.x, Z.x);
      Z.y = tfma(f, Zk.y, Z.y);
    }
    V out;
    out.x = Y.y - Z.y;     // -i (Y - Z)
    out.y = -(Y.x - Z.x);
    collapse(y, i, j, out);
    return out;
  }
};

// Right-hand-side provider of the sparse path: every entry of drho/dt from
// the ELL rows of H_eff and C_n (Me::rhs).  The solver calls
//   store(buf, idx, i, j, v)  for every entry of a stage input it writes,
//   publish(team)             once all entries of that input are written,
//   prepare(y, t)             before the entries of f(y) at time t are evaluated,
//   f(y, i, j)                for each entry.
// A provider that precomputes products (the tensor-core path) does its work
// in publish/prepare; here they reduce to a team barrier and nothing.
template <typename T>
struct SparseRhs {
  using V = typename CT<T>::V;
  static constexpr bool kCanFail = false;
  Me<T> me;
  double *coef;  // shared memory, kTdMax values
  __device__ SparseRhs(const MeArgs &a, const V *val, double *coef_ = nullptr) : me(a, val), coef(coef_) {
    me.tdcoef = coef_;
  }
  __device__ __forceinline__ void store(V *buf, int64_t idx, int, int, V v) { buf[idx] = v; }
  template <typename Team> __device__ __forceinline__ void publish(Team &team) { team.sync(); }
  // the coefficients of the time-dependent terms at the time of this
  // right-hand side (the previous phase ended with a team barrier)
  __device__ __forceinline__ void prepare(const V *, double t) {
    if (me.a.n_td > 0) {
      me.td_eval(t, coef);
      __syncthreads();
    }
  }
  __device__ __forceinline__ V f(const V *__restrict__ y, int i, int j) const { return me.rhs(y, i, j); }
  __device__ __forceinline__ int failed() const { return 0; }
};

// Slot of the CTA total in the reduction scratch sh (after one row of
// kMePartialMax per warp); sh holds kMePartialMax * (warps + 1) doubles.
__device__ __forceinline__ int sh_total() { return kMePartialMax * (int)(blockDim.x >> 5); }

// Sum over the CTA of nv values per thread; returns the totals in
// sh[sh_total() + 0..nv).
__device__ __forceinline__ void block_sum(double *v, int nv, double *sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  for (int q = 0; q < nv; ++q) {
    double x = v[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) sh[warp * kMePartialMax + q] = x;
  }
  __syncthreads();
  if (threadIdx.x < nv) {
    double x = 0.0;
    for (int w = 0; w < nw; ++w) x += sh[w * kMePartialMax + threadIdx.x];
    sh[sh_total() + threadIdx.x] = x;
  }
  __syncthreads();
}

// Grid-wide sum of nv values per thread, identical in every CTA.  Ends with
// the totals in tot[0..nv) (shared memory).
__device__ __forceinline__ void grid_sum(double *v, int nv, double *sh, double *partial, double *tot,
                         cg::grid_group &grid) {
  block_sum(v, nv, sh);
  if (threadIdx.x < nv)
    partial[(int64_t)blockIdx.x * kMePartialMax + threadIdx.x] = sh[sh_total() + threadIdx.x];
  grid.sync();
  // warp 0 of every CTA adds the partials of all CTAs in the same order
  if (threadIdx.x < 32) {
    for (int q = 0; q < nv; ++q) {
      double x = 0.0;
      for (int b = threadIdx.x; b < (int)gridDim.x; b += 32)
        x += partial[(int64_t)b * kMePartialMax + q];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      if (threadIdx.x == 0) tot[q] = x;
    }
  }
  __syncthreads();
}

// Team of the cooperative launch: all threads of the grid.
struct GridTeam {
  cg::grid_group grid;
  int64_t tid, stride;
  double *partial;
  __device__ GridTeam(double *partial_)
      : grid(cg::this_grid()), tid((int64_t)blockIdx.x * blockDim.x + threadIdx.x),
        stride((int64_t)gridDim.x * blockDim.x), partial(partial_) {}
  __device__ __forceinline__ void sync() { grid.sync(); }
  __device__ __forceinline__ void sum(double *v, int nv, double *sh, double *tot) {
    grid_sum(v, nv, sh, partial, tot, grid);
  }
  __device__ __forceinline__ bool first_block() const { return blockIdx.x == 0; }
};

// Team of one CTA (the batched kernel).
struct BlockTeam {
  int64_t tid, stride;
  __device__ BlockTeam() : tid(threadIdx.x), stride(blockDim.x) {}
  __device__ __forceinline__ void sync() { __syncthreads(); }
  __device__ __forceinline__ void sum(double *v, int nv, double *sh, double *tot) {
    block_sum(v, nv, sh);
    if (threadIdx.x < nv) tot[threadIdx.x] = sh[sh_total() + threadIdx.x];
    __syncthreads();
  }
  __device__ __forceinline__ bool first_block() const { return true; }
};

// Step-size controller of the master-equation solvers: the shared FP64 rule
// for the FP64 solvers; the same rule evaluated in FP32 for the mixed solvers
// (as in the mixed Monte-Carlo kernel), which keeps FP64 pow off every
// thread's path.
template <typename T>
__device__ __forceinline__ double me_control(double h, double err, bool accepted,
                                             bool after_reject, bool clipped, double hprop) {
  if constexpr (sizeof(T) == 8) {
    return dp_control(h, err, accepted, after_reject, clipped, hprop);
  } else {
    const float p = __powf((float)err, -0.2f);
    if (accepted) {
      const float facmax = after_reject ? 1.f : 5.f;
      const float fac = (err == 0.0) ? facmax : fminf(facmax, fmaxf(0.2f, 0.9f * p));
      double hn = h * (double)fac;
      if (clipped && hn < hprop) hn = hprop;
      return hn;
    }
    return h * (double)fmaxf(0.2f, 0.9f * p);
  }
}

// Scaled RMS error from the sum of squares over the 2n real components: in
// FP64 for the FP64 solvers, in FP32 for the mixed ones (an FP32 state's
// error estimate carries no more digits).
template <typename T>
__device__ __forceinline__ double me_error(double sum_sq, int64_t n) {
  if constexpr (sizeof(T) == 8) return sqrt(sum_sq / (2.0 * (double)n));
  else return (double)sqrtf((float)sum_sq * (0.5f / (float)n));
}

// The solve of one system by a team with the right-hand side of the provider
// rhs; sh[kMePartialMax * (warps + 1)] and tot[kMePartialMax] are
// shared-memory scratch of the calling CTA.
template <typename T, typename Team, typename Rhs>
__device__ void me_solve(const MeArgs &a, Team &team, Rhs &rhs, double *sh, double *tot) {
  using V = typename CT<T>::V;

  const int d = a.ops.d;
  const int64_t n = (int64_t)d * d;
  V *base = reinterpret_cast<V *>(a.work);
  V *rho = base, *ynew = base + n, *buf0 = base + 2 * n, *buf1 = base + 3 * n;
  V *k[7];
#pragma unroll
  for (int s = 0; s < 7; ++s) k[s] = base + (4 + s) * n;
  const int64_t tid = team.tid;
  const int64_t stride = team.stride;
  double v[kMePartialMax];

  // ---- initial state: rho0 = |psi><psi| / <psi|psi> or the given matrix
  double scale = 1.0;
  if (a.state_is_ket) {
    v[0] = 0.0;
    for (int64_t i = tid; i < d; i += stride)
      v[0] += a.state0[i].x * a.state0[i].x + a.state0[i].y * a.state0[i].y;
    team.sum(v, 1, sh, tot);
    if (!(tot[0] > 0.0)) {
      if (tid == 0) set_status(a.status, QT_ENORM);
      return;
    }
    scale = 1.0 / tot[0];
  }
  for (int64_t idx = tid; idx < n; idx += stride) {
    const int i = (int)(idx / d), j = (int)(idx % d);
    double2 r;
    if (a.state_is_ket) {
      const double2 p = a.state0[i], q = a.state0[j];  // p conj(q)
      r = make_double2((p.x * q.x + p.y * q.y) * scale, (p.y * q.x - p.x * q.y) * scale);
    } else {
      r = a.state0[idx];
    }
    rhs.store(rho, idx, i, j, cmake<V>(r.x, r.y));
  }
  rhs.publish(team);

  unsigned long long n_acc = 0, n_rej = 0, n_rhs = 0;
  auto eval = [&](const V *y, V *out, double te) {
    rhs.prepare(y, te);
    for (int64_t idx = tid; idx < n; idx += stride)
      out[idx] = rhs.f(y, (int)(idx / d), (int)(idx % d));
    ++n_rhs;
  };
  // Expectation values Tr(O rho) and the optional state copy at output m.
  const V *val = sizeof(T) == 8 ? reinterpret_cast<const V *>(a.ops.val64)
                                : reinterpret_cast<const V *>(a.ops.val32);
  auto output = [&](int m, const V *y) {
    if (a.states)
      for (int64_t idx = tid; idx < n; idx += stride)
        a.states[(int64_t)m * n + idx] = make_double2((double)y[idx].x, (double)y[idx].y);
    for (int e0 = 0; e0 < a.n_e; e0 += kMePartialMax / 2) {
      const int ne = min(a.n_e - e0, kMePartialMax / 2);
      for (int q = 0; q < 2 * ne; ++q) v[q] = 0.0;
      for (int64_t i = tid; i < d; i += stride) {
        for (int e = 0; e < ne; ++e) {
          const int op = 1 + a.n_c + e0 + e;
          const int w = a.ops.w[op];
          const int64_t off = a.ops.off[op];
          for (int s = 0; s < w; ++s) {
            const int64_t p = off + (int64_t)s * d + i;
            const V o = val[p];
            const V r = y[(int64_t)__ldg(a.ops.col + p) * d + i];  // O[i,c] rho[c,i]
            v[2 * e] += (double)o.x * r.x - (double)o.y * r.y;
            v[2 * e + 1] += (double)o.x * r.y + (double)o.y * r.x;
          }
        }
      }
      team.sum(v, 2 * ne, sh, tot);
      if (team.first_block() && threadIdx.x < ne)
        a.expect[(int64_t)m * a.n_e + e0 + threadIdx.x] =
            make_double2(tot[2 * threadIdx.x], tot[2 * threadIdx.x + 1]);
      team.sync();  // tot / partial are reused by the next reduction
    }
  };

  eval(rho, k[0], a.tlist[0]);
  output(0, rho);
  int status = QT_OK;
  if (a.n_t > 1) {
    double t = a.tlist[0];
    double hprop = a.h0;
    if (!(hprop > 0.0)) {
      // Hairer-Norsett-Wanner starting step (k[1], buf0 as scratch)
      team.sync();  // k[0] complete
      v[0] = v[1] = 0.0;
      for (int64_t idx = tid; idx < n; idx += stride) {
        const V r = rho[idx], f = k[0][idx];
        const double sx = a.atol + a.rtol * fabs((double)r.x);
        const double sy = a.atol + a.rtol * fabs((double)r.y);
        v[0] += ((double)r.x / sx) * ((double)r.x / sx) + ((double)r.y / sy) * ((double)r.y / sy);
        v[1] += ((double)f.x / sx) * ((double)f.x / sx) + ((double)f.y / sy) * ((double)f.y / sy);
      }
      team.sum(v, 2, sh, tot);
      const double nr = 2.0 * (double)n;
      const double d0 = sqrt(tot[0] / nr), d1 = sqrt(tot[1] / nr);
      const double h0 = (d0 < 1e-5 || d1 < 1e-5) ? 1e-6 : 0.01 * d0 / d1;
      for (int64_t idx = tid; idx < n; idx += stride) {
        const V r = rho[idx], f = k[0][idx];
        rhs.store(buf0, idx, (int)(idx / d), (int)(idx % d),
                  cmake<V>((double)r.x + h0 * (double)f.x, (double)r.y + h0 * (double)f.y));
      }
      rhs.publish(team);
      eval(buf0, k[1], t + h0);
      v[0] = 0.0;
      for (int64_t idx = tid; idx < n; idx += stride) {
        const V r = rho[idx];
        const double sx = a.atol + a.rtol * fabs((double)r.x);
        const double sy = a.atol + a.rtol * fabs((double)r.y);
        const double ex = ((double)k[1][idx].x - (double)k[0][idx].x) / sx;
        const double ey = ((double)k[1][idx].y - (double)k[0][idx].y) / sy;
        v[0] += ex * ex + ey * ey;
      }
      team.sum(v, 1, sh, tot);
      const double d2 = sqrt(tot[0] / nr) / h0;
      const double dm = fmax(d1, d2);
      const double h1 = (dm <= 1e-15) ? fmax(1e-6, h0 * 1e-3) : pow(0.01 / dm, 0.2);
      hprop = fmin(100.0 * h0, h1);
    }
    bool after_reject = false;
    for (int m = 1; m < a.n_t && status == QT_OK; ++m) {
      const double tk = a.tlist[m];
      int64_t attempts = 0;
      while (t < tk) {
        if (attempts++ >= a.max_steps) { status = QT_ESTEP; break; }
        const bool clipped = hprop >= tk - t;
        const double h = clipped ? tk - t : hprop;
        if (!clipped && h < dp_hmin(t, tk)) { status = QT_ESTEP; break; }
        const T ht = (T)h;
        // stage 2 input
        for (int64_t idx = tid; idx < n; idx += stride) {
          const V r = rho[idx], f0 = k[0][idx];
          V y;
          y.x = fma(ht, DPW<T>::a21 * f0.x, r.x);
          y.y = fma(ht, DPW<T>::a21 * f0.y, r.y);
          rhs.store(buf0, idx, (int)(idx / d), (int)(idx % d), y);
        }
        rhs.publish(team);
        // stages 2..6, each fused with the next stage input
#pragma unroll 1
        for (int st = 1; st <= 5; ++st) {
          const V *in = (st & 1) ? buf0 : buf1;
          V *nxt = (st == 5) ? ynew : ((st & 1) ? buf1 : buf0);
          rhs.prepare(in, stage_time(t, kDpC[st], h));
          for (int64_t idx = tid; idx < n; idx += stride) {
            const int i = (int)(idx / d), j = (int)(idx % d);
            const V f = rhs.f(in, i, j);
            k[st][idx] = f;
            T ax, ay;
            const V f0 = k[0][idx];
            const V r = rho[idx];
#define QT_A(c, K) ax = fma((T)(c), (K).x, ax); ay = fma((T)(c), (K).y, ay);
            if (st == 1) {
              ax = DPW<T>::a31 * f0.x; ay = DPW<T>::a31 * f0.y; QT_A(DPW<T>::a32, f)
            } else if (st == 2) {
              ax = DPW<T>::a41 * f0.x; ay = DPW<T>::a41 * f0.y; QT_A(DPW<T>::a42, k[1][idx])
              QT_A(DPW<T>::a43, f)
            } else if (st == 3) {
              ax = DPW<T>::a51 * f0.x; ay = DPW<T>::a51 * f0.y; QT_A(DPW<T>::a52, k[1][idx])
              QT_A(DPW<T>::a53, k[2][idx]) QT_A(DPW<T>::a54, f)
            } else if (st == 4) {
              ax = DPW<T>::a61 * f0.x; ay = DPW<T>::a61 * f0.y; QT_A(DPW<T>::a62, k[1][idx])
              QT_A(DPW<T>::a63, k[2][idx]) QT_A(DPW<T>::a64, k[3][idx]) QT_A(DPW<T>::a65, f)
            } else {
              ax = DPW<T>::b1 * f0.x; ay = DPW<T>::b1 * f0.y; QT_A(DPW<T>::b3, k[2][idx])
              QT_A(DPW<T>::b4, k[3][idx]) QT_A(DPW<T>::b5, k[4][idx]) QT_A(DPW<T>::b6, f)
            }
            V y;
            y.x = fma(ht, ax, r.x);
            y.y = fma(ht, ay, r.y);
            rhs.store(nxt, idx, i, j, y);
          }
          ++n_rhs;
          rhs.publish(team);
        }
        // k7 = f(ynew) fused with the error norm
        rhs.prepare(ynew, t + h);
        v[0] = 0.0;
        {
          const T at = (T)a.atol, rt = (T)a.rtol;
          T acc = (T)0;
          for (int64_t idx = tid; idx < n; idx += stride) {
            const V f = rhs.f(ynew, (int)(idx / d), (int)(idx % d));
            k[6][idx] = f;
            const V f0 = k[0][idx];
            T ax = DPW<T>::e1 * f0.x, ay = DPW<T>::e1 * f0.y;
            QT_A(DPW<T>::e3, k[2][idx]) QT_A(DPW<T>::e4, k[3][idx]) QT_A(DPW<T>::e5, k[4][idx])
            QT_A(DPW<T>::e6, k[5][idx]) QT_A(DPW<T>::e7, f)
#undef QT_A
            ax *= ht;
            ay *= ht;
            const V r = rho[idx], yn = ynew[idx];
            const T sx = at + rt * fmax(fabs(r.x), fabs(yn.x));
            const T sy = at + rt * fmax(fabs(r.y), fabs(yn.y));
            const T qx = ax / sx, qy = ay / sy;
            acc = fma(qx, qx, acc);
            acc = fma(qy, qy, acc);
          }
          v[0] = (double)acc;
        }
        ++n_rhs;
        if constexpr (Rhs::kCanFail) {
          // a provider whose bounded device waits ran out reports it here, in
          // the same reduction as the error norm, so that every CTA stops
          v[1] = (double)rhs.failed();
          team.sum(v, 2, sh, tot);
          if (tot[1] != 0.0) { status = QT_ETIMEOUT; break; }
        } else {
          team.sum(v, 1, sh, tot);
        }
        const double err = me_error<T>(tot[0], n);
        if (!isfinite(err)) { status = QT_ENUMERIC; break; }
        if (err <= 1.0) {
          hprop = me_control<T>(h, err, true, after_reject, clipped, hprop);
          after_reject = false;
          t = clipped ? tk : t + h;
          V *sw = rho; rho = ynew; ynew = sw;
          sw = k[0]; k[0] = k[6]; k[6] = sw;
          ++n_acc;
        } else {
          hprop = me_control<T>(h, err, false, after_reject, clipped, hprop);
          after_reject = true;
          ++n_rej;
        }
        team.sync();  // tot is rewritten by the next reduction
      }
      if (status != QT_OK) break;
      output(m, rho);
    }
  }
  if constexpr (Rhs::kCanFail) {
    // a run with no step still reports a provider failure
    if (status == QT_OK) {
      v[0] = (double)rhs.failed();
      team.sum(v, 1, sh, tot);
      if (tot[0] != 0.0) status = QT_ETIMEOUT;
    }
  }
  if (status != QT_OK && tid == 0) set_status(a.status, status);
  if (tid == 0) {
    atomicAdd(a.counters + 0, n_acc);
    atomicAdd(a.counters + 1, n_rej);
    atomicAdd(a.counters + 2, n_rhs);
  }
}

// One evaluation of drho/dt: a.rhs_in (FP64, d*d) -> a.rhs_out (FP64), with
// the state rounded to the provider's type first.
template <typename T, typename Team, typename Rhs>
__device__ void me_rhs_once(const MeArgs &a, Team &team, Rhs &rhs, double *sh, double *tot) {
  using V = typename CT<T>::V;
  const int d = a.ops.d;
  const int64_t n = (int64_t)d * d;
  V *y = reinterpret_cast<V *>(a.work);
  for (int64_t idx = team.tid; idx < n; idx += team.stride) {
    const double2 r = a.rhs_in[idx];
    rhs.store(y, idx, (int)(idx / d), (int)(idx % d), cmake<V>(r.x, r.y));
  }
  rhs.publish(team);
  rhs.prepare(y, a.rhs_t);
  for (int64_t idx = team.tid; idx < n; idx += team.stride) {
    const V f = rhs.f(y, (int)(idx / d), (int)(idx % d));
    a.rhs_out[idx] = make_double2((double)f.x, (double)f.y);
  }
  if constexpr (Rhs::kCanFail) {
    double v[1] = {(double)rhs.failed()};
    team.sum(v, 1, sh, tot);
    if (tot[0] != 0.0 && team.tid == 0) set_status(a.status, QT_ETIMEOUT);
  }
}

}  // namespace

}  // namespace qt
