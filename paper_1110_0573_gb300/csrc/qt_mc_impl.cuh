// qt_mc_impl.cuh -- persistent Monte-Carlo wave-function kernel (paper
// section 3.2), instantiated per precision by qt_mc_f64.cu and qt_mc_f32.cu.
//
// One group of G lanes (G = 32: one warp) integrates one trajectory at a
// time and then takes the next trajectory index from a device counter, until
// the range is exhausted.  Lane l of a group owns rows l, l + G, ..., l + (R-1) G
// of the state: every Dormand-Prince stage vector of the trajectory lives in
// that lane's registers for the whole run, so a trajectory never leaves the
// chip.  H_eff = H - (i/2) sum_n C_n^dag C_n (Eq. (heff)) is applied as an
// ELLPACK product: each lane keeps the stored entries of its own rows in
// registers (template W > 0) or reads them through the read-only cache
// (W == 0), and gathers the needed state components from a per-group copy of
// the vector in shared memory.
//
// Per trajectory the kernel runs steps I-IV of the paper's algorithm:
//   I    r = U(seed, j, k, 0);
//   II   adaptive Dormand-Prince steps of d psi/dt = -i H_eff psi; after each
//        accepted step <psi|psi> is compared with r; at a crossing the jump
//        time is bracketed by bisection on trial steps of length (tau - t)
//        from the accepted state (t, psi);
//   III  p_n = ||C_n psi(tau)||^2 (Eq. (pcn)), r2 = U(seed, j, k, 1), the
//        smallest n with sum_{i<=n} p_i >= r2 sum_i p_i (Eq. (mc3)),
//        psi <- C_n psi / sqrt(p_n) (Eq. (project));
//   IV   k <- k + 1, new r, continue from tau.
// At each output time the normalised expectations <psi|O_m|psi>/<psi|psi> are
// accumulated in FP64 (per CTA in shared memory, flushed once at the end).
//
// Precision: T = double runs everything in FP64.  T = float keeps the state
// and the stages in complex FP32 and does in FP64: t and h, the norm-decay
// comparison (an FP32 sum decides only when it is provably on the same side
// of r as the FP64 sum of the same values; otherwise the FP64 sum is formed),
// the collapse weights, the renormalisation and the expectation values.
#pragma once

#include "qt_device.cuh"
#include "qt_internal.h"

namespace qt {

namespace {

constexpr int kBlock = 128;

template <typename T, int G, int R, int W>
struct Traj {
  using V = typename CT<T>::V;
  static constexpr int WR = W > 0 ? W : 1;

  const McArgs &a;
  const int lane;
  const unsigned mask;
  const int d;
  V *ybuf;
  const V *val;      // operator values in the kernel's precision
  int wh;            // ELL width of H_eff
  float inv2d;       // 1 / (2 d)
  V hv[R][WR];       // this lane's H_eff entries (W > 0)
  int hc[R][WR];
  // statistics of this group (kept by every lane, flushed by lane 0)
  unsigned long long n_acc = 0, n_rej = 0, n_rhs = 0, n_bis = 0, n_jmp = 0, n_near = 0;

  __device__ Traj(const McArgs &a_, int lane_, unsigned mask_, V *ybuf_, const V *val_)
      : a(a_), lane(lane_), mask(mask_), d(a_.ops.d), ybuf(ybuf_), val(val_) {
    wh = a.ops.w[0];
    inv2d = 1.0f / (float)(2 * d);
    if (W > 0) {
      const int64_t off = a.ops.off[0];
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const int row = lane + q * G;
#pragma unroll
        for (int s = 0; s < WR; ++s) {
          if (row < d && s < wh) {
            hv[q][s] = val[off + (int64_t)s * d + row];
            hc[q][s] = a.ops.col[off + (int64_t)s * d + row];
          } else {
            hv[q][s] = cmake<V>(0.0, 0.0);
            hc[q][s] = 0;
          }
        }
      }
    }
  }

  __device__ __forceinline__ int row(int q) const { return lane + q * G; }

  // Publish y to the group's shared buffer.
  __device__ __forceinline__ void publish(const V (&y)[R]) {
    __syncwarp(mask);
#pragma unroll
    for (int q = 0; q < R; ++q)
      if (row(q) < d) ybuf[row(q)] = y[q];
    __syncwarp(mask);
  }

  // k = -i H_eff y.
  __device__ __forceinline__ void rhs(const V (&y)[R], V (&k)[R]) {
    publish(y);
    ++n_rhs;
#pragma unroll
    for (int q = 0; q < R; ++q) {
      V acc = cmake<V>(0.0, 0.0);
      if (W > 0) {
#pragma unroll
        for (int s = 0; s < WR; ++s)
          if (s < wh) cmac(acc, hv[q][s], ybuf[hc[q][s]]);
      } else if (row(q) < d) {
        const int64_t off = a.ops.off[0];
        for (int s = 0; s < wh; ++s) {
          const int64_t p = off + (int64_t)s * d + row(q);
          cmac(acc, val[p], ybuf[__ldg(a.ops.col + p)]);
        }
      }
      k[q].x = acc.y;   // -i (x + i y) = y - i x
      k[q].y = -acc.x;
    }
  }

  // (op y) for this lane's rows, op = index into the operator table; y must
  // already be published.
  __device__ __forceinline__ V apply_row(int op, int q) const {
    V acc = cmake<V>(0.0, 0.0);
    const int r = row(q);
    if (r >= d) return acc;
    const int w = a.ops.w[op];
    const int64_t off = a.ops.off[op];
    for (int s = 0; s < w; ++s) {
      const int64_t p = off + (int64_t)s * d + r;
      cmac(acc, val[p], ybuf[__ldg(a.ops.col + p)]);
    }
    return acc;
  }

  // <y|y> summed in FP64 over the group.
  __device__ __forceinline__ double norm2_64(const V (&y)[R]) const {
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const double x = (double)y[q].x, z = (double)y[q].y;
      s = fma(x, x, s);
      s = fma(z, z, s);
    }
    return group_sum<G>(s, mask);
  }

  // Is <y|y> <= r?  Decided as the FP64 sum of the stored values decides it.
  __device__ __forceinline__ bool below(const V (&y)[R], double r, double &n2) const {
    if constexpr (sizeof(T) == 8) {
      n2 = norm2_64(y);
      return n2 <= r;
    }
    float s = 0.f;
#pragma unroll
    for (int q = 0; q < R; ++q) {
      s = fmaf((float)y[q].x, (float)y[q].x, s);
      s = fmaf((float)y[q].y, (float)y[q].y, s);
    }
    s = group_sum<G>(s, mask);
    n2 = (double)s;
    // The FP32 sum of 2R products per lane and log2(G) tree levels is within
    // (2R + log2 G + 2) * 2^-24 of the exact sum; 1e-5 leaves a wide margin.
    if (fabs(n2 - r) > 1e-5 * r) return n2 <= r;
    n2 = norm2_64(y);
    return n2 <= r;
  }

  // One Dormand-Prince step of length h from (psi, k[0] = f(psi)).  Writes the
  // 5th-order solution to ynew; with want_err evaluates k[6] = f(ynew) and
  // returns the scaled RMS error norm, else returns 0.
  __device__ __forceinline__ T step(const V (&psi)[R], V (&k)[7][R], T h, V (&ynew)[R],
                                    bool want_err) {
    const T ht = h;
    V yt[R];
#define QT_STAGE(EXPR)                                   \
  _Pragma("unroll") for (int q = 0; q < R; ++q) {        \
    T ax, ay;                                            \
    EXPR;                                                \
    yt[q].x = fma(ht, ax, psi[q].x);                     \
    yt[q].y = fma(ht, ay, psi[q].y);                     \
  }
#define QT_ACC(c, j)                  \
  ax = fma((T)(c), k[j][q].x, ax);    \
  ay = fma((T)(c), k[j][q].y, ay);
    QT_STAGE(ax = (T)DP::a21 * k[0][q].x; ay = (T)DP::a21 * k[0][q].y)
    rhs(yt, k[1]);
    QT_STAGE(ax = (T)DP::a31 * k[0][q].x; ay = (T)DP::a31 * k[0][q].y; QT_ACC(DP::a32, 1))
    rhs(yt, k[2]);
    QT_STAGE(ax = (T)DP::a41 * k[0][q].x; ay = (T)DP::a41 * k[0][q].y; QT_ACC(DP::a42, 1)
                 QT_ACC(DP::a43, 2))
    rhs(yt, k[3]);
    QT_STAGE(ax = (T)DP::a51 * k[0][q].x; ay = (T)DP::a51 * k[0][q].y; QT_ACC(DP::a52, 1)
                 QT_ACC(DP::a53, 2) QT_ACC(DP::a54, 3))
    rhs(yt, k[4]);
    QT_STAGE(ax = (T)DP::a61 * k[0][q].x; ay = (T)DP::a61 * k[0][q].y; QT_ACC(DP::a62, 1)
                 QT_ACC(DP::a63, 2) QT_ACC(DP::a64, 3) QT_ACC(DP::a65, 4))
    rhs(yt, k[5]);
#pragma unroll
    for (int q = 0; q < R; ++q) {
      T ax = (T)DP::b1 * k[0][q].x, ay = (T)DP::b1 * k[0][q].y;
      QT_ACC(DP::b3, 2) QT_ACC(DP::b4, 3) QT_ACC(DP::b5, 4) QT_ACC(DP::b6, 5)
      ynew[q].x = fma(ht, ax, psi[q].x);
      ynew[q].y = fma(ht, ay, psi[q].y);
    }
#undef QT_STAGE
    if (!want_err) return (T)0;
    rhs(ynew, k[6]);
    T sum = (T)0;
    const T at = (T)a.atol, rt = (T)a.rtol;
#pragma unroll
    for (int q = 0; q < R; ++q) {
      if (row(q) >= d) continue;
      T ax = (T)DP::e1 * k[0][q].x, ay = (T)DP::e1 * k[0][q].y;
      QT_ACC(DP::e3, 2) QT_ACC(DP::e4, 3) QT_ACC(DP::e5, 4) QT_ACC(DP::e6, 5) QT_ACC(DP::e7, 6)
      ax *= ht;
      ay *= ht;
      const T sx = at + rt * fmax(fabs(psi[q].x), fabs(ynew[q].x));
      const T sy = at + rt * fmax(fabs(psi[q].y), fabs(ynew[q].y));
      T qx, qy;
      if constexpr (sizeof(T) == 8) {
        qx = ax / sx;
        qy = ay / sy;
      } else {
        qx = (T)__fdividef((float)ax, (float)sx);
        qy = (T)__fdividef((float)ay, (float)sy);
      }
      sum = fma(qx, qx, sum);
      sum = fma(qy, qy, sum);
    }
#undef QT_ACC
    sum = group_sum<G>(sum, mask);
    if constexpr (sizeof(T) == 8) {
      return sqrt(sum / (double)(2 * d));
    } else {
      return sqrtf(sum * inv2d);
    }
  }

  // Step-size controller in the scalar precision of the kernel: the FP64
  // kernel uses the shared FP64 rule; the mixed kernel the same rule in FP32.
  __device__ __forceinline__ T control(T h, T err, bool accepted, bool after_reject,
                                       bool clipped, T hprop) const {
    if constexpr (sizeof(T) == 8) {
      return dp_control(h, err, accepted, after_reject, clipped, hprop);
    } else {
      const float p = __powf(err, -0.2f);
      if (accepted) {
        const float facmax = after_reject ? 1.f : 5.f;
        const float fac = (err == 0.f) ? facmax : fminf(facmax, fmaxf(0.2f, 0.9f * p));
        float hn = h * fac;
        if (clipped && hn < hprop) hn = hprop;
        return hn;
      }
      return h * fmaxf(0.2f, 0.9f * p);
    }
  }

  // Hairer-Norsett-Wanner starting step; k[0] = f(psi).  Uses k[1].
  __device__ double initial_step(const V (&psi)[R], V (&k)[7][R]) {
    double s0 = 0.0, s1 = 0.0;
#pragma unroll
    for (int q = 0; q < R; ++q) {
      if (row(q) >= d) continue;
      const double scx = a.atol + a.rtol * fabs((double)psi[q].x);
      const double scy = a.atol + a.rtol * fabs((double)psi[q].y);
      s0 += ((double)psi[q].x / scx) * ((double)psi[q].x / scx) +
            ((double)psi[q].y / scy) * ((double)psi[q].y / scy);
      s1 += ((double)k[0][q].x / scx) * ((double)k[0][q].x / scx) +
            ((double)k[0][q].y / scy) * ((double)k[0][q].y / scy);
    }
    const double n = 2.0 * d;
    const double d0 = sqrt(group_sum<G>(s0, mask) / n);
    const double d1 = sqrt(group_sum<G>(s1, mask) / n);
    const double h0 = (d0 < 1e-5 || d1 < 1e-5) ? 1e-6 : 0.01 * d0 / d1;
    V yt[R];
#pragma unroll
    for (int q = 0; q < R; ++q) {
      yt[q].x = (T)((double)psi[q].x + h0 * (double)k[0][q].x);
      yt[q].y = (T)((double)psi[q].y + h0 * (double)k[0][q].y);
    }
    rhs(yt, k[1]);
    double s2 = 0.0;
#pragma unroll
    for (int q = 0; q < R; ++q) {
      if (row(q) >= d) continue;
      const double scx = a.atol + a.rtol * fabs((double)psi[q].x);
      const double scy = a.atol + a.rtol * fabs((double)psi[q].y);
      const double ex = ((double)k[1][q].x - (double)k[0][q].x) / scx;
      const double ey = ((double)k[1][q].y - (double)k[0][q].y) / scy;
      s2 += ex * ex + ey * ey;
    }
    const double d2 = sqrt(group_sum<G>(s2, mask) / n) / h0;
    const double dm = fmax(d1, d2);
    const double h1 = (dm <= 1e-15) ? fmax(1e-6, h0 * 1e-3) : pow(0.01 / dm, 0.2);
    return fmin(100.0 * h0, h1);
  }

  // Normalised expectation values of psi at output index m, added in FP64 to
  // the sums over trajectories.  The FP64 kernel forms each trajectory's
  // value in FP64; the mixed kernel forms <psi|O|psi> and <psi|psi> of its
  // FP32 state by an FP32 tree over the group (relative error ~1e-7, below
  // the state's own) and converts the ratio to FP64 for the accumulation.
  __device__ void output(int m, const V (&psi)[R], int64_t j, double *acc_smem) {
    if (a.n_e == 0) return;
    publish(psi);
    using A = T;  // per-trajectory accumulation type
    A nn = 0;
#pragma unroll
    for (int q = 0; q < R; ++q) {
      nn = fma((A)psi[q].x, (A)psi[q].x, nn);
      nn = fma((A)psi[q].y, (A)psi[q].y, nn);
    }
    nn = group_sum<G>(nn, mask);
    for (int e = 0; e < a.n_e; ++e) {
      const int op = 1 + a.n_c + e;
      A er = 0, ei = 0;
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const V o = apply_row(op, q);  // (O psi)_row
        er = fma((A)psi[q].x, (A)o.x, er);  // conj(psi) * (O psi)
        er = fma((A)psi[q].y, (A)o.y, er);
        ei = fma((A)psi[q].x, (A)o.y, ei);
        ei = fma(-(A)psi[q].y, (A)o.x, ei);
      }
      er = group_sum<G>(er, mask);
      ei = group_sum<G>(ei, mask);
      if (lane == 0) {
        const double vr = (double)(er / nn), vi = (double)(ei / nn);
        const int idx = m * a.n_e + e;
        if (acc_smem) {
          atomicAdd(acc_smem + 2 * idx, vr);
          atomicAdd(acc_smem + 2 * idx + 1, vi);
        } else {
          atomicAdd(&a.expect_sum[idx].x, vr);
          atomicAdd(&a.expect_sum[idx].y, vi);
        }
        if (a.traj_expect)
          a.traj_expect[(j * a.n_t + m) * a.n_e + e] = make_double2(vr, vi);
      }
    }
  }

  // ||C_n y||^2 (FP64 accumulation); y must already be published.
  __device__ __forceinline__ double weight(int n) const {
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const V c = apply_row(1 + n, q);
      s += (double)c.x * (double)c.x + (double)c.y * (double)c.y;
    }
    return group_sum<G>(s, mask);
  }

  // Steps III of the algorithm at the state y = psi(tau).  Returns false on
  // a numerical error.
  __device__ bool collapse(const V (&y)[R], V (&psi)[R], uint64_t gtraj, int64_t jk,
                           double tau, double t_lo_out, double t_hi_out) {
    publish(y);
    double psum = 0.0;
    int last_pos = -1;
    for (int n = 0; n < a.n_c; ++n) {
      const double p = weight(n);
      psum += p;
      if (p > 0.0) last_pos = n;
    }
    if (!(psum > 0.0) || !isfinite(psum)) return false;
    const double r2 = uniform52(a.seed, gtraj, (uint64_t)jk, 1);
    const double target = r2 * psum;
    int chosen = -1;
    double pc = 0.0, cum = 0.0;
    int64_t degenerate = 0;
    for (int n = 0; n < a.n_c; ++n) {
      const double p = weight(n);
      cum += p;
      if (fabs(cum - target) < 1e-5 * psum) degenerate |= 1;
      if (chosen < 0 && cum >= target) { chosen = n; pc = p; }
    }
    if (chosen < 0) { chosen = last_pos; pc = weight(chosen); }
    const double tscale = 1e-5 * fmax(1.0, fabs(tau));
    if (fabs(tau - t_lo_out) < tscale || fabs(tau - t_hi_out) < tscale) degenerate |= 2;
    const double inv = 1.0 / sqrt(pc);
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const V c = apply_row(1 + chosen, q);
      psi[q].x = (T)((double)c.x * inv);
      psi[q].y = (T)((double)c.y * inv);
    }
    if (lane == 0) {
      const unsigned long long slot = atomicAdd(a.n_jumps, 1ULL);
      if (a.jumps && (int64_t)slot < a.jump_cap) {
        qt_jump rec;
        rec.traj = (int64_t)gtraj;
        rec.k = jk;
        rec.channel = chosen;
        rec.tau = tau;
        rec.degenerate = degenerate;
        a.jumps[slot] = rec;
      }
    }
    ++n_jmp;
    return true;
  }

  // One whole trajectory (local index j).  Returns false after recording an
  // error in a.status.
  __device__ bool run(int64_t j, double *acc_smem) {
    const uint64_t gtraj = (uint64_t)(a.traj_begin + j);
    V psi[R];
#pragma unroll
    for (int q = 0; q < R; ++q) {
      if (row(q) < d) {
        const double2 p = a.psi0[row(q)];
        psi[q] = cmake<V>(p.x, p.y);
      } else {
        psi[q] = cmake<V>(0.0, 0.0);
      }
    }
    int64_t jk = 0;
    double r = uniform52(a.seed, gtraj, 0, 0);
    output(0, psi, j, acc_smem);
    if (a.n_t == 1) return true;

    // Time.  The FP64 kernel keeps the absolute time t in u (base tb = 0), as
    // the oracle does.  The mixed kernel keeps an FP32 offset u from the start
    // tb of the current output interval, so that its per-step control runs in
    // FP32; absolute FP64 times are formed only to search a jump time.
    constexpr bool kOff = sizeof(T) == 4;
    V k[7][R];
    rhs(psi, k[0]);
    T hprop = (T)((a.h0 > 0.0) ? a.h0 : initial_step(psi, k));
    bool after_reject = false;
    double tb = 0.0;
    T u = kOff ? (T)0 : (T)a.tlist[0];
    for (int m = 1; m < a.n_t; ++m) {
      const double tk = a.tlist[m];
      const double tprev = a.tlist[m - 1];
      if constexpr (kOff) {
        tb = tprev;
        u = (T)0;
      }
      const T L = kOff ? (T)(tk - tprev) : (T)tk;
      const T hmin_off = (T)(16.0f * 1.1920929e-7f) * L;
      int64_t attempts = 0;
      while (u < L) {
        if (attempts++ >= a.max_steps) { set_status(a.status, QT_ESTEP); return false; }
        const bool clipped = hprop >= L - u;
        const T h = clipped ? L - u : hprop;
        if (!clipped && (kOff ? h < hmin_off : h < (T)dp_hmin((double)u, tk))) {
          set_status(a.status, QT_ESTEP);
          return false;
        }
        V ynew[R];
        const T err = step(psi, k, h, ynew, true);
        if (!isfinite(err)) { set_status(a.status, QT_ENUMERIC); return false; }
        if (err > (T)1) {
          hprop = control(h, err, false, after_reject, clipped, hprop);
          after_reject = true;
          ++n_rej;
          continue;
        }
        hprop = control(h, err, true, after_reject, clipped, hprop);
        after_reject = false;
        ++n_acc;
        const T unew = clipped ? L : u + h;
        double n2;
        if (!below(ynew, r, n2)) {
          if (!isfinite(n2)) { set_status(a.status, QT_ENUMERIC); return false; }
#pragma unroll
          for (int q = 0; q < R; ++q) { psi[q] = ynew[q]; k[0][q] = k[6][q]; }
          u = unew;
          continue;
        }
        // Step II: bracket <psi(tau)|psi(tau)> = r in (t0, tnew], in FP64.
        // An FP32 state resolves its norm to ~1e-7, so the mixed kernel does
        // not narrow the bracket below 1e-9 max(1, |t|).
        const double t0 = tb + (double)u;
        double lo = t0, hi = clipped ? tk : tb + (double)unew;
        const double tol =
            (kOff ? fmax(a.bisect_tol, 1e-9) : a.bisect_tol) * fmax(1.0, fabs(t0));
        for (int it = 0; it < 64 && hi - lo > tol; ++it) {
          const double mid = lo + 0.5 * (hi - lo);
          V ytr[R];
          step(psi, k, (T)(mid - t0), ytr, false);
          ++n_bis;
          double nt2;
          if (below(ytr, r, nt2)) {
            hi = mid;
#pragma unroll
            for (int q = 0; q < R; ++q) ynew[q] = ytr[q];
          } else {
            lo = mid;
          }
        }
        // Steps III and IV.
        if (!collapse(ynew, psi, gtraj, jk, hi, tprev, tk)) {
          set_status(a.status, QT_ENUMERIC);
          return false;
        }
        ++jk;
        r = uniform52(a.seed, gtraj, (uint64_t)jk, 0);
        u = (hi == tk) ? L : (T)(hi - tb);
        rhs(psi, k[0]);
      }
      output(m, psi, j, acc_smem);
    }
    double n2 = norm2_64(psi);
    if (fabs(n2 - r) < 1e-5 * r) ++n_near;
    return true;
  }
};

template <typename T, int G, int R, int W>
__global__ void __launch_bounds__(kBlock) mc_kernel(const __grid_constant__ McArgs a) {
  using V = typename CT<T>::V;
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int groups = kBlock / G;
  const int grp = threadIdx.x / G;
  const int lane = threadIdx.x % G;
  const unsigned mask = group_mask<G>();
  V *ybuf = reinterpret_cast<V *>(smem) + grp * (G * R);
  const int nacc = a.n_t * a.n_e * 2;
  double *acc_smem = nullptr;
  const size_t ybytes = (size_t)groups * G * R * sizeof(V);
  const bool use_smem_acc = nacc > 0 && nacc * sizeof(double) <= 24 * 1024;
  if (use_smem_acc) {
    acc_smem = reinterpret_cast<double *>(smem + ((ybytes + 15) / 16) * 16);
    for (int i = threadIdx.x; i < nacc; i += blockDim.x) acc_smem[i] = 0.0;
  }
  __syncthreads();

  const V *val = sizeof(T) == 8 ? reinterpret_cast<const V *>(a.ops.val64)
                                : reinterpret_cast<const V *>(a.ops.val32);
  Traj<T, G, R, W> tr(a, lane, mask, ybuf, val);
  const int64_t ntraj = a.ntraj;
  const int leader = (threadIdx.x & 31) / G * G;
  for (;;) {
    // lane 0 takes the next index; an error anywhere ends the hand-out
    unsigned long long j = 0;
    if (lane == 0) {
      j = atomicAdd(a.work, 1ULL);
      if (*(volatile int *)a.status != 0) j = (unsigned long long)ntraj;
    }
    j = __shfl_sync(mask, j, leader);
    if ((int64_t)j >= ntraj) break;
    if (!tr.run((int64_t)j, acc_smem)) break;
  }
  if (lane == 0) {
    atomicAdd(a.counters + 0, tr.n_acc);
    atomicAdd(a.counters + 1, tr.n_rej);
    atomicAdd(a.counters + 2, tr.n_rhs);
    atomicAdd(a.counters + 3, tr.n_bis);
    atomicAdd(a.counters + 4, tr.n_jmp);
    atomicAdd(a.counters + 5, tr.n_near);
  }
  __syncthreads();
  if (use_smem_acc) {
    double *dst = reinterpret_cast<double *>(a.expect_sum);
    for (int i = threadIdx.x; i < nacc; i += blockDim.x)
      if (acc_smem[i] != 0.0) atomicAdd(dst + i, acc_smem[i]);
  }
}

template <typename T, int G, int R, int W>
cudaError_t launch_inst(const McArgs &a, cudaStream_t s) {
  using V = typename CT<T>::V;
  auto kern = mc_kernel<T, G, R, W>;
  constexpr int groups = kBlock / G;
  size_t ybytes = (size_t)groups * G * R * sizeof(V);
  size_t smem = ((ybytes + 15) / 16) * 16;
  const size_t nacc = (size_t)a.n_t * a.n_e * 2;
  if (nacc > 0 && nacc * sizeof(double) <= 24 * 1024) smem += nacc * sizeof(double);
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBlock, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  int64_t want = (a.ntraj + groups - 1) / groups;
  int64_t grid = (int64_t)sms * per_sm;
  if (want < grid) grid = want;
  if (grid < 1) grid = 1;
  kern<<<(unsigned)grid, kBlock, smem, s>>>(a);
  return cudaGetLastError();
}

// Instances: (rows per lane R, register-resident H_eff width W; 0 = cached
// global reads).
template <typename T>
cudaError_t dispatch(const McArgs &a, int R, int W, cudaStream_t s) {
  if (R == 1) {
    if (W == 4) return launch_inst<T, 32, 1, 4>(a, s);
    if (W == 16) return launch_inst<T, 32, 1, 16>(a, s);
    return launch_inst<T, 32, 1, 0>(a, s);
  }
  if (R == 2) {
    if (W == 4) return launch_inst<T, 32, 2, 4>(a, s);
    if (W == 8) return launch_inst<T, 32, 2, 8>(a, s);
    return launch_inst<T, 32, 2, 0>(a, s);
  }
  if (W == 4) return launch_inst<T, 32, 4, 4>(a, s);
  return launch_inst<T, 32, 4, 0>(a, s);
}

void choose(int d, int w, int &R, int &W) {
  R = d <= 32 ? 1 : (d <= 64 ? 2 : 4);
  if (R == 1) W = w <= 4 ? 4 : (w <= 16 ? 16 : 0);
  else if (R == 2) W = w <= 4 ? 4 : (w <= 8 ? 8 : 0);
  else W = w <= 4 ? 4 : 0;
}

}  // namespace

}  // namespace qt
