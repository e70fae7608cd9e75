// qt_adjoint.cu -- gradients of a master-equation loss by the discrete
// adjoint (an extension beyond the paper's solvers; the forward problem is
// Eq. (master_equation) of section 3.1).
//
// The generator of segment s is
//   F_s(rho) = -i [H0 + Omega_s Hd, rho]
//              + sum_k gamma_k (A_k rho A_k^dag - 1/2 {A_k^dag A_k, rho}),
// Omega_s constant on each segment of length t_seg, and the loss
//   L = Re Tr(P1 rho(T)) + Re q(T),   dq/dt = Tr(P2 rho),
// q carried by the same Runge-Kutta stages as rho.  The forward pass is the
// adaptive Dormand-Prince solve of the library's controller with the segment
// ends as output times; it records every accepted step length (the frozen
// grid) and rho at the segment ends.  The backward pass walks the segments in
// reverse: it recomputes the segment's states from its checkpoint, then for
// each step (last first) recomputes the stage inputs Y_l and applies the
// adjoint of the step,
//   nu_i  = h b_i lambda + sum_{l>i} h a_li mu_l,
//   mu_i  = F^dag(nu_i) + h b_i P2,
//   lambda <- lambda + sum_l mu_l,        lambda(T) = P1,
//   dL/dOmega_s += Re <nu_i, -i [Hd, Y_i]>,
//   dL/dgamma_k += Re <nu_i, A_k Y_i A_k^dag - 1/2 {A_k^dag A_k, Y_i}>,
// with F^dag(X) = i [H, X] + sum_k gamma_k (A_k^dag X A_k - 1/2 {A_k^dag A_k, X})
// and <X, Y> = Tr(X^dag Y).  This is the exact derivative of the discrete map,
// so it agrees with finite differences taken on the same grid.
//
// One CTA integrates one parameter vector; everything is FP64.
#include "qt_device.cuh"
#include "qt_internal.h"

namespace qt {

namespace {

constexpr int kAdjBlock = 256;
constexpr int kAdjRed = 16;  // reduction slots per warp

struct AdjIdx {  // operator indices in the table
  int nk;
  __device__ int H0() const { return 0; }
  __device__ int Hd() const { return 1; }
  __device__ int A(int k) const { return 2 + k; }
  __device__ int Ad(int k) const { return 2 + nk + k; }
  __device__ int N(int k) const { return 2 + 2 * nk + k; }
  __device__ int P1() const { return 2 + 3 * nk; }
  __device__ int P2() const { return 3 + 3 * nk; }
};

__device__ __forceinline__ double2 cj(double2 v) { return make_double2(v.x, -v.y); }
__device__ __forceinline__ double2 cadd(double2 a, double2 b) {
  return make_double2(a.x + b.x, a.y + b.y);
}
__device__ __forceinline__ double2 cscale(double2 a, double s) {
  return make_double2(a.x * s, a.y * s);
}

// (Op M)_ij - (M Op^dag)_ij for Hermitian Op (sign = -1) or + (sign = +1).
__device__ __forceinline__ double2 lr(const OpTable &t, int o, const double2 *M, int i, int j,
                                      int d, double sign) {
  const int w = t.w[o];
  const int64_t off = t.off[o];
  double2 acc = make_double2(0.0, 0.0);
  for (int s = 0; s < w; ++s) {
    const int64_t pi = off + (int64_t)s * d + i;
    cmac(acc, t.val64[pi], M[(int64_t)t.col[pi] * d + j]);
    const int64_t pj = off + (int64_t)s * d + j;
    double2 m = M[(int64_t)i * d + t.col[pj]];
    double2 v = cj(t.val64[pj]);
    double2 pr = make_double2(0.0, 0.0);
    cmac(pr, m, v);
    acc.x += sign * pr.x;
    acc.y += sign * pr.y;
  }
  return acc;
}

// (A M A^dag)_ij from the ELL rows i and j of A.
__device__ __forceinline__ double2 sand(const OpTable &t, int o, const double2 *M, int i, int j,
                                        int d) {
  const int w = t.w[o];
  const int64_t off = t.off[o];
  double2 acc = make_double2(0.0, 0.0);
  for (int s = 0; s < w; ++s) {
    const int64_t ps = off + (int64_t)s * d + i;
    const double2 u = t.val64[ps];
    const double2 *row = M + (int64_t)t.col[ps] * d;
    double2 inner = make_double2(0.0, 0.0);
    for (int r = 0; r < w; ++r) {
      const int64_t pt = off + (int64_t)r * d + j;
      cmac(inner, row[t.col[pt]], cj(t.val64[pt]));
    }
    cmac(acc, u, inner);
  }
  return acc;
}

// Entry (i, j) of the generator (dagger = 0) or of its adjoint (dagger = 1).
__device__ __forceinline__ double2 gen(const OpTable &t, AdjIdx ix, double omega,
                                       const double *gam, int dagger, const double2 *M, int i,
                                       int j, int d) {
  double2 c = lr(t, ix.H0(), M, i, j, d, -1.0);
  const double2 cd = lr(t, ix.Hd(), M, i, j, d, -1.0);
  c.x += omega * cd.x;
  c.y += omega * cd.y;
  // -i c (generator) or +i c (adjoint)
  double2 out = dagger ? make_double2(-c.y, c.x) : make_double2(c.y, -c.x);
  for (int k = 0; k < ix.nk; ++k) {
    const double2 s = sand(t, dagger ? ix.Ad(k) : ix.A(k), M, i, j, d);
    const double2 an = lr(t, ix.N(k), M, i, j, d, 1.0);
    out.x += gam[k] * (s.x - 0.5 * an.x);
    out.y += gam[k] * (s.y - 0.5 * an.y);
  }
  return out;
}

// Entry (i, j) of a (Hermitian, ELL) operator as a dense matrix.
__device__ __forceinline__ double2 dense_entry(const OpTable &t, int o, int i, int j, int d) {
  const int w = t.w[o];
  const int64_t off = t.off[o];
  double2 acc = make_double2(0.0, 0.0);
  for (int s = 0; s < w; ++s) {
    const int64_t p = off + (int64_t)s * d + i;
    if (t.col[p] == j) acc = cadd(acc, t.val64[p]);
  }
  return acc;
}

// Tr(P M) restricted to this thread's rows.
__device__ __forceinline__ double2 trace_rows(const OpTable &t, int o, const double2 *M, int d) {
  double2 acc = make_double2(0.0, 0.0);
  const int w = t.w[o];
  const int64_t off = t.off[o];
  for (int r = threadIdx.x; r < d; r += blockDim.x)
    for (int s = 0; s < w; ++s) {
      const int64_t p = off + (int64_t)s * d + r;
      cmac(acc, t.val64[p], M[(int64_t)t.col[p] * d + r]);
    }
  return acc;
}

// Sum over the CTA of nv doubles per thread; totals returned to every thread.
__device__ void cta_sum(double *v, int nv, double *sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  for (int q = 0; q < nv; ++q) {
    double x = v[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) sh[warp * kAdjRed + q] = x;
  }
  __syncthreads();
  for (int q = 0; q < nv; ++q) {
    double x = 0.0;
    for (int w = 0; w < nw; ++w) x += sh[w * kAdjRed + q];
    v[q] = x;
  }
  __syncthreads();
}

struct Buffers {
  double2 *rho, *rnew, *Y[6], *K[7], *nu[6], *mu[6], *lam, *seg;
};

__device__ Buffers buffers(const AdjArgs &a, int64_t n) {
  double2 *W = a.work + (int64_t)blockIdx.x * a.slots * n;
  Buffers B;
  B.rho = W;
  B.rnew = W + n;
  for (int i = 0; i < 6; ++i) B.Y[i] = W + (2 + i) * n;
  for (int i = 0; i < 7; ++i) B.K[i] = W + (8 + i) * n;
  for (int i = 0; i < 6; ++i) B.nu[i] = W + (15 + i) * n;
  for (int i = 0; i < 6; ++i) B.mu[i] = W + (21 + i) * n;
  B.lam = W + 27 * n;
  B.seg = W + 28 * n;  // a.maxs + 1 states of the current segment
  return B;
}

// Stage inputs and derivatives of one Dormand-Prince step of length h from
// x (K[0] = F(x) must be in place); writes Y[0..5], K[1..5] and xnew.
__device__ void dp_stages(const AdjArgs &a, AdjIdx ix, double omega, const double *gam, double h,
                          const double2 *x, Buffers &B, double2 *xnew, int d, int64_t n) {
  const double A[6][5] = {{0, 0, 0, 0, 0},
                          {DP::a21, 0, 0, 0, 0},
                          {DP::a31, DP::a32, 0, 0, 0},
                          {DP::a41, DP::a42, DP::a43, 0, 0},
                          {DP::a51, DP::a52, DP::a53, DP::a54, 0},
                          {DP::a61, DP::a62, DP::a63, DP::a64, DP::a65}};
  const double Bw[6] = {DP::b1, 0.0, DP::b3, DP::b4, DP::b5, DP::b6};
  for (int64_t e = threadIdx.x; e < n; e += blockDim.x) B.Y[0][e] = x[e];
#pragma unroll 1
  for (int st = 1; st < 6; ++st) {
    for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
      double ar = 0.0, ai = 0.0;
      for (int j = 0; j < st; ++j) {
        ar += A[st][j] * B.K[j][e].x;
        ai += A[st][j] * B.K[j][e].y;
      }
      B.Y[st][e] = make_double2(x[e].x + h * ar, x[e].y + h * ai);
    }
    __syncthreads();
    for (int64_t e = threadIdx.x; e < n; e += blockDim.x)
      B.K[st][e] = gen(a.ops, ix, omega, gam, 0, B.Y[st], (int)(e / d), (int)(e % d), d);
    __syncthreads();
  }
  for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
    double ar = 0.0, ai = 0.0;
    for (int j = 0; j < 6; ++j) {
      ar += Bw[j] * B.K[j][e].x;
      ai += Bw[j] * B.K[j][e].y;
    }
    xnew[e] = make_double2(x[e].x + h * ar, x[e].y + h * ai);
  }
  __syncthreads();
}

// Forward solve of one parameter vector: adaptive (recording the grid and
// the segment checkpoints) or on the recorded grid (a.fixed, loss only).
__global__ void __launch_bounds__(kAdjBlock) adjoint_forward_kernel(const __grid_constant__ AdjArgs a) {
  __shared__ double sh[32 * kAdjRed];
  const int b = blockIdx.x;
  const int d = a.ops.d;
  const int64_t n = (int64_t)d * d;
  const AdjIdx ix{a.nk};
  Buffers B = buffers(a, n);
  const double *om = a.omega + (int64_t)b * a.n_seg;
  const double *gam = a.gamma + (int64_t)b * a.nk;
  int *nsteps = a.nsteps + (int64_t)b * a.n_seg;
  double *hgrid = a.hgrid + (int64_t)b * a.n_seg * a.maxs;
  double2 *ckpt = a.ckpt + (int64_t)b * (a.n_seg + 1) * n;
  const double Bw[6] = {DP::b1, 0.0, DP::b3, DP::b4, DP::b5, DP::b6};
  const double Ew[7] = {DP::e1, 0.0, DP::e3, DP::e4, DP::e5, DP::e6, DP::e7};
  double2 *rho = B.rho, *rnew = B.rnew;
  for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
    rho[e] = a.rho0[e];
    if (!a.fixed) ckpt[e] = a.rho0[e];
  }
  __syncthreads();
  double qx = 0.0, qy = 0.0;  // this thread's share of q
  double hprop = 0.0;
  bool after_reject = false;
  int status = QT_OK;
  unsigned long long n_acc = 0, n_rej = 0, n_rhs = 0;
  double v[4];
  for (int s = 0; s < a.n_seg && status == QT_OK; ++s) {
    const double w = om[s];
    for (int64_t e = threadIdx.x; e < n; e += blockDim.x)
      B.K[0][e] = gen(a.ops, ix, w, gam, 0, rho, (int)(e / d), (int)(e % d), d);
    ++n_rhs;
    __syncthreads();
    if (!a.fixed && s == 0) {
      // Hairer-Norsett-Wanner starting step
      v[0] = v[1] = 0.0;
      for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
        const double2 r = rho[e], f = B.K[0][e];
        const double sx = a.atol + a.rtol * fabs(r.x), sy = a.atol + a.rtol * fabs(r.y);
        v[0] += (r.x / sx) * (r.x / sx) + (r.y / sy) * (r.y / sy);
        v[1] += (f.x / sx) * (f.x / sx) + (f.y / sy) * (f.y / sy);
      }
      cta_sum(v, 2, sh);
      const double d0 = sqrt(v[0] / (2.0 * n)), d1 = sqrt(v[1] / (2.0 * n));
      const double h0 = (d0 < 1e-5 || d1 < 1e-5) ? 1e-6 : 0.01 * d0 / d1;
      for (int64_t e = threadIdx.x; e < n; e += blockDim.x)
        rnew[e] = make_double2(rho[e].x + h0 * B.K[0][e].x, rho[e].y + h0 * B.K[0][e].y);
      __syncthreads();
      for (int64_t e = threadIdx.x; e < n; e += blockDim.x)
        B.K[1][e] = gen(a.ops, ix, w, gam, 0, rnew, (int)(e / d), (int)(e % d), d);
      ++n_rhs;
      __syncthreads();
      v[0] = 0.0;
      for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
        const double2 r = rho[e];
        const double sx = a.atol + a.rtol * fabs(r.x), sy = a.atol + a.rtol * fabs(r.y);
        const double ex = (B.K[1][e].x - B.K[0][e].x) / sx, ey = (B.K[1][e].y - B.K[0][e].y) / sy;
        v[0] += ex * ex + ey * ey;
      }
      cta_sum(v, 1, sh);
      const double d2 = sqrt(v[0] / (2.0 * n)) / h0;
      const double dm = fmax(d1, d2);
      const double h1 = (dm <= 1e-15) ? fmax(1e-6, h0 * 1e-3) : pow(0.01 / dm, 0.2);
      hprop = fmin(100.0 * h0, h1);
    }
    double u = 0.0;
    int ns = 0;
    int64_t attempts = 0;
    const int fixed_ns = a.fixed ? nsteps[s] : 0;
    while (a.fixed ? (ns < fixed_ns) : (u < a.t_seg)) {
      if (attempts++ >= a.max_steps) { status = QT_ESTEP; break; }
      double h;
      bool clipped = false;
      if (a.fixed) {
        h = hgrid[ns];
        if (ns > 0) {  // K[0] = F(rho) of this step (no first-same-as-last here)
          for (int64_t e = threadIdx.x; e < n; e += blockDim.x)
            B.K[0][e] = gen(a.ops, ix, w, gam, 0, rho, (int)(e / d), (int)(e % d), d);
          ++n_rhs;
          __syncthreads();
        }
      } else {
        clipped = hprop >= a.t_seg - u;
        h = clipped ? a.t_seg - u : hprop;
      }
      dp_stages(a, ix, w, gam, h, rho, B, rnew, d, n);
      n_rhs += 5;
      bool accept = true;
      if (!a.fixed) {
        for (int64_t e = threadIdx.x; e < n; e += blockDim.x)
          B.K[6][e] = gen(a.ops, ix, w, gam, 0, rnew, (int)(e / d), (int)(e % d), d);
        ++n_rhs;
        __syncthreads();
        v[0] = 0.0;
        for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
          double ex = 0.0, ey = 0.0;
          for (int j = 0; j < 7; ++j) {
            ex += Ew[j] * B.K[j][e].x;
            ey += Ew[j] * B.K[j][e].y;
          }
          ex *= h;
          ey *= h;
          const double sx = a.atol + a.rtol * fmax(fabs(rho[e].x), fabs(rnew[e].x));
          const double sy = a.atol + a.rtol * fmax(fabs(rho[e].y), fabs(rnew[e].y));
          v[0] += (ex / sx) * (ex / sx) + (ey / sy) * (ey / sy);
        }
        cta_sum(v, 1, sh);
        const double err = sqrt(v[0] / (2.0 * n));
        if (!isfinite(err)) { status = QT_ENUMERIC; break; }
        accept = err <= 1.0;
        hprop = dp_control(h, err, accept, after_reject, clipped, hprop);
        after_reject = !accept;
      }
      if (accept) {
        // q += h sum_i b_i Tr(P2 Y_i), this thread's rows
        for (int j = 0; j < 6; ++j) {
          if (Bw[j] == 0.0) continue;
          const double2 tr = trace_rows(a.ops, ix.P2(), B.Y[j], d);
          qx += h * Bw[j] * tr.x;
          qy += h * Bw[j] * tr.y;
        }
        if (!a.fixed) {
          if (ns >= a.maxs) { status = QT_ESTEP; break; }
          if (threadIdx.x == 0) hgrid[(int64_t)s * a.maxs + ns] = h;
          u = clipped ? a.t_seg : u + h;
          double2 *sw = B.K[0];
          B.K[0] = B.K[6];
          B.K[6] = sw;
        }
        double2 *sw = rho;
        rho = rnew;
        rnew = sw;
        ++ns;
        ++n_acc;
      } else {
        ++n_rej;
      }
      __syncthreads();
    }
    if (a.fixed) hgrid += a.maxs;
    if (status != QT_OK) break;
    if (!a.fixed) {
      if (threadIdx.x == 0) nsteps[s] = ns;
      for (int64_t e = threadIdx.x; e < n; e += blockDim.x) ckpt[(int64_t)(s + 1) * n + e] = rho[e];
    }
    __syncthreads();
  }
  const double2 t1 = trace_rows(a.ops, ix.P1(), rho, d);
  v[0] = t1.x + qx;
  cta_sum(v, 1, sh);
  if (threadIdx.x == 0) {
    if (status != QT_OK) set_status(a.status, status);
    a.loss[b] = v[0];
    atomicAdd(a.counters + 0, n_acc);
    atomicAdd(a.counters + 1, n_rej);
    atomicAdd(a.counters + 2, n_rhs);
  }
}

// Backward pass of one parameter vector on its recorded grid.
__global__ void __launch_bounds__(kAdjBlock) adjoint_backward_kernel(const __grid_constant__ AdjArgs a) {
  __shared__ double sh[32 * kAdjRed];
  const int b = blockIdx.x;
  const int d = a.ops.d;
  const int64_t n = (int64_t)d * d;
  const AdjIdx ix{a.nk};
  Buffers B = buffers(a, n);
  const double *om = a.omega + (int64_t)b * a.n_seg;
  const double *gam = a.gamma + (int64_t)b * a.nk;
  const int *nsteps = a.nsteps + (int64_t)b * a.n_seg;
  const double *hgrid = a.hgrid + (int64_t)b * a.n_seg * a.maxs;
  const double2 *ckpt = a.ckpt + (int64_t)b * (a.n_seg + 1) * n;
  const double Bw[6] = {DP::b1, 0.0, DP::b3, DP::b4, DP::b5, DP::b6};
  const double Aw[6][6] = {{0, 0, 0, 0, 0, 0},
                           {DP::a21, 0, 0, 0, 0, 0},
                           {DP::a31, DP::a32, 0, 0, 0, 0},
                           {DP::a41, DP::a42, DP::a43, 0, 0, 0},
                           {DP::a51, DP::a52, DP::a53, DP::a54, 0, 0},
                           {DP::a61, DP::a62, DP::a63, DP::a64, DP::a65, 0}};
  const double scale = a.dloss ? a.dloss[b] : 1.0;
  // lambda(T) = P1
  for (int64_t e = threadIdx.x; e < n; e += blockDim.x)
    B.lam[e] = dense_entry(a.ops, ix.P1(), (int)(e / d), (int)(e % d), d);
  __syncthreads();
  double ggam[8];
  for (int k = 0; k < 8; ++k) ggam[k] = 0.0;
  double v[8];
  for (int s = a.n_seg - 1; s >= 0; --s) {
    const double w = om[s];
    const int ns = nsteps[s];
    const double *hs = hgrid + (int64_t)s * a.maxs;
    // states of the segment from its checkpoint
    for (int64_t e = threadIdx.x; e < n; e += blockDim.x) B.seg[e] = ckpt[(int64_t)s * n + e];
    __syncthreads();
    for (int m = 0; m < ns; ++m) {
      const double2 *x = B.seg + (int64_t)m * n;
      for (int64_t e = threadIdx.x; e < n; e += blockDim.x)
        B.K[0][e] = gen(a.ops, ix, w, gam, 0, x, (int)(e / d), (int)(e % d), d);
      __syncthreads();
      dp_stages(a, ix, w, gam, hs[m], x, B, B.seg + (int64_t)(m + 1) * n, d, n);
    }
    double gom = 0.0;
    for (int m = ns - 1; m >= 0; --m) {
      const double h = hs[m];
      const double2 *x = B.seg + (int64_t)m * n;
      for (int64_t e = threadIdx.x; e < n; e += blockDim.x)
        B.K[0][e] = gen(a.ops, ix, w, gam, 0, x, (int)(e / d), (int)(e % d), d);
      __syncthreads();
      dp_stages(a, ix, w, gam, h, x, B, B.rnew, d, n);
      for (int i = 5; i >= 0; --i) {
        for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
          double2 acc = cscale(B.lam[e], h * Bw[i]);
          for (int l = i + 1; l < 6; ++l) acc = cadd(acc, cscale(B.mu[l][e], h * Aw[l][i]));
          B.nu[i][e] = acc;
        }
        __syncthreads();
        for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
          const int r = (int)(e / d), c = (int)(e % d);
          double2 m2 = gen(a.ops, ix, w, gam, 1, B.nu[i], r, c, d);
          if (Bw[i] != 0.0) m2 = cadd(m2, cscale(dense_entry(a.ops, ix.P2(), r, c, d), h * Bw[i]));
          B.mu[i][e] = m2;
          // parameter derivatives at Y_i: Re <nu_i, dF/dtheta (Y_i)>
          const double2 nv = B.nu[i][e];
          const double2 cd = lr(a.ops, ix.Hd(), B.Y[i], r, c, d, -1.0);  // [Hd, Y]
          // -i cd = (cd.y, -cd.x)
          gom += nv.x * cd.y - nv.y * cd.x;
          for (int k = 0; k < a.nk; ++k) {
            const double2 sd = sand(a.ops, ix.A(k), B.Y[i], r, c, d);
            const double2 an = lr(a.ops, ix.N(k), B.Y[i], r, c, d, 1.0);
            const double dx = sd.x - 0.5 * an.x, dy = sd.y - 0.5 * an.y;
            ggam[k] += nv.x * dx + nv.y * dy;
          }
        }
        __syncthreads();
      }
      for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
        double2 acc = B.lam[e];
        for (int l = 0; l < 6; ++l) acc = cadd(acc, B.mu[l][e]);
        B.lam[e] = acc;
      }
      __syncthreads();
    }
    v[0] = gom;
    cta_sum(v, 1, sh);
    if (threadIdx.x == 0) a.g_omega[(int64_t)b * a.n_seg + s] = scale * v[0];
  }
  for (int k = 0; k < a.nk; ++k) v[k] = ggam[k];
  cta_sum(v, a.nk, sh);
  if (threadIdx.x == 0)
    for (int k = 0; k < a.nk; ++k) a.g_gamma[(int64_t)b * a.nk + k] = scale * v[k];
}

}  // namespace

size_t adjoint_slots(int maxs) { return 28 + (size_t)maxs + 1; }

cudaError_t launch_adjoint_forward(const AdjArgs &a, cudaStream_t s) {
  adjoint_forward_kernel<<<a.batch, kAdjBlock, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_backward(const AdjArgs &a, cudaStream_t s) {
  adjoint_backward_kernel<<<a.batch, kAdjBlock, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace qt
