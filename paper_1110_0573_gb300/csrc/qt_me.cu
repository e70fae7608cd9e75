// qt_me.cu -- master-equation solver (paper section 3.1, Eq. (master_equation)).
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
// The whole Dormand-Prince integration runs inside one cooperative launch.
// Every CTA executes the same control flow: the stage combinations are
// element-wise and fused into the phase that produced the last stage, one
// grid-wide barrier separates the stages, and the error norm and the
// expectation values are reduced through per-CTA partial sums that every CTA
// then adds in the same fixed order, so all CTAs take identical decisions.
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

template <typename T>
struct Me {
  using V = typename CT<T>::V;
  const MeArgs &a;
  const int d;
  const int64_t n;  // d * d
  const V *val;

  __device__ Me(const MeArgs &a_, const V *val_)
      : a(a_), d(a_.ops.d), n((int64_t)a_.ops.d * a_.ops.d), val(val_) {}

  // drho/dt at entry (i, j) of the state y.
  __device__ __forceinline__ V rhs(const V *__restrict__ y, int i, int j) const {
    const int w0 = a.ops.w[0];
    const int64_t off0 = a.ops.off[0];
    V Y = cmake<V>(0.0, 0.0), Z = cmake<V>(0.0, 0.0);
    for (int s = 0; s < w0; ++s) {
      const int64_t pi = off0 + (int64_t)s * d + i;
      cmac(Y, val[pi], y[(int64_t)__ldg(a.ops.col + pi) * d + j]);
      const int64_t pj = off0 + (int64_t)s * d + j;
      cmac(Z, y[(int64_t)i * d + __ldg(a.ops.col + pj)], cconj(val[pj]));
    }
    V out;
    out.x = Y.y - Z.y;     // -i (Y - Z)
    out.y = -(Y.x - Z.x);
    for (int c = 1; c <= a.n_c; ++c) {
      const int wc = a.ops.w[c];
      const int64_t offc = a.ops.off[c];
      for (int s = 0; s < wc; ++s) {
        const int64_t ps = offc + (int64_t)s * d + i;
        const V u = val[ps];
        const V *yrow = y + (int64_t)__ldg(a.ops.col + ps) * d;
        V inner = cmake<V>(0.0, 0.0);
        for (int t = 0; t < wc; ++t) {
          const int64_t pt = offc + (int64_t)t * d + j;
          cmac(inner, yrow[__ldg(a.ops.col + pt)], cconj(val[pt]));
        }
        cmac(out, u, inner);
      }
    }
    return out;
  }
};

// Sum over the CTA of nv values per thread; returns the totals in sh[0..nv).
__device__ void block_sum(double *v, int nv, double *sh) {
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
    sh[kMePartialMax * 8 + threadIdx.x] = x;
  }
  __syncthreads();
}

// Grid-wide sum of nv values per thread, identical in every CTA.  Ends with
// the totals in tot[0..nv) (shared memory).
__device__ void grid_sum(double *v, int nv, double *sh, double *partial, double *tot,
                         cg::grid_group &grid) {
  block_sum(v, nv, sh);
  if (threadIdx.x < nv)
    partial[(int64_t)blockIdx.x * kMePartialMax + threadIdx.x] = sh[kMePartialMax * 8 + threadIdx.x];
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

template <typename T>
__global__ void __launch_bounds__(kMeBlock) me_kernel(const __grid_constant__ MeArgs a) {
  using V = typename CT<T>::V;
  cg::grid_group grid = cg::this_grid();
  __shared__ double sh[kMePartialMax * 8 + kMePartialMax];
  __shared__ double tot[kMePartialMax];

  const V *val = sizeof(T) == 8 ? reinterpret_cast<const V *>(a.ops.val64)
                                : reinterpret_cast<const V *>(a.ops.val32);
  Me<T> me(a, val);
  const int d = me.d;
  const int64_t n = me.n;
  V *base = reinterpret_cast<V *>(a.work);
  V *rho = base, *ynew = base + n, *buf0 = base + 2 * n, *buf1 = base + 3 * n;
  V *k[7];
#pragma unroll
  for (int s = 0; s < 7; ++s) k[s] = base + (4 + s) * n;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  double v[kMePartialMax];

  // ---- initial state: rho0 = |psi><psi| / <psi|psi> or the given matrix
  double scale = 1.0;
  if (a.state_is_ket) {
    v[0] = 0.0;
    for (int64_t i = tid; i < d; i += stride)
      v[0] += a.state0[i].x * a.state0[i].x + a.state0[i].y * a.state0[i].y;
    grid_sum(v, 1, sh, a.partial, tot, grid);
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
    rho[idx] = cmake<V>(r.x, r.y);
  }
  grid.sync();

  unsigned long long n_acc = 0, n_rej = 0, n_rhs = 0;
  auto eval = [&](const V *y, V *out) {
    for (int64_t idx = tid; idx < n; idx += stride)
      out[idx] = me.rhs(y, (int)(idx / d), (int)(idx % d));
    ++n_rhs;
  };
  // Expectation values Tr(O rho) and the optional state copy at output m.
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
      grid_sum(v, 2 * ne, sh, a.partial, tot, grid);
      if (blockIdx.x == 0 && threadIdx.x < ne)
        a.expect[(int64_t)m * a.n_e + e0 + threadIdx.x] =
            make_double2(tot[2 * threadIdx.x], tot[2 * threadIdx.x + 1]);
      grid.sync();  // tot / partial are reused by the next reduction
    }
  };

  eval(rho, k[0]);
  output(0, rho);
  if (a.n_t > 1) {
    double t = a.tlist[0];
    double hprop = a.h0;
    if (!(hprop > 0.0)) {
      // Hairer-Norsett-Wanner starting step (k[1], buf0 as scratch)
      grid.sync();  // k[0] complete
      v[0] = v[1] = 0.0;
      for (int64_t idx = tid; idx < n; idx += stride) {
        const V r = rho[idx], f = k[0][idx];
        const double sx = a.atol + a.rtol * fabs((double)r.x);
        const double sy = a.atol + a.rtol * fabs((double)r.y);
        v[0] += ((double)r.x / sx) * ((double)r.x / sx) + ((double)r.y / sy) * ((double)r.y / sy);
        v[1] += ((double)f.x / sx) * ((double)f.x / sx) + ((double)f.y / sy) * ((double)f.y / sy);
      }
      grid_sum(v, 2, sh, a.partial, tot, grid);
      const double nr = 2.0 * (double)n;
      const double d0 = sqrt(tot[0] / nr), d1 = sqrt(tot[1] / nr);
      const double h0 = (d0 < 1e-5 || d1 < 1e-5) ? 1e-6 : 0.01 * d0 / d1;
      for (int64_t idx = tid; idx < n; idx += stride) {
        const V r = rho[idx], f = k[0][idx];
        buf0[idx] = cmake<V>((double)r.x + h0 * (double)f.x, (double)r.y + h0 * (double)f.y);
      }
      grid.sync();
      eval(buf0, k[1]);
      v[0] = 0.0;
      for (int64_t idx = tid; idx < n; idx += stride) {
        const V r = rho[idx];
        const double sx = a.atol + a.rtol * fabs((double)r.x);
        const double sy = a.atol + a.rtol * fabs((double)r.y);
        const double ex = ((double)k[1][idx].x - (double)k[0][idx].x) / sx;
        const double ey = ((double)k[1][idx].y - (double)k[0][idx].y) / sy;
        v[0] += ex * ex + ey * ey;
      }
      grid_sum(v, 1, sh, a.partial, tot, grid);
      const double d2 = sqrt(tot[0] / nr) / h0;
      const double dm = fmax(d1, d2);
      const double h1 = (dm <= 1e-15) ? fmax(1e-6, h0 * 1e-3) : pow(0.01 / dm, 0.2);
      hprop = fmin(100.0 * h0, h1);
    }
    bool after_reject = false;
    int status = QT_OK;
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
          y.x = fma(ht, (T)DP::a21 * f0.x, r.x);
          y.y = fma(ht, (T)DP::a21 * f0.y, r.y);
          buf0[idx] = y;
        }
        grid.sync();
        // stages 2..6, each fused with the next stage input
#pragma unroll 1
        for (int st = 1; st <= 5; ++st) {
          const V *in = (st & 1) ? buf0 : buf1;
          V *nxt = (st == 5) ? ynew : ((st & 1) ? buf1 : buf0);
          for (int64_t idx = tid; idx < n; idx += stride) {
            const V f = me.rhs(in, (int)(idx / d), (int)(idx % d));
            k[st][idx] = f;
            T ax, ay;
            const V f0 = k[0][idx];
            const V r = rho[idx];
#define QT_A(c, K) ax = fma((T)(c), (K).x, ax); ay = fma((T)(c), (K).y, ay);
            if (st == 1) {
              ax = (T)DP::a31 * f0.x; ay = (T)DP::a31 * f0.y; QT_A(DP::a32, f)
            } else if (st == 2) {
              ax = (T)DP::a41 * f0.x; ay = (T)DP::a41 * f0.y; QT_A(DP::a42, k[1][idx])
              QT_A(DP::a43, f)
            } else if (st == 3) {
              ax = (T)DP::a51 * f0.x; ay = (T)DP::a51 * f0.y; QT_A(DP::a52, k[1][idx])
              QT_A(DP::a53, k[2][idx]) QT_A(DP::a54, f)
            } else if (st == 4) {
              ax = (T)DP::a61 * f0.x; ay = (T)DP::a61 * f0.y; QT_A(DP::a62, k[1][idx])
              QT_A(DP::a63, k[2][idx]) QT_A(DP::a64, k[3][idx]) QT_A(DP::a65, f)
            } else {
              ax = (T)DP::b1 * f0.x; ay = (T)DP::b1 * f0.y; QT_A(DP::b3, k[2][idx])
              QT_A(DP::b4, k[3][idx]) QT_A(DP::b5, k[4][idx]) QT_A(DP::b6, f)
            }
            V y;
            y.x = fma(ht, ax, r.x);
            y.y = fma(ht, ay, r.y);
            nxt[idx] = y;
          }
          ++n_rhs;
          grid.sync();
        }
        // k7 = f(ynew) fused with the error norm
        v[0] = 0.0;
        {
          const T at = (T)a.atol, rt = (T)a.rtol;
          T acc = (T)0;
          for (int64_t idx = tid; idx < n; idx += stride) {
            const V f = me.rhs(ynew, (int)(idx / d), (int)(idx % d));
            k[6][idx] = f;
            const V f0 = k[0][idx];
            T ax = (T)DP::e1 * f0.x, ay = (T)DP::e1 * f0.y;
            QT_A(DP::e3, k[2][idx]) QT_A(DP::e4, k[3][idx]) QT_A(DP::e5, k[4][idx])
            QT_A(DP::e6, k[5][idx]) QT_A(DP::e7, f)
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
        grid_sum(v, 1, sh, a.partial, tot, grid);
        const double err = sqrt(tot[0] / (2.0 * (double)n));
        if (!isfinite(err)) { status = QT_ENUMERIC; break; }
        if (err <= 1.0) {
          hprop = dp_control(h, err, true, after_reject, clipped, hprop);
          after_reject = false;
          t = clipped ? tk : t + h;
          V *sw = rho; rho = ynew; ynew = sw;
          sw = k[0]; k[0] = k[6]; k[6] = sw;
          ++n_acc;
        } else {
          hprop = dp_control(h, err, false, after_reject, clipped, hprop);
          after_reject = true;
          ++n_rej;
        }
        grid.sync();  // tot is rewritten by the next reduction
      }
      if (status != QT_OK) break;
      output(m, rho);
    }
    if (status != QT_OK && tid == 0) set_status(a.status, status);
  }
  if (tid == 0) {
    atomicAdd(a.counters + 0, n_acc);
    atomicAdd(a.counters + 1, n_rej);
    atomicAdd(a.counters + 2, n_rhs);
  }
}

template <typename T>
int grid_for(int d) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, me_kernel<T>, kMeBlock, 0) !=
      cudaSuccess)
    return -1;
  if (per_sm < 1) return -1;
  const int64_t n = (int64_t)d * d;
  int64_t want = (n + kMeBlock - 1) / kMeBlock;
  int64_t cap = (int64_t)sms * per_sm;
  return (int)(want < cap ? want : cap);
}

}  // namespace

int me_grid(int d, int precision) {
  return precision == QT_MIXED ? grid_for<float>(d) : grid_for<double>(d);
}

size_t me_workspace_bytes(int d, int precision, int grid) {
  const size_t elem = precision == QT_MIXED ? sizeof(float2) : sizeof(double2);
  return 11 * (size_t)d * d * elem + (size_t)grid * kMePartialMax * sizeof(double) + 256;
}

cudaError_t launch_me(const MeArgs &a, int precision, cudaStream_t s) {
  void *args[] = {const_cast<MeArgs *>(&a)};
  if (precision == QT_MIXED)
    return cudaLaunchCooperativeKernel((const void *)me_kernel<float>, dim3(a.grid),
                                       dim3(kMeBlock), args, 0, s);
  return cudaLaunchCooperativeKernel((const void *)me_kernel<double>, dim3(a.grid),
                                     dim3(kMeBlock), args, 0, s);
}

}  // namespace qt
