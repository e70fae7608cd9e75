// qt_me_herm.cuh -- master-equation solver for Hermitian states (paper
// section 3.1, Eq. (master_equation)) on the whole grid of a cooperative
// launch.
//
// A density matrix and every Runge-Kutta stage built from it are Hermitian,
// and so is the right-hand side.  In the effective-Hamiltonian form
//   d rho/dt = -i (Y - Y^dag) + sum_n C_n rho C_n^dag,   Y = H_eff rho,
// because rho H_eff^dag = (H_eff rho^dag)^dag = Y^dag.  So each right-hand
// side is evaluated in two phases:
//   1. the product Y = H_eff y of the stage input y, by a product provider:
//      a sparse ELL product on the CUDA cores (SpmmY below) or a dense
//      tensor-core GEMM (qt_me_tc.cu);
//   2. a combine phase over pairs of 32 x 32 tiles (I, J), I <= J: the two
//      tiles of Y are staged in shared memory, each upper-triangle entry
//      (i <= j) gets -i (Y_ij - conj(Y_ji)) plus its collapse terms, fused
//      with the Dormand-Prince stage combination; a new stage input is
//      written at (i, j) and, as its exact conjugate, at (j, i).
// The stage derivatives k_s are stored and read only in the upper triangle.
// Every value at (j, i) is the conjugate of the one at (i, j) bit for bit, so
// the error norm over all 2 d^2 reals is the diagonal plus twice the strictly
// upper part.
#pragma once

#include "qt_me_impl.cuh"

namespace qt {

namespace {

constexpr int kHT = 32;              // tile edge of the combine phase
constexpr int kHTP = kHT + 1;        // padded row of a staged tile

// Bytes of shared memory the combine phase needs for element type V with
// n_cslots collapse slots and n_cterms terms staged (0, 0: not staged).
template <typename V>
constexpr size_t herm_smem_bytes(int n_cslots, int n_cterms) {
  return (3 * kHT * kHTP * sizeof(V) + (size_t)n_cslots * kHT * (2 * sizeof(V) + 2 * sizeof(int)) +
          (size_t)n_cterms * sizeof(int2) + 15) / 16 * 16;
}

// Pair p of the upper triangle of the nt x nt tile grid, row-major.
__device__ __forceinline__ void tile_pair(int p, int nt, int &I, int &J) {
  int i = 0;
  while (p >= nt - i) {
    p -= nt - i;
    ++i;
  }
  I = i;
  J = i + p;
}

// Product provider on the CUDA cores: the entries of Y = H_eff y are formed
// from the ELL rows of H_eff inside the combine phase, by the CTA that
// consumes them (kFusedY: no product buffer, no grid barrier).
template <typename T>
struct SpmmY {
  using V = typename CT<T>::V;
  static constexpr bool kCanFail = false;
  static constexpr bool kFusedY = true;
  const MeArgs &a;
  const V *val;
  const int d, w0, off0;
  double *coef;  // f_k at the current stage time (shared memory, kTdMax values)
  __device__ SpmmY(const MeArgs &a_, const V *val_, double *coef_)
      : a(a_), val(val_), d(a_.ops.d), w0(a_.ops.w[0]), off0((int)a_.ops.off[0]), coef(coef_) {}
  __device__ __forceinline__ int ystride() const { return d; }
  __device__ __forceinline__ const V *product() const { return nullptr; }
  __device__ __forceinline__ const V *collapse_product() const { return nullptr; }
  __device__ __forceinline__ void store(V *buf, int idx, int, int, V v) { buf[idx] = v; }
  __device__ __forceinline__ void publish(GridTeam &team) { team.sync(); }
  __device__ __forceinline__ int failed() const { return 0; }
  // the coefficients of the time-dependent terms at the stage time t (the
  // previous phase ended with a grid barrier)
  __device__ __forceinline__ void prepare(GridTeam &, const V *, double t) {
    if (a.n_td > 0) {
      if ((int)threadIdx.x < a.n_td) coef[threadIdx.x] = td_coef_at(a, (int)threadIdx.x, t);
      __syncthreads();
    }
  }

  // Y_ij = sum_s H_eff[i, c_s] y[c_s, j] (0 outside the matrix), with eight
  // independent gathers in flight; plus sum_k f_k(t) (H_k y)_ij.
  __device__ __forceinline__ V entry(const V *__restrict__ y, int i, int j) const {
    V acc = cmake<V>(0.0, 0.0);
    if (i >= d || j >= d) return acc;
    const int *__restrict__ col = a.ops.col;
    for (int k = 0; k < a.n_td; ++k) {
      const int op = a.td_op0 + k;
      const int wk = a.ops.w[op], offk = (int)a.ops.off[op];
      V hk = cmake<V>(0.0, 0.0);
      for (int s = 0; s < wk; ++s) {
        const int p = offk + s * d + i;
        cmac(hk, val[p], y[__ldg(col + p) * d + j]);
      }
      const T f = (T)coef[k];
      acc.x = tfma(f, hk.x, acc.x);
      acc.y = tfma(f, hk.y, acc.y);
    }
    int s = 0;
    for (; s + 8 <= w0; s += 8) {
      const int p = off0 + s * d + i;
      int c[8];
      V g[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) c[u] = __ldg(col + p + u * d);
#pragma unroll
      for (int u = 0; u < 8; ++u) g[u] = y[c[u] * d + j];
#pragma unroll
      for (int u = 0; u < 8; ++u) cmac(acc, val[p + u * d], g[u]);
    }
    for (; s < w0; ++s) {
      const int p = off0 + s * d + i;
      cmac(acc, val[p], y[__ldg(col + p) * d + j]);
    }
    return acc;
  }
};

template <typename T, typename Prod>
struct HermSolver {
  using V = typename CT<T>::V;
  const MeArgs &a;
  GridTeam &team;
  Prod &prod;
  Me<T> me;  // collapse terms read from global memory (operators too large to stage)
  const V *val;
  // shared memory: [2][kHT][kHTP] tiles of Y, [kHT][kHTP] mirror staging,
  // then the collapse slots of the pair's rows and columns and the terms
  V *Ys, *rs_val, *cs_val;
  int2 *terms;
  int *rs_col, *cs_col;
  const int d, nt, n_pairs, ns, nterm;

  __device__ HermSolver(const MeArgs &a_, GridTeam &team_, Prod &prod_, const V *val_, V *smem)
      : a(a_), team(team_), prod(prod_), me(a_, val_), val(val_), Ys(smem), d(a_.ops.d),
        nt((a_.ops.d + kHT - 1) / kHT), n_pairs(nt * (nt + 1) / 2), ns(a_.n_cslots),
        nterm(a_.n_cterms) {
    rs_val = Ys + 3 * kHT * kHTP;
    cs_val = rs_val + ns * kHT;
    terms = reinterpret_cast<int2 *>(cs_val + ns * kHT);
    rs_col = reinterpret_cast<int *>(terms + nterm);
    cs_col = rs_col + ns * kHT;
  }

  // Collapse slots of rows i0.. and columns j0.. (conjugated) and the term
  // list into shared memory.
  __device__ void stage_collapse(int i0, int j0) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int q = warp; q < ns; q += nw) {
      const int base = __ldg(a.cslot_off + q);
      const int i = i0 + lane, j = j0 + lane;
      rs_val[q * kHT + lane] = i < d ? val[base + i] : cmake<V>(0.0, 0.0);
      rs_col[q * kHT + lane] = i < d ? __ldg(a.ops.col + base + i) : 0;
      cs_val[q * kHT + lane] = j < d ? cconj(val[base + j]) : cmake<V>(0.0, 0.0);
      cs_col[q * kHT + lane] = j < d ? __ldg(a.ops.col + base + j) : 0;
    }
    for (int k = threadIdx.x; k < nterm; k += blockDim.x) terms[k] = __ldg(a.cterms + k);
  }

  // sum_n (C_n y C_n^dag) at (i0 + r, j0 + lane) from the staged slots.
  __device__ __forceinline__ void collapse_staged(const V *__restrict__ y, int r, int lane,
                                                  V &out) const {
    V acc = cmake<V>(0.0, 0.0);
    int k = 0;
    for (; k + 8 <= nterm; k += 8) {  // eight independent gathers in flight
      int2 tm[8];
      V g[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        tm[u] = terms[k + u];
        g[u] = y[rs_col[tm[u].x * kHT + r] * d + cs_col[tm[u].y * kHT + lane]];
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const V p = rs_val[tm[u].x * kHT + r], q = cs_val[tm[u].y * kHT + lane];
        V pq;
        pq.x = p.x * q.x - p.y * q.y;
        pq.y = p.x * q.y + p.y * q.x;
        cmac(acc, pq, g[u]);
      }
    }
    for (; k < nterm; ++k) {
      const int2 tm = terms[k];
      const V g = y[rs_col[tm.x * kHT + r] * d + cs_col[tm.y * kHT + lane]];
      const V p = rs_val[tm.x * kHT + r], q = cs_val[tm.y * kHT + lane];
      V pq;
      pq.x = p.x * q.x - p.y * q.y;
      pq.y = p.x * q.y + p.y * q.x;
      cmac(acc, pq, g);
    }
    out.x += acc.x;
    out.y += acc.y;
  }

  // Runs body(i, j, idx, f) for every upper-triangle entry, with f the
  // right-hand side at (i, j) of the state y whose product Y the provider
  // holds (f is not computed when with_f is false).  body returns whether it
  // produced a value v (written through the provider at (i, j) and as conj(v)
  // at (j, i) into out).
  template <bool with_f, typename Body>
  __device__ void phase(const V *__restrict__ y, V *out, Body &&body) {
    const V *Y = prod.product();
    const V *Wc = prod.collapse_product();  // dense collapse terms, when the provider has them
    const int ys = prod.ystride();
    V *t0 = Ys, *t1 = Ys + kHT * kHTP, *ms = Ys + 2 * kHT * kHTP;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int p = blockIdx.x; p < n_pairs; p += gridDim.x) {
      int I, J;
      tile_pair(p, nt, I, J);
      const int i0 = I * kHT, j0 = J * kHT;
      if (with_f) {
        // the tiles Y[i0.., j0..] and Y[j0.., i0..] (rows coalesced)
        for (int r = warp; r < kHT; r += nw) {
          const int ia = i0 + r, ja = j0 + lane, ib = j0 + r, jb = i0 + lane;
          if constexpr (Prod::kFusedY) {
            t0[r * kHTP + lane] = prod.entry(y, ia, ja);
            t1[r * kHTP + lane] = prod.entry(y, ib, jb);
          } else {
            t0[r * kHTP + lane] = (ia < d && ja < d) ? Y[ia * ys + ja] : cmake<V>(0.0, 0.0);
            t1[r * kHTP + lane] = (ib < d && jb < d) ? Y[ib * ys + jb] : cmake<V>(0.0, 0.0);
          }
        }
        if (ns > 0 && !Wc) stage_collapse(i0, j0);
        __syncthreads();
      }
      for (int r = warp; r < kHT; r += nw) {
        const int i = i0 + r, j = j0 + lane;
        bool wrote = false;
        if (i < d && j < d && j >= i) {
          V f = cmake<V>(0.0, 0.0);
          if (with_f) {
            const V yij = t0[r * kHTP + lane], yji = t1[lane * kHTP + r];
            f.x = yij.y + yji.y;  // -i (Y_ij - conj(Y_ji))
            f.y = yji.x - yij.x;
            if (Wc) {
              const V w = Wc[i * ys + j];
              f.x += w.x;
              f.y += w.y;
            } else if (ns > 0) {
              collapse_staged(y, r, lane, f);
            } else {
              me.collapse(y, i, j, f);
            }
          }
          V v;
          wrote = body(i, j, i * d + j, f, v);
          if (wrote) {
            prod.store(out, i * d + j, i, j, v);
            ms[r * kHTP + lane] = v;
          }
        }
        if (!wrote) ms[r * kHTP + lane] = cmake<V>(0.0, 0.0);
      }
      if (out) {
        __syncthreads();
        // mirror: (j, i) for the entries above written, rows j coalesced in i
        for (int r = warp; r < kHT; r += nw) {
          const int j = j0 + r, i = i0 + lane;
          if (i < d && j < d && j > i) {
            V v = ms[lane * kHTP + r];
            v.y = -v.y;  // conjugate in the state's own precision
            prod.store(out, j * d + i, j, i, v);
          }
        }
      }
      __syncthreads();  // the staged tiles are reused by the next pair
    }
  }
};

// The solve on the grid for a Hermitian initial state (a ket, or a density
// matrix the caller has found Hermitian); workspace: rho, ynew, two stage
// inputs, k1..k7 (upper triangles), d*d each.
template <typename T, typename Prod>
__device__ void me_solve_herm(const MeArgs &a, GridTeam &team, Prod &prod, const typename CT<T>::V *val,
                              typename CT<T>::V *tiles, double *sh, double *tot) {
  using V = typename CT<T>::V;
  HermSolver<T, Prod> hs(a, team, prod, val, tiles);
  const int d = a.ops.d;
  const int n = d * d;
  V *base = reinterpret_cast<V *>(a.work);
  V *rho = base, *ynew = base + n, *buf0 = base + 2 * n, *buf1 = base + 3 * n;
  V *k[7];
#pragma unroll
  for (int s = 0; s < 7; ++s) k[s] = base + (4 + s) * n;
  double v[kMePartialMax];

  // ---- initial state: rho0 = |psi><psi| / <psi|psi>, or the Hermitian part
  // of the given matrix (equal to it up to rounding)
  double scale = 1.0;
  if (a.state_is_ket) {
    v[0] = 0.0;
    for (int64_t i = team.tid; i < d; i += team.stride)
      v[0] += a.state0[i].x * a.state0[i].x + a.state0[i].y * a.state0[i].y;
    team.sum(v, 1, sh, tot);
    if (!(tot[0] > 0.0)) {
      if (team.tid == 0) set_status(a.status, QT_ENORM);
      return;
    }
    scale = 1.0 / tot[0];
  }
  hs.template phase<false>(nullptr, rho, [&](int i, int j, int idx, V, V &out) {
    double2 r;
    if (a.state_is_ket) {
      const double2 p = a.state0[i], q = a.state0[j];  // p conj(q)
      r = make_double2((p.x * q.x + p.y * q.y) * scale, (p.y * q.x - p.x * q.y) * scale);
    } else {
      const double2 u = a.state0[idx], w = a.state0[j * d + i];
      r = make_double2(0.5 * (u.x + w.x), 0.5 * (u.y - w.y));
    }
    if (i == j) r.y = 0.0;
    out = cmake<V>(r.x, r.y);
    return true;
  });
  prod.publish(team);

  unsigned long long n_acc = 0, n_rej = 0, n_rhs = 0;
  // k_out = f(y) on the upper triangle
  auto eval = [&](const V *y, V *kout, double te) {
    prod.prepare(team, y, te);
    hs.template phase<true>(y, nullptr, [&](int, int, int idx, V f, V &) {
      kout[idx] = f;
      return false;
    });
    ++n_rhs;
  };
  auto output = [&](int m, const V *y) {
    if (a.states)
      for (int64_t idx = team.tid; idx < n; idx += team.stride)
        a.states[(int64_t)m * n + idx] = make_double2((double)y[idx].x, (double)y[idx].y);
    for (int e0 = 0; e0 < a.n_e; e0 += kMePartialMax / 2) {
      const int ne = min(a.n_e - e0, kMePartialMax / 2);
      for (int q = 0; q < 2 * ne; ++q) v[q] = 0.0;
      for (int64_t i = team.tid; i < d; i += team.stride) {
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
      team.sync();
    }
  };

  eval(rho, k[0], a.tlist[0]);
  output(0, rho);
  int status = QT_OK;
  if (a.n_t > 1) {
    double t = a.tlist[0];
    double hprop = a.h0;
    if (!(hprop > 0.0)) {
      // Hairer-Norsett-Wanner starting step
      team.sync();  // k[0] complete
      v[0] = v[1] = 0.0;
      {
        // in the state's precision (FP64 for the FP64 solver, as the oracle)
        const T at = (T)a.atol, rt = (T)a.rtol;
        T s0 = (T)0, s1 = (T)0;
        hs.template phase<false>(nullptr, nullptr, [&](int i, int j, int idx, V, V &) {
          const V r = rho[idx], f = k[0][idx];
          const T sx = at + rt * tabs(r.x), sy = at + rt * tabs(r.y);
          const T wt = i == j ? (T)1 : (T)2;
          s0 += wt * ((r.x / sx) * (r.x / sx) + (r.y / sy) * (r.y / sy));
          s1 += wt * ((f.x / sx) * (f.x / sx) + (f.y / sy) * (f.y / sy));
          return false;
        });
        v[0] = (double)s0;
        v[1] = (double)s1;
      }
      team.sum(v, 2, sh, tot);
      const double nr = 2.0 * (double)n;
      const double d0 = sqrt(tot[0] / nr), d1 = sqrt(tot[1] / nr);
      const double h0 = (d0 < 1e-5 || d1 < 1e-5) ? 1e-6 : 0.01 * d0 / d1;
      hs.template phase<false>(nullptr, buf0, [&](int, int, int idx, V, V &out) {
        const V r = rho[idx], f = k[0][idx];
        out = cmake<V>((double)r.x + h0 * (double)f.x, (double)r.y + h0 * (double)f.y);
        return true;
      });
      prod.publish(team);
      eval(buf0, k[1], t + h0);
      team.sync();
      {
        const T at = (T)a.atol, rt = (T)a.rtol;
        T s2 = (T)0;
        hs.template phase<false>(nullptr, nullptr, [&](int i, int j, int idx, V, V &) {
          const V r = rho[idx];
          const T sx = at + rt * tabs(r.x), sy = at + rt * tabs(r.y);
          const T ex = (k[1][idx].x - k[0][idx].x) / sx;
          const T ey = (k[1][idx].y - k[0][idx].y) / sy;
          s2 += (i == j ? (T)1 : (T)2) * (ex * ex + ey * ey);
          return false;
        });
        v[0] = (double)s2;
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
        hs.template phase<false>(nullptr, buf0, [&](int, int, int idx, V, V &y) {
          const V r = rho[idx], f0 = k[0][idx];
          y.x = fma(ht, DPW<T>::a21 * f0.x, r.x);
          y.y = fma(ht, DPW<T>::a21 * f0.y, r.y);
          return true;
        });
        prod.publish(team);
        // stages 2..6, each fused with the next stage input
#pragma unroll 1
        for (int st = 1; st <= 5; ++st) {
          const V *in = (st & 1) ? buf0 : buf1;
          V *nxt = (st == 5) ? ynew : ((st & 1) ? buf1 : buf0);
          prod.prepare(team, in, stage_time(t, kDpC[st], h));
          hs.template phase<true>(in, nxt, [&](int, int, int idx, V f, V &y) {
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
            y.x = fma(ht, ax, r.x);
            y.y = fma(ht, ay, r.y);
            return true;
          });
          ++n_rhs;
          prod.publish(team);
        }
        // k7 = f(ynew) fused with the error norm
        prod.prepare(team, ynew, t + h);
        v[0] = 0.0;
        {
          const T at = (T)a.atol, rt = (T)a.rtol;
          T acc = (T)0;
          hs.template phase<true>(ynew, nullptr, [&](int i, int j, int idx, V f, V &) {
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
            const T wt = i == j ? (T)1 : (T)2;
            acc = fma(wt * qx, qx, acc);
            acc = fma(wt * qy, qy, acc);
            return false;
          });
          v[0] = (double)acc;
        }
        ++n_rhs;
        if constexpr (Prod::kCanFail) {
          v[1] = (double)prod.failed();
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
  if constexpr (Prod::kCanFail) {
    if (status == QT_OK) {
      v[0] = (double)prod.failed();
      team.sum(v, 1, sh, tot);
      if (tot[0] != 0.0) status = QT_ETIMEOUT;
    }
  }
  if (status != QT_OK && team.tid == 0) set_status(a.status, status);
  if (team.tid == 0) {
    atomicAdd(a.counters + 0, n_acc);
    atomicAdd(a.counters + 1, n_rej);
    atomicAdd(a.counters + 2, n_rhs);
  }
}

// Whether the d x d matrix m is Hermitian within kHermTol2; the same answer
// in every CTA of the grid.
__device__ bool herm_check(const double2 *m, int d, GridTeam &team, double *sh, double *tot) {
  double v[2] = {0.0, 0.0};
  const int64_t n = (int64_t)d * d;
  for (int64_t idx = team.tid; idx < n; idx += team.stride) {
    const int i = (int)(idx / d), j = (int)(idx - (int64_t)i * d);
    const double2 u = m[idx], w = m[(int64_t)j * d + i];
    const double dx = u.x - w.x, dy = u.y + w.y;
    v[0] += dx * dx + dy * dy;
    v[1] += u.x * u.x + u.y * u.y;
  }
  team.sum(v, 2, sh, tot);
  const bool ok = tot[0] <= kHermTol2 * tot[1];
  team.sync();  // tot is rewritten by the next reduction
  return ok;
}

// One evaluation of drho/dt on the Hermitian path (a.rhs_in -> a.rhs_out,
// both triangles written).
template <typename T, typename Prod>
__device__ void me_rhs_once_herm(const MeArgs &a, GridTeam &team, Prod &prod,
                                 const typename CT<T>::V *val, typename CT<T>::V *tiles) {
  using V = typename CT<T>::V;
  HermSolver<T, Prod> hs(a, team, prod, val, tiles);
  const int d = a.ops.d;
  V *y = reinterpret_cast<V *>(a.work);
  hs.template phase<false>(nullptr, y, [&](int i, int j, int idx, V, V &out) {
    const double2 u = a.rhs_in[idx], w = a.rhs_in[j * d + i];
    out = cmake<V>(0.5 * (u.x + w.x), i == j ? 0.0 : 0.5 * (u.y - w.y));
    return true;
  });
  prod.publish(team);
  prod.prepare(team, y, a.rhs_t);
  hs.template phase<true>(y, nullptr, [&](int i, int j, int idx, V f, V &) {
    a.rhs_out[idx] = make_double2((double)f.x, (double)f.y);
    a.rhs_out[j * d + i] = make_double2((double)f.x, -(double)f.y);
    return false;
  });
}

}  // namespace

}  // namespace qt
