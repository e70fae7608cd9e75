// qt_ss.cu -- steady state of the master equation (the paper's steadystate,
// section 5 function list): the density matrix rho with L(rho) = 0 and
// Tr rho = 1, for a Liouvillian L with a unique stationary state.
//
// The constraint is folded into an invertible operator:
//   A(x) = L(x) + w Tr(x) I,    A(rho) = w I,
// (A(x) = 0 forces Tr x = 0, as Tr L(x) = 0, hence L(x) = 0 and x = 0 when the
// null space of L is spanned by rho).  A x = w I is solved matrix-free by
// restarted GMRES(m) (Saad and Schultz 1986) with a diagonal (Jacobi) right
// preconditioner, in one cooperative launch:
//  * every application of A is the general master-equation right-hand side
//    of qt_me_impl.cuh plus the trace term;
//  * the m + 1 basis vectors live in device memory; each CTA owns a
//    contiguous chunk of the d*d entries and keeps its chunk of the vector
//    being orthogonalised in shared memory;
//  * classical Gram-Schmidt with one reorthogonalisation (two passes): each
//    pass forms all inner products at once (per-CTA partials, one CTA per
//    product adds them in a fixed order), so an Arnoldi step costs five grid
//    barriers whatever its length;
//  * the Givens rotations of the least-squares problem are applied by one
//    warp of CTA 0 to blocks of 16 Hessenberg columns at once (a lane per
//    column), so the residual estimate is known every 16 steps, after one
//    grid barrier; the iteration stops at the first column that met the
//    tolerance (the few steps taken past it are discarded).
// The result is (x + x^dag) / 2 scaled to unit trace.
#include "qt_me_impl.cuh"

namespace qt {

namespace {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  const double den = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / den, (a.y * b.x - a.x * b.y) / den);
}
__device__ __forceinline__ double2 cscale(double2 a, double s) {
  return make_double2(a.x * s, a.y * s);
}
__device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }

// Diagonal entry (i, i) of table operator op (ELL rows; padding adds zero).
__device__ __forceinline__ double2 ell_diag(const OpTable &ops, int op, int i) {
  double2 acc = make_double2(0.0, 0.0);
  const int d = ops.d;
  const int w = ops.w[op];
  const int64_t off = ops.off[op];
  for (int s = 0; s < w; ++s) {
    const int64_t p = off + (int64_t)s * d + i;
    if (__ldg(ops.col + p) == i) {
      const double2 v = ops.val64[p];
      acc.x += v.x;
      acc.y += v.y;
    }
  }
  return acc;
}

constexpr int kGmRot = 16;  // Hessenberg columns rotated together (<= 32)

// Givens rotations of the Hessenberg columns jb0..je (at most kGmRot,
// stored unrotated in R with leading dimension m + 1), by one warp with a
// lane per column: first the rotations of the earlier columns, each applied
// to all the block's columns at once, then the block's own rotations in
// order, each formed by its column's lane and applied by the lanes of the
// later columns.  Updates the rotated right-hand side gg and writes ctl[0] =
// the first column whose residual estimate is <= lim (-1 if none), ctl[1] =
// that estimate (else the last one).
__device__ void givens_block(const GmArgs &g, int m, int jb0, int je, double *cs, double2 *sn,
                             double2 *gg, double lim, int lane) {
  const int64_t ld = m + 1;
  const int c = jb0 + lane;
  const bool mine = c <= je;
  double2 *col = g.R + (int64_t)(mine ? c : jb0) * ld;
  double2 cur = mine ? col[0] : make_double2(0.0, 0.0);
  for (int q = 0; q < jb0; ++q) {
    const double cq = cs[q];
    const double2 sq = sn[q];
    if (mine) {
      // [c s; -conj(s) c] applied to rows (q, q+1)
      const double2 h1 = col[q + 1];
      const double2 t0 = cmul(sq, h1), t1 = cmul(make_double2(sq.x, -sq.y), cur);
      col[q] = make_double2(cq * cur.x + t0.x, cq * cur.y + t0.y);
      cur = make_double2(cq * h1.x - t1.x, cq * h1.y - t1.y);
    }
  }
  double conv = -1.0, rconv = 0.0, last = 0.0;
  for (int q = jb0; q <= je; ++q) {
    double cq = 0.0;
    double2 sq = make_double2(0.0, 0.0);
    if (c == q) {
      const double hn = col[q + 1].x;
      const double aa = sqrt(cabs2(cur));
      const double nu = sqrt(aa * aa + hn * hn);
      double2 ph;
      if (aa == 0.0) {
        cq = 0.0;
        sq = make_double2(1.0, 0.0);
        ph = make_double2(1.0, 0.0);
      } else {
        cq = aa / nu;
        ph = cscale(cur, 1.0 / aa);
        sq = cscale(ph, hn / nu);
      }
      col[q] = cscale(ph, nu);
    }
    const int src = q - jb0;
    cq = __shfl_sync(0xffffffffu, cq, src);
    sq.x = __shfl_sync(0xffffffffu, sq.x, src);
    sq.y = __shfl_sync(0xffffffffu, sq.y, src);
    if (mine && c > q) {
      const double2 h1 = col[q + 1];
      const double2 t0 = cmul(sq, h1), t1 = cmul(make_double2(sq.x, -sq.y), cur);
      col[q] = make_double2(cq * cur.x + t0.x, cq * cur.y + t0.y);
      cur = make_double2(cq * h1.x - t1.x, cq * h1.y - t1.y);
    }
    if (lane == 0) {
      cs[q] = cq;
      sn[q] = sq;
      const double2 g0 = gg[q];
      const double2 t = cmul(make_double2(sq.x, -sq.y), g0);
      gg[q + 1] = make_double2(-t.x, -t.y);
      gg[q] = cscale(g0, cq);
      last = sqrt(cabs2(gg[q + 1]));
      if (conv < 0.0 && last <= lim) {
        conv = (double)q;
        rconv = last;
      }
    }
  }
  if (lane == 0) {
    g.ctl[0] = conv;
    g.ctl[1] = conv >= 0.0 ? rconv : last;
  }
}

__global__ void __launch_bounds__(kGmBlock, 1) gmres_kernel(const __grid_constant__ MeArgs a,
                                                            const __grid_constant__ GmArgs g) {
  extern __shared__ double2 dsm[];
  const int m = g.m;
  double2 *wv = dsm;             // this CTA's chunk of the vector being built
  double2 *hs = wv + g.chunk;    // Hessenberg column (m + 2)
  double2 *hp = hs + m + 2;      // coefficients of one Gram-Schmidt pass (m + 1)
  double2 *sn = hp + m + 1;      // Givens sines (m)
  double2 *gg = sn + m;          // rotated right-hand side (m + 1)
  double2 *red = gg + m + 1;     // per-warp partial sums, kGmBlock (small chunks)
  double *cs = reinterpret_cast<double *>(red + kGmBlock);  // Givens cosines (m)
  __shared__ double sh[kMePartialMax * (kGmBlock / 32) + kMePartialMax];
  __shared__ double tot[kMePartialMax];
  __shared__ double tdcoef[kTdMax];
  cg::grid_group grid = cg::this_grid();
  const int d = a.ops.d;
  const int64_t n = (int64_t)d * d;
  const int64_t c0 = (int64_t)blockIdx.x * g.chunk;
  const int64_t c1 = c0 + g.chunk < n ? c0 + g.chunk : n;
  const int nl = c1 > c0 ? (int)(c1 - c0) : 0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const bool small = g.chunk <= 32;  // at most a warp's width of entries per CTA
  SparseRhs<double> L(a, reinterpret_cast<const double2 *>(a.ops.val64), tdcoef);
  int half = 0;
  // consecutive sums alternate between the two halves of each CTA's partial
  // slots (a CTA that runs ahead never overwrites partials still being read)
  auto gsum = [&](double *vals, int nv) {
    grid_sum(vals, nv, sh, a.partial + (half & 1) * (kMePartialMax / 2), tot, grid);
    ++half;
  };

  // ---- diagonal of L, trace weight w = mean |L_(ij),(ij)|, preconditioner
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int l = threadIdx.x; l < nl; l += blockDim.x) {
    const int64_t idx = c0 + l;
    const int i = (int)(idx / d), j = (int)(idx - (int64_t)i * d);
    const double2 hi = ell_diag(a.ops, 0, i), hj = ell_diag(a.ops, 0, j);
    // -i H_eff,ii + i conj(H_eff,jj) + sum_n C_n,ii conj(C_n,jj)
    double2 D = make_double2(hi.y + hj.y, hj.x - hi.x);
    for (int c = 1; c <= a.n_c; ++c) {
      const double2 ci = ell_diag(a.ops, c, i), cj = ell_diag(a.ops, c, j);
      const double2 t = cmul(ci, make_double2(cj.x, -cj.y));
      D.x += t.x;
      D.y += t.y;
    }
    g.minv[idx] = D;
    acc[0] += sqrt(cabs2(D));
  }
  gsum(acc, 1);
  double w = tot[0] / (double)n;
  if (!(w > 0.0) || !isfinite(w)) w = 1.0;
  const double bnorm = w * sqrt((double)d);  // ||w I||_F
  for (int l = threadIdx.x; l < nl; l += blockDim.x) {
    const int64_t idx = c0 + l;
    double2 M = g.minv[idx];
    if (idx % (d + 1) == 0) M.x += w;
    if (!(sqrt(cabs2(M)) >= 1e-3 * w)) M = make_double2(w, 0.0);
    g.minv[idx] = cdiv(make_double2(1.0, 0.0), M);
    g.x[idx] = make_double2(idx % (d + 1) == 0 ? 1.0 / (double)d : 0.0, 0.0);
  }
  grid.sync();

  int64_t it = 0;
  unsigned long long n_mv = 0;
  int status = QT_OK;
  double resid = 0.0;
  for (;;) {  // restarts
    // Tr x (x is complete: every path here follows a barrier)
    acc[0] = acc[1] = 0.0;
    for (int l = threadIdx.x; l < nl; l += blockDim.x)
      if ((c0 + l) % (d + 1) == 0) { acc[0] += g.x[c0 + l].x; acc[1] += g.x[c0 + l].y; }
    gsum(acc, 2);
    const double2 trx = make_double2(tot[0], tot[1]);
    // r = w I - A x into wv; z = M^-1 r into zu; ||r||^2, Tr z
    L.prepare(g.x, 0.0);
    acc[0] = acc[1] = acc[2] = 0.0;
    for (int l = threadIdx.x; l < nl; l += blockDim.x) {
      const int64_t idx = c0 + l;
      const int i = (int)(idx / d), j = (int)(idx - (int64_t)i * d);
      const double2 f = L.f(g.x, i, j);
      double2 rr = make_double2(-f.x, -f.y);
      if (i == j) { rr.x += w * (1.0 - trx.x); rr.y -= w * trx.y; }
      wv[l] = rr;
      const double2 z = cmul(g.minv[idx], rr);
      g.zu[idx] = z;
      acc[0] += cabs2(rr);
      if (i == j) { acc[1] += z.x; acc[2] += z.y; }
    }
    ++n_mv;
    gsum(acc, 3);
    const double beta = sqrt(tot[0]);
    double2 trzu = make_double2(tot[1], tot[2]);
    resid = beta;
    if (!isfinite(beta)) { status = QT_ENUMERIC; break; }
    if (beta <= g.tol * bnorm) break;
    if (it >= g.max_iter) { status = QT_ESTEP; break; }
    if (threadIdx.x == 0) {
      gg[0] = make_double2(beta, 0.0);
      for (int q = 1; q <= m; ++q) gg[q] = make_double2(0.0, 0.0);
    }
    double hprev = beta;
    int k = 0, jb0 = 0;
    for (int jj = 0; jj < m && it < g.max_iter; ++jj) {
      ++it;
      const double inv = 1.0 / hprev;
      // v_jj = wv / hprev; wv = A z_jj = (L(zu) + w Tr(zu) I) / hprev
      double2 *vj = g.V + (int64_t)jj * n + c0;
      L.prepare(g.zu, 0.0);
      for (int l = threadIdx.x; l < nl; l += blockDim.x) {
        const int64_t idx = c0 + l;
        const int i = (int)(idx / d), j = (int)(idx - (int64_t)i * d);
        vj[l] = cscale(wv[l], inv);
        double2 f = L.f(g.zu, i, j);
        if (i == j) { f.x += w * trzu.x; f.y += w * trzu.y; }
        wv[l] = cscale(f, inv);
      }
      ++n_mv;
      __syncthreads();
      // two passes of classical Gram-Schmidt against v_0 .. v_jj
      for (int pass = 0; pass < 2; ++pass) {
        if (small) {
          // a thread per basis vector over the CTA's few entries
          for (int i = threadIdx.x; i <= jj; i += blockDim.x) {
            const double2 *vi = g.V + (int64_t)i * n + c0;
            double ax = 0.0, ay = 0.0;
            for (int l = 0; l < nl; ++l) {
              const double2 v = vi[l], u = wv[l];
              ax += v.x * u.x + v.y * u.y;
              ay += v.x * u.y - v.y * u.x;
            }
            g.pd[(int64_t)blockIdx.x * (m + 1) + i] = make_double2(ax, ay);
          }
        } else {
          // a warp per basis vector, lanes over the CTA's entries
          for (int i = warp; i <= jj; i += nw) {
            const double2 *vi = g.V + (int64_t)i * n + c0;
            double ax = 0.0, ay = 0.0;
            for (int l = lane; l < nl; l += 32) {
              const double2 v = vi[l], u = wv[l];
              ax += v.x * u.x + v.y * u.y;
              ay += v.x * u.y - v.y * u.x;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
              ax += __shfl_xor_sync(0xffffffffu, ax, o);
              ay += __shfl_xor_sync(0xffffffffu, ay, o);
            }
            if (lane == 0) g.pd[(int64_t)blockIdx.x * (m + 1) + i] = make_double2(ax, ay);
          }
        }
        grid.sync();
        // inner product i summed over the CTAs by CTA i mod grid, in CTA order
        for (int i = blockIdx.x; i <= jj; i += gridDim.x) {
          double v2[2] = {0.0, 0.0};
          for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
            const double2 q = g.pd[(int64_t)b * (m + 1) + i];
            v2[0] += q.x;
            v2[1] += q.y;
          }
          block_sum(v2, 2, sh);
          if (threadIdx.x == 0)
            g.hcol[i] = make_double2(sh[sh_total()], sh[sh_total() + 1]);
          __syncthreads();
        }
        grid.sync();
        for (int i = threadIdx.x; i <= jj; i += blockDim.x) {
          const double2 q = g.hcol[i];
          hp[i] = q;
          hs[i] = pass ? make_double2(hs[i].x + q.x, hs[i].y + q.y) : q;
        }
        __syncthreads();
        // wv -= sum_i hp_i v_i; after the second pass also z = M^-1 wv,
        // ||wv||^2 and Tr z.  Few entries per CTA: warp w adds the basis
        // vectors i = w, w + nw, ... for lane = entry, then the warps' sums
        // are combined in shared memory.
        if (small) {
          double2 part = make_double2(0.0, 0.0);
          if (lane < nl)
            for (int i = warp; i <= jj; i += nw) {
              const double2 t = cmul(hp[i], g.V[(int64_t)i * n + c0 + lane]);
              part.x += t.x;
              part.y += t.y;
            }
          red[warp * 32 + lane] = part;
          __syncthreads();
        }
        for (int l = threadIdx.x; l < nl; l += blockDim.x) {
          double2 u = wv[l];
          if (small) {
            for (int w2 = 0; w2 < nw; ++w2) {
              u.x -= red[w2 * 32 + l].x;
              u.y -= red[w2 * 32 + l].y;
            }
          } else {
            for (int i = 0; i <= jj; ++i) {
              const double2 t = cmul(hp[i], g.V[(int64_t)i * n + c0 + l]);
              u.x -= t.x;
              u.y -= t.y;
            }
          }
          wv[l] = u;
          if (pass == 1) {
            const int64_t idx = c0 + l;
            const double2 z = cmul(g.minv[idx], u);
            g.zu[idx] = z;
            acc[0] += cabs2(u);
            if (idx % (d + 1) == 0) { acc[1] += z.x; acc[2] += z.y; }
          }
        }
        if (pass == 0) {
          __syncthreads();
          acc[0] = acc[1] = acc[2] = 0.0;
        }
      }
      gsum(acc, 3);
      const double hnew = sqrt(tot[0]);
      trzu = make_double2(tot[1], tot[2]);
      // the new Hessenberg column, unrotated, into column jj of R (CTA 0); its
      // Givens rotations are applied a block of columns at a time
      if (blockIdx.x == 0) {
        for (int q = threadIdx.x; q <= jj; q += blockDim.x) g.R[(int64_t)jj * (m + 1) + q] = hs[q];
        if (threadIdx.x == 0) g.R[(int64_t)jj * (m + 1) + jj + 1] = make_double2(hnew, 0.0);
      }
      k = jj + 1;
      hprev = hnew;
      const bool block_end = jj + 1 - jb0 == kGmRot || jj + 1 == m || it >= g.max_iter ||
                             !(hnew > 0.0) || !isfinite(hnew);
      if (!block_end) continue;
      if (blockIdx.x == 0) {
        __syncthreads();  // this CTA's column writes are complete
        if (warp == 0) givens_block(g, m, jb0, jj, cs, sn, gg, g.tol * bnorm, lane);
      }
      grid.sync();
      const double conv = g.ctl[0];
      resid = g.ctl[1];
      if (!isfinite(resid)) { status = QT_ENUMERIC; break; }
      if (conv >= 0.0) { k = (int)conv + 1; break; }
      if (!(hnew > 0.0)) break;
      jb0 = jj + 1;
    }
    if (status != QT_OK) break;
    // y = R^-1 g by back substitution (CTA 0), then x += M^-1 (V y)
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      for (int i = k - 1; i >= 0; --i) {
        double2 s = gg[i];
        for (int q = i + 1; q < k; ++q) {
          const double2 t = cmul(g.R[(int64_t)q * (m + 1) + i], g.y[q]);
          s.x -= t.x;
          s.y -= t.y;
        }
        g.y[i] = cdiv(s, g.R[(int64_t)i * (m + 1) + i]);
      }
    }
    grid.sync();
    for (int i = threadIdx.x; i < k; i += blockDim.x) hp[i] = g.y[i];
    __syncthreads();
    for (int l = threadIdx.x; l < nl; l += blockDim.x) {
      const int64_t idx = c0 + l;
      double2 u = make_double2(0.0, 0.0);
      for (int i = 0; i < k; ++i) {
        const double2 t = cmul(hp[i], g.V[(int64_t)i * n + idx]);
        u.x += t.x;
        u.y += t.y;
      }
      const double2 dx = cmul(g.minv[idx], u);
      g.x[idx] = make_double2(g.x[idx].x + dx.x, g.x[idx].y + dx.y);
    }
    grid.sync();
  }
  // rho = (x + x^dag) / 2 / Tr x
  acc[0] = 0.0;
  for (int l = threadIdx.x; l < nl; l += blockDim.x)
    if ((c0 + l) % (d + 1) == 0) acc[0] += g.x[c0 + l].x;
  gsum(acc, 1);
  const double trx = tot[0];
  if (status == QT_OK && !(fabs(trx) > 0.0 && isfinite(trx))) status = QT_ENUMERIC;
  const double inv = 1.0 / trx;
  for (int l = threadIdx.x; l < nl; l += blockDim.x) {
    const int64_t idx = c0 + l;
    const int i = (int)(idx / d), j = (int)(idx - (int64_t)i * d);
    const double2 u = g.x[idx], t = g.x[(int64_t)j * d + i];
    g.rho_out[idx] = make_double2(0.5 * (u.x + t.x) * inv, 0.5 * (u.y - t.y) * inv);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (status != QT_OK) set_status(a.status, status);
    atomicAdd(a.counters + 0, (unsigned long long)it);
    atomicAdd(a.counters + 2, n_mv);
    if (g.info) {
      g.info[0] = resid / bnorm;
      g.info[1] = w;
      g.info[2] = (double)it;
    }
  }
}

}  // namespace

size_t gmres_smem_bytes(int chunk, int m) {
  return (size_t)chunk * sizeof(double2) +
         (size_t)(m + 2 + m + 1 + m + m + 1 + kGmBlock) * sizeof(double2) +
         (size_t)m * sizeof(double);
}

int gmres_grid(size_t smem) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
  if (cudaFuncSetAttribute(gmres_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return -1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gmres_kernel, kGmBlock, smem) !=
      cudaSuccess)
    return -1;
  if (per_sm < 1) return -1;
  return sms * per_sm;
}

cudaError_t launch_gmres(const MeArgs &a, const GmArgs &g, int grid, size_t smem,
                         cudaStream_t s) {
  cudaError_t e =
      cudaFuncSetAttribute(gmres_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  void *args[] = {const_cast<MeArgs *>(&a), const_cast<GmArgs *>(&g)};
  return cudaLaunchCooperativeKernel((const void *)gmres_kernel, dim3(grid), dim3(kGmBlock), args,
                                     smem, s);
}

}  // namespace qt

// ---------------------------------------------------------------------------
// Propagator steady state (the paper's propagator_steadystate): the fixed
// point of rho -> V(T) rho, by repeated master-equation solves over one
// period T.  These kernels form the start state I/d and the change
// ||rho_{k+1} - rho_k||_F of one period.
namespace qt {

namespace {

__global__ void identity_state_kernel(double2 *rho, int d) {
  const int64_t n = (int64_t)d * d;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
       idx += (int64_t)gridDim.x * blockDim.x)
    rho[idx] = make_double2(idx % (d + 1) == 0 ? 1.0 / (double)d : 0.0, 0.0);
}

// One CTA (a fixed summation order): out = sqrt(sum |a - b|^2).
__global__ void __launch_bounds__(1024) diff_norm_kernel(const double2 *a, const double2 *b,
                                                         int64_t n, double *out) {
  __shared__ double part[32];
  double s = 0.0;
  for (int64_t idx = threadIdx.x; idx < n; idx += blockDim.x) {
    const double2 u = a[idx], v = b[idx];
    const double dx = u.x - v.x, dy = u.y - v.y;
    s = fma(dx, dx, fma(dy, dy, s));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) *out = sqrt(s);
  }
}

__global__ void set_status_kernel(int *status, int code) { set_status(status, code); }

}  // namespace

cudaError_t launch_set_status(int *status, int code, cudaStream_t s) {
  set_status_kernel<<<1, 1, 0, s>>>(status, code);
  return cudaGetLastError();
}

cudaError_t launch_identity_state(double2 *rho, int d, cudaStream_t s) {
  const int64_t n = (int64_t)d * d;
  const int64_t blocks = (n + 255) / 256;
  identity_state_kernel<<<(unsigned)(blocks < 1024 ? blocks : 1024), 256, 0, s>>>(rho, d);
  return cudaGetLastError();
}

cudaError_t launch_diff_norm(const double2 *a, const double2 *b, int64_t n, double *out,
                             cudaStream_t s) {
  diff_norm_kernel<<<1, 1024, 0, s>>>(a, b, n, out);
  return cudaGetLastError();
}

}  // namespace qt
