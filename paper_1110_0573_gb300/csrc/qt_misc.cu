// qt_misc.cu -- small kernels around the solvers: expectation values of a
// batch of states (the paper's expect(), section 2), normalisation of the
// initial ket (Qobj.unit()), and the hand-over of device-side statistics.
#include "qt_device.cuh"
#include "qt_internal.h"

namespace qt {

namespace {

constexpr int kExpBlock = 128;

// One CTA per state.  Kets: <psi|O|psi> = sum_i conj(psi_i) (O psi)_i.
// Density matrices: Tr(O rho) = sum_i sum_s O[i, c_s] rho[c_s, i].  FP64.
__global__ void __launch_bounds__(kExpBlock)
    expect_kernel(const __grid_constant__ OpTable ops, int op, const double2 *states,
                  int is_ket, int64_t batch, double2 *out) {
  __shared__ double sh[2 * (kExpBlock / 32)];
  const int d = ops.d;
  const int w = ops.w[op];
  const int64_t off = ops.off[op];
  for (int64_t b = blockIdx.x; b < batch; b += gridDim.x) {
    double re = 0.0, im = 0.0;
    if (is_ket) {
      const double2 *psi = states + b * d;
      for (int i = threadIdx.x; i < d; i += blockDim.x) {
        double2 acc = make_double2(0.0, 0.0);
        for (int s = 0; s < w; ++s) {
          const int64_t p = off + (int64_t)s * d + i;
          cmac(acc, ops.val64[p], psi[ops.col[p]]);
        }
        const double2 x = psi[i];
        re += x.x * acc.x + x.y * acc.y;
        im += x.x * acc.y - x.y * acc.x;
      }
    } else {
      const double2 *rho = states + b * (int64_t)d * d;
      for (int i = threadIdx.x; i < d; i += blockDim.x) {
        for (int s = 0; s < w; ++s) {
          const int64_t p = off + (int64_t)s * d + i;
          const double2 o = ops.val64[p];
          const double2 r = rho[(int64_t)ops.col[p] * d + i];
          re += o.x * r.x - o.y * r.y;
          im += o.x * r.y + o.y * r.x;
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      re += __shfl_xor_sync(0xffffffffu, re, o);
      im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    const int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { sh[2 * warp] = re; sh[2 * warp + 1] = im; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double sr = 0.0, si = 0.0;
      for (int q = 0; q < kExpBlock / 32; ++q) { sr += sh[2 * q]; si += sh[2 * q + 1]; }
      out[b] = make_double2(sr, si);
    }
    __syncthreads();
  }
}

constexpr int kNormaliseBlock = 256;

// out = in / ||in|| (one CTA); status QT_ENORM for a zero or non-finite norm.
__global__ void normalise_kernel(const double2 *in, double2 *out, int d, int *status,
                                 const double *tlist, int n_t, double *ivl_tb, float *ivl_len) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < d; i += blockDim.x) s += in[i].x * in[i].x + in[i].y * in[i].y;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += sh[q];
    sh[0] = t;
    if (!(t > 0.0) || !isfinite(t)) set_status(status, QT_ENORM);
  }
  __syncthreads();
  const double inv = 1.0 / sqrt(sh[0]);
  for (int i = threadIdx.x; i < d; i += blockDim.x)
    out[i] = make_double2(in[i].x * inv, in[i].y * inv);
  // the output intervals: each starts where the previous one ended (a serial
  // recurrence, run by thread 0 on output times staged in shared memory by
  // the whole block, blockDim.x at a time)
  if (ivl_len) {
    __shared__ double tl[kNormaliseBlock];
    double tb = tlist[0];
    for (int base = 1; base < n_t; base += kNormaliseBlock) {
      __syncthreads();
      if (base + (int)threadIdx.x < n_t) tl[threadIdx.x] = tlist[base + threadIdx.x];
      __syncthreads();
      if (threadIdx.x == 0) {
        const int e = min(kNormaliseBlock, n_t - base);
        for (int j = 0; j < e; ++j) {
          const float len = (float)(tl[j] - tb);
          ivl_tb[base + j] = tb;
          ivl_len[base + j] = len;
          tb = tb + (double)len;
        }
      }
    }
  }
}

__global__ void finalize_kernel(const unsigned long long *c, const int *status,
                                const unsigned long long *n_jumps, qt_stats *st) {
  st->accepted = (int64_t)c[0];
  st->rejected = (int64_t)c[1];
  st->rhs_evals = (int64_t)c[2];
  st->bisect_iters = (int64_t)c[3];
  st->jumps = (int64_t)c[4];
  st->near_miss = (int64_t)c[5];
  st->status = *status;
  st->reserved = 0;
  (void)n_jumps;
}

}  // namespace

cudaError_t launch_expect(const OpTable &ops, int op_index, const double2 *states, int is_ket,
                          int64_t batch, double2 *out, cudaStream_t s) {
  if (batch <= 0) return cudaSuccess;
  const int64_t grid = batch < 65535 ? batch : 65535;
  expect_kernel<<<(unsigned)grid, kExpBlock, 0, s>>>(ops, op_index, states, is_ket, batch, out);
  return cudaGetLastError();
}

cudaError_t launch_normalise(const double2 *in, double2 *out, int d, int *status,
                             cudaStream_t s, const double *tlist, int n_t, double *ivl_tb,
                             float *ivl_len) {
  normalise_kernel<<<1, kNormaliseBlock, 0, s>>>(in, out, d, status, tlist, n_t, ivl_tb, ivl_len);
  return cudaGetLastError();
}

cudaError_t launch_finalize_stats(const unsigned long long *counters, const int *status,
                                  const unsigned long long *n_jumps, qt_stats *stats,
                                  cudaStream_t s) {
  finalize_kernel<<<1, 1, 0, s>>>(counters, status, n_jumps, stats);
  return cudaGetLastError();
}

}  // namespace qt
