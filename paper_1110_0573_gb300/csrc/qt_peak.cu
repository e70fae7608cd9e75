// qt_peak.cu -- FMA throughput of this GPU, measured: the FP32 and FP64
// arithmetic roofs against which the ALU-bound solver kernels are reported.
//
// Every thread runs kChains independent multiply-add chains (no chain waits
// on another, so the pipes, not the latency, bound the rate) for `iters`
// rounds of kUnroll steps; the grid fills every SM to the occupancy limit.
// kinds:
//   QT_PEAK_FP32    scalar FFMA          (2 flop per lane and instruction)
//   QT_PEAK_FP32X2  packed fma.rn.f32x2  (4 flop per lane and instruction)
//   QT_PEAK_FP64    DFMA                 (2 flop per lane and instruction)
// The values stay bounded (x <- x a + b with |a| < 1), and the result is
// stored only when it equals a value it cannot reach, so nothing is dead.
#include <cstdio>
#include <string>

#include "qt_internal.h"

namespace {

constexpr int kPeakBlock = 256;
constexpr int kChains = 8;
constexpr int kUnroll = 16;

__device__ __forceinline__ unsigned long long pack2(float x, float y) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(x), "f"(y));
  return r;
}

__device__ __forceinline__ float2 unpack2(unsigned long long v) {
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
  return r;
}

template <int KIND>
__global__ void __launch_bounds__(kPeakBlock) fma_peak_kernel(double *sink, int iters, double a64,
                                                              double b64) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  double total = 0.0;
  if constexpr (KIND == QT_PEAK_FP64) {
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1e-3 * (t + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int u = 0; u < kUnroll; ++u)
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a64, b64);
    }
#pragma unroll
    for (int c = 0; c < kChains; ++c) total += x[c];
  } else if constexpr (KIND == QT_PEAK_FP32) {
    const float a = (float)a64, b = (float)b64;
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1e-3f * (float)(t + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int u = 0; u < kUnroll; ++u)
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
    }
#pragma unroll
    for (int c = 0; c < kChains; ++c) total += (double)x[c];
  } else {
    const unsigned long long a2 = pack2((float)a64, (float)a64), b2 = pack2((float)b64, (float)b64);
    unsigned long long x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = pack2(1e-3f * (float)(t + c), 2e-3f * (float)(t + c));
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int u = 0; u < kUnroll; ++u)
#pragma unroll
        for (int c = 0; c < kChains; ++c)
          asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[c]) : "l"(a2), "l"(b2));
    }
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
      const float2 v = unpack2(x[c]);
      total += (double)v.x + (double)v.y;
    }
  }
  if (total == -1.0) sink[t] = total;  // unreachable: |x| stays below b / (1 - a)
}

template <int KIND>
int run_peak(int64_t iters, int reps, double *flop_per_s, double *flop_per_launch,
             double *ms_per_launch, cudaStream_t s) {
  auto kern = fma_peak_kernel<KIND>;
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPeakBlock, 0);
  if (e != cudaSuccess) return qt::set_error(QT_ECUDA, cudaGetErrorString(e));
  if (per_sm < 1) per_sm = 1;
  const int grid = sms * per_sm;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return qt::set_error(QT_ECUDA, "cudaEventCreate failed");
  }
  kern<<<grid, kPeakBlock, 0, s>>>(nullptr, (int)iters, 0.999999, 1e-6);  // warm-up
  e = cudaEventRecord(e0, s);
  for (int r = 0; r < reps && e == cudaSuccess; ++r) {
    kern<<<grid, kPeakBlock, 0, s>>>(nullptr, (int)iters, 0.999999, 1e-6);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return qt::set_error(QT_ECUDA, cudaGetErrorString(e));
  const double lanes_flop = KIND == QT_PEAK_FP32X2 ? 4.0 : 2.0;
  const double per_launch =
      (double)grid * kPeakBlock * (double)iters * kUnroll * kChains * lanes_flop;
  const double sec = ms / 1e3 / reps;
  if (flop_per_launch) *flop_per_launch = per_launch;
  if (ms_per_launch) *ms_per_launch = sec * 1e3;
  if (flop_per_s) *flop_per_s = per_launch / sec;
  return QT_OK;
}

}  // namespace

extern "C" int qt_fma_peak(int kind, int64_t iters, int reps, double *flop_per_s,
                           double *flop_per_launch, double *ms_per_launch, void *stream) {
  if (iters < 1 || iters > (1 << 30) || reps < 1 || reps > 10000 || !flop_per_s)
    return qt::set_error(QT_EINVAL, "qt_fma_peak: need 1 <= iters <= 2^30, 1 <= reps <= 10000 "
                                    "and a non-null flop_per_s");
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || n < 1)
    return qt::set_error(QT_ENODEV, "no usable CUDA device");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  switch (kind) {
    case QT_PEAK_FP32:
      return run_peak<QT_PEAK_FP32>(iters, reps, flop_per_s, flop_per_launch, ms_per_launch, s);
    case QT_PEAK_FP32X2:
      return run_peak<QT_PEAK_FP32X2>(iters, reps, flop_per_s, flop_per_launch, ms_per_launch, s);
    case QT_PEAK_FP64:
      return run_peak<QT_PEAK_FP64>(iters, reps, flop_per_s, flop_per_launch, ms_per_launch, s);
    default:
      return qt::set_error(QT_EINVAL, "qt_fma_peak: unknown kind");
  }
}
