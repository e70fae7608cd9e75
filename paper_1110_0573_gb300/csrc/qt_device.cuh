// qt_device.cuh -- device-side building blocks shared by the libqt kernels:
// complex helpers, the counter-based random numbers, the Dormand-Prince
// coefficients and warp-group reductions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace qt {

// ------------------------------------------------------------ complex types
template <typename T> struct CT;
template <> struct CT<float> { using V = float2; };
template <> struct CT<double> { using V = double2; };

template <typename V> __device__ __forceinline__ V cmake(double re, double im);
template <> __device__ __forceinline__ float2 cmake<float2>(double re, double im) {
  return make_float2((float)re, (float)im);
}
template <> __device__ __forceinline__ double2 cmake<double2>(double re, double im) {
  return make_double2(re, im);
}

// Explicitly typed scalar helpers, so that FP32 code never widens to FP64.
__device__ __forceinline__ float tfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double tfma(double a, double b, double c) { return fma(a, b, c); }
// Both components of a complex value scaled and accumulated: y + s x (one
// packed two-lane FP32 instruction on sm_100 and later), y * s.
__device__ __forceinline__ float2 vfma(float s, float2 x, float2 y) {
  return __ffma2_rn(make_float2(s, s), x, y);
}
__device__ __forceinline__ double2 vfma(double s, double2 x, double2 y) {
  return make_double2(fma(s, x.x, y.x), fma(s, x.y, y.y));
}
__device__ __forceinline__ float2 vmul(float s, float2 x) { return __fmul2_rn(make_float2(s, s), x); }
__device__ __forceinline__ double2 vmul(double s, double2 x) { return make_double2(s * x.x, s * x.y); }
__device__ __forceinline__ float2 vadd(float2 x, float2 y) { return __fadd2_rn(x, y); }
__device__ __forceinline__ double2 vadd(double2 x, double2 y) { return make_double2(x.x + y.x, x.y + y.y); }

// The hardware's approximate FP32 reciprocal, square root, base-2 logarithm
// and power of two (PTX rcp/sqrt/lg2/ex2 .approx.ftz: a few ulp, subnormals
// flushed), for the step-size control of the mixed kernels, where a few ulp
// do not matter and the correctly rounded forms cost extra instructions.
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float sqrt_approx(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float lg2_approx(float x) {
  float r;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float ex2_approx(float x) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// s = fl(a + b) and e = (a + b) - s exactly (Knuth's TwoSum, six
// round-to-nearest additions that the compiler may neither fuse nor reorder).
__device__ __forceinline__ float two_sum(float a, float b, float &e) {
  const float s = __fadd_rn(a, b);
  const float bp = __fsub_rn(s, a);
  const float ap = __fsub_rn(s, bp);
  e = __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp));
  return s;
}
// The same for both components of a complex value with packed two-lane
// instructions (each difference u - v as the single rounding of -1 v + u).
__device__ __forceinline__ float2 two_sum(float2 a, float2 b, float2 &e) {
  const float2 m1 = make_float2(-1.f, -1.f);
  const float2 s = __fadd2_rn(a, b);
  const float2 bp = __ffma2_rn(m1, a, s);
  const float2 ap = __ffma2_rn(m1, bp, s);
  e = __fadd2_rn(__ffma2_rn(m1, ap, a), __ffma2_rn(m1, bp, b));
  return s;
}
__device__ __forceinline__ float tabs(float a) { return fabsf(a); }
__device__ __forceinline__ double tabs(double a) { return fabs(a); }
__device__ __forceinline__ float tmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double tmax(double a, double b) { return fmax(a, b); }

// acc += v * x (complex)
__device__ __forceinline__ void cmac(float2 &acc, float2 v, float2 x) {
  acc.x = fmaf(v.x, x.x, acc.x);
  acc.x = fmaf(-v.y, x.y, acc.x);
  acc.y = fmaf(v.x, x.y, acc.y);
  acc.y = fmaf(v.y, x.x, acc.y);
}
__device__ __forceinline__ void cmac(double2 &acc, double2 v, double2 x) {
  acc.x = fma(v.x, x.x, acc.x);
  acc.x = fma(-v.y, x.y, acc.x);
  acc.y = fma(v.x, x.y, acc.y);
  acc.y = fma(v.y, x.x, acc.y);
}

// A sum of complex products v x.  FP32: two packed halves, p = sum v.x x and
// r = sum v.y x (one two-lane multiply-add each per product, no operand
// shuffles), so that sum v x = (p.x - r.y, p.y + r.x).  FP64: cmac in the
// order above.
template <typename V> struct CAcc;
template <> struct CAcc<float2> {
  float2 p = {0.f, 0.f}, r = {0.f, 0.f};
  __device__ __forceinline__ void mac(float2 v, float2 x) {
    p = __ffma2_rn(make_float2(v.x, v.x), x, p);
    r = __ffma2_rn(make_float2(v.y, v.y), x, r);
  }
  __device__ __forceinline__ float2 get() const { return make_float2(p.x - r.y, p.y + r.x); }
};
template <> struct CAcc<double2> {
  double2 s = {0.0, 0.0};
  __device__ __forceinline__ void mac(double2 v, double2 x) { cmac(s, v, x); }
  __device__ __forceinline__ double2 get() const { return s; }
};

// ------------------------------------------------- Philox4x32-10 (Salmon et al.)
// Ten rounds of the Philox S-box: words 0 and 2 are multiplied by two odd
// 32-bit constants; the new words are (hi(w2*M1)^w1^k0, lo(w2*M1),
// hi(w0*M0)^w3^k1, lo(w0*M0)); the key advances by the golden-ratio and
// sqrt(3)-1 Weyl increments between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) { k.x += 0x9E3779B9u; k.y += 0xBB67AE85u; }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// Uniform in (0, 1) for jump k of trajectory traj: counter (traj, k, stream,
// 0), key = seed; 52 random bits m, U = (m + 1/2) 2^-52 (exact in FP64).
__device__ __forceinline__ double uniform52(uint64_t seed, uint64_t traj, uint64_t k,
                                            uint32_t stream) {
  uint4 x = philox4x32_10(make_uint4((uint32_t)traj, (uint32_t)k, stream, 0u),
                          make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
  double m = (double)(x.x >> 6) * 67108864.0 + (double)(x.y >> 6);
  return (m + 0.5) * (1.0 / 4503599627370496.0);
}

// ------------------------------------------- Dormand-Prince 5(4) coefficients
// Dormand & Prince (1980).  a_ij of the stages 2..7 (row 7 = 5th-order
// weights, first-same-as-last) and e_j = b5_j - b4_j for the error estimate.
struct DP {
  static constexpr double c2 = 1.0 / 5, c3 = 3.0 / 10, c4 = 4.0 / 5, c5 = 8.0 / 9;
  static constexpr double a21 = 1.0 / 5;
  static constexpr double a31 = 3.0 / 40, a32 = 9.0 / 40;
  static constexpr double a41 = 44.0 / 45, a42 = -56.0 / 15, a43 = 32.0 / 9;
  static constexpr double a51 = 19372.0 / 6561, a52 = -25360.0 / 2187, a53 = 64448.0 / 6561,
                          a54 = -212.0 / 729;
  static constexpr double a61 = 9017.0 / 3168, a62 = -355.0 / 33, a63 = 46732.0 / 5247,
                          a64 = 49.0 / 176, a65 = -5103.0 / 18656;
  static constexpr double b1 = 35.0 / 384, b3 = 500.0 / 1113, b4 = 125.0 / 192,
                          b5 = -2187.0 / 6784, b6 = 11.0 / 84;
  // embedded 4th-order weights
  static constexpr double d1 = 5179.0 / 57600, d3 = 7571.0 / 16695, d4 = 393.0 / 640,
                          d5 = -92097.0 / 339200, d6 = 187.0 / 2100, d7 = 1.0 / 40;
  static constexpr double e1 = b1 - d1, e3 = b3 - d3, e4 = b4 - d4, e5 = b5 - d5,
                          e6 = b6 - d6, e7 = 0.0 - d7;
};

// The coefficients in the arithmetic precision T of a kernel.  FP64: the
// values above.  FP32: each value rounded to FP32, except one coefficient per
// row, chosen so that the exact sum of the row's FP32 coefficients is the
// row's target again (a_ij summed over j = c_i, sum b_j = 1, sum e_j = 0).
// Rounding every coefficient separately leaves sum b_j = 1 + 3 2^-27: every
// step then advances the solution by h (1 + 2.2e-8), a drift of the solution
// against its time of 2.2e-8 t; rows 5 and 6 would miss c_5, c_6 by 2.3e-7
// and 2.7e-7.  Rows 2 to 4 round to within 1.2e-8 of c_i as they are.
template <typename T> struct DPW;
template <> struct DPW<double> : DP {};
// x rounded to FP32, as a double (exact)
__host__ __device__ constexpr double dp_r32(double x) { return (double)(float)x; }
template <> struct DPW<float> {
  static constexpr float a21 = (float)DP::a21;
  static constexpr float a31 = (float)DP::a31, a32 = (float)DP::a32;
  static constexpr float a41 = (float)DP::a41, a42 = (float)DP::a42, a43 = (float)DP::a43;
  static constexpr float a51 = (float)DP::a51, a52 = (float)DP::a52, a53 = (float)DP::a53,
                         a54 = (float)(DP::c5 - (dp_r32(DP::a51) + dp_r32(DP::a52) + dp_r32(DP::a53)));
  static constexpr float a61 = (float)DP::a61, a62 = (float)DP::a62, a63 = (float)DP::a63,
                         a64 = (float)DP::a64,
                         a65 = (float)(1.0 - (dp_r32(DP::a61) + dp_r32(DP::a62) + dp_r32(DP::a63) + dp_r32(DP::a64)));
  static constexpr float b3 = (float)DP::b3, b4 = (float)DP::b4, b5 = (float)DP::b5,
                         b6 = (float)DP::b6,
                         b1 = (float)(1.0 - (dp_r32(DP::b3) + dp_r32(DP::b4) + dp_r32(DP::b5) + dp_r32(DP::b6)));
  static constexpr float e1 = (float)DP::e1, e3 = (float)DP::e3, e4 = (float)DP::e4,
                         e5 = (float)DP::e5, e6 = (float)DP::e6,
                         e7 = (float)(-(dp_r32(DP::e1) + dp_r32(DP::e3) + dp_r32(DP::e4) + dp_r32(DP::e5) + dp_r32(DP::e6)));
};

// Step-size controller shared by both solvers (see qt.h): returns the next
// proposal after a step of length h with error norm err.
__device__ __forceinline__ double dp_control(double h, double err, bool accepted,
                                             bool after_reject, bool clipped, double hprop) {
  if (accepted) {
    double facmax = after_reject ? 1.0 : 5.0;
    double fac = (err == 0.0) ? facmax : fmin(facmax, fmax(0.2, 0.9 * pow(err, -0.2)));
    double hn = h * fac;
    if (clipped && hn < hprop) hn = hprop;
    return hn;
  }
  return h * fmax(0.2, 0.9 * pow(err, -0.2));
}

__device__ __forceinline__ double dp_hmin(double t, double tnext) {
  return 16.0 * 2.220446049250313e-16 * fmax(fabs(t), fabs(tnext));
}

// ------------------------------------------ time-dependent coefficients
// f(t) of one term (paper section 4.3, H(t) = H + sum_k f_k(t) H_k): linear
// between knots (kt[i], kv[i]), i = a0 .. b0, the end values outside.  The
// operation order (w = (t - t_i) / (t_i+1 - t_i), f = v_i + w (v_i+1 - v_i),
// each rounded separately) is the same in every solver, so that the FP64
// solvers see bit-identical coefficients.
__device__ __forceinline__ double td_piecewise(const double *kt, const double *kv, int64_t a0,
                                               int64_t b0, double t) {
  if (t <= kt[a0]) return kv[a0];
  if (t >= kt[b0]) return kv[b0];
  int64_t lo = a0, hi = b0;  // kt[lo] < t <= kt[hi]
  while (hi - lo > 1) {
    const int64_t mid = (lo + hi) >> 1;
    if (kt[mid] < t) lo = mid; else hi = mid;
  }
  const double w = __ddiv_rn(__dsub_rn(t, kt[lo]), __dsub_rn(kt[hi], kt[lo]));
  return __dadd_rn(kv[lo], __dmul_rn(w, __dsub_rn(kv[hi], kv[lo])));
}

// Stage time t + c h with the product and the sum rounded separately.
__device__ __forceinline__ double stage_time(double t, double c, double h) {
  return __dadd_rn(t, __dmul_rn(c, h));
}

// ------------------------------------------------------ warp-group helpers
// A group is G consecutive lanes of one warp (G = 8, 16 or 32).
template <int G> __device__ __forceinline__ unsigned group_mask() {
  if constexpr (G == 32) {
    return 0xffffffffu;
  } else {
    const unsigned lane = threadIdx.x & 31u;
    return ((1u << G) - 1u) << (lane / G * G);
  }
}

template <int G, typename X> __device__ __forceinline__ X group_sum(X v, unsigned mask) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o);
  return v;
}

// Record the first error code (0 = no error yet).
__device__ __forceinline__ void set_status(int *status, int code) {
  atomicCAS(status, 0, code);
}

}  // namespace qt
