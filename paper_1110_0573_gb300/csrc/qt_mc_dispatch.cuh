// qt_mc_dispatch.cuh -- which instance of the Monte-Carlo kernel of
// qt_mc_impl.cuh runs a given system: rows per lane and register-resident
// H_eff width from the dimension and the widest H_eff row.
#pragma once

#include "qt_mc_impl.cuh"

namespace qt {

namespace {

// Instances.  Warp groups: rows per lane R and register-resident H_eff width
// W (0 = read through the read-only cache).  CTA-wide groups (dimensions
// above 128): 256 or 512 threads with 4 rows each, H_eff read through the
// read-only cache (it stays L1/L2 resident and is shared by the CTAs of an
// SM).
// The instances are spread over three translation units per precision (warp
// groups here, time-dependent and CTA-wide ones in qt_mc_f*_td.cu and
// qt_mc_f*_wide.cu) and a fourth for the mixed dictionary instances
// (qt_mc_f32_dict.cu), so that they compile in parallel.

// Mixed precision, dimensions 129..1024 with a dictionary H_eff of at most
// 160 KB: two rows per thread and the operator in shared memory (no operator
// traffic from L2 in the right-hand sides).  These instances compile in a
// unit of their own (qt_mc_f32_dict.cu).
constexpr size_t kDictSmemMax = 160 * 1024;

inline bool use_dict(const McArgs &a) {
  return a.dict_code && a.ops.d > 128 && a.ops.d <= 1024 && a.n_td == 0 &&
         dict_bytes(a.dict_w, a.ops.d, a.dict_nv) <= kDictSmemMax;
}

template <typename T>
cudaError_t dispatch_dict(const McArgs &a, cudaStream_t s) {
  const int d = a.ops.d;
  if (a.dict_groups > 0) {  // entries grouped by value
    if (d <= 512) return launch_inst<T, 256, 2, -2, true>(a, s);
    return launch_inst<T, 512, 2, -2, true>(a, s);
  }
  if (d <= 512) return launch_inst<T, 256, 2, -1, true>(a, s);
  return launch_inst<T, 512, 2, -1, true>(a, s);
}

// Dimensions above 2048 (stages in global memory) and time-independent
// dimensions 129..2048 without a dictionary: CTA-wide groups.
template <typename T>
cudaError_t dispatch_wide(const McArgs &a, cudaStream_t s) {
  const int d = a.ops.d;
  if (d > 2048) return launch_inst<T, kBigG, kBigR, 0, true, false, true>(a, s);
  if (d > 1024) return launch_inst<T, 512, 4, 0, true>(a, s);
  return launch_inst<T, 256, 4, 0, true>(a, s);
}

// Time-dependent Hamiltonians (dimension <= 1024): H_eff in registers when
// its rows hold at most 4 entries, else read through the read-only cache.
template <typename T>
cudaError_t dispatch_td(const McArgs &a, int R, int W, cudaStream_t s) {
  if (a.ops.d > 128) return launch_inst<T, 256, 4, 0, true, true>(a, s);
  if (R == 1) {
    if (W == 4) return launch_inst<T, 32, 1, 4, false, true>(a, s);
    return launch_inst<T, 32, 1, 0, false, true>(a, s);
  }
  if (R == 2) {
    if (W == 3) return launch_inst<T, 32, 2, 3, false, true>(a, s);
    if (W == 4) return launch_inst<T, 32, 2, 4, false, true>(a, s);
    return launch_inst<T, 32, 2, 0, false, true>(a, s);
  }
  if (W == 4) return launch_inst<T, 32, 4, 4, false, true>(a, s);
  return launch_inst<T, 32, 4, 0, false, true>(a, s);
}

// Time-independent warp groups (dimension <= 128).
template <typename T>
cudaError_t dispatch_warp(const McArgs &a, int R, int W, cudaStream_t s) {
  if (R == 1) {
    if (W == 4) return launch_inst<T, 32, 1, 4, false>(a, s);
    if (W == 16) return launch_inst<T, 32, 1, 16, false>(a, s);
    return launch_inst<T, 32, 1, 0, false>(a, s);
  }
  if (R == 2) {
    if (W == 3) return launch_inst<T, 32, 2, 3, false>(a, s);
    if (W == 4) return launch_inst<T, 32, 2, 4, false>(a, s);
    if (W == 8) return launch_inst<T, 32, 2, 8, false>(a, s);
    return launch_inst<T, 32, 2, 0, false>(a, s);
  }
  if (W == 4) return launch_inst<T, 32, 4, 4, false>(a, s);
  return launch_inst<T, 32, 4, 0, false>(a, s);
}

// Which unit runs a system.
enum class McUnit { kWarp, kTd, kWide };
inline McUnit mc_unit(const McArgs &a) {
  if (a.ops.d > 2048) return McUnit::kWide;
  if (a.n_td > 0) return McUnit::kTd;
  return a.ops.d > 128 ? McUnit::kWide : McUnit::kWarp;
}

inline void choose(int d, int w, int &R, int &W) {
  R = d <= 32 ? 1 : (d <= 64 ? 2 : 4);
  if (R == 1) W = w <= 4 ? 4 : (w <= 16 ? 16 : 0);
  else if (R == 2) W = w <= 3 ? 3 : (w <= 4 ? 4 : (w <= 8 ? 8 : 0));
  else W = w <= 4 ? 4 : 0;
}

}  // namespace

}  // namespace qt
