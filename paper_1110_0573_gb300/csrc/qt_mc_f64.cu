// qt_mc_f64.cu -- FP64 warp-group instances of the Monte-Carlo kernel and the
// launchers.
#include "qt_mc_dispatch.cuh"

namespace qt {

cudaError_t launch_mc_f64(const McArgs &a, cudaStream_t s) {
  int R, W;
  choose(a.ops.d, a.heff_w, R, W);
  switch (mc_unit(a)) {
    case McUnit::kWide: return launch_mc_f64_wide(a, s);
    case McUnit::kTd: return launch_mc_f64_td(a, R, W, s);
    default: return dispatch_warp<double>(a, R, W, s);
  }
}

int mc_supported(int d, int w_heff, int precision, int group) {
  (void)w_heff;
  (void)precision;
  if (group != 0 && group != 32) return 0;
  return d >= 1 && d <= kBigG * kBigR;
}

size_t mc_stage_slab_bytes(int precision) {
  return (size_t)7 * kBigG * kBigR * (precision == QT_MIXED ? sizeof(float2) : sizeof(double2));
}

int mc_stage_ctas() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
  return sms;  // one CTA of kBigG threads per SM
}

cudaError_t launch_mc(const McArgs &a, int precision, int group, cudaStream_t s) {
  (void)group;
  return precision == QT_MIXED ? launch_mc_f32(a, s) : launch_mc_f64(a, s);
}

}  // namespace qt
