// qt_mc_f32.cu -- mixed-precision warp-group instances of the Monte-Carlo
// kernel (complex FP32 state, FP64 norm decisions, weights and expectations)
// and the mixed launcher.
#include "qt_mc_dispatch.cuh"

namespace qt {

cudaError_t launch_mc_f32(const McArgs &a, cudaStream_t s) {
  int R, W;
  choose(a.ops.d, a.heff_w, R, W);
  switch (mc_unit(a)) {
    case McUnit::kWide: return use_dict(a) ? launch_mc_f32_dict(a, s) : launch_mc_f32_wide(a, s);
    case McUnit::kTd: return launch_mc_f32_td(a, R, W, s);
    default: return dispatch_warp<float>(a, R, W, s);
  }
}

}  // namespace qt
