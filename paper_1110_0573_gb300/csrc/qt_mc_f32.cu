// qt_mc_f32.cu -- mixed-precision instances of the Monte-Carlo kernel
// (complex FP32 state, FP64 norm decisions, weights and expectations).
#include "qt_mc_dispatch.cuh"

namespace qt {

cudaError_t launch_mc_f32(const McArgs &a, cudaStream_t s) {
  int R, W;
  choose(a.ops.d, a.heff_w, R, W);
  return dispatch<float>(a, R, W, s);
}

}  // namespace qt
