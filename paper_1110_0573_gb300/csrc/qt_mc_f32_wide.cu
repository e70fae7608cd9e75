// qt_mc_f32_wide.cu -- mixed-precision CTA-wide instances of the Monte-Carlo kernel.
#include "qt_mc_dispatch.cuh"

namespace qt {

cudaError_t launch_mc_f32_wide(const McArgs &a, cudaStream_t s) { return dispatch_wide<float>(a, s); }

}  // namespace qt
