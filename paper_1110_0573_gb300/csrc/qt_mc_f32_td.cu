// qt_mc_f32_td.cu -- mixed-precision time-dependent instances of the Monte-Carlo kernel.
#include "qt_mc_dispatch.cuh"

namespace qt {

cudaError_t launch_mc_f32_td(const McArgs &a, int R, int W, cudaStream_t s) { return dispatch_td<float>(a, R, W, s); }

}  // namespace qt
