// qt_mc_f64_td.cu -- FP64 time-dependent instances of the Monte-Carlo kernel.
#include "qt_mc_dispatch.cuh"

namespace qt {

cudaError_t launch_mc_f64_td(const McArgs &a, int R, int W, cudaStream_t s) { return dispatch_td<double>(a, R, W, s); }

}  // namespace qt
