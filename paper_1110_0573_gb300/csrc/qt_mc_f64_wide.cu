// qt_mc_f64_wide.cu -- FP64 CTA-wide instances of the Monte-Carlo kernel.
#include "qt_mc_dispatch.cuh"

namespace qt {

cudaError_t launch_mc_f64_wide(const McArgs &a, cudaStream_t s) { return dispatch_wide<double>(a, s); }

}  // namespace qt
