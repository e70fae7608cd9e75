// qt_mc_f32_dict.cu -- mixed-precision CTA-wide instances of the Monte-Carlo
// kernel with H_eff as a dictionary in shared memory (plain codes, or entries
// grouped by value).
#include "qt_mc_dispatch.cuh"

namespace qt {

cudaError_t launch_mc_f32_dict(const McArgs &a, cudaStream_t s) { return dispatch_dict<float>(a, s); }

}  // namespace qt
