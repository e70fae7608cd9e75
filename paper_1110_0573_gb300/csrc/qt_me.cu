// qt_me.cu -- the master-equation solver as one cooperative launch over the
// whole grid (the team of qt_me_impl.cuh is the grid).
#include "qt_me_impl.cuh"

namespace qt {

namespace {

template <typename T>
__global__ void __launch_bounds__(kMeBlock) me_kernel(const __grid_constant__ MeArgs a) {
  __shared__ double sh[kMePartialMax * 8 + kMePartialMax];
  __shared__ double tot[kMePartialMax];
  GridTeam team(a.partial);
  SparseRhs<T> rhs(a, sizeof(T) == 8 ? reinterpret_cast<const typename CT<T>::V *>(a.ops.val64)
                                     : reinterpret_cast<const typename CT<T>::V *>(a.ops.val32));
  if (a.rhs_in)
    me_rhs_once<T>(a, team, rhs, sh, tot);
  else
    me_solve<T>(a, team, rhs, sh, tot);
}

template <typename T>
int grid_for(int d) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, me_kernel<T>, kMeBlock, 0) !=
      cudaSuccess)
    return -1;
  if (per_sm < 1) return -1;
  const int64_t n = (int64_t)d * d;
  int64_t want = (n + kMeBlock - 1) / kMeBlock;
  int64_t cap = (int64_t)sms * per_sm;
  return (int)(want < cap ? want : cap);
}

}  // namespace

int me_grid(int d, int precision) {
  return precision == QT_MIXED ? grid_for<float>(d) : grid_for<double>(d);
}

size_t me_workspace_bytes(int d, int precision, int grid) {
  const size_t elem = precision == QT_MIXED ? sizeof(float2) : sizeof(double2);
  return 11 * (size_t)d * d * elem + (size_t)grid * kMePartialMax * sizeof(double) + 256;
}

cudaError_t launch_me(const MeArgs &a, int precision, cudaStream_t s) {
  void *args[] = {const_cast<MeArgs *>(&a)};
  if (precision == QT_MIXED)
    return cudaLaunchCooperativeKernel((const void *)me_kernel<float>, dim3(a.grid),
                                       dim3(kMeBlock), args, 0, s);
  return cudaLaunchCooperativeKernel((const void *)me_kernel<double>, dim3(a.grid),
                                     dim3(kMeBlock), args, 0, s);
}

}  // namespace qt
