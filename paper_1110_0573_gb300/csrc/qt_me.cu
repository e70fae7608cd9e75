// qt_me.cu -- the master-equation solver as one cooperative launch over the
// whole grid: the Hermitian-state solver of qt_me_herm.cuh with the sparse
// product on the CUDA cores, or the general solver of qt_me_impl.cuh (no
// symmetry assumed) for non-Hermitian initial matrices and on request.
#include "qt_me_herm.cuh"

namespace qt {

namespace {

template <typename T>
__global__ void __launch_bounds__(kMeBlock) me_kernel(const __grid_constant__ MeArgs a) {
  using V = typename CT<T>::V;
  extern __shared__ double2 dyn_smem[];  // tiles of the Hermitian combine phase
  __shared__ double sh[kMePartialMax * (kMeBlock / 32) + kMePartialMax];
  __shared__ double tot[kMePartialMax];
  __shared__ double tdcoef[kTdMax];
  GridTeam team(a.partial);
  const V *val = sizeof(T) == 8 ? reinterpret_cast<const V *>(a.ops.val64)
                                : reinterpret_cast<const V *>(a.ops.val32);
  bool herm = a.herm == 1;
  if (a.herm == 2) {
    const double2 *m = a.rhs_in ? a.rhs_in : a.state0;
    herm = (!a.rhs_in && a.state_is_ket) || herm_check(m, a.ops.d, team, sh, tot);
  }
  if (herm) {
    SpmmY<T> prod(a, val, tdcoef);
    V *tiles = reinterpret_cast<V *>(dyn_smem);
    if (a.rhs_in)
      me_rhs_once_herm<T>(a, team, prod, val, tiles);
    else
      me_solve_herm<T>(a, team, prod, val, tiles, sh, tot);
  } else {
    SparseRhs<T> rhs(a, val, tdcoef);
    if (a.rhs_in)
      me_rhs_once<T>(a, team, rhs, sh, tot);
    else
      me_solve<T>(a, team, rhs, sh, tot);
  }
}

// Small systems: the general solver on one CTA (team barriers are
// __syncthreads, no grid-wide synchronisation).
template <typename T>
__global__ void __launch_bounds__(kMeBlock) me_block_kernel(const __grid_constant__ MeArgs a) {
  using V = typename CT<T>::V;
  __shared__ double sh[kMePartialMax * (kMeBlock / 32) + kMePartialMax];
  __shared__ double tot[kMePartialMax];
  __shared__ double tdcoef[kTdMax];
  BlockTeam team;
  const V *val = sizeof(T) == 8 ? reinterpret_cast<const V *>(a.ops.val64)
                                : reinterpret_cast<const V *>(a.ops.val32);
  SparseRhs<T> rhs(a, val, tdcoef);
  if (a.rhs_in)
    me_rhs_once<T>(a, team, rhs, sh, tot);
  else
    me_solve<T>(a, team, rhs, sh, tot);
}

template <typename T>
size_t dyn_bytes(int n_cslots, int n_cterms) {
  return herm_smem_bytes<typename CT<T>::V>(n_cslots, n_cterms);
}

template <typename T>
int grid_for(int d, bool herm, int n_cslots, int n_cterms) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
  const size_t dyn = herm ? dyn_bytes<T>(n_cslots, n_cterms) : 0;
  if (cudaFuncSetAttribute(me_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn) !=
      cudaSuccess)
    return -1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, me_kernel<T>, kMeBlock, dyn) !=
      cudaSuccess)
    return -1;
  if (per_sm < 1) return -1;
  const int64_t n = (int64_t)d * d;
  const int64_t nt = (d + kHT - 1) / kHT;
  int64_t want = herm ? nt * (nt + 1) / 2 : (n + kMeBlock - 1) / kMeBlock;
  int64_t cap = (int64_t)sms * per_sm;
  return (int)(want < cap ? want : cap);
}

}  // namespace

int me_grid(int d, int precision) {
  return precision == QT_MIXED ? grid_for<float>(d, false, 0, 0) : grid_for<double>(d, false, 0, 0);
}

int me_herm_grid(int d, int precision, int n_cslots, int n_cterms) {
  return precision == QT_MIXED ? grid_for<float>(d, true, n_cslots, n_cterms)
                               : grid_for<double>(d, true, n_cslots, n_cterms);
}

size_t me_workspace_bytes(int d, int precision, int grid) {
  const size_t elem = precision == QT_MIXED ? sizeof(float2) : sizeof(double2);
  return 11 * (size_t)d * d * elem + (size_t)grid * kMePartialMax * sizeof(double) + 256;
}

template <typename T>
cudaError_t launch_me_t(const MeArgs &a, cudaStream_t s) {
  if (a.single_cta) {
    me_block_kernel<T><<<1, kMeBlock, 0, s>>>(a);
    return cudaGetLastError();
  }
  const size_t dyn = a.herm ? dyn_bytes<T>(a.n_cslots, a.n_cterms) : 0;
  cudaError_t e =
      cudaFuncSetAttribute(me_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
  if (e != cudaSuccess) return e;
  void *args[] = {const_cast<MeArgs *>(&a)};
  return cudaLaunchCooperativeKernel((const void *)me_kernel<T>, dim3(a.grid), dim3(kMeBlock),
                                     args, dyn, s);
}

cudaError_t launch_me(const MeArgs &a, int precision, cudaStream_t s) {
  return precision == QT_MIXED ? launch_me_t<float>(a, s) : launch_me_t<double>(a, s);
}

}  // namespace qt
