// qt_corr.cu -- two-time correlation functions <A(t + tau) B(t)> by the
// quantum regression theorem (the ODE form of the paper's correlation
// functions, section 5 function list): with rho(t_k) from one master-equation
// solve, X_k = B rho(t_k) is evolved over tau by the same Lindblad generator
// and C(t_k, tau_j) = Tr[A X_k(t_k + tau_j)].
//
// Small systems: one CTA per X_k (the general solver of qt_me_impl.cuh on a
// CTA team), X_k and the shifted output times formed by the CTA itself.
// Larger systems: corr_prepare_kernel forms one X_k and its times, and the
// cooperative solver of qt_me.cu evolves it.
//
// The same one-CTA-per-start-matrix scheme gives the propagator (the paper's
// propagator): every matrix unit evolved, its states scattered into the
// columns of U(t_k).
#include "qt_me_impl.cuh"

namespace qt {

namespace {

// X = B rho_k (FP64; B is table operator b_op in ELL rows) and the output
// times t_k + tau_j of the k-th evolution, by threads tid, tid + stride, ...
__device__ __forceinline__ void corr_prepare(const OpTable &ops, const CorrArgs &c, int k,
                                             double2 *X, double *times, int64_t tid,
                                             int64_t stride) {
  const int d = ops.d;
  const int64_t n = (int64_t)d * d;
  const double2 *rho = c.rho_t + (int64_t)k * n;
  const int w = ops.w[c.b_op];
  const int64_t off = ops.off[c.b_op];
  for (int64_t idx = tid; idx < n; idx += stride) {
    const int i = (int)(idx / d), j = (int)(idx - (int64_t)i * d);
    double2 acc = make_double2(0.0, 0.0);
    for (int s = 0; s < w; ++s) {
      const int64_t p = off + (int64_t)s * d + i;
      cmac(acc, ops.val64[p], rho[(int64_t)__ldg(ops.col + p) * d + j]);
    }
    X[idx] = acc;
  }
  const double tk = c.tlist[k];
  for (int64_t j = tid; j < c.n_tau; j += stride) times[j] = __dadd_rn(tk, c.taulist[j]);
}

__global__ void corr_prepare_kernel(const __grid_constant__ OpTable ops,
                                    const __grid_constant__ CorrArgs c, int k, double2 *X,
                                    double *times) {
  corr_prepare(ops, c, k, X, times, (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
               (int64_t)gridDim.x * blockDim.x);
}

// CTA b evolves X_k for k = b, b + grid, ...; its slab of a.work holds the
// solver workspace, X_k and the times.  a carries the tau evolution (n_t =
// n_tau, expect = the correlation array, general solver).
template <typename T>
__global__ void __launch_bounds__(kMeBlock) corr_block_kernel(const __grid_constant__ MeArgs a,
                                                              const __grid_constant__ CorrArgs c) {
  using V = typename CT<T>::V;
  __shared__ MeArgs m;
  __shared__ double sh[kMePartialMax * (kMeBlock / 32) + kMePartialMax];
  __shared__ double tot[kMePartialMax];
  __shared__ double tdcoef[kTdMax];
  const V *val = sizeof(T) == 8 ? reinterpret_cast<const V *>(a.ops.val64)
                                : reinterpret_cast<const V *>(a.ops.val32);
  char *slab = reinterpret_cast<char *>(a.work) + (size_t)blockIdx.x * c.ws_stride;
  double2 *X = reinterpret_cast<double2 *>(slab + c.x_off);
  double *times = reinterpret_cast<double *>(slab + c.times_off);
  for (int k = blockIdx.x; k < c.n_t; k += gridDim.x) {
    corr_prepare(a.ops, c, k, X, times, threadIdx.x, blockDim.x);
    if (threadIdx.x == 0) {
      m = a;
      m.state0 = X;
      m.tlist = times;
      m.expect = a.expect + (int64_t)k * a.n_t * a.n_e;
      m.work = slab;
    }
    __syncthreads();
    BlockTeam team;
    SparseRhs<T> rhs(m, val, tdcoef);
    me_solve<T>(m, team, rhs, sh, tot);
    __syncthreads();  // m, X and times are rewritten for the next k
  }
}

// The propagator: CTA b evolves the matrix units E_k (k = a d + b') for
// k = b, b + grid, ... from tlist[0] by the general solver and scatters each
// output state rho_k(t_m) into column k of U(t_m): U[m][ij][k].
template <typename T>
__global__ void __launch_bounds__(kMeBlock) prop_block_kernel(const __grid_constant__ MeArgs a,
                                                              const __grid_constant__ PropArgs p) {
  using V = typename CT<T>::V;
  __shared__ MeArgs m;
  __shared__ double sh[kMePartialMax * (kMeBlock / 32) + kMePartialMax];
  __shared__ double tot[kMePartialMax];
  __shared__ double tdcoef[kTdMax];
  const V *val = sizeof(T) == 8 ? reinterpret_cast<const V *>(a.ops.val64)
                                : reinterpret_cast<const V *>(a.ops.val32);
  const int64_t n = (int64_t)a.ops.d * a.ops.d;
  char *slab = reinterpret_cast<char *>(a.work) + (size_t)blockIdx.x * p.ws_stride;
  double2 *X = reinterpret_cast<double2 *>(slab + p.x_off);
  double2 *st = reinterpret_cast<double2 *>(slab + p.st_off);
  for (int64_t k = blockIdx.x; k < n; k += gridDim.x) {
    for (int64_t idx = threadIdx.x; idx < n; idx += blockDim.x)
      X[idx] = make_double2(idx == k ? 1.0 : 0.0, 0.0);
    if (threadIdx.x == 0) {
      m = a;
      m.state0 = X;
      m.states = st;
      m.work = slab;
    }
    __syncthreads();
    BlockTeam team;
    SparseRhs<T> rhs(m, val, tdcoef);
    me_solve<T>(m, team, rhs, sh, tot);
    __syncthreads();
    for (int t = 0; t < a.n_t; ++t)
      for (int64_t idx = threadIdx.x; idx < n; idx += blockDim.x)
        p.U[((int64_t)t * n + idx) * n + k] = st[(int64_t)t * n + idx];
    __syncthreads();  // m, X and st are rewritten for the next k
  }
}

template <typename T>
int prop_grid_t(int64_t units) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, prop_block_kernel<T>, kMeBlock, 0) !=
      cudaSuccess)
    return -1;
  if (per_sm < 1) return -1;
  const int64_t cap = (int64_t)sms * per_sm;
  return (int)(units < cap ? units : cap);
}

template <typename T>
int corr_grid_t(int n_t) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, corr_block_kernel<T>, kMeBlock, 0) !=
      cudaSuccess)
    return -1;
  if (per_sm < 1) return -1;
  const int cap = sms * per_sm;
  return n_t < cap ? n_t : cap;
}

}  // namespace

int corr_block_grid(int n_t, int precision) {
  return precision == QT_MIXED ? corr_grid_t<float>(n_t) : corr_grid_t<double>(n_t);
}

cudaError_t launch_corr_block(const MeArgs &a, const CorrArgs &c, int grid, int precision,
                              cudaStream_t s) {
  if (precision == QT_MIXED)
    corr_block_kernel<float><<<grid, kMeBlock, 0, s>>>(a, c);
  else
    corr_block_kernel<double><<<grid, kMeBlock, 0, s>>>(a, c);
  return cudaGetLastError();
}

int prop_block_grid(int64_t units, int precision) {
  return precision == QT_MIXED ? prop_grid_t<float>(units) : prop_grid_t<double>(units);
}

cudaError_t launch_prop_block(const MeArgs &a, const PropArgs &p, int grid, int precision,
                              cudaStream_t s) {
  if (precision == QT_MIXED)
    prop_block_kernel<float><<<grid, kMeBlock, 0, s>>>(a, p);
  else
    prop_block_kernel<double><<<grid, kMeBlock, 0, s>>>(a, p);
  return cudaGetLastError();
}

cudaError_t launch_corr_prepare(const OpTable &ops, const CorrArgs &c, int k, double2 *X,
                                double *times, cudaStream_t s) {
  const int64_t n = (int64_t)ops.d * ops.d;
  const int64_t blocks = (n + 255) / 256;
  corr_prepare_kernel<<<(unsigned)(blocks < 2048 ? blocks : 2048), 256, 0, s>>>(ops, c, k, X,
                                                                              times);
  return cudaGetLastError();
}

}  // namespace qt
