// qt_batch.cu -- many independent problems of uneven dimension in one
// persistent launch.
//
// Persistent CTAs of 256 threads take work items from a device counter, in
// the order the host sorted them (largest estimated cost first):
//   * a master-equation item (paper section 3.1) is solved by the whole CTA
//     with the team-generic solver of qt_me_impl.cuh (the team is the CTA;
//     its Dormand-Prince buffers live in the CTA's slice of the workspace);
//   * a Monte-Carlo item (paper section 3.2) is a block of trajectories of
//     one problem; the CTA's eight warps take its trajectories one at a time
//     and integrate them with the warp-group trajectory code of
//     qt_mc_impl.cuh.
// Nothing is allocated at solve time, so the launch can be captured in a
// CUDA graph.
#include "qt_mc_impl.cuh"
#include "qt_me_impl.cuh"

namespace qt {

namespace {

constexpr int kBatchWarps = kBatchBlock / 32;

template <typename T>
struct BatchShared {
  double sh[kMePartialMax * 8 + kMePartialMax];
  double tot[kMePartialMax];
  MeArgs me;
  McArgs mc[kBatchWarps];
  GroupScalars gs[kBatchWarps][2];  // one per trajectory group (half-warps when G = 16)
  typename CT<T>::V ybuf[kBatchWarps][128];  // per group two copies (Traj::publish)
  // mixed precision: the FP32 remainders of each warp's H_eff (64 rows x 4)
  typename CT<T>::V hlo[kBatchWarps][sizeof(T) == 4 ? 64 * 4 : 1];
  // mixed precision: each warp's two buffers of lo psi (64 rows each)
  typename CT<T>::V lpb[kBatchWarps][sizeof(T) == 4 ? 2 * 64 : 1];
  unsigned long long item;
};

// Integrates the trajectories of one Monte-Carlo item on this warp: groups
// of G lanes (the whole warp, or its two halves for small dimensions), each
// group one trajectory at a time with R rows per lane.
template <typename T, int G, int R, int W>
__device__ void batch_mc_warp(const BatchArgs &a, const BatchProblem &P, const McArgs &m,
                              unsigned long long it, int64_t n, BatchShared<T> &sm, int warp,
                              int lane) {
  using V = typename CT<T>::V;
  static_assert(G == 32 || G == 16, "trajectory groups of 32 or 16 lanes");
  static_assert(G * R <= 64, "state buffer of 64 rows per warp");
  const int grp = lane / G, glane = lane % G;
  const unsigned mask = group_mask<G>();
  const V *val = sizeof(T) == 8 ? reinterpret_cast<const V *>(P.ops.val64)
                                : reinterpret_cast<const V *>(P.ops.val32);
  V *hlo = nullptr;
  if constexpr (sizeof(T) == 4 && W > 0) {
    static_assert(G * R * W <= 64 * 4, "remainder buffer too small");
    hlo = sm.hlo[warp];  // rows 0 .. G R - 1, shared by the warp's groups
    const V *vlo = reinterpret_cast<const V *>(P.ops.val32lo);
    const int d = P.ops.d, wh = P.ops.w[0];
    const int64_t off0 = P.ops.off[0];
    for (int i = lane; i < G * R * W; i += 32) {
      const int r = i / W;
      // the register slot order of Traj: own-column slot first
      const int sl = heff_swapped_slot(
          i - r * W, r < d ? heff_own_slot(P.ops.col, off0, d, wh, r, W) : -1);
      hlo[i] = (r < d && sl < wh) ? vlo[off0 + (int64_t)sl * d + r] : cmake<V>(0.0, 0.0);
    }
    __syncwarp();
  }
  Traj<T, G, R, W, false, false, false> tr(
      m, glane, mask, sm.ybuf[warp] + grp * (2 * G * R), val, val, P.ops.col, P.ops.w, P.opoff32,
      &sm.gs[warp][grp], hlo,
      sizeof(T) == 4 ? sm.lpb[warp] + grp * (2 * G * R) + glane : nullptr);
  for (;;) {
    unsigned long long j = 0;
    if (glane == 0) {
      j = atomicAdd(a.item_work + it, 1ULL);
      if (*(volatile int *)a.status != 0) j = (unsigned long long)n;
    }
    j = __shfl_sync(mask, j, grp * G);
    if ((int64_t)j >= n) break;
    const bool ok = tr.run((int64_t)j);
    tr.flush_stats();
    if (!ok) break;
  }
}

template <typename T>
__global__ void __launch_bounds__(kBatchBlock, (sizeof(T) == 4 ? 2 : 1)) batch_kernel(const __grid_constant__ BatchArgs a) {
  __shared__ BatchShared<T> sm;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (;;) {
    if (threadIdx.x == 0) {
      unsigned long long it = atomicAdd(a.next_item, 1ULL);
      if (*(volatile int *)a.status != 0) it = (unsigned long long)a.n_items;
      sm.item = it;
    }
    __syncthreads();
    const unsigned long long it = sm.item;
    __syncthreads();
    if (it >= (unsigned long long)a.n_items) break;
    const BatchItem item = a.items[it];
    const BatchProblem &P = a.probs[item.problem];
    const int64_t out_off = P.expect_off * (int64_t)a.n_t;
    if (P.kind == QT_KIND_ME) {
      if (threadIdx.x == 0) {
        MeArgs &m = sm.me;
        m.ops = P.ops;
        m.n_c = P.n_c;
        m.n_e = P.n_e;
        m.n_t = a.n_t;
        m.grid = 1;
        m.tlist = a.tlist;
        m.rtol = a.rtol;
        m.atol = a.atol;
        m.h0 = a.h0;
        m.max_steps = a.max_steps;
        m.expect = a.expect + out_off;
        m.states = nullptr;
        m.counters = a.prob_counters + 6 * (int64_t)item.problem;
        m.status = a.status;
        m.state0 = P.state0;
        m.state_is_ket = P.state_is_ket;
        m.work = reinterpret_cast<char *>(a.ws) + (size_t)blockIdx.x * a.ws_stride;
        m.partial = nullptr;
        m.rhs_in = nullptr;
        m.rhs_out = nullptr;
        m.n_td = 0;
      }
      __syncthreads();
      BlockTeam team;
      SparseRhs<T> rhs(sm.me, sizeof(T) == 8
                                  ? reinterpret_cast<const typename CT<T>::V *>(sm.me.ops.val64)
                                  : reinterpret_cast<const typename CT<T>::V *>(sm.me.ops.val32));
      me_solve<T>(sm.me, team, rhs, sm.sh, sm.tot);
      __syncthreads();
    } else {
      if (lane == 0) {
        McArgs &m = sm.mc[warp];
        m.ops = P.ops;
        m.heff_w = 0;
        m.stage_aux = 0;
        m.aux_begin = 0;
        m.aux_slots = 0;
        m.n_c = P.n_c;
        m.n_e = P.n_e;
        m.n_t = a.n_t;
        m.psi0 = P.state0;
        m.tlist = a.tlist;
        m.traj_begin = item.traj_begin;
        m.ntraj = item.ntraj;
        m.seed = P.seed;
        m.rtol = a.rtol;
        m.atol = a.atol;
        m.h0 = a.h0;
        m.bisect_tol = a.bisect_tol;
        m.max_steps = a.max_steps;
        m.expect_sum = a.expect + out_off;
        m.traj_expect = nullptr;
        m.jumps = nullptr;
        m.jump_cap = 0;
        m.n_jumps = a.n_jumps;
        m.counters = a.prob_counters + 6 * (int64_t)item.problem;
        m.status = a.status;
        m.work = nullptr;
        m.n_td = 0;
        m.ivl_tb = nullptr;  // the kernel forms the output intervals itself
        m.ivl_len = nullptr;
      }
      __syncwarp();
      // lanes per trajectory and rows per lane by dimension: half-warp
      // groups for dimensions up to a.small_group_dim (chosen by the tuner),
      // else whole warps with one row per lane up to 32, two above
      const int wh = P.ops.w[0], d = P.ops.d;
      if (wh <= 4) {
        if (d <= a.small_group_dim && d <= 16)
          batch_mc_warp<T, 16, 1, 4>(a, P, sm.mc[warp], it, item.ntraj, sm, warp, lane);
        else if (d <= a.small_group_dim)
          batch_mc_warp<T, 16, 2, 4>(a, P, sm.mc[warp], it, item.ntraj, sm, warp, lane);
        else if (d <= 32)
          batch_mc_warp<T, 32, 1, 4>(a, P, sm.mc[warp], it, item.ntraj, sm, warp, lane);
        else
          batch_mc_warp<T, 32, 2, 4>(a, P, sm.mc[warp], it, item.ntraj, sm, warp, lane);
      } else {
        batch_mc_warp<T, 32, 2, 0>(a, P, sm.mc[warp], it, item.ntraj, sm, warp, lane);
      }
      __syncthreads();
    }
  }
}

// Monte-Carlo outputs: sums -> means; per-problem statistics summed into the
// batch's counters.
__global__ void batch_finalize_kernel(const __grid_constant__ BatchArgs a) {
  for (int p = blockIdx.x; p < a.n_problems; p += gridDim.x) {
    if (threadIdx.x < 6) atomicAdd(a.counters + threadIdx.x, a.prob_counters[6 * (int64_t)p + threadIdx.x]);
    const BatchProblem &P = a.probs[p];
    if (P.kind != QT_KIND_MC || P.ntraj <= 0) continue;
    const double inv = 1.0 / (double)P.ntraj;
    double2 *e = a.expect + P.expect_off * (int64_t)a.n_t;
    for (int i = threadIdx.x; i < a.n_t * P.n_e; i += blockDim.x) {
      e[i].x *= inv;
      e[i].y *= inv;
    }
  }
}

template <typename T>
int grid_for_batch() {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel<T>, kBatchBlock, 0) !=
      cudaSuccess)
    return -1;
  if (per_sm < 1) return -1;
  return sms * per_sm;
}

}  // namespace

int batch_grid(int precision) {
  return precision == QT_MIXED ? grid_for_batch<float>() : grid_for_batch<double>();
}

size_t batch_ws_stride(int dmax, int precision) {
  const size_t elem = precision == QT_MIXED ? sizeof(float2) : sizeof(double2);
  return ((11 * (size_t)dmax * dmax * elem + 255) / 256) * 256;
}

cudaError_t launch_batch(const BatchArgs &a, int precision, int grid, cudaStream_t s) {
  if (precision == QT_MIXED)
    batch_kernel<float><<<grid, kBatchBlock, 0, s>>>(a);
  else
    batch_kernel<double><<<grid, kBatchBlock, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_batch_finalize(const BatchArgs &a, cudaStream_t s) {
  const int grid = a.n_problems < 1024 ? (a.n_problems > 0 ? a.n_problems : 1) : 1024;
  batch_finalize_kernel<<<grid, 128, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace qt
