// qt_me_tc.cu -- the master equation (paper section 3.1, Eq. (master_equation))
// with its Hamiltonian products on the tensor cores.
//
// The right-hand side in effective-Hamiltonian form is
//   d rho/dt = -i (H_eff rho - rho H_eff^dag) + sum_n C_n rho C_n^dag.
// For a Hermitian state y, rho H_eff^dag = (H_eff y)^dag, so one product
// Y = H_eff y gives both Hamiltonian terms: -i (Y - Y^dag).  Y is computed as
// one real GEMM (layout in qt_internal.h, TcArgs) with BF16 operands split
// into hi + lo pieces and FP32 accumulation in tensor memory:
//   Y ~ A_hi B_hi^T + A_hi B_lo^T + A_lo B_hi^T
// (the dropped A_lo B_lo^T term and the rounding of lo are O(2^-17) relative
// to sum |A||B|).  Sparse collapse operators (one or two entries per row, as
// in the workloads) keep their terms C_n y C_n^dag on the ELL rows in the
// combine phase.  When one of them is at least kTcDenseCWidth wide, all their
// terms are dense products on the tensor cores too, as two more GEMMs of the
// same form (TcArgs): T = [C_1; ...; C_nc] y in the same tile loop as Y, then
// W = [T_1 ... T_nc] [C_1 ... C_nc]^dag = sum_n C_n y C_n^dag after a grid
// barrier, and the combine phase adds W.
//
// Everything runs in one cooperative launch with one CTA of 512 threads per
// SM, reusing the Hermitian-state Dormand-Prince solver of qt_me_herm.cuh
// with the product provider below:
//   store    writes a stage-input entry in FP32 and its BF16 hi/lo B entries;
//   publish  proxy fence + grid barrier (the B planes are read by TMA next);
//   prepare  the GEMM phase: each CTA computes 128 x 128 tiles of Y --
//            warp 0 issues TMA loads of A_hi, A_lo, B_hi, B_lo (64-wide K
//            blocks, 3-stage mbarrier pipeline), warp 1 issues tcgen05.mma
//            (M = 128, N = 128, K = 16, three products per K step) into a
//            TMEM accumulator, and all 16 warps move the accumulator to Y;
//            then a grid barrier.
// The combine phase of qt_me_herm.cuh then forms -i (Y_ij - conj(Y_ji)) +
// sum_n (C_n y C_n^dag)_ij on the upper triangle.
// Every wait on an mbarrier is bounded (1 s); a wait that runs out marks the
// CTA failed, the solver stops at its next error-norm reduction with
// QT_ETIMEOUT, in-flight copies are waited for (bounded) and TMEM is freed.
#include <cuda_bf16.h>

#include "qt_me_herm.cuh"
#include "qt_tc.cuh"

namespace qt {

namespace {

constexpr int kTcBlock = 512;
constexpr int kTcWarps = kTcBlock / 32;
constexpr int kTcStages = 3;
constexpr int kTcBM = 128, kTcBN = 128, kTcBK = 64;  // tile and K block (elements)
constexpr int kTcTileBytes = 128 * kTcBK * 2;         // one 128 x 64 BF16 tile
constexpr int kTcStageBytes = 4 * kTcTileBytes;       // A_hi, A_lo, B_hi, B_lo
constexpr uint32_t kTcCols = 128;                     // TMEM columns (FP32 accumulator)
constexpr uint64_t kTcWaitNs = 1000000000ull;         // bound of every mbarrier wait

struct TcCtl {
  uint64_t full[kTcStages];
  uint64_t empty[kTcStages];
  uint64_t accum;
  uint32_t tmem;
  int failed;
};

constexpr size_t kTcShBytes = sizeof(double) * kMePartialMax * (kTcWarps + 1);
constexpr size_t kTcSmemBytes = 1024 + (size_t)kTcStages * kTcStageBytes + sizeof(TcCtl) +
                                kTcShBytes + sizeof(double) * kMePartialMax;
static_assert(kTcSmemBytes <= 232448, "shared memory of the tensor-core kernel");
// the combine phase reuses the pipeline stages for its tiles and staged
// collapse operators (no copy is in flight then)
static_assert(herm_smem_bytes<float2>(kCSlotsMax, kCTermsMax) <= (size_t)kTcStages * kTcStageBytes,
              "combine-phase shared memory");

__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16 &hi, __nv_bfloat16 &lo) {
  hi = __float2bfloat16_rn(x);
  lo = __float2bfloat16_rn(x - __bfloat162float(hi));  // x - hi is exact in FP32
}

struct TcY {
  using V = float2;
  static constexpr bool kCanFail = true;
  static constexpr bool kFusedY = false;
  const TcArgs &t;
  uint8_t *stages;
  TcCtl *ctl;
  const int dp;
  // pipeline state: producer (warp 0, lane 0), MMA issuer (warp 1, lane 0),
  // accumulator phase (all threads)
  uint32_t ps = 0, pph = 0, cs = 0, cph = 0, aph = 0;
  uint32_t pending = 0, pending_par = 0;  // producer: stages with a load in flight, their parity

  __device__ TcY(const TcArgs &t_, uint8_t *stages_, TcCtl *ctl_)
      : t(t_), stages(stages_), ctl(ctl_), dp(t_.dp) {}

  __device__ __forceinline__ const V *product() const { return t.Y; }
  __device__ __forceinline__ int ystride() const { return dp; }
  // sum_n C_n y C_n^dag as a dense [dp][dp] array when the collapse
  // operators are dense (else null: the combine phase forms them sparsely)
  __device__ __forceinline__ const V *collapse_product() const { return t.nc ? t.W : nullptr; }

  __device__ __forceinline__ void store(V *buf, int idx, int i, int j, V v) {
    buf[idx] = v;
    __nv_bfloat16 hx, lx, hz, lz;
    split_bf16(v.x, hx, lx);
    split_bf16(v.y, hz, lz);
    const int64_t r0 = (int64_t)(2 * i) * (2 * dp) + 2 * j, r1 = r0 + 2 * dp;
    __nv_bfloat162 *bh = reinterpret_cast<__nv_bfloat162 *>(t.b_hi_ptr);
    __nv_bfloat162 *bl = reinterpret_cast<__nv_bfloat162 *>(t.b_lo_ptr);
    bh[r0 >> 1] = __halves2bfloat162(hx, hz);
    bh[r1 >> 1] = __halves2bfloat162(__hneg(hz), hx);
    bl[r0 >> 1] = __halves2bfloat162(lx, lz);
    bl[r1 >> 1] = __halves2bfloat162(__hneg(lz), lx);
  }

  __device__ __forceinline__ void publish(GridTeam &tm) {
    tc::fence_proxy_async_global();
    tm.sync();
  }

  __device__ __forceinline__ int failed() const { return *(volatile int *)&ctl->failed; }

  __device__ void fail() { *(volatile int *)&ctl->failed = 1; }

  // TMA producer of one tile: nk K blocks of A_hi, A_lo (rows m0..) and
  // B_hi, B_lo (rows n0..) from the given maps.
  __device__ void produce(const CUtensorMap *ah, const CUtensorMap *al, const CUtensorMap *bh,
                          const CUtensorMap *bl, int m0, int n0, int nk) {
    tc::fence_proxy_async_global();
    for (int kb = 0; kb < nk; ++kb) {
      if (!tc::mbar_wait(&ctl->empty[ps], pph ^ 1u, kTcWaitNs)) { fail(); return; }
      uint8_t *s = stages + ps * kTcStageBytes;
      uint64_t *bar = &ctl->full[ps];
      tc::mbar_arrive_expect_tx(bar, kTcStageBytes);
      const int x = kb * kTcBK;
      tc::tma_load_2d(s, ah, bar, x, m0);
      tc::tma_load_2d(s + kTcTileBytes, al, bar, x, m0);
      tc::tma_load_2d(s + 2 * kTcTileBytes, bh, bar, x, n0);
      tc::tma_load_2d(s + 3 * kTcTileBytes, bl, bar, x, n0);
      pending |= 1u << ps;
      pending_par = (pending_par & ~(1u << ps)) | (pph << ps);
      if (++ps == kTcStages) { ps = 0; pph ^= 1u; }
    }
  }

  // MMA issuer of one tile: three products per K step of 16.
  __device__ void issue(int nk) {
    constexpr uint32_t idesc = tc::idesc_bf16_f32(kTcBM, kTcBN);
    for (int kb = 0; kb < nk; ++kb) {
      if (!tc::mbar_wait(&ctl->full[cs], cph, kTcWaitNs)) { fail(); return; }
      tc::fence_after_sync();
      const uint32_t s = tc::smem_u32(stages + cs * kTcStageBytes);
#pragma unroll
      for (int kk = 0; kk < kTcBK / 16; ++kk) {
        const uint64_t ah = tc::sw128_desc(s + kk * 32);
        const uint64_t al = tc::sw128_desc(s + kTcTileBytes + kk * 32);
        const uint64_t bh = tc::sw128_desc(s + 2 * kTcTileBytes + kk * 32);
        const uint64_t bl = tc::sw128_desc(s + 3 * kTcTileBytes + kk * 32);
        tc::mma_bf16(ctl->tmem, ah, bh, idesc, (kb | kk) != 0);
        tc::mma_bf16(ctl->tmem, ah, bl, idesc, 1u);
        tc::mma_bf16(ctl->tmem, al, bh, idesc, 1u);
      }
      tc::mma_commit(&ctl->empty[cs]);  // frees the stage once these MMAs are done
      if (++cs == kTcStages) { cs = 0; cph ^= 1u; }
    }
    tc::mma_commit(&ctl->accum);
  }

  // One 128 x 128 tile of a GEMM: the pipeline for it, then the epilogue
  // moves the accumulator out of TMEM.  job 0: Y = H_eff y into Y; job 1:
  // rows m0.. of T = [C_1; ...] y into the T planes (BF16 hi/lo, row m of
  // C_n y at row m, columns of block n); job 2: W = T [C ...]^dag into W.
  __device__ void tile(int job, int m0, int n0, int nk) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool live = failed() == 0;  // uniform: changes only before the barrier below
    if (live) {
      if (warp == 0 && lane == 0) {
        if (job == 0) produce(&t.a_hi, &t.a_lo, &t.b_hi, &t.b_lo, m0, n0, nk);
        else if (job == 1) produce(&t.c_hi, &t.c_lo, &t.b_hi, &t.b_lo, m0, n0, nk);
        else produce(&t.t_hi, &t.t_lo, &t.cc_hi, &t.cc_lo, m0, n0, nk);
      } else if (warp == 1 && lane == 0) {
        issue(nk);
      }
    }
    bool ok = live && tc::mbar_wait(&ctl->accum, aph, kTcWaitNs);
    aph ^= 1u;
    __syncwarp();
    tc::fence_after_sync();
    ok = __all_sync(0xffffffffu, ok);
    if (ok) {
      // warp w reads TMEM lanes 32 (w % 4) .. +31 (tile rows), columns
      // 32 (w / 4) .. +31 (16 complex entries)
      const int q = warp & 3, cgrp = warp >> 2;
      uint32_t r[32];
      tc::tmem_ld_32cols(ctl->tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(32 * cgrp), r);
      const int row = m0 + 32 * q + lane;
      const int k0 = (n0 >> 1) + 16 * cgrp;  // first complex column
      if (job == 1) {
        const int n = row / dp, m = row - n * dp;
        const int64_t kc = 2 * (int64_t)t.nc * dp;
        __nv_bfloat162 *th = reinterpret_cast<__nv_bfloat162 *>(t.t_hi_ptr + (int64_t)m * kc) +
                             (int64_t)n * dp + k0;
        __nv_bfloat162 *tl = reinterpret_cast<__nv_bfloat162 *>(t.t_lo_ptr + (int64_t)m * kc) +
                             (int64_t)n * dp + k0;
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          __nv_bfloat16 hx, lx, hz, lz;
          split_bf16(__uint_as_float(r[2 * u]), hx, lx);
          split_bf16(__uint_as_float(r[2 * u + 1]), hz, lz);
          th[u] = __halves2bfloat162(hx, hz);
          tl[u] = __halves2bfloat162(lx, lz);
        }
      } else {
        float2 *out = job == 0 ? t.Y : t.W;
        float4 *dst = reinterpret_cast<float4 *>(out + (int64_t)row * dp + k0);
#pragma unroll
        for (int u = 0; u < 8; ++u)
          dst[u] = make_float4(__uint_as_float(r[4 * u]), __uint_as_float(r[4 * u + 1]),
                               __uint_as_float(r[4 * u + 2]), __uint_as_float(r[4 * u + 3]));
      }
    } else if (lane == 0) {
      fail();
    }
    tc::fence_before_sync();
    __syncthreads();  // the accumulator is free for the next tile
  }

  // The GEMM phase: Y = H_eff y for the y whose B planes were published last
  // and, with dense collapse operators, T = [C_1; ...] y in the same tile loop
  // and then W = sum_n C_n y C_n^dag.
  __device__ void prepare(GridTeam &team, const V *, double) {
    // the combine phase used the stage buffers through the generic proxy;
    // order that before the TMA writes and tensor-core reads below
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    const int n_m = dp / kTcBM, n_n = 2 * dp / kTcBN, nk = 2 * dp / kTcBK;
    const int n_y = n_m * n_n, n_t = t.nc * n_m * n_n;
    for (int u = blockIdx.x; u < n_y + n_t; u += gridDim.x) {
      const int job = u < n_y ? 0 : 1, v = u < n_y ? u : u - n_y;
      tile(job, (v / n_n) * kTcBM, (v % n_n) * kTcBN, nk);
    }
    if (t.nc) {
      // the T planes were written through the generic proxy and are read by
      // TMA in the next GEMM
      tc::fence_proxy_async_global();
      team.sync();
      const int nk2 = 2 * t.nc * dp / kTcBK;
      for (int v = blockIdx.x; v < n_y; v += gridDim.x)
        tile(2, (v / n_n) * kTcBM, (v % n_n) * kTcBN, nk2);
    }
    team.sync();
  }

  // Kernel exit: after a failure, wait (bounded) for the loads still in
  // flight and for the last MMAs before TMEM is released.
  __device__ void finish() {
    if (failed() == 0) return;
    if (threadIdx.x == 0) {
      for (int s = 0; s < kTcStages; ++s)
        if (pending & (1u << s))
          (void)tc::mbar_wait(&ctl->full[s], (pending_par >> s) & 1u, kTcWaitNs);
    }
    if (threadIdx.x == 32) {
      tc::mma_commit(&ctl->accum);
      (void)tc::mbar_wait(&ctl->accum, aph, kTcWaitNs);
    }
  }
};

__global__ void __launch_bounds__(kTcBlock, 1)
    me_tc_kernel(const __grid_constant__ MeArgs a, const __grid_constant__ TcArgs t) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *base = reinterpret_cast<uint8_t *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint8_t *stages = base;
  TcCtl *ctl = reinterpret_cast<TcCtl *>(base + (size_t)kTcStages * kTcStageBytes);
  double *sh = reinterpret_cast<double *>(ctl + 1);
  double *tot = sh + kMePartialMax * (kTcWarps + 1);
  const int warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kTcStages; ++s) {
      tc::mbar_init(&ctl->full[s], 1);
      tc::mbar_init(&ctl->empty[s], 1);
    }
    tc::mbar_init(&ctl->accum, 1);
    ctl->failed = 0;
    tc::fence_barrier_init();
    tc::tma_prefetch_map(&t.a_hi);
    tc::tma_prefetch_map(&t.a_lo);
    tc::tma_prefetch_map(&t.b_hi);
    tc::tma_prefetch_map(&t.b_lo);
  }
  if (warp == 0) tc::tmem_alloc(&ctl->tmem, kTcCols);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();

  GridTeam team(a.partial);
  TcY prod(t, stages, ctl);
  float2 *tiles = reinterpret_cast<float2 *>(stages);  // combine phase only
  bool herm = a.herm == 1;
  if (a.herm == 2) {
    const double2 *m = a.rhs_in ? a.rhs_in : a.state0;
    herm = (!a.rhs_in && a.state_is_ket) || herm_check(m, a.ops.d, team, sh, tot);
  }
  if (!herm) {
    if (team.tid == 0) set_status(a.status, QT_ENONHERM);
  } else if (a.rhs_in) {
    me_rhs_once_herm<float>(a, team, prod, a.ops.val32, tiles);
  } else {
    me_solve_herm<float>(a, team, prod, a.ops.val32, tiles, sh, tot);
  }
  prod.finish();

  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(ctl->tmem, kTcCols);
}

}  // namespace

int me_tc_grid() {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
  if (cudaFuncSetAttribute(me_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kTcSmemBytes) != cudaSuccess)
    return -1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, me_tc_kernel, kTcBlock,
                                                    kTcSmemBytes) != cudaSuccess)
    return -1;
  if (per_sm < 1) return -1;
  return sms;  // one CTA per SM (the shared-memory pipeline allows no more)
}

cudaError_t launch_me_tc(const MeArgs &a, const TcArgs &t, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(me_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kTcSmemBytes);
  if (e != cudaSuccess) return e;
  void *args[] = {const_cast<MeArgs *>(&a), const_cast<TcArgs *>(&t)};
  return cudaLaunchCooperativeKernel((const void *)me_tc_kernel, dim3(a.grid), dim3(kTcBlock),
                                     args, kTcSmemBytes, s);
}

}  // namespace qt
