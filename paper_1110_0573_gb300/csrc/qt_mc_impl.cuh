// qt_mc_impl.cuh -- persistent Monte-Carlo wave-function kernel (paper
// section 3.2), instantiated per precision by qt_mc_f64.cu and qt_mc_f32.cu.
//
// One group of G threads integrates one trajectory at a time and then takes
// the next trajectory index from a device counter, until the range is
// exhausted.  A group is one warp (G = 32, dimensions up to 128) or a whole
// CTA (template BLK, G = 256 or 512 threads, dimensions up to 2048; the group
// barrier is then __syncthreads and the reductions go through shared memory).  Lane l of a group owns rows l, l + G, ..., l + (R-1) G
// of the state: every Dormand-Prince stage vector of the trajectory lives in
// that lane's registers for the whole run, so a trajectory never leaves the
// chip.  H_eff = H - (i/2) sum_n C_n^dag C_n (Eq. (heff)) is applied as an
// ELLPACK product: each lane keeps the stored entries of its own rows in
// registers (template W > 0) or reads them through the read-only cache
// (W == 0), and gathers the needed state components from a per-group copy of
// the vector in shared memory.  The collapse and observable operators are
// staged in shared memory once per CTA when they fit.
//
// Per trajectory the kernel runs steps I-IV of the paper's algorithm:
//   I    r = U(seed, j, k, 0);
//   II   adaptive Dormand-Prince steps of d psi/dt = -i H_eff psi; after each
//        accepted step <psi|psi> is compared with r; at a crossing the jump
//        time is located on trial steps of length (tau - t) from the
//        accepted state (t, psi);
//   III  p_n = ||C_n psi(tau)||^2 (Eq. (pcn)), r2 = U(seed, j, k, 1), the
//        smallest n with sum_{i<=n} p_i >= r2 sum_i p_i (Eq. (mc3)),
//        psi <- C_n psi / sqrt(p_n) (Eq. (project));
//   IV   k <- k + 1, new r, continue from tau.
// At each output time the normalised expectations <psi|O_m|psi>/<psi|psi>
// are added in FP64 to the sums over trajectories.
//
// Precision: T = double runs everything in FP64 and follows the oracle's
// order of operations.  T = float keeps the state, the stages and the step
// control in FP32 and uses FP64 for the absolute times, the jump-time
// search, the norm-decay comparison (an FP32 sum decides only when it is
// provably on the same side of r as the FP64 sum of the same values), the
// collapse weights, the renormalisation factor and the sums over
// trajectories.
#pragma once

#include <type_traits>

#include "qt_device.cuh"
#include "qt_internal.h"

namespace qt {

namespace {

constexpr int kBlock = 128;
// dimensions 2049 .. kBigG * kBigR: one CTA of kBigG threads per trajectory,
// kBigR rows per thread, the stage vectors in global memory
constexpr int kBigG = 512, kBigR = 10;

// The linear piece of a time-dependent coefficient around tb + s, looked up
// in FP64 (paper section 4.3, H(t) = H + sum_k f_k(t) H_k with f_k piecewise
// linear between the knots kt[a0..b0], constant outside): {f at offset 0,
// slope, first offset, last offset} relative to tb, and f at offset s.  Out
// of line: it is the slow path of every stage's coefficient, and a copy
// inlined into each stage of each step made the time-dependent kernels
// overflow the instruction cache.
template <typename T>
struct TdPiece {
  T f0, slope, lo, hi, f;
};

template <typename T>
__device__ __noinline__ TdPiece<T> td_lookup_piece(const double *kt, const double *kv, int64_t a0,
                                                   int64_t b0, double tb, T s) {
  const double t = tb + (double)s;
  double f0, slope, lo, hi;
  if (t <= kt[a0]) {
    f0 = kv[a0]; slope = 0.0; lo = -1e300; hi = kt[a0] - tb;
  } else if (t >= kt[b0]) {
    f0 = kv[b0]; slope = 0.0; lo = kt[b0] - tb; hi = 1e300;
  } else {
    int64_t lo_i = a0, hi_i = b0;  // kt[lo_i] < t < kt[hi_i]
    while (hi_i - lo_i > 1) {
      const int64_t mid = (lo_i + hi_i) >> 1;
      if (kt[mid] < t) lo_i = mid; else hi_i = mid;
    }
    slope = (kv[hi_i] - kv[lo_i]) / (kt[hi_i] - kt[lo_i]);
    f0 = kv[lo_i] + slope * (tb - kt[lo_i]);
    lo = kt[lo_i] - tb;
    hi = kt[hi_i] - tb;
  }
  TdPiece<T> p;
  p.f0 = (T)f0;
  p.slope = (T)slope;
  p.lo = (T)fmax(lo, -3e38);
  p.hi = (T)fmin(hi, 3e38);
  p.f = (T)(f0 + slope * (double)s);
  return p;
}

// FP64 scalars of one group's current trajectory.
struct GroupScalars {
  double r;                 // pending jump threshold
  double tb;                // base of the time offsets
  unsigned long long next;  // trajectory index handed to a CTA-wide group
  double red[16];           // CTA-wide reduction slots (one per warp)
  // time-dependent terms: the linear piece of f_k in use, as
  // {f at offset 0, slope, first offset, last offset} relative to tb
  double tdd[kTdMax][4];
  float tdf[kTdMax][4];
};

// Shared-memory layout of one CTA (host and device agree on it).
struct McSmem {
  size_t ybuf;   // per-group state copies
  size_t gscal;  // GroupScalars per group
  size_t opw;    // int  w[n_ops]
  size_t opoff;  // int  off[n_ops] relative to the staged block
  size_t val;    // V    staged values of operators 1..n_ops-1
  size_t col;    // int  staged columns
  size_t hlo;    // V    FP32 remainders of this lane's H_eff entries, [row][W]
  size_t lpb;    // V    per group two buffers of lo psi (mixed), [2][R][G]
  size_t dict;   //      dictionary H_eff: codes, diagonal [2][d], table [2][nv]
  size_t redv;   // T    CTA-wide groups: per-warp partial sums of the outputs [16][16]
  size_t total;
};

// Bytes of a dictionary H_eff staged in shared memory (McArgs::dict_*), and
// the offsets of its diagonal and table within them.
__host__ __device__ inline size_t dict_code_bytes(int w, int d) {
  return ((size_t)w * d * sizeof(uint32_t) + 15) / 16 * 16;
}
__host__ __device__ inline size_t dict_bytes(int w, int d, int nv) {
  return dict_code_bytes(w, d) + 2 * (size_t)d * sizeof(float2) + 2 * (size_t)nv * sizeof(float2);
}

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) / 16 * 16; }

template <typename V>
__host__ __device__ inline McSmem mc_smem_layout(int groups, int G, int R, int n_ops,
                                                 int64_t aux_slots, bool staged,
                                                 int hlo_slots = 0, size_t dict_b = 0) {
  McSmem l;
  l.ybuf = 0;
  // warp groups: two copies per group, [group][copy][G R]; a CTA-wide group:
  // one, and one zero entry past it (row G R), the padding column of a
  // grouped dictionary H_eff
  size_t p = align16(((size_t)groups * G * R * (groups == 1 ? 1 : 2) + (groups == 1 ? 1 : 0)) *
                     sizeof(V));
  l.gscal = p;
  p = align16(p + (size_t)groups * sizeof(GroupScalars));
  l.opw = p;
  p = align16(p + (size_t)n_ops * sizeof(int));
  l.opoff = p;
  p = align16(p + (size_t)n_ops * sizeof(int));
  l.val = p;
  if (staged) p = align16(p + (size_t)aux_slots * sizeof(V));
  l.col = p;
  if (staged) p = align16(p + (size_t)aux_slots * sizeof(int));
  l.hlo = p;
  p = align16(p + (size_t)hlo_slots * sizeof(V));
  l.lpb = p;
  if (sizeof(V) == 8) p = align16(p + (size_t)groups * 2 * G * R * sizeof(V));
  l.dict = p;
  p = align16(p + dict_b);
  l.redv = p;
  if (groups == 1) p = align16(p + 16 * 16 * sizeof(double));
  l.total = p;
  return l;
}

// Storage of the seven Dormand-Prince stage vectors of a trajectory: this
// lane's rows in registers, or (dimensions above 2048, where they do not
// fit) in a per-CTA slab of global memory that stays L2-resident, stage j of
// row lane + q G at base[j * stride + lane + q G].
template <typename V, int R>
struct RegStages {
  V k[7][R];
  __device__ __forceinline__ V (&operator[](int j))[R] { return k[j]; }
};

template <typename V, int G>
struct GlobalRow {
  V *p;
  __device__ __forceinline__ V &operator[](int q) const { return p[q * G]; }
};

template <typename V, int G>
struct GlobalStages {
  V *base;
  int stride;
  __device__ __forceinline__ GlobalRow<V, G> operator[](int j) const {
    return GlobalRow<V, G>{base + (int64_t)j * stride};
  }
};

// Mixed register instances (W > 0): slot 0 of each row of H_eff is made its
// own-column slot, so that the right-hand side takes that product from the
// thread's own state entry instead of the shared copy.  The host gives every
// row of H_eff such a slot (the diagonal entry, or a zero padding entry).
// heff_own_slot: the first of the nw register slots of row r whose column is
// r (slots at or beyond the ELL width w hold column 0), or -1.
__device__ __forceinline__ int heff_own_slot(const int *col, int64_t off0, int d, int w, int r,
                                             int nw) {
  for (int s = 0; s < nw; ++s) {
    const int c = s < w ? col[off0 + (int64_t)s * d + r] : 0;
    if (c == r) return s;
  }
  return -1;
}
// The ELL slot held in register slot sl once slot 0 and slot p swap places.
__host__ __device__ constexpr int heff_swapped_slot(int sl, int p) {
  return p <= 0 ? sl : (sl == 0 ? p : (sl == p ? 0 : sl));
}

template <typename T, int G, int R, int W, bool BLK, bool TD, bool GST = false>
struct Traj {
  using V = typename CT<T>::V;
  static constexpr int WR = W > 0 ? W : 1;

  const McArgs &a;
  const int lane;
  const unsigned mask;
  const int d;
  V *ybuf;           // the group's shared copies of published vectors: copy 0
                     // at ybuf, copy 1 at ybuf + kYD (see publish())
  const V *val;      // operator values in the kernel's precision (global)
  const V *aval;     // values of operators 1.. (shared when staged)
  const int *acol;   // columns of operators 1..
  const int *opw;    // ELL width per operator (shared)
  const int *opoff;  // slot offset per operator relative to aval/acol
  int wh;            // ELL width of H_eff
  float inv2d;       // 1 / (2 d)
  T atol_t, rtol_t;  // tolerances in the kernel's precision
  V hv[R][WR];       // this lane's H_eff entries (W > 0)
  int hc[R][WR];
  // mixed kernel: the FP32 remainders of the same entries (H_eff = hv + hl to
  // ~2^-48), so that the operator carries no systematic FP32 rounding
  const V *vlo;      // remainders of all operator values (mixed kernel)
  const V *hlo;      // this CTA's shared copy of the remainders of H_eff,
                     // [row][WR] (register instances; null: read vlo)
  V *lpb;            // mixed: this lane's two shared buffers of -i lo psi,
                     // buffer c row q at lpb[(c R + q) G]
  int lpc = 0;       // the buffer holding lo psi of the current state
  // W < 0: H_eff as a dictionary in shared memory (see McArgs::dict_code):
  // codes [dict_w][d], diagonal hi/lo [2][d], value table hi/lo [2][nv]
  const uint32_t *dcode = nullptr;
  const V *ddiag = nullptr, *dtab = nullptr;
  T *redv = nullptr;  // CTA-wide groups: [warp][value] partial sums of the outputs
  // the first time-dependent term: its ELL rows in registers when at most 4
  // wide (tw0 >= 0), and its current linear piece {f at offset 0, slope,
  // first offset, last offset} (every thread of the group holds the same)
  static constexpr int TR = (TD && W > 0) ? 4 : 1;
  V tv[R][TR];
  int tc[R][TR];
  int tw0 = -1;
  T p0[4];
  // statistics of the current trajectory (kept by every lane, added to the
  // global counters by lane 0 when the trajectory ends)
  unsigned n_acc = 0, n_rej = 0, n_rhs = 0, n_bis = 0, n_jmp = 0, n_near = 0;
  GroupScalars *gs;  // per-group FP64 scalars kept out of the step loop's registers

  __device__ Traj(const McArgs &a_, int lane_, unsigned mask_, V *ybuf_, const V *val_,
                  const V *aval_, const int *acol_, const int *opw_, const int *opoff_,
                  GroupScalars *gs_, const V *hlo_ = nullptr, V *lpb_ = nullptr,
                  const unsigned char *dict_ = nullptr)
      : a(a_), lane(lane_), mask(mask_), d(a_.ops.d), ybuf(ybuf_), val(val_), aval(aval_),
        acol(acol_), opw(opw_), opoff(opoff_), gs(gs_), hlo(hlo_), lpb(lpb_) {
    if (dict_) {
      dcode = reinterpret_cast<const uint32_t *>(dict_);
      ddiag = reinterpret_cast<const V *>(dict_ + dict_code_bytes(a_.dict_w, a_.ops.d));
      dtab = ddiag + 2 * a_.ops.d;
    }
    vlo = sizeof(T) == 4 ? reinterpret_cast<const V *>(a_.ops.val32lo) : nullptr;
    wh = opw[0];
    inv2d = 1.0f / (float)(2 * d);
    atol_t = (T)a_.atol;
    rtol_t = (T)a_.rtol;
    if (W > 0) {
      const int64_t off = a.ops.off[0];
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const int row = lane + q * G;
#pragma unroll
        for (int s = 0; s < WR; ++s) {
          if (row < d && s < wh) {
            hv[q][s] = val[off + (int64_t)s * d + row];
            hc[q][s] = a.ops.col[off + (int64_t)s * d + row];
          } else {
            hv[q][s] = cmake<V>(0.0, 0.0);
            hc[q][s] = 0;
          }
        }
        if constexpr (sizeof(T) == 4) {  // the own-column slot to slot 0
          int p = -1;
#pragma unroll
          for (int s = WR - 1; s >= 0; --s)
            if (hc[q][s] == row) p = s;
          if (row < d && p < 0) set_status(a.status, QT_EINVAL);
#pragma unroll
          for (int s = 1; s < WR; ++s)
            if (p == s) {
              const V tv0 = hv[q][0];
              const int tc0 = hc[q][0];
              hv[q][0] = hv[q][s];
              hc[q][0] = hc[q][s];
              hv[q][s] = tv0;
              hc[q][s] = tc0;
            }
        }
      }
    }
    if constexpr (TD && W > 0) {
      if (a.n_td > 0 && opw[a.td_op0] <= TR) {
        tw0 = opw[a.td_op0];
        const int off = opoff[a.td_op0];
#pragma unroll
        for (int q = 0; q < R; ++q) {
          const int row = lane + q * G;
#pragma unroll
          for (int s = 0; s < TR; ++s) {
            if (row < d && s < tw0) {
              tv[q][s] = aval[off + s * d + row];
              tc[q][s] = acol[off + s * d + row];
            } else {
              tv[q][s] = cmake<V>(0.0, 0.0);
              tc[q][s] = 0;
            }
          }
        }
      }
    }
    p0[0] = p0[1] = (T)0;
    p0[2] = (T)1;
    p0[3] = (T)-1;
  }

  __device__ __forceinline__ int row(int q) const { return lane + q * G; }

  // Distance of a warp group's copy 1 from its copy 0 (a CTA-wide group has
  // one copy), and copy B.
  static constexpr int kYD = BLK ? 0 : G * R;
  template <int B> __device__ __forceinline__ V *ycopy() const { return ybuf + B * kYD; }

  // Group barrier: the warp's lanes, or the whole CTA.
  __device__ __forceinline__ void sync() const {
    if constexpr (BLK) {
      __syncthreads();
    } else {
      __syncwarp(mask);
    }
  }

  // Sum over the group, identical on every thread of the group.
  template <typename X> __device__ __forceinline__ X gsum(X v) const {
    if constexpr (!BLK) {
      return group_sum<G>(v, mask);
    } else {
      v = group_sum<32>(v, 0xffffffffu);
      X *slot = reinterpret_cast<X *>(gs->red);
      __syncthreads();
      if ((threadIdx.x & 31) == 0) slot[threadIdx.x >> 5] = v;
      __syncthreads();
      X t = slot[0];
#pragma unroll
      for (int i = 1; i < G / 32; ++i) t += slot[i];
      return t;
    }
  }

  // Two FP32 sums over the group at once (the same additions, in the same
  // order, as gsum of each).
  __device__ __forceinline__ void gsum2(float &x, float &y) const {
    if constexpr (!BLK) {
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) {
        x += __shfl_xor_sync(mask, x, o);
        y += __shfl_xor_sync(mask, y, o);
      }
    } else {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        x += __shfl_xor_sync(0xffffffffu, x, o);
        y += __shfl_xor_sync(0xffffffffu, y, o);
      }
      float *slot = reinterpret_cast<float *>(gs->red);  // 32 floats: [x][16], [y][16]
      __syncthreads();
      if ((threadIdx.x & 31) == 0) {
        slot[threadIdx.x >> 5] = x;
        slot[16 + (threadIdx.x >> 5)] = y;
      }
      __syncthreads();
      float tx = slot[0], ty = slot[16];
#pragma unroll
      for (int i = 1; i < G / 32; ++i) {
        tx += slot[i];
        ty += slot[16 + i];
      }
      x = tx;
      y = ty;
    }
  }

  // Adds this trajectory's statistics to the global counters.
  __device__ __forceinline__ void flush_stats() {
    if (lane == 0) {
      atomicAdd(a.counters + 0, (unsigned long long)n_acc);
      atomicAdd(a.counters + 1, (unsigned long long)n_rej);
      atomicAdd(a.counters + 2, (unsigned long long)n_rhs);
      atomicAdd(a.counters + 3, (unsigned long long)n_bis);
      atomicAdd(a.counters + 4, (unsigned long long)n_jmp);
      atomicAdd(a.counters + 5, (unsigned long long)n_near);
    }
    n_acc = n_rej = n_rhs = n_bis = n_jmp = n_near = 0;
  }

  // Writes an FP64 group scalar (lane 0 stores, the group synchronises).
  __device__ __forceinline__ void put(double &slot, double v) {
    sync();
    if (lane == 0) slot = v;
    sync();
  }

  // Publish y to copy B of the group's shared buffer.  The barrier before
  // the writes (lead) keeps them from overtaking the reads of the copy's
  // previous contents; the stage evaluations of step() alternate between
  // the copies, so there the barrier after the previous publish has already
  // ordered those reads.  Readers outside step() use copy 1, and every
  // publish to it leads with a barrier.
  template <int B = 1>
  __device__ __forceinline__ void publish(const V (&y)[R], bool lead = true) {
    if (BLK || lead) sync();
    V *yb = ycopy<B>();
#pragma unroll
    for (int q = 0; q < R; ++q)  // the buffer holds G * R rows; padded rows stay zero
      if (sizeof(T) == 4 || row(q) < d) yb[row(q)] = y[q];
    sync();
  }

  // The cached linear piece of the time-dependent coefficient k, in the
  // kernel's precision.
  __device__ __forceinline__ T *td_piece(int k) const {
    if constexpr (sizeof(T) == 8) return reinterpret_cast<T *>(gs->tdd[k]);
    else return reinterpret_cast<T *>(gs->tdf[k]);
  }

  // Forget the cached pieces (the base time tb changed).
  __device__ __forceinline__ void td_reset() {
    if constexpr (TD) {
      p0[2] = (T)1;
      p0[3] = (T)-1;
      sync();
      if (lane == 0)
        for (int k = 0; k < a.n_td; ++k) {
          T *c = td_piece(k);
          c[2] = (T)1;
          c[3] = (T)-1;
        }
      sync();
    }
  }

  // f_k at time tb + s (piecewise linear between knots, constant outside;
  // paper section 4.3 with H(t) = H + sum_k f_k(t) H_k): from the cached piece
  // when s lies in it, else the piece around tb + s is looked up in FP64.
  __device__ __forceinline__ T td_coef(int k, T s) {
    if constexpr (sizeof(T) == 8) {
      // FP64 kernel: s is the absolute time; the oracle's evaluation order
      return td_piecewise(a.td_t, a.td_v, a.td_off[k], a.td_off[k + 1] - 1, (double)s);
    }
    // the piece around tb + s: looked up in FP64 when s leaves the cached one
    auto lookup = [&](T (&c)[4]) {
      const TdPiece<T> p =
          td_lookup_piece<T>(a.td_t, a.td_v, a.td_off[k], a.td_off[k + 1] - 1, gs->tb, s);
      c[0] = p.f0;
      c[1] = p.slope;
      c[2] = p.lo;
      c[3] = p.hi;
      return p.f;
    };
    if (k == 0) {
      // every thread of the group holds the same piece in registers
      if (!(s >= p0[2] && s <= p0[3])) return lookup(p0);
      return tfma(p0[1], s, p0[0]);
    }
    T *c = td_piece(k);
    if (!(s >= c[2] && s <= c[3])) {
      T nc[4];
      const T f = lookup(nc);
      sync();
      if (lane == 0)
        for (int q = 0; q < 4; ++q) c[q] = nc[q];
      sync();
      return f;
    }
    return tfma(c[1], s, c[0]);
  }

  // k = -i H_eff(tb + ts) y, with the time-dependent terms when TD.  With
  // LO (mixed kernel) also lo = (H_eff - fl32(H_eff)) y, the product with the
  // FP32 remainders of H_eff's entries (see step()).
  template <bool LO = false, typename KO>
  __device__ __forceinline__ void rhs(const V (&y)[R], KO &&k, T ts, int lobuf = 0) {
    T f0 = (T)0;
    if constexpr (TD) {
      if (a.n_td > 0) f0 = td_coef(0, ts);
    }
    ++n_rhs;
    rhs_f<LO, 1>(y, k, ts, f0, lobuf);
  }

  // The same with the coefficient of the first time-dependent term given;
  // with LO the remainder product goes to buffer lobuf of lpb.  (Not counted
  // in n_rhs: step() counts its evaluations at once.)
  template <bool LO = false, int B = 1, typename KO>
  __device__ __forceinline__ void rhs_f(const V (&y)[R], KO &&k, T ts, T f0, int lobuf = 0,
                                        bool lead = true) {
    constexpr bool kLo = LO && sizeof(T) == 4;
    publish<B>(y, lead);
    const V *yb = ycopy<B>();
    if constexpr (W == -2) {
      // grouped dictionary H_eff: the diagonal times this thread's own
      // entry, then per value the sum of the gathered entries, times the
      // value.  The thread's rows walk the slots together, so that each slot
      // issues R independent code-then-entry loads.
      CAcc<V> acc[R];  // the products with H_eff
      CAcc<V> acl[R];  // the products with the remainders of its entries (kLo)
      const int nv = a.dict_nv;
      bool in[R];
#pragma unroll
      for (int q = 0; q < R; ++q) {
        in[q] = row(q) < d;
        if (in[q]) {
          acc[q].mac(ddiag[row(q)], y[q]);
          if constexpr (kLo) acl[q].mac(ddiag[d + row(q)], y[q]);
        }
      }
      int s = 0;
      for (int g = 0; g < a.dict_groups; ++g) {
        const int e = a.dict_gend[g];
        V sum[R];
#pragma unroll
        for (int q = 0; q < R; ++q) sum[q] = cmake<V>(0.0, 0.0);
#pragma unroll 4
        for (; s < e; ++s)  // padding, and rows beyond d: column d, a zero entry
#pragma unroll
          for (int q = 0; q < R; ++q)
            sum[q] = vadd(sum[q], yb[in[q] ? dcode[s * d + row(q)] : (uint32_t)d]);
#pragma unroll
        for (int q = 0; q < R; ++q) {
          acc[q].mac(dtab[g + 1], sum[q]);
          if constexpr (kLo) acl[q].mac(dtab[nv + g + 1], sum[q]);
        }
      }
#pragma unroll
      for (int q = 0; q < R; ++q) {
        if constexpr (kLo) {  // stored as -i lo y
          const V lo = acl[q].get();
          lpb[(lobuf * R + q) * G] = cmake<V>(lo.y, -lo.x);
        }
        const V hy = acc[q].get();
        k[q].x = hy.y;  // -i (x + i y) = y - i x
        k[q].y = -hy.x;
      }
    } else {
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const V yq = y[q];
      CAcc<V> acc;  // the product with H_eff
      CAcc<V> acl;  // the product with the remainders of its entries (kLo)
      if constexpr (W == -1) {
        // dictionary H_eff: the diagonal times this thread's own entry, then
        // the off-diagonal entries as codes (column, value index)
        if (row(q) < d) {
          const int r = row(q);
          acc.mac(ddiag[r], y[q]);
          if constexpr (kLo) acl.mac(ddiag[d + r], y[q]);
          const int nv = a.dict_nv;
          const int dw = a.dict_w;
#pragma unroll 4
          for (int s = 0; s < dw; ++s) {
            const uint32_t c = dcode[s * d + r];
            const V yc = yb[c & 0xffffu];
            acc.mac(dtab[c >> 16], yc);
            if constexpr (kLo) acl.mac(dtab[nv + (c >> 16)], yc);
          }
        }
      } else if (W > 0) {
#pragma unroll
        for (int s = 0; s < WR; ++s)  // mixed: padded slots hold 0 at column 0
          if (sizeof(T) == 4 || s < wh) {
            // mixed: slot 0 is the row's own column (this thread's entry)
            const V y = (sizeof(T) == 4 && s == 0) ? yq : yb[hc[q][s]];
            acc.mac(hv[q][s], y);
            if constexpr (kLo) acl.mac(hlo[row(q) * WR + s], y);
          }
      } else if (row(q) < d) {
        const int64_t off = a.ops.off[0];
        for (int s = 0; s < wh; ++s) {
          const int64_t p = off + (int64_t)s * d + row(q);
          const V y = yb[__ldg(a.ops.col + p)];
          acc.mac(__ldg(val + p), y);
          if constexpr (kLo) acl.mac(__ldg(vlo + p), y);
        }
      }
      if constexpr (kLo) {  // stored as -i lo y
        const V lo = acl.get();
        lpb[(lobuf * R + q) * G] = cmake<V>(lo.y, -lo.x);
      }
      const V hy = acc.get();
      k[q].x = hy.y;   // -i (x + i y) = y - i x
      k[q].y = -hy.x;
    }
    }
    if constexpr (TD) {
      for (int t = 0; t < a.n_td; ++t) {
        const T f = t == 0 ? f0 : td_coef(t, ts);
#pragma unroll
        for (int q = 0; q < R; ++q) {
          V hy;
          if (t == 0 && tw0 >= 0) {
            CAcc<V> acd;  // mixed: two packed multiply-adds per entry
#pragma unroll
            for (int s = 0; s < TR; ++s)
              if (s < tw0) acd.mac(tv[q][s], yb[tc[q][s]]);
            hy = acd.get();
          } else {
            hy = apply_row<B>(a.td_op0 + t, q);
          }
          k[q].x = tfma(f, hy.y, k[q].x);
          k[q].y = tfma(-f, hy.x, k[q].y);
        }
      }
    }
  }

  // (op y) for this lane's row q, op >= 1; y must already be published (to
  // copy B).
  template <int B = 1>
  __device__ __forceinline__ V apply_row(int op, int q) const {
    V acc = cmake<V>(0.0, 0.0);
    const int r = row(q);
    if (r >= d) return acc;
    const int w = opw[op];
    const int off = opoff[op];
    for (int s = 0; s < w; ++s) {
      const int p = off + s * d + r;
      cmac(acc, aval[p], ycopy<B>()[acol[p]]);
    }
    return acc;
  }

  // This thread's part of <y|y> in FP32 (the mixed kernel's norm test).
  __device__ __forceinline__ float norm2_32(const V (&y)[R]) const {
    if constexpr (sizeof(T) == 4) {  // both components packed, added at the end
      float2 s = make_float2(0.f, 0.f);
#pragma unroll
      for (int q = 0; q < R; ++q) s = __ffma2_rn(y[q], y[q], s);
      return s.x + s.y;
    } else {
      float s = 0.f;
#pragma unroll
      for (int q = 0; q < R; ++q) {
        s = fmaf((float)y[q].x, (float)y[q].x, s);
        s = fmaf((float)y[q].y, (float)y[q].y, s);
      }
      return s;
    }
  }

  // <y|y> summed in FP64 over the group.
  __device__ __forceinline__ double norm2_64(const V (&y)[R]) const {
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const double x = (double)y[q].x, z = (double)y[q].y;
      s = fma(x, x, s);
      s = fma(z, z, s);
    }
    return gsum(s);
  }

  // <y + c|y + c> summed in FP64 over the group (the compensated state of
  // the mixed kernel: y + c is exact in FP64).
  __device__ __forceinline__ double norm2_64c(const V (&y)[R], const V (&c)[R]) const {
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const double x = (double)y[q].x + (double)c[q].x, z = (double)y[q].y + (double)c[q].y;
      s = fma(x, x, s);
      s = fma(z, z, s);
    }
    return gsum(s);
  }

  // Is <y|y> <= r?  The FP64 kernel decides with the FP64 sum of its values.
  // The mixed kernel forms the FP32 sum of the stored values and decides with
  // it when it lies outside [rlo, rhi] = r (1 -/+ 1e-5): the FP32 sum of 2R
  // products per lane and log2(G) tree levels is within (2R + log2 G + 2)
  // 2^-24 of the exact sum, and the remainders c change it by ~2^-24, both far
  // inside that band.  Inside the band it decides with the FP64 sum of the
  // compensated state y + c.  n2 receives <y|y> (FP64 when formed, else the
  // FP32 sum) when want_n2; s32 receives the FP32 sum (mixed kernel only).
  // pre: the FP32 group sum already formed (by step()), or null.
  template <bool want_n2>
  __device__ __forceinline__ bool below(const V (&y)[R], const V (&c)[R], float rlo, float rhi,
                                        double &n2, float &s32,
                                        const float *pre = nullptr) const {
    if constexpr (sizeof(T) == 8) {
      n2 = norm2_64(y);
      return n2 <= gs->r;
    } else {
      float s;
      if (pre) {
        s = *pre;
      } else {
        s = norm2_32(y);
        s = gsum(s);
      }
      s32 = s;
      if (s < rlo) {
        if (want_n2) n2 = (double)s;
        return true;
      }
      if (s > rhi) {
        if (want_n2) n2 = (double)s;
        return false;
      }
      if (!(s == s)) {  // NaN: report it, decide "not below"
        n2 = (double)s;
        return false;
      }
      n2 = norm2_64c(y, c);
      return n2 <= gs->r;
    }
  }

  // Offset of the stage at c h of a step from u0 (the FP64 kernel rounds the
  // product and the sum separately, as the oracle's stage times).
  __device__ __forceinline__ T stage_off(T u0, double c, T h) const {
    if constexpr (sizeof(T) == 8) return stage_time(u0, c, h);
    else return tfma((T)c, h, u0);
  }

  // One Dormand-Prince step of length h from (psi, k[0] = f(psi)).  Writes the
  // 5th-order solution to ynew; with want_err evaluates k[6] = f(ynew) and
  // returns the scaled RMS error norm, else returns 0.
  //
  // Mixed kernel: the stages use the FP32 entries of H_eff.  Their rounding
  // (relative 2^-24) is a fixed perturbation of the Hamiltonian whose effect
  // grows with the phase |H| t; the step adds it back to first order as
  // -i h lo(psi), lo = H_eff - fl32(H_eff) (FP32 remainders of the entries),
  // formed once per step with the last stage evaluation of the previous one
  // (lo psi from buffer lpc of lpb; lo ynew to the other buffer).  What
  // remains is O(h |H|) of the remainder's effect.  The update itself is
  // compensated (psi + cps carries the integrated state to ~2^-48).
  template <typename KS>
  __device__ __forceinline__ T step(const V (&psi)[R], const V (&cps)[R], KS &k, T u0, T h,
                                    V (&ynew)[R], V (&cnew)[R], bool want_err,
                                    float *n2sum = nullptr) {
    const T ht = h;
    n_rhs += want_err ? 6 : 5;
    V yt[R];
    // stage input psi + h (c_1 k_1 + ... ): both components of each complex
    // entry with one packed multiply-add per coefficient
#define QT_STAGE(EXPR)                                   \
  _Pragma("unroll") for (int q = 0; q < R; ++q) {        \
    V acs;                                               \
    EXPR;                                                \
    yt[q] = vfma(ht, acs, psi[q]);                       \
  }
#define QT_ACC(c, j) acs = vfma((T)(c), k[j][q], acs);
    // coefficient of the first time-dependent term at a stage offset: from
    // the cached piece when the whole step lies in it
    bool fast = true;
    if constexpr (TD) fast = sizeof(T) == 4 && u0 >= p0[2] && u0 + ht <= p0[3];
    auto coef = [&](T so) -> T {
      if constexpr (!TD) {
        return (T)0;
      } else {
        if (a.n_td == 0) return (T)0;
        return fast ? tfma(p0[1], so, p0[0]) : td_coef(0, so);
      }
    };
    QT_STAGE(acs = vmul(DPW<T>::a21, k[0][q]))
    // the stage inputs go to copies 0, 1, 0, 1, 0 and ynew to copy 1; only a
    // trial step (no ynew) can follow one that wrote copy 0 last
    { const T so = stage_off(u0, DP::c2, ht); rhs_f<false, 0>(yt, k[1], so, coef(so), 0, !want_err); }
    QT_STAGE(acs = vmul(DPW<T>::a31, k[0][q]); QT_ACC(DPW<T>::a32, 1))
    { const T so = stage_off(u0, DP::c3, ht); rhs_f<false, 1>(yt, k[2], so, coef(so), 0, false); }
    QT_STAGE(acs = vmul(DPW<T>::a41, k[0][q]); QT_ACC(DPW<T>::a42, 1) QT_ACC(DPW<T>::a43, 2))
    { const T so = stage_off(u0, DP::c4, ht); rhs_f<false, 0>(yt, k[3], so, coef(so), 0, false); }
    QT_STAGE(acs = vmul(DPW<T>::a51, k[0][q]); QT_ACC(DPW<T>::a52, 1) QT_ACC(DPW<T>::a53, 2)
                 QT_ACC(DPW<T>::a54, 3))
    { const T so = stage_off(u0, DP::c5, ht); rhs_f<false, 1>(yt, k[4], so, coef(so), 0, false); }
    QT_STAGE(acs = vmul(DPW<T>::a61, k[0][q]); QT_ACC(DPW<T>::a62, 1) QT_ACC(DPW<T>::a63, 2)
                 QT_ACC(DPW<T>::a64, 3) QT_ACC(DPW<T>::a65, 4))
    const T s_end = u0 + ht;
    rhs_f<false, 0>(yt, k[5], s_end, coef(s_end), 0, false);
#pragma unroll
    for (int q = 0; q < R; ++q) {
      V acs = vmul(DPW<T>::b1, k[0][q]);
      QT_ACC(DPW<T>::b3, 2) QT_ACC(DPW<T>::b4, 3) QT_ACC(DPW<T>::b5, 4) QT_ACC(DPW<T>::b6, 5)
      if constexpr (sizeof(T) == 4) {
        acs = vadd(acs, lpb[(lpc * R + q) * G]);  // + (-i lo psi)
        // compensated update: the increment carries the remainder of the
        // previous updates, and the rounding error of this one is kept
        const V inc = vfma(ht, acs, cps[q]);
        ynew[q].x = two_sum(psi[q].x, inc.x, cnew[q].x);
        ynew[q].y = two_sum(psi[q].y, inc.y, cnew[q].y);
      } else {
        ynew[q].x = tfma(ht, acs.x, psi[q].x);
        ynew[q].y = tfma(ht, acs.y, psi[q].y);
        cnew[q] = cmake<V>(0.0, 0.0);
      }
    }
#undef QT_STAGE
    if (!want_err) return (T)0;
    rhs_f<true, 1>(ynew, k[6], s_end, coef(s_end), lpc ^ 1, false);
    T sum = (T)0;
    V sum2 = cmake<V>(0.0, 0.0);  // mixed: the sums of both components, packed
    const T at = atol_t, rt = rtol_t;
#pragma unroll
    for (int q = 0; q < R; ++q) {
      if (row(q) >= d) continue;
      V acs = vmul(DPW<T>::e1, k[0][q]);
      QT_ACC(DPW<T>::e3, 2) QT_ACC(DPW<T>::e4, 3) QT_ACC(DPW<T>::e5, 4) QT_ACC(DPW<T>::e6, 5)
      QT_ACC(DPW<T>::e7, 6)
      acs = vmul(ht, acs);
      const V mx = cmake<V>(tmax(tabs(psi[q].x), tabs(ynew[q].x)), tmax(tabs(psi[q].y), tabs(ynew[q].y)));
      if constexpr (sizeof(T) == 8) {
        const T qx = acs.x / tfma(rt, mx.x, at);
        const T qy = acs.y / tfma(rt, mx.y, at);
        sum = tfma(qx, qx, sum);
        sum = tfma(qy, qy, sum);
      } else {
        const V sc = vfma(rt, mx, cmake<V>(at, at));  // atol + rtol max(|psi|, |ynew|)
        const V qv = __fmul2_rn(acs, make_float2(rcp_approx(sc.x), rcp_approx(sc.y)));
        sum2 = __ffma2_rn(qv, qv, sum2);
      }
    }
    if constexpr (sizeof(T) == 4) sum = sum2.x + sum2.y;
#undef QT_ACC
    if constexpr (sizeof(T) == 4) {
      // mixed: <ynew|ynew> for the norm test in the same reduction
      float ns = norm2_32(ynew);
      gsum2(sum, ns);
      if (n2sum) *n2sum = ns;
    } else {
      sum = gsum(sum);
    }
    if constexpr (sizeof(T) == 8) {
      return sqrt(sum / (double)(2 * d));
    } else {
      return sqrt_approx(sum * inv2d);
    }
  }

  // Step-size controller in the scalar precision of the kernel: the FP64
  // kernel uses the shared FP64 rule; the mixed kernel the same rule in FP32.
  __device__ __forceinline__ T control(T h, T err, bool accepted, bool after_reject,
                                       bool clipped, T hprop) const {
    if constexpr (sizeof(T) == 8) {
      return dp_control(h, err, accepted, after_reject, clipped, hprop);
    } else {
      const float p = ex2_approx(-0.2f * lg2_approx(err));  // err^(-1/5)
      if (accepted) {
        const float facmax = after_reject ? 1.f : 5.f;
        const float fac = (err == 0.f) ? facmax : fminf(facmax, fmaxf(0.2f, 0.9f * p));
        float hn = h * fac;
        if (clipped && hn < hprop) hn = hprop;
        return hn;
      }
      return h * fmaxf(0.2f, 0.9f * p);
    }
  }

  // Hairer-Norsett-Wanner starting step; k[0] = f(psi).  Uses k[1].
  template <typename KS>
  __device__ double initial_step(const V (&psi)[R], KS &k, T u0) {
    double s0 = 0.0, s1 = 0.0;
#pragma unroll
    for (int q = 0; q < R; ++q) {
      if (row(q) >= d) continue;
      const double scx = a.atol + a.rtol * fabs((double)psi[q].x);
      const double scy = a.atol + a.rtol * fabs((double)psi[q].y);
      s0 += ((double)psi[q].x / scx) * ((double)psi[q].x / scx) +
            ((double)psi[q].y / scy) * ((double)psi[q].y / scy);
      s1 += ((double)k[0][q].x / scx) * ((double)k[0][q].x / scx) +
            ((double)k[0][q].y / scy) * ((double)k[0][q].y / scy);
    }
    const double n = 2.0 * d;
    const double d0 = sqrt(gsum(s0) / n);
    const double d1 = sqrt(gsum(s1) / n);
    const double h0 = (d0 < 1e-5 || d1 < 1e-5) ? 1e-6 : 0.01 * d0 / d1;
    V yt[R];
#pragma unroll
    for (int q = 0; q < R; ++q) {
      yt[q].x = (T)((double)psi[q].x + h0 * (double)k[0][q].x);
      yt[q].y = (T)((double)psi[q].y + h0 * (double)k[0][q].y);
    }
    rhs(yt, k[1], u0 + (T)h0);
    double s2 = 0.0;
#pragma unroll
    for (int q = 0; q < R; ++q) {
      if (row(q) >= d) continue;
      const double scx = a.atol + a.rtol * fabs((double)psi[q].x);
      const double scy = a.atol + a.rtol * fabs((double)psi[q].y);
      const double ex = ((double)k[1][q].x - (double)k[0][q].x) / scx;
      const double ey = ((double)k[1][q].y - (double)k[0][q].y) / scy;
      s2 += ex * ex + ey * ey;
    }
    const double d2 = sqrt(gsum(s2) / n) / h0;
    const double dm = fmax(d1, d2);
    const double h1 = (dm <= 1e-15) ? fmax(1e-6, h0 * 1e-3) : pow(0.01 / dm, 0.2);
    return fmin(100.0 * h0, h1);
  }

  // Normalised expectation values of psi at output index m, added in FP64 to
  // the sums over trajectories (global FP64 atomics, one lane per value).
  // The FP64 kernel forms each trajectory's value in FP64 as the oracle does
  // (<psi|O|psi> * (1 / <psi|psi>)); the mixed kernel forms <psi|O|psi> and
  // <psi|psi> of its FP32 state by FP32 trees over the group (relative error
  // ~1e-7, below that of the state itself).
  __device__ void output(int m, const V (&psi)[R], int64_t j) {
    if (a.n_e == 0) return;
    publish(psi);
    T nn = 0;
#pragma unroll
    for (int q = 0; q < R; ++q) {
      nn = tfma(psi[q].x, psi[q].x, nn);
      nn = tfma(psi[q].y, psi[q].y, nn);
    }
    nn = gsum(nn);
    const T inv = (T)1 / nn;
    double *sum = reinterpret_cast<double *>(a.expect_sum);
    double *tex = reinterpret_cast<double *>(a.traj_expect);
    if constexpr (BLK) {
      // CTA-wide group: the partial sums of up to 8 observables at once,
      // reduced over the warps in one pass (two barriers per 8 observables
      // instead of four per observable)
      const int warp = threadIdx.x >> 5, wl = threadIdx.x & 31;
      for (int e0 = 0; e0 < a.n_e; e0 += 8) {
        const int ne = min(a.n_e - e0, 8);
        T v[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] = 0;
        for (int e = 0; e < ne; ++e) {
          const int op = 1 + a.n_c + e0 + e;
          T er = 0, ei = 0;
#pragma unroll
          for (int q = 0; q < R; ++q) {
            const V o = apply_row(op, q);
            er = tfma(psi[q].x, o.x, er);
            er = tfma(psi[q].y, o.y, er);
            ei = tfma(psi[q].x, o.y, ei);
            ei = tfma(-psi[q].y, o.x, ei);
          }
#pragma unroll
          for (int k = 0; k < 16; ++k) {  // v[2e], v[2e+1] without dynamic indexing
            if (k == 2 * e) v[k] = er;
            if (k == 2 * e + 1) v[k] = ei;
          }
        }
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] = group_sum<32>(v[k], 0xffffffffu);
        __syncthreads();
        if (wl == 0)
#pragma unroll
          for (int k = 0; k < 16; ++k) redv[warp * 16 + k] = v[k];
        __syncthreads();
        if ((int)threadIdx.x < 2 * ne) {
          T t = 0;
          for (int w = 0; w < G / 32; ++w) t += redv[w * 16 + threadIdx.x];
          const int64_t idx = 2 * ((int64_t)m * a.n_e + e0) + threadIdx.x;
          const double val = (double)(t * inv);
          atomicAdd(sum + idx, val);
          if (tex) tex[2 * ((j * a.n_t + m) * a.n_e + e0) + threadIdx.x] = val;
        }
      }
      return;
    }
    for (int e0 = 0; e0 < a.n_e; e0 += G / 2) {
      const int ne = min(a.n_e - e0, G / 2);
      T mine = 0;  // lane 2e holds Re, lane 2e+1 Im of observable e0 + e
      for (int e = 0; e < ne; ++e) {
        const int op = 1 + a.n_c + e0 + e;
        T er = 0, ei = 0;
#pragma unroll
        for (int q = 0; q < R; ++q) {
          const V o = apply_row(op, q);  // (O psi)_row
          er = tfma(psi[q].x, o.x, er);  // conj(psi) * (O psi)
          er = tfma(psi[q].y, o.y, er);
          ei = tfma(psi[q].x, o.y, ei);
          ei = tfma(-psi[q].y, o.x, ei);
        }
        er = gsum(er);
        ei = gsum(ei);
        if (lane == 2 * e) mine = er * inv;
        if (lane == 2 * e + 1) mine = ei * inv;
      }
      if (lane < 2 * ne) {
        const int64_t idx = 2 * ((int64_t)m * a.n_e + e0) + lane;
        const double v = (double)mine;
        atomicAdd(sum + idx, v);
        if (tex) tex[2 * ((j * a.n_t + m) * a.n_e + e0) + lane] = v;
      }
    }
  }

  // ||C_n y||^2: per-lane partial in the state precision, FP64 across lanes;
  // y must already be published.
  __device__ __forceinline__ double weight(int n) const {
    T s = 0;
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const V c = apply_row(1 + n, q);
      s = tfma(c.x, c.x, s);
      s = tfma(c.y, c.y, s);
    }
    return gsum((double)s);
  }

  // Step III of the algorithm at the state y = psi(tau).  Returns false on a
  // numerical error.
  __device__ bool collapse(const V (&y)[R], V (&psi)[R], uint64_t gtraj, int64_t jk,
                           double tau, double t_lo_out, double t_hi_out) {
    publish(y);
    const double r2 = uniform52(a.seed, gtraj, (uint64_t)jk, 1);
    const int nc = a.n_c;
    int chosen = -1;
    double psum = 0.0, pc = 0.0;
    int64_t degenerate = 0;
    bool done = false;
    if constexpr (!BLK) {
     if (nc <= G) {
      // lane n keeps p_n; an inclusive scan over the lanes gives the
      // cumulative sums of Eq. (mc3)
      double mine = 0.0;
      for (int n = 0; n < nc; ++n) {
        const double p = weight(n);
        if (lane == n) mine = p;
      }
      double cum = mine;
#pragma unroll
      for (int o = 1; o < G; o <<= 1) {
        const double v = __shfl_up_sync(mask, cum, o, G);
        if (lane >= o) cum += v;
      }
      const int base = (threadIdx.x & 31) / G * G;
      psum = __shfl_sync(mask, cum, base + nc - 1);
      if (!(psum > 0.0) || !isfinite(psum)) return false;
      const double target = r2 * psum;
      const unsigned gbits = (G == 32) ? 0xffffffffu : ((1u << G) - 1u);
      const unsigned ge = (__ballot_sync(mask, lane < nc && cum >= target) >> base) & gbits;
      const unsigned nearb =
          (__ballot_sync(mask, lane < nc && fabs(cum - target) < 1e-5 * psum) >> base) & gbits;
      const unsigned pos = (__ballot_sync(mask, lane < nc && mine > 0.0) >> base) & gbits;
      if (nearb) degenerate |= 1;
      chosen = ge ? __ffs(ge) - 1 : (31 - __clz(pos));  // round-off fallback: last p > 0
      pc = __shfl_sync(mask, mine, base + chosen);
      done = true;
     }
    }
    if (!done) {
      int last_pos = -1;
      for (int n = 0; n < nc; ++n) {
        const double p = weight(n);
        psum += p;
        if (p > 0.0) last_pos = n;
      }
      if (!(psum > 0.0) || !isfinite(psum)) return false;
      const double target = r2 * psum;
      double cum = 0.0;
      for (int n = 0; n < nc; ++n) {
        const double p = weight(n);
        cum += p;
        if (fabs(cum - target) < 1e-5 * psum) degenerate |= 1;
        if (chosen < 0 && cum >= target) { chosen = n; pc = p; }
      }
      if (chosen < 0) { chosen = last_pos; pc = weight(chosen); }
    }
    const double tscale = 4e-6 * fmax(1.0, fabs(tau));
    if (fabs(tau - t_lo_out) < tscale || fabs(tau - t_hi_out) < tscale) degenerate |= 2;
    const T inv = (T)rsqrt(pc);
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const V c = apply_row(1 + chosen, q);
      psi[q].x = c.x * inv;
      psi[q].y = c.y * inv;
    }
    if (lane == 0) {
      const unsigned long long slot = atomicAdd(a.n_jumps, 1ULL);
      if (a.jumps && (int64_t)slot < a.jump_cap) {
        qt_jump rec;
        rec.traj = (int64_t)gtraj;
        rec.k = jk;
        rec.channel = chosen;
        rec.tau = tau;
        rec.degenerate = degenerate;
        a.jumps[slot] = rec;
      }
    }
    ++n_jmp;
    return true;
  }

  // One whole trajectory (local index j).  Returns false after recording an
  // error in a.status.
  __device__ bool run(int64_t j) {
    const uint64_t gtraj = (uint64_t)(a.traj_begin + j);
    V psi[R];
#pragma unroll
    for (int q = 0; q < R; ++q) {
      if (row(q) < d) {
        const double2 p = a.psi0[row(q)];
        psi[q] = cmake<V>(p.x, p.y);
      } else {
        psi[q] = cmake<V>(0.0, 0.0);
      }
    }
    // mixed kernel: the rounding remainder of psi carried by the compensated
    // update (psi + cps is the integrated state to ~2^-48)
    V cps[R];
#pragma unroll
    for (int q = 0; q < R; ++q) cps[q] = cmake<V>(0.0, 0.0);
    int64_t jk = 0;
    {
      const double r0 = uniform52(a.seed, gtraj, 0, 0);
      put(gs->r, r0);
    }
    float rlo = (float)(gs->r * (1.0 - 1e-5)), rhi = (float)(gs->r * (1.0 + 1e-5));
    output(0, psi, j);
    if (a.n_t == 1) return true;

    // Time.  The FP64 kernel keeps the absolute time t in u (base tb = 0), as
    // the oracle does.  The mixed kernel keeps an FP32 offset u from the start
    // tb of the current output interval, so that its per-step control runs in
    // FP32; absolute FP64 times are formed only to search a jump time.  An
    // interval starts where the previous one ended (tb + L, the FP32 length
    // actually integrated), so the rounding of the lengths to FP32 does not
    // accumulate over the intervals.  Without time-dependent terms the
    // starts and lengths come from the table of a.ivl_tb / a.ivl_len (no
    // FP64 arithmetic per interval), else they are formed here.  The FP64
    // scalars (r, tb) live in the group's shared slot, so that no FP64 value
    // is carried through the step loop.
    constexpr bool kOff = sizeof(T) == 4;
    std::conditional_t<GST, GlobalStages<V, G>, RegStages<V, R>> k;
    if constexpr (GST)
      k = GlobalStages<V, G>{reinterpret_cast<V *>(a.stage_ws) +
                                 (int64_t)blockIdx.x * 7 * (G * R) + lane,
                             G * R};
    T u = kOff ? (T)0 : (T)a.tlist[0];
    put(gs->tb, kOff ? a.tlist[0] : 0.0);
    td_reset();
    lpc = 0;
    rhs<true>(psi, k[0], u, lpc);
    T hprop = (T)((a.h0 > 0.0) ? a.h0 : initial_step(psi, k, u));
    bool after_reject = false;
    T n2_cur = (T)1;  // <psi|psi> of the current state (approximate in FP32)
    T L = (T)0;
    for (int m = 1; m < a.n_t; ++m) {
      if constexpr (kOff) {
        if (!TD && a.ivl_len) {
          L = __ldg(a.ivl_len + m);  // the interval table (same values)
        } else {
          const double tstart = (m == 1) ? a.tlist[0] : gs->tb + (double)L;
          put(gs->tb, tstart);
          td_reset();
          L = (T)(a.tlist[m] - tstart);
        }
        u = (T)0;
      } else {
        L = (T)a.tlist[m];
      }
      const T hmin_off = (T)(16.0f * 1.1920929e-7f) * L;
      int attempts = 0;
      while (u < L) {
        if (attempts++ >= a.max_steps) { set_status(a.status, QT_ESTEP); return false; }
        const bool clipped = hprop >= L - u;
        const T h = clipped ? L - u : hprop;
        if constexpr (kOff) {
          if (!clipped && h < hmin_off) { set_status(a.status, QT_ESTEP); return false; }
        } else {
          if (!clipped && h < (T)dp_hmin((double)u, a.tlist[m])) {
            set_status(a.status, QT_ESTEP);
            return false;
          }
        }
        V ynew[R], cnew[R];
        float n2sum = 0.f;  // mixed: <ynew|ynew> in FP32, formed by step()
        const T err = step(psi, cps, k, u, h, ynew, cnew, true, &n2sum);
        if (!isfinite(err)) { set_status(a.status, QT_ENUMERIC); return false; }
        if (err > (T)1) {
          hprop = control(h, err, false, after_reject, clipped, hprop);
          after_reject = true;
          ++n_rej;
          continue;
        }
        hprop = control(h, err, true, after_reject, clipped, hprop);
        after_reject = false;
        ++n_acc;
        const T unew = clipped ? L : u + h;
        double n2 = 0.0;
        float s32 = 0.f;
        if (!below<sizeof(T) == 8>(ynew, cnew, rlo, rhi, n2, s32,
                                   sizeof(T) == 4 ? &n2sum : nullptr)) {
          if constexpr (sizeof(T) == 8) {
            if (!isfinite(n2)) { set_status(a.status, QT_ENUMERIC); return false; }
            n2_cur = n2;
          } else {
            // a finite error norm implies a finite state; keep its FP32 norm
            n2_cur = s32;
          }
#pragma unroll
          for (int q = 0; q < R; ++q) {
            psi[q] = ynew[q];
            cps[q] = cnew[q];
            k[0][q] = k[6][q];
          }
          lpc ^= 1;  // lo ynew became lo psi
          u = unew;
          continue;
        }
        // Step II: locate tau in (t0, tnew] with <psi(tau)|psi(tau)> = r, in
        // FP64 time.  Each trial state is one Dormand-Prince step of length
        // tau - t0 from the accepted (t0, psi); f(tau) = <psi(tau)|psi(tau)> - r
        // is positive at t0 and <= 0 at tnew.  The bracket is narrowed by the
        // Illinois variant of regula falsi, with a bisection step whenever two
        // consecutive trials fail to halve it; it stops when narrower than
        // bisect_tol max(1, |t0|) (the mixed kernel does not go below
        // 1e-9 max(1, |t0|): an FP32 state resolves its norm to ~1e-7).  The
        // result is tau = the upper end of the bracket, where f <= 0, as with
        // plain bisection, and agrees with it to within the tolerance.
        const double tk = a.tlist[m], tprev = a.tlist[m - 1];
        const double tb = (kOff && !TD && a.ivl_len) ? a.ivl_tb[m] : gs->tb, r = gs->r;
        const double t0 = tb + (double)u;
        double hi;
        if constexpr (kOff) {
          // Mixed kernel: the bracket is kept as FP32 offsets s in [0, h] from
          // the FP64 step start t0 (resolution h 2^-24, ~1e-9 for the steps of
          // an FP32 state), tau = t0 + s formed in FP64 at the end.  The
          // decisions f(s) <= 0 are the FP64-exact ones of below(); f values
          // only place the next trial.
          const float rf = (float)r;
          float slo = 0.f, shi = h, flo = n2_cur - rf, fhi = s32 - rf;
          if (!(flo > 0.f)) flo = 1e-30f;
          const float tol =
              fmaxf((float)(fmax(a.bisect_tol, 1e-9) * fmax(1.0, fabs(t0))), 4.f * shi * 1.1920929e-7f);
          int side = 0, slow = 0;
          for (int it = 0; it < 64 && shi - slo > tol; ++it) {
            const float w = shi - slo;
            float c;
            if (slow >= 2) {
              c = slo + 0.5f * w;
              slow = 0;
            } else {
              c = shi - w * (fhi / (fhi - flo));
              const float e = 0.5f * tol;
              c = fminf(fmaxf(c, slo + e), shi - e);
              if (!(c > slo && c < shi)) c = slo + 0.5f * w;
            }
            V ytr[R], ctr[R];
            step(psi, cps, k, u, (T)c, ytr, ctr, false);
            ++n_bis;
            double nc2 = 0.0;
            float sc = 0.f;
            const bool b = below<false>(ytr, ctr, rlo, rhi, nc2, sc);
            // f at the trial: the FP64 difference when the band forced the FP64
            // sum (n2 = nc2), else the FP32 one
            const bool band = !(sc < rlo) && !(sc > rhi);
            const float fc = band ? (float)(nc2 - r) : sc - rf;
            if (b) {
              shi = c;
              fhi = fc;
              if (side == -1) flo *= 0.5f;
              side = -1;
#pragma unroll
              for (int q = 0; q < R; ++q) ynew[q] = ytr[q];
            } else {
              slo = c;
              flo = (fc > 0.f) ? fc : 1e-30f;
              if (side == 1) fhi *= 0.5f;
              side = 1;
            }
            slow = (shi - slo > 0.5f * w) ? slow + 1 : 0;
          }
          hi = (clipped && shi == h) ? tk : t0 + (double)shi;
        } else {
          // FP64 kernel: the same search in FP64 absolute time.
          hi = clipped ? tk : tb + (double)unew;
          double lo = t0;
          double flo = (double)n2_cur - r, fhi = n2 - r;
          if (!(flo > 0.0)) flo = 1e-300;
          const double tol = a.bisect_tol * fmax(1.0, fabs(t0));
          int side = 0, slow = 0;
          for (int it = 0; it < 64 && hi - lo > tol; ++it) {
            const double w = hi - lo;
            double c;
            if (slow >= 2) {
              c = lo + 0.5 * w;
              slow = 0;
            } else {
              c = hi - w * (fhi / (fhi - flo));
              const double e = 0.5 * tol;
              c = fmin(fmax(c, lo + e), hi - e);
              if (!(c > lo && c < hi)) c = lo + 0.5 * w;
            }
            V ytr[R], ctr[R];
            step(psi, cps, k, u, (T)(c - t0), ytr, ctr, false);
            ++n_bis;
            double nc2 = 0.0;
            float sc = 0.f;
            if (below<true>(ytr, ctr, rlo, rhi, nc2, sc)) {
              hi = c;
              fhi = nc2 - r;
              if (side == -1) flo *= 0.5;
              side = -1;
#pragma unroll
              for (int q = 0; q < R; ++q) ynew[q] = ytr[q];
            } else {
              lo = c;
              flo = nc2 - r;
              if (!(flo > 0.0)) flo = 1e-300;
              if (side == 1) fhi *= 0.5;
              side = 1;
            }
            slow = (hi - lo > 0.5 * w) ? slow + 1 : 0;
          }
        }
        // Steps III and IV.
        if (!collapse(ynew, psi, gtraj, jk, hi, tprev, tk)) {
          set_status(a.status, QT_ENUMERIC);
          return false;
        }
        ++jk;
        const double rn = uniform52(a.seed, gtraj, (uint64_t)jk, 0);
        put(gs->r, rn);
        rlo = (float)(rn * (1.0 - 1e-5));
        rhi = (float)(rn * (1.0 + 1e-5));
        n2_cur = (T)1;
#pragma unroll
        for (int q = 0; q < R; ++q) cps[q] = cmake<V>(0.0, 0.0);
        u = (hi == tk) ? L : (T)(hi - tb);
        rhs<true>(psi, k[0], u, lpc);
      }
      output(m, psi, j);
    }
    const double n2 = norm2_64(psi), rr = gs->r;
    if (fabs(n2 - rr) < 1e-5 * rr) ++n_near;
    return true;
  }
};

// Resident CTAs per SM the register allocation is sized for: the small mixed
// instances fit 128 registers (16 warps per SM); the FP64 and wide instances
// keep up to 255 registers rather than spill.
// Threads per CTA: four warp groups, or one CTA-wide group of G threads.
template <int G, bool BLK>
__host__ __device__ constexpr int mc_block() {
  return BLK ? G : kBlock;
}

// Resident CTAs per SM the register allocation is sized for: the small mixed
// instances fit 128 registers (16 warps per SM; 168 and 12 warps with the
// time-dependent terms); the FP64 and wide instances keep up to 255 registers
// rather than spill; a CTA-wide group runs one CTA.
template <typename T, int G, int R, int W, bool BLK, bool TD>
__host__ __device__ constexpr int mc_min_blocks() {
  return BLK ? ((W < 0 && G == 256) ? 2 : 1)
             : ((sizeof(T) == 4 && R <= 2 && W <= 4) ? (TD ? 3 : 4) : 2);
}

template <typename T, int G, int R, int W, bool BLK, bool TD, bool GST>
__global__ void __launch_bounds__((mc_block<G, BLK>()), (mc_min_blocks<T, G, R, W, BLK, TD>()))
    mc_kernel(const __grid_constant__ McArgs a) {
  using V = typename CT<T>::V;
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int NT = mc_block<G, BLK>();
  constexpr int groups = NT / G;
  const int grp = threadIdx.x / G;
  const int lane = threadIdx.x % G;
  const unsigned mask = BLK ? 0xffffffffu : group_mask<(BLK ? 32 : G)>();
  const int n_ops = a.ops.n_ops;
  const int64_t aux_begin = a.aux_begin;
  constexpr int HLO = (sizeof(T) == 4 && W > 0) ? G * R * W : 0;
  const size_t DB = W < 0 ? dict_bytes(a.dict_w, a.ops.d, a.dict_nv) : 0;
  const McSmem L =
      mc_smem_layout<V>(groups, G, R, n_ops, a.aux_slots, a.stage_aux != 0, HLO, DB);
  V *ybuf = reinterpret_cast<V *>(smem + L.ybuf) + grp * (G * R) * (BLK ? 1 : 2);
  int *opw = reinterpret_cast<int *>(smem + L.opw);
  int *opoff = reinterpret_cast<int *>(smem + L.opoff);
  const V *val = sizeof(T) == 8 ? reinterpret_cast<const V *>(a.ops.val64)
                                : reinterpret_cast<const V *>(a.ops.val32);
  const V *aval;
  const int *acol;
  for (int i = threadIdx.x; i < n_ops; i += blockDim.x) {
    opw[i] = a.ops.w[i];
    opoff[i] = (int)(a.ops.off[i] - (a.stage_aux ? aux_begin : 0));
  }
  if (a.stage_aux) {
    V *sv = reinterpret_cast<V *>(smem + L.val);
    int *sc = reinterpret_cast<int *>(smem + L.col);
    for (int64_t i = threadIdx.x; i < a.aux_slots; i += blockDim.x) {
      sv[i] = val[aux_begin + i];
      sc[i] = a.ops.col[aux_begin + i];
    }
    aval = sv;
    acol = sc;
  } else {
    aval = val;
    acol = a.ops.col;
  }
  if constexpr (W < 0) {
    // the dictionary H_eff, copied as it is laid out in global memory
    const uint4 *src = reinterpret_cast<const uint4 *>(a.dict_code);
    uint4 *dst = reinterpret_cast<uint4 *>(smem + L.dict);
    for (size_t i = threadIdx.x; i < DB / 16; i += blockDim.x) dst[i] = src[i];
    if (threadIdx.x == 0) reinterpret_cast<V *>(smem + L.ybuf)[G * R] = cmake<V>(0.0, 0.0);
  }
  V *hlo = nullptr;
  if constexpr (HLO > 0) {
    // the FP32 remainders of H_eff, row-major per row so that lane l reads
    // rows l + q G at fixed offsets; padded rows and slots hold 0
    hlo = reinterpret_cast<V *>(smem + L.hlo);
    const V *vlo = reinterpret_cast<const V *>(a.ops.val32lo);
    const int d = a.ops.d, wh = a.heff_w;
    const int64_t off0 = a.ops.off[0];
    for (int i = threadIdx.x; i < HLO; i += blockDim.x) {
      const int r = i / W;
      // the register slot order of Traj: own-column slot first
      const int sl = heff_swapped_slot(
          i - r * W, r < d ? heff_own_slot(a.ops.col, off0, d, wh, r, W) : -1);
      hlo[i] = (r < d && sl < wh) ? vlo[off0 + (int64_t)sl * d + r] : cmake<V>(0.0, 0.0);
    }
  }
  __syncthreads();

  GroupScalars *gs = reinterpret_cast<GroupScalars *>(smem + L.gscal) + grp;
  V *lpb = sizeof(T) == 4 ? reinterpret_cast<V *>(smem + L.lpb) + grp * (2 * G * R) + lane
                          : nullptr;
  Traj<T, G, R, W, BLK, TD, GST> tr(a, lane, mask, ybuf, val, aval, acol, opw, opoff, gs, hlo,
                                    lpb, W < 0 ? smem + L.dict : nullptr);
  if constexpr (BLK) tr.redv = reinterpret_cast<T *>(smem + L.redv);
  const int64_t ntraj = a.ntraj;
  for (;;) {
    // lane 0 takes the next index; an error anywhere ends the hand-out
    unsigned long long j = 0;
    if (lane == 0) {
      j = atomicAdd(a.work, 1ULL);
      if (*(volatile int *)a.status != 0) j = (unsigned long long)ntraj;
    }
    if constexpr (BLK) {
      if (lane == 0) gs->next = j;
      __syncthreads();
      j = gs->next;
      __syncthreads();
    } else {
      const int leader = (threadIdx.x & 31) / G * G;
      j = __shfl_sync(mask, j, leader);
    }
    if ((int64_t)j >= ntraj) break;
    const bool ok = tr.run((int64_t)j);
    tr.flush_stats();
    if (!ok) break;
  }
}

template <typename T, int G, int R, int W, bool BLK, bool TD = false, bool GST = false>
cudaError_t launch_inst(const McArgs &a_in, cudaStream_t s) {
  using V = typename CT<T>::V;
  auto kern = mc_kernel<T, G, R, W, BLK, TD, GST>;
  constexpr int NT = mc_block<G, BLK>();
  constexpr int groups = NT / G;
  McArgs a = a_in;
  // stage the collapse and observable operators when they fit in 40 KB
  const size_t aux_bytes = (size_t)a.aux_slots * (sizeof(V) + sizeof(int));
  a.stage_aux = (a.ops.n_ops > 1 && a.aux_slots > 0 && aux_bytes <= 40 * 1024) ? 1 : 0;
  constexpr int HLO = (sizeof(T) == 4 && W > 0) ? G * R * W : 0;
  const size_t DB = W < 0 ? dict_bytes(a.dict_w, a.ops.d, a.dict_nv) : 0;
  const McSmem L =
      mc_smem_layout<V>(groups, G, R, a.ops.n_ops, a.aux_slots, a.stage_aux != 0, HLO, DB);
  const size_t smem = L.total;
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  if (smem > 48 * 1024) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  int64_t want = (a.ntraj + groups - 1) / groups;
  int64_t grid = (int64_t)sms * per_sm;
  if (want < grid) grid = want;
  if (grid < 1) grid = 1;
  if (GST && grid > a.stage_ctas) grid = a.stage_ctas;  // one stage slab per CTA
  kern<<<(unsigned)grid, NT, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

}  // namespace qt
