// qt_host.cpp -- host side of libqt: argument validation, operator packing
// (CSR/dense -> canonical CSR -> ELLPACK), the effective Hamiltonian of the
// paper's Eq. (heff), device-resident systems, and the C ABI of qt.h.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "qt_internal.h"

using cplx = std::complex<double>;

namespace {

thread_local std::string g_err;

int fail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define QT_CK(call)                                                                  \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess)                                                           \
      return fail(e_ == cudaErrorMemoryAllocation ? QT_ENOMEM : QT_ECUDA, "%s: %s", #call, \
                  cudaGetErrorString(e_));                                           \
  } while (0)

int ensure_device() {
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess || n < 1)
    return fail(QT_ENODEV, "no usable CUDA device: %s",
                e == cudaSuccess ? "device count is 0" : cudaGetErrorString(e));
  return QT_OK;
}

// Device buffer released on scope exit.
struct DevBuf {
  void *p = nullptr;
  DevBuf() = default;
  DevBuf(const DevBuf &) = delete;
  DevBuf &operator=(const DevBuf &) = delete;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
  int alloc(size_t bytes) {
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
      p = nullptr;
      return fail(QT_ENOMEM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    }
    return QT_OK;
  }
  template <typename X> X *as() const { return reinterpret_cast<X *>(p); }
};

struct StreamGuard {
  cudaStream_t s = nullptr;
  ~StreamGuard() {
    if (s) cudaStreamDestroy(s);
  }
};

// FP32 values as hi + lo pairs: out[q] = fl32(v), out[n + q] = fl32(v - out[q])
// (n = v.size()), so that hi + lo carries v to ~2^-48 relative.
void split_fp32(const std::vector<double2> &v, std::vector<float2> &out) {
  const size_t n = v.size();
  for (size_t q = 0; q < n; ++q) {
    const float hx = (float)v[q].x, hy = (float)v[q].y;
    out[q] = make_float2(hx, hy);
    out[n + q] = make_float2((float)(v[q].x - (double)hx), (float)(v[q].y - (double)hy));
  }
}

// ------------------------------------------------------------ canonical CSR
struct Csr {
  int d = 0;
  std::vector<int64_t> ptr;
  std::vector<int> col;
  std::vector<cplx> val;
};

// Validates op and converts it to CSR with sorted, merged columns and no
// explicit zeros.  expect_dim < 0 accepts any positive dimension.
int to_csr(const qt_op *op, int expect_dim, const char *what, Csr &out) {
  if (!op) return fail(QT_EINVAL, "%s: null operator", what);
  if (op->dim <= 0) return fail(QT_EINVAL, "%s: dim %d must be positive", what, op->dim);
  if (expect_dim >= 0 && op->dim != expect_dim)
    return fail(QT_EINVAL, "%s: dim %d does not match %d", what, op->dim, expect_dim);
  const int d = op->dim;
  out.d = d;
  out.ptr.assign(d + 1, 0);
  out.col.clear();
  out.val.clear();
  if (op->fmt == QT_DENSE) {
    if (!op->values) return fail(QT_EINVAL, "%s: null dense values", what);
    for (int i = 0; i < d; ++i) {
      for (int j = 0; j < d; ++j) {
        const qt_c128 v = op->values[(size_t)i * d + j];
        if (!std::isfinite(v.re) || !std::isfinite(v.im))
          return fail(QT_EINVAL, "%s: non-finite entry (%d, %d)", what, i, j);
        if (v.re != 0.0 || v.im != 0.0) {
          out.col.push_back(j);
          out.val.emplace_back(v.re, v.im);
        }
      }
      out.ptr[i + 1] = (int64_t)out.col.size();
    }
    return QT_OK;
  }
  if (op->fmt != QT_CSR) return fail(QT_EINVAL, "%s: unknown format %d", what, op->fmt);
  if (op->nnz < 0) return fail(QT_EINVAL, "%s: negative nnz", what);
  if (!op->indptr || (op->nnz > 0 && (!op->indices || !op->values)))
    return fail(QT_EINVAL, "%s: null CSR array", what);
  if (op->indptr[0] != 0 || op->indptr[d] != op->nnz)
    return fail(QT_EINVAL, "%s: indptr must start at 0 and end at nnz", what);
  std::vector<std::pair<int, cplx>> row;
  for (int i = 0; i < d; ++i) {
    const int64_t a = op->indptr[i], b = op->indptr[i + 1];
    if (b < a || b > op->nnz) return fail(QT_EINVAL, "%s: indptr not monotone at row %d", what, i);
    row.clear();
    for (int64_t p = a; p < b; ++p) {
      const int c = op->indices[p];
      if (c < 0 || c >= d) return fail(QT_EINVAL, "%s: column %d out of range in row %d", what, c, i);
      const qt_c128 v = op->values[p];
      if (!std::isfinite(v.re) || !std::isfinite(v.im))
        return fail(QT_EINVAL, "%s: non-finite value in row %d", what, i);
      row.emplace_back(c, cplx(v.re, v.im));
    }
    std::sort(row.begin(), row.end(),
              [](const std::pair<int, cplx> &x, const std::pair<int, cplx> &y) { return x.first < y.first; });
    for (size_t q = 0; q < row.size();) {
      int c = row[q].first;
      cplx s = 0.0;
      while (q < row.size() && row[q].first == c) s += row[q++].second;
      if (s != cplx(0.0, 0.0)) {
        out.col.push_back(c);
        out.val.push_back(s);
      }
    }
    out.ptr[i + 1] = (int64_t)out.col.size();
  }
  return QT_OK;
}

// H_eff = H - (i/2) sum_n C_n^dag C_n (paper Eq. (heff), hbar = 1), in FP64.
// Row i of C^dag C is sum over the entries (k, i) of C of conj(C_ki) * row k.
// H_eff as a dictionary: diagonal, and off-diagonal entries as column plus
// an index into the table of their distinct values (exact FP64 equality;
// entry 0 is zero and pads short rows).  Returns false when the values do not
// fit the table or the dimension does not fit 16-bit columns.
struct DictOp {
  int w = 0;
  std::vector<uint32_t> code;  // [w][d]
  std::vector<double2> diag;   // [d]
  std::vector<double2> tab;    // [nv]
  // grouped form (groups > 0): the slots of value index g + 1 are the range
  // [gend[g - 1], gend[g]) of every row, holding its columns (d: padding)
  int groups = 0;
  int gend[qt::kDictMaxGroups] = {};
};

// Regroups a dictionary by value: when every row's entries of one value fit
// a common slot range and the padded width stays within 5/4 of the plain
// one, the codes become plain columns ordered by value (padding column d, a
// zero entry of the state copy), so a right-hand side sums the gathered
// entries of each value and multiplies once per value.
void group_dictionary(int d, DictOp &D) {
  const int ng = (int)D.tab.size() - 1;
  if (ng < 1 || ng > qt::kDictMaxGroups) return;
  std::vector<int> gw(ng, 0);
  std::vector<int> cnt(ng);
  for (int i = 0; i < d; ++i) {
    std::fill(cnt.begin(), cnt.end(), 0);
    for (int s = 0; s < D.w; ++s) {
      const uint32_t c = D.code[(size_t)s * d + i];
      if ((c >> 16) != 0) ++cnt[(c >> 16) - 1];
    }
    for (int g = 0; g < ng; ++g) gw[g] = std::max(gw[g], cnt[g]);
  }
  // A value whose entries (i, j) take few distinct masks i ^ j (a spin
  // chain's bit flips) gives each mask a slot of its own: the rows of a warp
  // then gather r ^ m for one m per slot, a permutation within each aligned
  // block of 32 entries (no shared-memory bank conflicts).
  std::vector<std::vector<int>> masks(ng);
  std::vector<char> fixed(ng, 1);
  for (int i = 0; i < d; ++i)
    for (int s = 0; s < D.w; ++s) {
      const uint32_t c = D.code[(size_t)s * d + i];
      const int g = (int)(c >> 16) - 1;
      if (g < 0 || !fixed[g]) continue;
      const int m = i ^ (int)(c & 0xffffu);
      if (std::find(masks[g].begin(), masks[g].end(), m) == masks[g].end()) {
        masks[g].push_back(m);
        if (4 * (int)masks[g].size() > 5 * gw[g]) fixed[g] = 0;
      }
    }
  std::vector<int> width(ng);
  int total = 0;
  for (int g = 0; g < ng; ++g) {
    if (fixed[g]) std::sort(masks[g].begin(), masks[g].end());
    width[g] = fixed[g] ? (int)masks[g].size() : gw[g];
    total += width[g];
  }
  if (4 * total > 5 * D.w) {  // the mask slots widen the rows too much
    total = 0;
    for (int g = 0; g < ng; ++g) {
      fixed[g] = 0;
      width[g] = gw[g];
      total += gw[g];
    }
  }
  if (4 * total > 5 * D.w) return;
  std::vector<int> start(ng, 0);
  for (int g = 1; g < ng; ++g) start[g] = start[g - 1] + width[g - 1];
  std::vector<uint32_t> code((size_t)total * d, (uint32_t)d);
  for (int i = 0; i < d; ++i) {
    std::fill(cnt.begin(), cnt.end(), 0);
    for (int s = 0; s < D.w; ++s) {
      const uint32_t c = D.code[(size_t)s * d + i];
      const int g = (int)(c >> 16) - 1;
      if (g < 0) continue;
      const int col = (int)(c & 0xffffu);
      const int k = fixed[g] ? (int)(std::find(masks[g].begin(), masks[g].end(), i ^ col) -
                                     masks[g].begin())
                             : cnt[g]++;
      code[(size_t)(start[g] + k) * d + i] = (uint32_t)col;
    }
  }
  int e = 0;
  for (int g = 0; g < ng; ++g) D.gend[g] = (e += width[g]);
  D.code.swap(code);
  D.w = total;
  D.groups = ng;
}

bool dictionary_form(const Csr &A, int max_values, DictOp &out) {
  const int d = A.d;
  if (d > 65536) return false;
  std::vector<std::pair<std::pair<double, double>, int>> seen;  // small: linear search is fine
  out.tab.assign(1, make_double2(0.0, 0.0));
  out.diag.assign(d, make_double2(0.0, 0.0));
  int w = 0;
  for (int i = 0; i < d; ++i) {
    int cnt = 0;
    for (int64_t p = A.ptr[i]; p < A.ptr[i + 1]; ++p) cnt += A.col[p] != i;
    w = std::max(w, cnt);
  }
  out.w = w;
  out.code.assign((size_t)w * d, 0u);
  for (int i = 0; i < d; ++i) {
    int s = 0;
    for (int64_t p = A.ptr[i]; p < A.ptr[i + 1]; ++p) {
      const int c = A.col[p];
      const cplx v = A.val[p];
      if (c == i) {
        out.diag[i] = make_double2(v.real(), v.imag());
        continue;
      }
      int idx = -1;
      for (const auto &e : seen)
        if (e.first.first == v.real() && e.first.second == v.imag()) { idx = e.second; break; }
      if (idx < 0) {
        if ((int)out.tab.size() >= max_values) return false;
        idx = (int)out.tab.size();
        out.tab.push_back(make_double2(v.real(), v.imag()));
        seen.push_back({{v.real(), v.imag()}, idx});
      }
      out.code[(size_t)s * d + i] = (uint32_t)c | ((uint32_t)idx << 16);
      ++s;
    }
    for (; s < w; ++s) out.code[(size_t)s * d + i] = (uint32_t)i;  // padding: value 0
  }
  return true;
}

Csr effective_hamiltonian(const Csr &H, const std::vector<Csr> &C) {
  const int d = H.d;
  std::vector<std::vector<std::pair<int, cplx>>> colsof(d);  // transpose lists, reused
  std::vector<cplx> acc(d, 0.0);
  std::vector<char> used(d, 0);
  std::vector<int> touched;
  std::vector<std::vector<std::pair<int, cplx>>> rows(d);
  for (int i = 0; i < d; ++i)
    for (int64_t p = H.ptr[i]; p < H.ptr[i + 1]; ++p) rows[i].emplace_back(H.col[p], H.val[p]);
  for (const Csr &c : C) {
    for (auto &v : colsof) v.clear();
    for (int k = 0; k < d; ++k)
      for (int64_t p = c.ptr[k]; p < c.ptr[k + 1]; ++p) colsof[c.col[p]].emplace_back(k, c.val[p]);
    for (int i = 0; i < d; ++i) {
      touched.clear();
      for (const auto &kv : colsof[i]) {
        const int k = kv.first;
        const cplx ck = std::conj(kv.second);
        for (int64_t p = c.ptr[k]; p < c.ptr[k + 1]; ++p) {
          const int j = c.col[p];
          if (!used[j]) { used[j] = 1; touched.push_back(j); acc[j] = 0.0; }
          acc[j] += ck * c.val[p];
        }
      }
      for (int j : touched) {
        rows[i].emplace_back(j, cplx(0.0, -0.5) * acc[j]);
        used[j] = 0;
      }
    }
  }
  Csr out;
  out.d = d;
  out.ptr.assign(d + 1, 0);
  for (int i = 0; i < d; ++i) {
    auto &r = rows[i];
    std::sort(r.begin(), r.end(),
              [](const std::pair<int, cplx> &x, const std::pair<int, cplx> &y) { return x.first < y.first; });
    for (size_t q = 0; q < r.size();) {
      int c = r[q].first;
      cplx s = 0.0;
      while (q < r.size() && r[q].first == c) s += r[q++].second;
      if (s != cplx(0.0, 0.0)) {
        out.col.push_back(c);
        out.val.push_back(s);
      }
    }
    out.ptr[i + 1] = (int64_t)out.col.size();
  }
  return out;
}

// Appends A in slot-major ELLPACK form (width = longest row, at least 1;
// padding entries are zeros in the row's own column).  With diag_slot every
// row gets a slot in its own column: the width grows by one when a longest
// row has no diagonal entry (the mixed Monte-Carlo kernels take the product
// with that slot from the thread's own state entry).
int ell_append(const Csr &A, std::vector<int> &cols, std::vector<double2> &vals,
               bool diag_slot = false) {
  const int d = A.d;
  int w = 1;
  for (int i = 0; i < d; ++i) {
    int n = (int)(A.ptr[i + 1] - A.ptr[i]);
    if (diag_slot) {
      bool has = false;
      for (int64_t p = A.ptr[i]; p < A.ptr[i + 1]; ++p) has = has || A.col[p] == i;
      if (!has) ++n;
    }
    w = std::max<int>(w, n);
  }
  const size_t base = cols.size();
  cols.resize(base + (size_t)w * d);
  vals.resize(base + (size_t)w * d);
  for (int s = 0; s < w; ++s)
    for (int i = 0; i < d; ++i) {
      const int64_t p = A.ptr[i] + s;
      const size_t q = base + (size_t)s * d + i;
      if (p < A.ptr[i + 1]) {
        cols[q] = A.col[p];
        vals[q] = make_double2(A.val[p].real(), A.val[p].imag());
      } else {
        cols[q] = i;
        vals[q] = make_double2(0.0, 0.0);
      }
    }
  return w;
}

int check_opts(const qt_opts *o) {
  if (!o) return fail(QT_EINVAL, "null options");
  if (!(o->rtol > 0.0) || !(o->atol >= 0.0) || !std::isfinite(o->rtol) || !std::isfinite(o->atol))
    return fail(QT_EINVAL, "tolerances must be rtol > 0, atol >= 0");
  if (o->max_steps < 1) return fail(QT_EINVAL, "max_steps must be >= 1");
  if (!(o->bisect_tol > 0.0)) return fail(QT_EINVAL, "bisect_tol must be > 0");
  if (o->precision != QT_FP64 && o->precision != QT_MIXED)
    return fail(QT_EINVAL, "unknown precision %d", o->precision);
  if (o->traj_block != 0 && o->traj_block != 32)
    return fail(QT_ENOTIMPL, "traj_block %d is not built (0 or 32)", o->traj_block);
  if (o->me_method != QT_ME_AUTO && o->me_method != QT_ME_SPARSE &&
      o->me_method != QT_ME_DENSE_TC)
    return fail(QT_EINVAL, "unknown me_method %d", o->me_method);
  if (o->me_method == QT_ME_DENSE_TC && o->precision != QT_MIXED)
    return fail(QT_EINVAL, "me_method QT_ME_DENSE_TC computes in BF16/FP32: precision must be QT_MIXED");
  return QT_OK;
}

int check_tlist_host(const double *tlist, int n_t) {
  if (!tlist || n_t < 1) return fail(QT_EINVAL, "tlist must hold at least one time");
  for (int k = 0; k < n_t; ++k)
    if (!std::isfinite(tlist[k])) return fail(QT_EINVAL, "tlist[%d] is not finite", k);
  for (int k = 1; k < n_t; ++k)
    if (!(tlist[k] > tlist[k - 1])) return fail(QT_EINVAL, "tlist must be strictly increasing");
  return QT_OK;
}

}  // namespace

// ------------------------------------------------------------------ systems
struct qt_system_s {
  int d = 0, n_c = 0, n_e = 0, n_ops = 0;
  int64_t total_slots = 0;
  std::vector<int> w_host;
  std::vector<int64_t> off_host;
  int *w_dev = nullptr;
  int64_t *off_dev = nullptr;
  int *col_dev = nullptr;
  double2 *v64_dev = nullptr;
  float2 *v32_dev = nullptr;
  unsigned long long *ctl = nullptr;  // counters[6], n_jumps, work, status
  double2 *psi_norm = nullptr;        // normalised initial ket
  void *ws = nullptr;
  size_t ws_bytes = 0;
  // H_eff in ELL form on the host (slot-major, as on the device), kept for
  // the dense operands of the tensor-core path, which are built on first use
  std::vector<int> heff_col;
  std::vector<double2> heff_val;
  // the collapse operators in ELL form on the host (slot-major), kept when one
  // of them is at least kTcDenseCWidth wide: the tensor-core path then forms
  // their terms as dense products
  std::vector<int> c_col, c_w;
  std::vector<int64_t> c_off;
  std::vector<double2> c_val;
  int dp = 0;  // 0 until the dense operands exist
  uint16_t *a_hi = nullptr, *a_lo = nullptr, *b_hi = nullptr, *b_lo = nullptr;
  uint16_t *c_planes = nullptr, *t_planes = nullptr, *cc_planes = nullptr;  // hi then lo
  float2 *wdense = nullptr;
  float2 *ydense = nullptr;
  qt::TcArgs tc;
  // time-dependent Hamiltonian terms: operators 1 + n_c + n_e + k, knots
  int n_td = 0;
  int64_t *td_off_dev = nullptr;
  double *td_t_dev = nullptr, *td_v_dev = nullptr;
  // collapse operators in slot/term form (device), when small enough to stage
  int n_cslots = 0, n_cterms = 0;
  int *cslot_off = nullptr;
  int2 *cterms = nullptr;
  // grow-only store of the correlation functions (the states rho(t_k), the
  // tau-evolution slabs) and of the propagator steady state
  void *aux = nullptr;
  size_t aux_bytes = 0;
  // H_eff as a dictionary (see McArgs), when its distinct off-diagonal values
  // are few: one device block of codes, diagonal and value table
  void *dict = nullptr;
  int dict_w = 0, dict_nv = 0, dict_groups = 0;
  // the output intervals of the mixed Monte-Carlo kernel (McArgs::ivl_tb,
  // ivl_len): ivl_cap FP64 starts then ivl_cap FP32 lengths, grown on demand
  void *ivl = nullptr;
  int ivl_cap = 0;
  int dict_gend[qt::kDictMaxGroups] = {};

  qt::OpTable table() const {
    qt::OpTable t;
    t.d = d;
    t.n_ops = n_ops;
    t.w = w_dev;
    t.off = off_dev;
    t.col = col_dev;
    t.val64 = v64_dev;
    t.val32 = v32_dev;
    t.val32lo = v32_dev ? v32_dev + total_slots : nullptr;
    return t;
  }
  unsigned long long *counters() const { return ctl; }
  unsigned long long *n_jumps() const { return ctl + 6; }
  unsigned long long *work() const { return ctl + 7; }
  int *status() const { return reinterpret_cast<int *>(ctl + 8); }
  ~qt_system_s() {
    for (void *p : {(void *)w_dev, (void *)off_dev, (void *)col_dev, (void *)v64_dev,
                    (void *)v32_dev, (void *)ctl, (void *)psi_norm, ws, (void *)a_hi,
                    (void *)a_lo, (void *)b_hi, (void *)b_lo, (void *)ydense,
                    (void *)cslot_off, (void *)cterms, (void *)td_off_dev, (void *)td_t_dev,
                    (void *)td_v_dev, aux, dict, (void *)c_planes, (void *)t_planes,
                    (void *)cc_planes, (void *)wdense, ivl})
      if (p) cudaFree(p);
  }
};

namespace {

constexpr size_t kCtlBytes = 16 * sizeof(unsigned long long);

int reset_ctl(qt_system s, cudaStream_t st) {
  QT_CK(cudaMemsetAsync(s->ctl, 0, kCtlBytes, st));
  return QT_OK;
}

int ensure_ws(qt_system s, size_t bytes) {
  if (s->ws_bytes >= bytes) return QT_OK;
  if (s->ws) {
    cudaFree(s->ws);
    s->ws = nullptr;
    s->ws_bytes = 0;
  }
  cudaError_t e = cudaMalloc(&s->ws, bytes);
  if (e != cudaSuccess) {
    s->ws = nullptr;
    return fail(QT_ENOMEM, "workspace of %zu bytes: %s", bytes, cudaGetErrorString(e));
  }
  s->ws_bytes = bytes;
  return QT_OK;
}

int ensure_ivl(qt_system s, int n_t) {
  if (s->ivl_cap >= n_t) return QT_OK;
  if (s->ivl) cudaFree(s->ivl);
  s->ivl = nullptr;
  s->ivl_cap = 0;
  cudaError_t e = cudaMalloc(&s->ivl, (size_t)n_t * (sizeof(double) + sizeof(float)));
  if (e != cudaSuccess) {
    s->ivl = nullptr;
    return fail(QT_ENOMEM, "interval table of %d entries: %s", n_t, cudaGetErrorString(e));
  }
  s->ivl_cap = n_t;
  return QT_OK;
}

int ensure_aux(qt_system s, size_t bytes) {
  if (s->aux_bytes >= bytes) return QT_OK;
  if (s->aux) cudaFree(s->aux);
  s->aux = nullptr;
  s->aux_bytes = 0;
  cudaError_t e = cudaMalloc(&s->aux, bytes);
  if (e != cudaSuccess) {
    s->aux = nullptr;
    return fail(QT_ENOMEM, "store of %zu bytes: %s", bytes, cudaGetErrorString(e));
  }
  s->aux_bytes = bytes;
  return QT_OK;
}

int finish_stats(qt_system s, qt_stats *stats_dev, int64_t *n_jumps_dev, cudaStream_t st) {
  if (stats_dev)
    QT_CK(qt::launch_finalize_stats(s->counters(), s->status(), s->n_jumps(), stats_dev, st));
  if (n_jumps_dev)
    QT_CK(cudaMemcpyAsync(n_jumps_dev, s->n_jumps(), sizeof(int64_t), cudaMemcpyDeviceToDevice, st));
  return QT_OK;
}

// Master-equation kernel arguments common to the solve and the one-shot
// right-hand side (times, outputs and the state are set by the caller).
void me_args(qt_system s, const qt_opts *o, int grid, void *ws, qt::MeArgs &a) {
  std::memset(&a, 0, sizeof a);
  a.ops = s->table();
  a.n_c = s->n_c;
  a.n_e = s->n_e;
  a.grid = grid;
  a.rtol = o->rtol;
  a.atol = o->atol;
  a.h0 = o->h0;
  a.max_steps = o->max_steps;
  a.counters = s->counters();
  a.status = s->status();
  a.work = ws;
  a.cslot_off = s->cslot_off;
  a.cterms = s->cterms;
  a.n_td = s->n_td;
  a.td_op0 = 1 + s->n_c + s->n_e;
  a.td_off = s->td_off_dev;
  a.td_t = s->td_t_dev;
  a.td_v = s->td_v_dev;
  a.n_cslots = s->n_cslots;
  a.n_cterms = s->n_cterms;
  const size_t elem = o->precision == QT_MIXED ? sizeof(float2) : sizeof(double2);
  const size_t state_bytes = 11 * (size_t)s->d * s->d * elem;
  a.partial = reinterpret_cast<double *>(reinterpret_cast<char *>(ws) +
                                         ((state_bytes + 255) / 256) * 256);
}

// Largest dimension of the Hermitian solvers (32-bit entry indices).
constexpr int kHermMaxDim = 46340;

int ensure_dense(qt_system s);

// Path, grid and workspace of a master-equation launch:
//   QT_ME_SPARSE    the general solver (no symmetry assumed);
//   QT_ME_AUTO      the Hermitian solver with the sparse product for a ket,
//                   or for a matrix the kernel finds Hermitian (else general);
//   QT_ME_DENSE_TC  the Hermitian solver with the tensor-core product
//                   (QT_ENONHERM from the device for a non-Hermitian matrix).
// Sparse solves of dimension <= kMeSmallDim run the general solver on one CTA.
int me_setup(qt_system s, const qt_opts *o, bool is_ket, qt::MeArgs &a) {
  const bool dense = o->me_method == QT_ME_DENSE_TC;
  const bool small = !dense && s->d <= qt::kMeSmallDim;
  const bool herm = dense || (o->me_method == QT_ME_AUTO && !small && s->d <= kHermMaxDim);
  if (dense && s->d > kHermMaxDim)
    return fail(QT_ENOTIMPL, "the tensor-core method is built for dim <= %d", kHermMaxDim);
  if (dense && s->n_td > 0)
    return fail(QT_ENOTIMPL, "the tensor-core method is built for time-independent Hamiltonians");
  int rc;
  if (dense && (rc = ensure_dense(s))) return rc;
  const int grid = small ? 1
                 : dense ? qt::me_tc_grid()
                 : (herm ? qt::me_herm_grid(s->d, o->precision, s->n_cslots, s->n_cterms)
                         : qt::me_grid(s->d, o->precision));
  if (grid <= 0) return fail(QT_ECUDA, "cannot size the cooperative launch");
  if ((rc = ensure_ws(s, qt::me_workspace_bytes(s->d, o->precision, grid)))) return rc;
  me_args(s, o, grid, s->ws, a);
  a.herm = herm ? (is_ket ? 1 : 2) : 0;
  a.single_cta = small ? 1 : 0;
  return QT_OK;
}

// BF16 of an FP32 value, rounded to nearest even (NaN kept quiet).
uint16_t bf16_rn(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) == 0x7f800000u) return (uint16_t)((u >> 16) | ((u & 0xffffu) ? 0x40u : 0u));
  u += 0x7fffu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}

float bf16_value(uint16_t h) {
  const uint32_t u = (uint32_t)h << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// A 2-D BF16 tensor map over rows x inner elements (row-major), tiles of
// 128 rows x 64 elements with 128-byte swizzling.
int make_map(CUtensorMap *m, void *ptr, uint64_t inner, uint64_t rows) {
  static EncodeTiledFn enc = nullptr;
  if (!enc) {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return fail(QT_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
    enc = reinterpret_cast<EncodeTiledFn>(fn);
  }
  const cuuint64_t dims[2] = {inner, rows};
  const cuuint64_t strides[1] = {inner * 2};
  const cuuint32_t box[2] = {64, 128};
  const cuuint32_t es[2] = {1, 1};
  const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, ptr, dims, strides, box, es,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(QT_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return QT_OK;
}

// BF16 hi/lo of x: hi = x rounded to BF16, lo = (x - hi) rounded to BF16.
void bf16_split(double x, uint16_t &hi, uint16_t &lo) {
  hi = bf16_rn((float)x);
  lo = bf16_rn((float)(x - (double)bf16_value(hi)));
}

// Dense collapse operators of the tensor-core path (TcArgs): the stacked C
// planes [nc dp][2dp] (A of T = C y), the planes of [C_1 ... C_nc] as B
// [2dp][2 nc dp] (B of W = T [C_1 ... C_nc]^dag), zeroed T planes
// [dp][2 nc dp], the W buffer and their tensor maps.
int ensure_dense_collapse(qt_system s, int dp) {
  const int d = s->d, nc = s->n_c;
  std::vector<double2> Cd((size_t)nc * dp * dp, make_double2(0.0, 0.0));  // C_n[m][k]
  for (int n = 0; n < nc; ++n)
    for (int q = 0; q < s->c_w[n]; ++q)
      for (int i = 0; i < d; ++i) {
        const size_t p = (size_t)s->c_off[n] + (size_t)q * d + i;  // padding carries 0
        double2 &c = Cd[((size_t)n * dp + i) * dp + s->c_col[p]];
        c.x += s->c_val[p].x;
        c.y += s->c_val[p].y;
      }
  const size_t kc = (size_t)2 * nc * dp;                 // inner extent of T and [C ...] planes
  const size_t c_elems = (size_t)nc * dp * 2 * dp;       // stacked C planes
  const size_t t_elems = (size_t)dp * kc;                // T planes
  const size_t cc_elems = (size_t)2 * dp * kc;           // [C_1 ... C_nc] as B
  std::vector<uint16_t> cp(2 * c_elems), ccp(2 * cc_elems);
  for (int n = 0; n < nc; ++n)
    for (size_t m = 0; m < (size_t)dp; ++m)
      for (size_t k = 0; k < (size_t)dp; ++k) {
        const double2 c = Cd[((size_t)n * dp + m) * dp + k];
        // A of the stacked C: row n dp + m, entries (Re, Im) of C_n[m][k]
        const size_t a = ((size_t)n * dp + m) * 2 * dp + 2 * k;
        bf16_split(c.x, cp[a], cp[c_elems + a]);
        bf16_split(c.y, cp[a + 1], cp[c_elems + a + 1]);
        // B of X = [C_1 ... C_nc]: X[m][n dp + k] = C_n[m][k] in rows 2m
        // (Re, Im) and 2m + 1 (-Im, Re)
        const size_t kk = 2 * ((size_t)n * dp + k);
        const size_t r0 = (2 * m) * kc + kk, r1 = (2 * m + 1) * kc + kk;
        bf16_split(c.x, ccp[r0], ccp[cc_elems + r0]);
        bf16_split(c.y, ccp[r0 + 1], ccp[cc_elems + r0 + 1]);
        bf16_split(-c.y, ccp[r1], ccp[cc_elems + r1]);
        bf16_split(c.x, ccp[r1 + 1], ccp[cc_elems + r1 + 1]);
      }
  auto dalloc = [&](void **p, size_t bytes) -> int {
    if (cudaMalloc(p, bytes) != cudaSuccess) {
      *p = nullptr;
      return fail(QT_ENOMEM, "cudaMalloc of %zu bytes for the dense collapse operands failed",
                  bytes);
    }
    return QT_OK;
  };
  int rc;
  if ((rc = dalloc((void **)&s->c_planes, 2 * c_elems * 2)) ||
      (rc = dalloc((void **)&s->t_planes, 2 * t_elems * 2)) ||
      (rc = dalloc((void **)&s->cc_planes, 2 * cc_elems * 2)) ||
      (rc = dalloc((void **)&s->wdense, (size_t)dp * dp * sizeof(float2))))
    return rc;
  QT_CK(cudaMemcpy(s->c_planes, cp.data(), 2 * c_elems * 2, cudaMemcpyHostToDevice));
  QT_CK(cudaMemcpy(s->cc_planes, ccp.data(), 2 * cc_elems * 2, cudaMemcpyHostToDevice));
  QT_CK(cudaMemset(s->t_planes, 0, 2 * t_elems * 2));
  if ((rc = make_map(&s->tc.c_hi, s->c_planes, 2 * (uint64_t)dp, (uint64_t)nc * dp)) ||
      (rc = make_map(&s->tc.c_lo, s->c_planes + c_elems, 2 * (uint64_t)dp, (uint64_t)nc * dp)) ||
      (rc = make_map(&s->tc.t_hi, s->t_planes, kc, dp)) ||
      (rc = make_map(&s->tc.t_lo, s->t_planes + t_elems, kc, dp)) ||
      (rc = make_map(&s->tc.cc_hi, s->cc_planes, kc, 2 * (uint64_t)dp)) ||
      (rc = make_map(&s->tc.cc_lo, s->cc_planes + cc_elems, kc, 2 * (uint64_t)dp)))
    return rc;
  s->tc.t_hi_ptr = s->t_planes;
  s->tc.t_lo_ptr = s->t_planes + t_elems;
  s->tc.W = s->wdense;
  s->tc.nc = nc;
  return QT_OK;
}

// The dense operands of the tensor-core path: H_eff as BF16 hi/lo planes of
// the real dp x 2dp matrix A (layout in qt_internal.h), zeroed B planes, the
// FP32 product buffer and the four tensor maps.
int ensure_dense(qt_system s) {
  if (s->dp) return QT_OK;
  const int d = s->d;
  const int dp = (d + 127) / 128 * 128;
  const int w = s->w_host[0];
  std::vector<double2> H((size_t)dp * dp, make_double2(0.0, 0.0));
  for (int q = 0; q < w; ++q)
    for (int i = 0; i < d; ++i) {
      const size_t p = (size_t)q * d + i;  // padding entries carry the value 0
      double2 &h = H[(size_t)i * dp + s->heff_col[p]];
      h.x += s->heff_val[p].x;
      h.y += s->heff_val[p].y;
    }
  const size_t a_elems = (size_t)dp * 2 * dp, b_elems = (size_t)2 * dp * 2 * dp;
  std::vector<uint16_t> ahi(a_elems), alo(a_elems);
  for (size_t m = 0; m < (size_t)dp; ++m)
    for (size_t k = 0; k < (size_t)dp; ++k) {
      const double2 h = H[m * dp + k];
      const double parts[2] = {h.x, h.y};
      for (int c = 0; c < 2; ++c) {
        const uint16_t hi = bf16_rn((float)parts[c]);
        const uint16_t lo = bf16_rn((float)(parts[c] - (double)bf16_value(hi)));
        ahi[m * 2 * dp + 2 * k + c] = hi;
        alo[m * 2 * dp + 2 * k + c] = lo;
      }
    }
  auto dalloc = [&](void **p, size_t bytes) -> int {
    if (cudaMalloc(p, bytes) != cudaSuccess) {
      *p = nullptr;
      return fail(QT_ENOMEM, "cudaMalloc of %zu bytes for the dense operands failed", bytes);
    }
    return QT_OK;
  };
  int rc;
  if ((rc = dalloc((void **)&s->a_hi, a_elems * 2)) || (rc = dalloc((void **)&s->a_lo, a_elems * 2)) ||
      (rc = dalloc((void **)&s->b_hi, b_elems * 2)) || (rc = dalloc((void **)&s->b_lo, b_elems * 2)) ||
      (rc = dalloc((void **)&s->ydense, (size_t)dp * dp * sizeof(float2))))
    return rc;
  QT_CK(cudaMemcpy(s->a_hi, ahi.data(), a_elems * 2, cudaMemcpyHostToDevice));
  QT_CK(cudaMemcpy(s->a_lo, alo.data(), a_elems * 2, cudaMemcpyHostToDevice));
  QT_CK(cudaMemset(s->b_hi, 0, b_elems * 2));  // rows and columns past d stay zero
  QT_CK(cudaMemset(s->b_lo, 0, b_elems * 2));
  std::memset(&s->tc, 0, sizeof s->tc);
  if ((rc = make_map(&s->tc.a_hi, s->a_hi, 2 * (uint64_t)dp, dp)) ||
      (rc = make_map(&s->tc.a_lo, s->a_lo, 2 * (uint64_t)dp, dp)) ||
      (rc = make_map(&s->tc.b_hi, s->b_hi, 2 * (uint64_t)dp, 2 * (uint64_t)dp)) ||
      (rc = make_map(&s->tc.b_lo, s->b_lo, 2 * (uint64_t)dp, 2 * (uint64_t)dp)))
    return rc;
  s->tc.b_hi_ptr = s->b_hi;
  s->tc.b_lo_ptr = s->b_lo;
  s->tc.Y = s->ydense;
  s->tc.dp = dp;
  if (!s->c_w.empty() && (rc = ensure_dense_collapse(s, dp))) return rc;
  s->dp = dp;
  return QT_OK;
}

}  // namespace

extern "C" {

void qt_opts_default(qt_opts *o) {
  if (!o) return;
  std::memset(o, 0, sizeof *o);
  o->rtol = 1e-8;
  o->atol = 1e-10;
  o->h0 = 0.0;
  o->max_steps = 1000000;
  o->bisect_tol = 1e-13;
  o->precision = QT_FP64;
  o->traj_block = 0;
  o->me_method = QT_ME_AUTO;
}

const char *qt_last_error(void) { return g_err.c_str(); }

const char *qt_version(void) { return "qt-gb300 0.1 (sm_103a)"; }

int qt_system_create(const qt_op *H, const qt_op *c_ops, int n_c, const qt_op *e_ops, int n_e,
                     qt_system *out) {
  return qt_system_create_td(H, nullptr, c_ops, n_c, e_ops, n_e, out);
}

int qt_system_create_td(const qt_op *H, const qt_td *td, const qt_op *c_ops, int n_c,
                        const qt_op *e_ops, int n_e, qt_system *out) {
  g_err.clear();
  if (!out) return fail(QT_EINVAL, "null output handle");
  *out = nullptr;
  if (n_c < 0 || n_e < 0) return fail(QT_EINVAL, "negative operator count");
  if ((n_c > 0 && !c_ops) || (n_e > 0 && !e_ops)) return fail(QT_EINVAL, "null operator list");
  const int n_td = td ? td->n_terms : 0;
  if (n_td < 0 || n_td > qt::kTdMax)
    return fail(QT_EINVAL, "time-dependent terms: 0..%d supported, got %d", qt::kTdMax, n_td);
  int64_t n_knots_total = 0;
  if (n_td > 0) {
    if (!td->H || !td->n_knots || !td->times || !td->values)
      return fail(QT_EINVAL, "time-dependent terms: null array");
    for (int k = 0; k < n_td; ++k) {
      if (td->n_knots[k] < 1) return fail(QT_EINVAL, "time-dependent term %d has no knots", k);
      for (int64_t q = 1; q < td->n_knots[k]; ++q)
        if (!(td->times[n_knots_total + q] > td->times[n_knots_total + q - 1]))
          return fail(QT_EINVAL, "time-dependent term %d: knot times must increase", k);
      for (int64_t q = 0; q < td->n_knots[k]; ++q)
        if (!std::isfinite(td->times[n_knots_total + q]) || !std::isfinite(td->values[n_knots_total + q]))
          return fail(QT_EINVAL, "time-dependent term %d: knot not finite", k);
      n_knots_total += td->n_knots[k];
    }
  }
  Csr Hc;
  int rc = to_csr(H, -1, "H", Hc);
  if (rc) return rc;
  const int d = Hc.d;
  std::vector<Csr> C(n_c), E(n_e);
  for (int n = 0; n < n_c; ++n) {
    char what[32];
    snprintf(what, sizeof what, "c_ops[%d]", n);
    if ((rc = to_csr(&c_ops[n], d, what, C[n]))) return rc;
  }
  for (int n = 0; n < n_e; ++n) {
    char what[32];
    snprintf(what, sizeof what, "e_ops[%d]", n);
    if ((rc = to_csr(&e_ops[n], d, what, E[n]))) return rc;
  }
  std::vector<Csr> Hk(n_td);
  for (int k = 0; k < n_td; ++k) {
    char what[32];
    snprintf(what, sizeof what, "td.H[%d]", k);
    if ((rc = to_csr(&td->H[k], d, what, Hk[k]))) return rc;
  }
  if ((rc = ensure_device())) return rc;

  std::vector<int> cols;
  std::vector<double2> vals;
  qt_system s = new (std::nothrow) qt_system_s();
  if (!s) return fail(QT_ENOMEM, "host allocation");
  s->d = d;
  s->n_c = n_c;
  s->n_e = n_e;
  s->n_td = n_td;
  s->n_ops = 1 + n_c + n_e + n_td;
  auto add = [&](const Csr &A, bool diag_slot = false) {
    s->off_host.push_back((int64_t)cols.size());
    s->w_host.push_back(ell_append(A, cols, vals, diag_slot));
  };
  const Csr heff = effective_hamiltonian(Hc, C);
  add(heff, true);
  DictOp dict;
  const bool have_dict = d > 128 && d <= 2048 && dictionary_form(heff, qt::kDictMaxValues, dict);
  if (have_dict) group_dictionary(d, dict);
  s->heff_col.assign(cols.begin(), cols.end());
  s->heff_val.assign(vals.begin(), vals.end());
  for (const Csr &c : C) add(c);
  {
    int wmax = 0;
    for (int n = 0; n < n_c; ++n) wmax = std::max(wmax, s->w_host[1 + n]);
    if (wmax >= qt::kTcDenseCWidth) {
      const int64_t b = s->off_host[1], e = (int64_t)cols.size();
      s->c_col.assign(cols.begin() + b, cols.begin() + e);
      s->c_val.assign(vals.begin() + b, vals.begin() + e);
      for (int n = 0; n < n_c; ++n) {
        s->c_off.push_back(s->off_host[1 + n] - b);
        s->c_w.push_back(s->w_host[1 + n]);
      }
    }
  }
  for (const Csr &e : E) add(e);
  for (const Csr &h : Hk) add(h);
  s->total_slots = (int64_t)cols.size();
  if (s->total_slots >= ((int64_t)1 << 31)) {
    delete s;
    return fail(QT_ENOTIMPL, "packed operators exceed 2^31 stored entries");
  }
  // FP32 copy of the values, then the FP32 remainders (hi + lo pairs)
  std::vector<float2> v32(2 * vals.size());
  split_fp32(vals, v32);

  auto up = [&](void **dst, const void *src, size_t bytes) -> int {
    cudaError_t e = cudaMalloc(dst, bytes ? bytes : 16);
    if (e != cudaSuccess) {
      *dst = nullptr;
      return fail(QT_ENOMEM, "cudaMalloc: %s", cudaGetErrorString(e));
    }
    if (bytes && src) {
      e = cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
      if (e != cudaSuccess) return fail(QT_ECUDA, "cudaMemcpy: %s", cudaGetErrorString(e));
    }
    return QT_OK;
  };
  if ((rc = up((void **)&s->w_dev, s->w_host.data(), s->w_host.size() * sizeof(int))) ||
      (rc = up((void **)&s->off_dev, s->off_host.data(), s->off_host.size() * sizeof(int64_t))) ||
      (rc = up((void **)&s->col_dev, cols.data(), cols.size() * sizeof(int))) ||
      (rc = up((void **)&s->v64_dev, vals.data(), vals.size() * sizeof(double2))) ||
      (rc = up((void **)&s->v32_dev, v32.data(), v32.size() * sizeof(float2))) ||
      (rc = up((void **)&s->ctl, nullptr, kCtlBytes)) ||
      (rc = up((void **)&s->psi_norm, nullptr, (size_t)d * sizeof(double2)))) {
    delete s;
    return rc;
  }
  if (n_td > 0) {
    std::vector<int64_t> koff(n_td + 1, 0);
    for (int k = 0; k < n_td; ++k) koff[k + 1] = koff[k] + td->n_knots[k];
    if ((rc = up((void **)&s->td_off_dev, koff.data(), koff.size() * sizeof(int64_t))) ||
        (rc = up((void **)&s->td_t_dev, td->times, (size_t)n_knots_total * sizeof(double))) ||
        (rc = up((void **)&s->td_v_dev, td->values, (size_t)n_knots_total * sizeof(double)))) {
      delete s;
      return rc;
    }
  }
  // collapse operators as slots and terms for the Hermitian combine phase
  std::vector<int> slot_off;
  std::vector<int2> terms;
  for (int c = 1; c <= n_c; ++c) {
    const int q0 = (int)slot_off.size();
    for (int q = 0; q < s->w_host[c]; ++q) slot_off.push_back((int)(s->off_host[c] + (int64_t)q * d));
    for (int a = 0; a < s->w_host[c]; ++a)
      for (int b = 0; b < s->w_host[c]; ++b) terms.push_back(make_int2(q0 + a, q0 + b));
  }
  if (!slot_off.empty() && (int)slot_off.size() <= qt::kCSlotsMax &&
      (int)terms.size() <= qt::kCTermsMax) {
    if ((rc = up((void **)&s->cslot_off, slot_off.data(), slot_off.size() * sizeof(int))) ||
        (rc = up((void **)&s->cterms, terms.data(), terms.size() * sizeof(int2)))) {
      delete s;
      return rc;
    }
    s->n_cslots = (int)slot_off.size();
    s->n_cterms = (int)terms.size();
  }
  if (have_dict) {
    // codes, then the diagonal and the table as FP32 hi values followed by
    // their FP32 remainders
    const size_t nc = dict.code.size(), nv = dict.tab.size();
    const size_t b_code = (nc * sizeof(uint32_t) + 15) / 16 * 16;
    std::vector<unsigned char> blob(b_code + 2 * (size_t)d * sizeof(float2) +
                                    2 * nv * sizeof(float2));
    std::memcpy(blob.data(), dict.code.data(), nc * sizeof(uint32_t));
    std::vector<float2> dg(2 * (size_t)d), tb(2 * nv);
    split_fp32(dict.diag, dg);
    split_fp32(dict.tab, tb);
    std::memcpy(blob.data() + b_code, dg.data(), dg.size() * sizeof(float2));
    std::memcpy(blob.data() + b_code + dg.size() * sizeof(float2), tb.data(),
                tb.size() * sizeof(float2));
    if ((rc = up(&s->dict, blob.data(), blob.size()))) {
      delete s;
      return rc;
    }
    s->dict_w = dict.w;
    s->dict_nv = (int)nv;
    s->dict_groups = dict.groups;
    for (int g = 0; g < dict.groups; ++g) s->dict_gend[g] = dict.gend[g];
  }
  // commit the preallocated workspace of qt_mesolve_dev_noalloc on this
  // device now, while device memory is being allocated anyway
  qt::noalloc_prepare();
  *out = s;
  return QT_OK;
}

int qt_system_destroy(qt_system s) {
  if (!s) return QT_OK;
  cudaDeviceSynchronize();
  delete s;
  return QT_OK;
}

int qt_system_dim(qt_system s) { return s ? s->d : QT_EINVAL; }

int qt_mcsolve_dev(qt_system s, const qt_c128 *psi0_dev, const double *tlist_dev, int n_t,
                   int64_t traj_begin, int64_t ntraj, uint64_t seed, const qt_opts *o,
                   qt_c128 *expect_sum_dev, qt_c128 *traj_expect_dev, qt_jump *jumps_dev,
                   int64_t jump_cap, int64_t *n_jumps_dev, qt_stats *stats_dev, void *stream) {
  g_err.clear();
  if (!s) return fail(QT_EINVAL, "null system");
  int rc = check_opts(o);
  if (rc) return rc;
  if (!psi0_dev || !tlist_dev || n_t < 1) return fail(QT_EINVAL, "psi0 and tlist are required");
  if (ntraj < 0 || traj_begin < 0) return fail(QT_EINVAL, "negative trajectory range");
  if (traj_begin + ntraj > ((int64_t)1 << 32))
    return fail(QT_EINVAL, "trajectory index beyond 2^32 (random counter width)");
  if (s->n_e > 0 && !expect_sum_dev) return fail(QT_EINVAL, "expect_sum_dev is required");
  if (jump_cap < 0 || (jump_cap > 0 && !jumps_dev)) return fail(QT_EINVAL, "bad jump buffer");
  if (!qt::mc_supported(s->d, s->w_host[0], o->precision, o->traj_block))
    return fail(QT_ENOTIMPL, "MC kernel for dim %d is not built (dim <= 5120)", s->d);
  if (s->n_td > 0 && s->d > 1024)
    return fail(QT_ENOTIMPL, "MC with time-dependent terms is built for dim <= 1024");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int64_t ntr = (s->n_c == 0 && ntraj > 0) ? 1 : ntraj;
  if ((rc = reset_ctl(s, st))) return rc;
  if (s->n_e > 0)
    QT_CK(cudaMemsetAsync(expect_sum_dev, 0, (size_t)n_t * s->n_e * sizeof(qt_c128), st));
  // the mixed kernel without time-dependent terms reads its output intervals
  // from a table formed once per solve
  double *ivl_tb = nullptr;
  float *ivl_len = nullptr;
  if (o->precision == QT_MIXED && s->n_td == 0 && n_t > 1 && ntr > 0) {
    if ((rc = ensure_ivl(s, n_t))) return rc;
    ivl_tb = static_cast<double *>(s->ivl);
    ivl_len = reinterpret_cast<float *>(ivl_tb + s->ivl_cap);
  }
  QT_CK(qt::launch_normalise(reinterpret_cast<const double2 *>(psi0_dev), s->psi_norm, s->d,
                             s->status(), st, tlist_dev, n_t, ivl_tb, ivl_len));
  qt::McArgs a;
  std::memset(&a, 0, sizeof a);
  a.ivl_tb = ivl_tb;
  a.ivl_len = ivl_len;
  a.ops = s->table();
  a.heff_w = s->w_host[0];
  a.aux_begin = s->n_ops > 1 ? s->off_host[1] : s->total_slots;
  a.aux_slots = s->total_slots - a.aux_begin;
  a.n_c = s->n_c;
  a.n_e = s->n_e;
  a.n_t = n_t;
  a.psi0 = s->psi_norm;
  a.tlist = tlist_dev;
  a.traj_begin = traj_begin;
  a.ntraj = ntr;
  a.seed = seed;
  a.rtol = o->rtol;
  a.atol = o->atol;
  a.h0 = o->h0;
  a.bisect_tol = o->bisect_tol;
  a.max_steps = o->max_steps;
  a.expect_sum = reinterpret_cast<double2 *>(expect_sum_dev);
  a.traj_expect = reinterpret_cast<double2 *>(traj_expect_dev);
  a.jumps = jumps_dev;
  a.jump_cap = jump_cap;
  a.n_jumps = s->n_jumps();
  a.counters = s->counters();
  a.status = s->status();
  a.work = s->work();
  a.n_td = s->n_td;
  a.td_op0 = 1 + s->n_c + s->n_e;
  a.td_off = s->td_off_dev;
  a.td_t = s->td_t_dev;
  a.td_v = s->td_v_dev;
  if (s->dict) {
    const size_t b_code = ((size_t)s->dict_w * s->d * sizeof(uint32_t) + 15) / 16 * 16;
    a.dict_code = reinterpret_cast<const uint32_t *>(s->dict);
    a.dict_diag = reinterpret_cast<const float2 *>(static_cast<char *>(s->dict) + b_code);
    a.dict_tab = a.dict_diag + 2 * (size_t)s->d;
    a.dict_w = s->dict_w;
    a.dict_nv = s->dict_nv;
    a.dict_groups = s->dict_groups;
    for (int g = 0; g < s->dict_groups; ++g) a.dict_gend[g] = s->dict_gend[g];
  }
  if (s->d > 2048) {
    // the stage vectors of one trajectory per CTA, in the system workspace
    const int ctas = qt::mc_stage_ctas();
    if (ctas <= 0) return fail(QT_ECUDA, "cannot size the trajectory launch");
    if ((rc = ensure_ws(s, (size_t)ctas * qt::mc_stage_slab_bytes(o->precision)))) return rc;
    a.stage_ws = s->ws;
    a.stage_ctas = ctas;
  }
  if (ntr > 0) QT_CK(qt::launch_mc(a, o->precision, o->traj_block, st));
  return finish_stats(s, stats_dev, n_jumps_dev, st);
}

int qt_mesolve_dev(qt_system s, const qt_c128 *state0_dev, int state_is_ket,
                   const double *tlist_dev, int n_t, const qt_opts *o, qt_c128 *expect_dev,
                   qt_c128 *states_dev, qt_stats *stats_dev, void *stream) {
  g_err.clear();
  if (!s) return fail(QT_EINVAL, "null system");
  int rc = check_opts(o);
  if (rc) return rc;
  if (!state0_dev || !tlist_dev || n_t < 1) return fail(QT_EINVAL, "state0 and tlist are required");
  if (s->n_e > 0 && !expect_dev) return fail(QT_EINVAL, "expect_dev is required");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  qt::MeArgs a;
  if ((rc = me_setup(s, o, state_is_ket != 0, a))) return rc;
  if ((rc = reset_ctl(s, st))) return rc;
  a.n_t = n_t;
  a.tlist = tlist_dev;
  a.expect = reinterpret_cast<double2 *>(expect_dev);
  a.states = reinterpret_cast<double2 *>(states_dev);
  a.state0 = reinterpret_cast<const double2 *>(state0_dev);
  a.state_is_ket = state_is_ket ? 1 : 0;
  QT_CK(o->me_method == QT_ME_DENSE_TC ? qt::launch_me_tc(a, s->tc, st)
                                       : qt::launch_me(a, o->precision, st));
  return finish_stats(s, stats_dev, nullptr, st);
}

int qt_me_rhs_dev(qt_system s, double t, const qt_c128 *rho_dev, qt_c128 *out_dev,
                  const qt_opts *o, qt_stats *stats_dev, void *stream) {
  g_err.clear();
  if (!s) return fail(QT_EINVAL, "null system");
  int rc = check_opts(o);
  if (rc) return rc;
  if (!rho_dev || !out_dev) return fail(QT_EINVAL, "rho_dev and out_dev are required");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  qt::MeArgs a;
  if ((rc = me_setup(s, o, false, a))) return rc;
  if ((rc = reset_ctl(s, st))) return rc;
  a.n_t = 1;
  a.rhs_in = reinterpret_cast<const double2 *>(rho_dev);
  a.rhs_out = reinterpret_cast<double2 *>(out_dev);
  a.rhs_t = t;
  QT_CK(o->me_method == QT_ME_DENSE_TC ? qt::launch_me_tc(a, s->tc, st)
                                       : qt::launch_me(a, o->precision, st));
  return finish_stats(s, stats_dev, nullptr, st);
}

int qt_correlation_2op_2t_dev(qt_system s, const qt_c128 *state0_dev, int state_is_ket,
                              const double *tlist_dev, int n_t, const double *taulist_dev,
                              int n_tau, int b_index, const qt_opts *o, qt_c128 *corr_dev,
                              qt_stats *stats_dev, void *stream) {
  g_err.clear();
  if (!s) return fail(QT_EINVAL, "null system");
  int rc = check_opts(o);
  if (rc) return rc;
  if (!state0_dev || !tlist_dev || !taulist_dev || n_t < 1 || n_tau < 1)
    return fail(QT_EINVAL, "state0, tlist and taulist are required");
  if (b_index < 0 || b_index >= s->n_e) return fail(QT_EINVAL, "observable index out of range");
  if (!corr_dev) return fail(QT_EINVAL, "corr_dev is required");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int d = s->d;
  const size_t n = (size_t)d * d;
  auto up = [](size_t b) { return (b + 255) / 256 * 256; };
  // store: rho(t_k) [n_t][d][d], the first solve's expectation values, then
  // either one CTA slab per CTA of the batched launch or one X_k + times
  const bool small = d <= qt::kMeSmallDim;
  const int grid = small ? qt::corr_block_grid(n_t, o->precision) : 0;
  if (small && grid <= 0) return fail(QT_ECUDA, "cannot size the correlation launch");
  const size_t elem = o->precision == QT_MIXED ? sizeof(float2) : sizeof(double2);
  qt::CorrArgs c;
  std::memset(&c, 0, sizeof c);
  c.x_off = up(11 * n * elem);
  c.times_off = c.x_off + up(n * sizeof(double2));
  c.ws_stride = c.times_off + up((size_t)n_tau * sizeof(double));
  const size_t states_bytes = up((size_t)n_t * n * sizeof(double2));
  const size_t exp_bytes = up((size_t)n_t * (s->n_e > 0 ? s->n_e : 1) * sizeof(double2));
  const size_t need = states_bytes + exp_bytes + (small ? (size_t)grid : 1) * c.ws_stride;
  if ((rc = ensure_aux(s, need))) return rc;
  char *base = reinterpret_cast<char *>(s->aux);
  double2 *rho_t = reinterpret_cast<double2 *>(base);
  double2 *exp0 = reinterpret_cast<double2 *>(base + states_bytes);
  char *slabs = base + states_bytes + exp_bytes;
  c.rho_t = rho_t;
  c.tlist = tlist_dev;
  c.taulist = taulist_dev;
  c.n_t = n_t;
  c.n_tau = n_tau;
  c.b_op = 1 + s->n_c + b_index;

  // X_k = B rho(t_k) over tau: the general solver (X_k is not Hermitian).
  // Both solves' workspace is sized before the first launch (a later growth
  // would free memory that the first solve may still be using).
  qt_opts o2 = *o;
  if (o2.me_method == QT_ME_DENSE_TC) o2.me_method = QT_ME_AUTO;
  qt::MeArgs a, b;
  if (!small && (rc = me_setup(s, &o2, false, b))) return rc;
  void *ws_before = s->ws;
  if ((rc = me_setup(s, o, state_is_ket != 0, a))) return rc;
  if (!small && s->ws != ws_before && (rc = me_setup(s, &o2, false, b))) return rc;

  // rho(t_k): the master equation with the caller's method
  if ((rc = reset_ctl(s, st))) return rc;
  a.n_t = n_t;
  a.tlist = tlist_dev;
  a.expect = exp0;
  a.states = rho_t;
  a.state0 = reinterpret_cast<const double2 *>(state0_dev);
  a.state_is_ket = state_is_ket ? 1 : 0;
  QT_CK(o->me_method == QT_ME_DENSE_TC ? qt::launch_me_tc(a, s->tc, st)
                                       : qt::launch_me(a, o->precision, st));

  // the tau evolutions
  double2 *corr = reinterpret_cast<double2 *>(corr_dev);
  if (small) {
    me_args(s, &o2, 1, slabs, b);
    b.n_t = n_tau;
    b.expect = corr;
    b.state_is_ket = 0;
    b.herm = 0;
    QT_CK(qt::launch_corr_block(b, c, grid, o->precision, st));
  } else {
    double2 *X = reinterpret_cast<double2 *>(slabs + c.x_off);
    double *times = reinterpret_cast<double *>(slabs + c.times_off);
    b.n_t = n_tau;
    b.tlist = times;
    b.states = nullptr;
    b.state0 = X;
    b.state_is_ket = 0;
    for (int k = 0; k < n_t; ++k) {
      QT_CK(qt::launch_corr_prepare(b.ops, c, k, X, times, st));
      b.expect = corr + (size_t)k * n_tau * s->n_e;
      QT_CK(qt::launch_me(b, o->precision, st));
    }
  }
  return finish_stats(s, stats_dev, nullptr, st);
}

int qt_steadystate_dev(qt_system s, double tol, int64_t max_iter, int krylov_dim,
                       qt_c128 *rho_dev, double *info_dev, qt_stats *stats_dev, void *stream) {
  g_err.clear();
  if (!s) return fail(QT_EINVAL, "null system");
  if (!rho_dev) return fail(QT_EINVAL, "rho_dev is required");
  if (!(tol > 0.0) || max_iter < 0) return fail(QT_EINVAL, "tol must be > 0 and max_iter >= 0");
  if (s->n_td > 0)
    return fail(QT_ENOTIMPL, "the steady state is defined for time-independent Hamiltonians");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int d = s->d;
  const size_t n = (size_t)d * d;
  int m = krylov_dim > 0 ? krylov_dim : 600;
  if (m > 4096) return fail(QT_EINVAL, "krylov_dim must be <= 4096");
  // the grid: every resident CTA; each owns a chunk of the d*d entries held
  // in shared memory (at most 200 KB per CTA)
  constexpr size_t kSmemMax = 200 * 1024;
  int grid = qt::gmres_grid(0);
  if (grid <= 0) return fail(QT_ECUDA, "cannot size the cooperative launch");
  int chunk = 0;
  size_t smem = 0;
  for (int pass = 0; pass < 2; ++pass) {
    chunk = (int)((n + grid - 1) / grid);
    smem = qt::gmres_smem_bytes(chunk, m);
    if (smem > kSmemMax)
      return fail(QT_ENOTIMPL,
                  "dim %d with krylov_dim %d needs %zu bytes of shared memory per CTA; use a "
                  "smaller krylov_dim or qt_propagator_steadystate",
                  d, m, smem);
    const int g2 = qt::gmres_grid(smem);
    if (g2 <= 0) return fail(QT_ECUDA, "cannot size the cooperative launch");
    if (g2 >= grid) break;
    grid = g2;  // fewer resident CTAs with this much shared memory: larger chunks
  }
  if (qt::gmres_grid(smem) < grid)
    return fail(QT_ENOTIMPL, "dim %d with krylov_dim %d does not fit one cooperative launch", d,
                m);
  int rc;
  // solver workspace (grid_sum partials) and the GMRES store
  if ((rc = ensure_ws(s, qt::me_workspace_bytes(d, QT_FP64, grid)))) return rc;
  auto up = [](size_t b) { return (b + 255) / 256 * 256; };
  const size_t vb = up(n * sizeof(double2));
  const size_t need = (size_t)(m + 1) * vb + 3 * vb + up((size_t)grid * (m + 1) * sizeof(double2)) +
                      up((size_t)(m + 1) * sizeof(double2)) +
                      up((size_t)(m + 1) * m * sizeof(double2)) + up((size_t)m * sizeof(double2)) +
                      256;
  if ((rc = ensure_aux(s, need))) return rc;
  char *p = reinterpret_cast<char *>(s->aux);
  qt::GmArgs g;
  g.tol = tol;
  g.max_iter = max_iter;
  g.m = m;
  g.chunk = chunk;
  g.V = reinterpret_cast<double2 *>(p);
  p += (size_t)(m + 1) * vb;
  g.x = reinterpret_cast<double2 *>(p);
  g.zu = reinterpret_cast<double2 *>(p + vb);
  g.minv = reinterpret_cast<double2 *>(p + 2 * vb);
  p += 3 * vb;
  g.pd = reinterpret_cast<double2 *>(p);
  p += up((size_t)grid * (m + 1) * sizeof(double2));
  g.hcol = reinterpret_cast<double2 *>(p);
  p += up((size_t)(m + 1) * sizeof(double2));
  g.R = reinterpret_cast<double2 *>(p);
  p += up((size_t)(m + 1) * m * sizeof(double2));
  g.y = reinterpret_cast<double2 *>(p);
  p += up((size_t)m * sizeof(double2));
  g.ctl = reinterpret_cast<double *>(p);
  g.rho_out = reinterpret_cast<double2 *>(rho_dev);
  g.info = info_dev;
  qt_opts o;
  qt_opts_default(&o);
  qt::MeArgs a;
  me_args(s, &o, grid, s->ws, a);
  if ((rc = reset_ctl(s, st))) return rc;
  QT_CK(qt::launch_gmres(a, g, grid, smem, st));
  return finish_stats(s, stats_dev, nullptr, st);
}

int qt_propagator_steadystate_dev(qt_system s, const qt_c128 *rho0_dev, double period,
                                  double tol, int64_t max_periods, const qt_opts *o,
                                  qt_c128 *rho_dev, double *info, qt_stats *stats_dev,
                                  void *stream) {
  g_err.clear();
  if (!s) return fail(QT_EINVAL, "null system");
  int rc = check_opts(o);
  if (rc) return rc;
  if (!rho_dev) return fail(QT_EINVAL, "rho_dev is required");
  if (!(period > 0.0) || !std::isfinite(period) || !(tol > 0.0) || max_periods < 1)
    return fail(QT_EINVAL, "period and tol must be > 0, max_periods >= 1");
  if (s->n_td > 0)
    return fail(QT_ENOTIMPL, "the propagator steady state is built for time-independent "
                             "Hamiltonians");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int d = s->d;
  const size_t n = (size_t)d * d;
  // store: tlist {0, T}, the change of the last period, states rho_k, rho_k+1
  const size_t need = 256 + 2 * n * sizeof(double2) + std::max<size_t>(s->n_e, 1) * 2 * sizeof(double2);
  if ((rc = ensure_aux(s, need))) return rc;
  char *base = reinterpret_cast<char *>(s->aux);
  double *tl = reinterpret_cast<double *>(base);
  double *dnorm = tl + 2;
  double2 *B = reinterpret_cast<double2 *>(base + 256);
  double2 *ex = B + 2 * n;
  qt::MeArgs a;
  if ((rc = me_setup(s, o, false, a))) return rc;
  if ((rc = reset_ctl(s, st))) return rc;
  const double hl[2] = {0.0, period};
  QT_CK(cudaMemcpyAsync(tl, hl, sizeof hl, cudaMemcpyHostToDevice, st));
  if (rho0_dev)
    QT_CK(cudaMemcpyAsync(B + n, rho0_dev, n * sizeof(double2), cudaMemcpyDeviceToDevice, st));
  else
    QT_CK(qt::launch_identity_state(B + n, d, st));
  a.n_t = 2;
  a.tlist = tl;
  a.expect = ex;
  a.states = B;  // rho_k is copied to B[0, n), rho_k+1 written to B[n, 2n)
  a.state0 = B + n;
  a.state_is_ket = 0;
  // the change per period falls geometrically until it meets the integration
  // error of one period; 50 periods without a new minimum end the loop there
  double h = 0.0, best = HUGE_VAL;
  int64_t k = 0, k_best = 0;
  bool stalled = false;
  for (; k < max_periods;) {
    QT_CK(o->me_method == QT_ME_DENSE_TC ? qt::launch_me_tc(a, s->tc, st)
                                         : qt::launch_me(a, o->precision, st));
    ++k;
    QT_CK(qt::launch_diff_norm(B, B + n, (int64_t)n, dnorm, st));
    int status = QT_OK;
    QT_CK(cudaMemcpyAsync(&h, dnorm, sizeof h, cudaMemcpyDeviceToHost, st));
    QT_CK(cudaMemcpyAsync(&status, s->status(), sizeof status, cudaMemcpyDeviceToHost, st));
    QT_CK(cudaStreamSynchronize(st));
    if (status != QT_OK || !std::isfinite(h) || h <= tol) break;
    if (h < best) {
      best = h;
      k_best = k;
    } else if (k - k_best >= 50) {
      stalled = true;
      break;
    }
  }
  QT_CK(cudaMemcpyAsync(rho_dev, B + n, n * sizeof(double2), cudaMemcpyDeviceToDevice, st));
  if (info) {
    info[0] = h;
    info[1] = (double)k;
  }
  if (!std::isfinite(h)) QT_CK(qt::launch_set_status(s->status(), QT_ENUMERIC, st));
  else if (h > tol) QT_CK(qt::launch_set_status(s->status(), QT_ESTEP, st));
  return finish_stats(s, stats_dev, nullptr, st);
}

int qt_propagator_dev(qt_system s, const double *tlist_dev, int n_t, const qt_opts *o,
                      qt_c128 *U_dev, qt_stats *stats_dev, void *stream) {
  g_err.clear();
  if (!s) return fail(QT_EINVAL, "null system");
  int rc = check_opts(o);
  if (rc) return rc;
  if (!tlist_dev || n_t < 1 || !U_dev) return fail(QT_EINVAL, "tlist and U are required");
  const int d = s->d;
  if (d > qt::kMeSmallDim)
    return fail(QT_ENOTIMPL, "the propagator is built for dim <= %d (dim^4 entries per time)",
                qt::kMeSmallDim);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int64_t n = (int64_t)d * d;
  const int grid = qt::prop_block_grid(n, o->precision);
  if (grid <= 0) return fail(QT_ECUDA, "cannot size the propagator launch");
  auto up = [](size_t b) { return (b + 255) / 256 * 256; };
  const size_t elem = o->precision == QT_MIXED ? sizeof(float2) : sizeof(double2);
  qt::PropArgs p;
  p.U = reinterpret_cast<double2 *>(U_dev);
  p.x_off = up(11 * (size_t)n * elem);
  p.st_off = p.x_off + up((size_t)n * sizeof(double2));
  p.ws_stride = p.st_off + up((size_t)n_t * n * sizeof(double2));
  if ((rc = ensure_aux(s, (size_t)grid * p.ws_stride))) return rc;
  qt_opts o2 = *o;
  if (o2.me_method == QT_ME_DENSE_TC) o2.me_method = QT_ME_AUTO;
  qt::MeArgs a;
  me_args(s, &o2, 1, s->aux, a);
  a.n_t = n_t;
  a.tlist = tlist_dev;
  a.expect = nullptr;
  a.states = nullptr;
  a.state_is_ket = 0;
  a.herm = 0;
  if ((rc = reset_ctl(s, st))) return rc;
  QT_CK(qt::launch_prop_block(a, p, grid, o->precision, st));
  return finish_stats(s, stats_dev, nullptr, st);
}

int qt_expect_dev(qt_system s, int e_index, const qt_c128 *states_dev, int is_ket,
                  int64_t batch, qt_c128 *out_dev, void *stream) {
  g_err.clear();
  if (!s) return fail(QT_EINVAL, "null system");
  if (e_index < 0 || e_index >= s->n_e) return fail(QT_EINVAL, "observable index out of range");
  if (batch < 0 || (batch > 0 && (!states_dev || !out_dev)))
    return fail(QT_EINVAL, "bad state batch");
  QT_CK(qt::launch_expect(s->table(), 1 + s->n_c + e_index,
                          reinterpret_cast<const double2 *>(states_dev), is_ket, batch,
                          reinterpret_cast<double2 *>(out_dev),
                          reinterpret_cast<cudaStream_t>(stream)));
  return QT_OK;
}

}  // extern "C"

namespace qt {

int set_error(int code, const char *msg) { return fail(code, "%s", msg); }

int mesolve_dev_ws(qt_system s, const qt_c128 *state0_dev, int state_is_ket,
                   const double *tlist_dev, int n_t, const qt_opts *o, qt_c128 *expect_dev,
                   qt_c128 *states_dev, qt_stats *stats_dev, void *stream, void *ws,
                   size_t ws_bytes) {
  g_err.clear();
  if (!s) return fail(QT_EINVAL, "null system");
  int rc = check_opts(o);
  if (rc) return rc;
  if (o->me_method == QT_ME_DENSE_TC)
    return fail(QT_ENOTIMPL, "the tensor-core method allocates its dense operands; it has no "
                             "preallocated-workspace form");
  if (!state0_dev || !tlist_dev || n_t < 1) return fail(QT_EINVAL, "state0 and tlist are required");
  if (s->n_e > 0 && !expect_dev) return fail(QT_EINVAL, "expect_dev is required");
  if (!ws) return fail(QT_EINVAL, "null workspace");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int grid = qt::me_grid(s->d, o->precision);
  if (grid <= 0) return fail(QT_ECUDA, "cannot size the cooperative launch");
  // sized for the largest grid the launch can use on any device, so that the
  // accepted dimensions do not depend on the device
  const int64_t d2 = (int64_t)s->d * s->d;
  const int worst = (int)std::max<int64_t>(grid, (d2 + 255) / 256);
  const size_t need = qt::me_workspace_bytes(s->d, o->precision, worst);
  if (need > ws_bytes)
    return fail(QT_EINVAL,
                "dim %d in %s precision needs %zu bytes of solver workspace; the "
                "preallocated workspace holds %zu bytes",
                s->d, o->precision == QT_MIXED ? "mixed" : "FP64", need, ws_bytes);
  if ((rc = reset_ctl(s, st))) return rc;
  qt::MeArgs a;
  me_args(s, o, grid, ws, a);
  a.n_t = n_t;
  a.tlist = tlist_dev;
  a.expect = reinterpret_cast<double2 *>(expect_dev);
  a.states = reinterpret_cast<double2 *>(states_dev);
  a.state0 = reinterpret_cast<const double2 *>(state0_dev);
  a.state_is_ket = state_is_ket ? 1 : 0;
  QT_CK(qt::launch_me(a, o->precision, st));
  return finish_stats(s, stats_dev, nullptr, st);
}

}  // namespace qt

extern "C" {

// ------------------------------------------------------------------ batches

}  // extern "C"

struct qt_batch_s {
  int n = 0, dmax = 1;
  std::vector<int> kind, dim, n_e, heff_w;
  std::vector<int64_t> ntraj, expect_base;  // expect offsets per unit n_t
  std::vector<double> me_cost;              // per master-equation item
  std::vector<double> mc_cost_per_traj;     // per trajectory of a Monte-Carlo item
  int64_t expect_units = 0;                 // sum of n_e
  std::vector<void *> dev;                  // every device allocation
  qt::BatchProblem *probs = nullptr;
  qt::BatchItem *items = nullptr;
  int items_cap = 0, n_items = 0, tb = 64;
  int small_group_dim = 0;                  // MC items up to this dim: half-warp groups
  double tuned_ms = 0.0;                    // the tuner's best time (0: not tuned)
  unsigned long long *ctl = nullptr;        // counters[6], n_jumps, next_item, status
  unsigned long long *item_work = nullptr;
  unsigned long long *prob_ctl = nullptr;   // [n][6] statistics per problem
  void *ws = nullptr;
  size_t ws_stride = 0;
  int grid = 0;
  ~qt_batch_s() {
    for (void *p : dev)
      if (p) cudaFree(p);
  }
  void *alloc(size_t bytes) {
    void *p = nullptr;
    if (cudaMalloc(&p, bytes ? bytes : 16) != cudaSuccess) return nullptr;
    dev.push_back(p);
    return p;
  }
  void release(void *p) {
    for (void *&q : dev)
      if (q == p) {
        cudaFree(q);
        q = nullptr;
      }
  }
};

namespace {

// Work items for Monte-Carlo blocks of tb trajectories, sorted by estimated
// cost, largest first.
int build_items(qt_batch b, int tb) {
  struct Item {
    qt::BatchItem it;
    double cost;
  };
  std::vector<Item> items;
  for (int p = 0; p < b->n; ++p) {
    if (b->kind[p] == QT_KIND_ME) {
      items.push_back({{p, 0, 0, 0}, b->me_cost[p]});
    } else {
      for (int64_t t0 = 0; t0 < b->ntraj[p]; t0 += tb) {
        const int64_t nb = std::min<int64_t>(tb, b->ntraj[p] - t0);
        items.push_back({{p, 0, t0, nb}, b->mc_cost_per_traj[p] * (double)nb});
      }
    }
  }
  std::stable_sort(items.begin(), items.end(),
                   [](const Item &x, const Item &y) { return x.cost > y.cost; });
  if ((int64_t)items.size() > b->items_cap) {
    // smaller blocks than the creation sized for: grow the item arrays
    if ((int64_t)items.size() >= ((int64_t)1 << 31)) return fail(QT_EINVAL, "too many work items");
    void *ni = b->alloc(items.size() * sizeof(qt::BatchItem));
    void *nw = b->alloc(items.size() * sizeof(unsigned long long));
    if (!ni || !nw) return fail(QT_ENOMEM, "device allocation of the work items failed");
    b->release(b->items);
    b->release(b->item_work);
    b->items = (qt::BatchItem *)ni;
    b->item_work = (unsigned long long *)nw;
    b->items_cap = (int)items.size();
  }
  std::vector<qt::BatchItem> flat(items.size());
  for (size_t i = 0; i < items.size(); ++i) flat[i] = items[i].it;
  if (!flat.empty())
    QT_CK(cudaMemcpy(b->items, flat.data(), flat.size() * sizeof(qt::BatchItem),
                     cudaMemcpyHostToDevice));
  b->n_items = (int)flat.size();
  b->tb = tb;
  return QT_OK;
}

}  // namespace

extern "C" {

int qt_batch_create(const qt_problem *problems, int n_problems, qt_batch *out) {
  g_err.clear();
  if (!out) return fail(QT_EINVAL, "null output handle");
  *out = nullptr;
  if (!problems || n_problems < 1) return fail(QT_EINVAL, "empty batch");
  int rc;
  std::vector<int> cols, w_all;
  std::vector<int64_t> off_all;
  std::vector<int> off32_all;
  std::vector<double2> vals, states;
  struct PInfo {
    int d, n_ops, wbase;
    int64_t sbase;
  };
  std::vector<PInfo> info(n_problems);
  qt_batch b = new (std::nothrow) qt_batch_s();
  if (!b) return fail(QT_ENOMEM, "host allocation");
  b->n = n_problems;
  int64_t item_bound = 0;
  for (int p = 0; p < n_problems; ++p) {
    const qt_problem &P = problems[p];
    char what[48];
    if (P.kind != QT_KIND_ME && P.kind != QT_KIND_MC) {
      delete b;
      return fail(QT_EINVAL, "problem %d: unknown kind %d", p, P.kind);
    }
    if (P.n_c < 0 || P.n_e < 0 || (P.n_c > 0 && !P.c_ops) || (P.n_e > 0 && !P.e_ops) ||
        !P.state0) {
      delete b;
      return fail(QT_EINVAL, "problem %d: bad operator list or state", p);
    }
    Csr Hc;
    snprintf(what, sizeof what, "problem %d H", p);
    if ((rc = to_csr(P.H, -1, what, Hc))) { delete b; return rc; }
    const int d = Hc.d;
    if (d > 64) {
      delete b;
      return fail(QT_ENOTIMPL, "problem %d: dim %d > 64 is not supported in a batch", p, d);
    }
    if (P.kind == QT_KIND_MC && !P.state_is_ket) {
      delete b;
      return fail(QT_EINVAL, "problem %d: Monte-Carlo problems start from a ket", p);
    }
    std::vector<Csr> C(P.n_c), E(P.n_e);
    for (int n = 0; n < P.n_c; ++n) {
      snprintf(what, sizeof what, "problem %d c_ops[%d]", p, n);
      if ((rc = to_csr(&P.c_ops[n], d, what, C[n]))) { delete b; return rc; }
    }
    for (int n = 0; n < P.n_e; ++n) {
      snprintf(what, sizeof what, "problem %d e_ops[%d]", p, n);
      if ((rc = to_csr(&P.e_ops[n], d, what, E[n]))) { delete b; return rc; }
    }
    PInfo &pi = info[p];
    pi.d = d;
    pi.n_ops = 1 + P.n_c + P.n_e;
    pi.wbase = (int)w_all.size();
    auto add = [&](const Csr &A, bool diag_slot = false) {
      const int64_t off = (int64_t)cols.size();
      w_all.push_back(ell_append(A, cols, vals, diag_slot));
      off_all.push_back(off);
      off32_all.push_back((int)off);
    };
    const Csr He = effective_hamiltonian(Hc, C);
    add(He, true);
    int wsum_c2 = 0;
    for (const Csr &c : C) {
      add(c);
      wsum_c2 += w_all.back() * w_all.back();
    }
    for (const Csr &e : E) add(e);
    // initial state: MC kets normalised here in FP64; ME states as given
    pi.sbase = (int64_t)states.size();
    const int64_t ns = P.state_is_ket ? d : (int64_t)d * d;
    double nrm = 0.0;
    for (int64_t i = 0; i < ns; ++i) nrm += P.state0[i].re * P.state0[i].re + P.state0[i].im * P.state0[i].im;
    if (!(nrm > 0.0) || !std::isfinite(nrm)) {
      delete b;
      return fail(QT_ENORM, "problem %d: zero or non-finite initial state", p);
    }
    const double sc = (P.kind == QT_KIND_MC) ? 1.0 / std::sqrt(nrm) : 1.0;
    for (int64_t i = 0; i < ns; ++i)
      states.push_back(make_double2(P.state0[i].re * sc, P.state0[i].im * sc));
    const int64_t nt = (P.kind == QT_KIND_MC) ? ((P.n_c == 0 && P.ntraj > 0) ? 1 : P.ntraj) : 0;
    if (P.kind == QT_KIND_MC && nt < 0) {
      delete b;
      return fail(QT_EINVAL, "problem %d: negative ntraj", p);
    }
    b->kind.push_back(P.kind);
    b->dim.push_back(d);
    b->n_e.push_back(P.n_e);
    b->heff_w.push_back(w_all[pi.wbase]);
    b->ntraj.push_back(nt);
    b->expect_base.push_back(b->expect_units);
    b->expect_units += P.n_e;
    b->me_cost.push_back((double)d * d * (2.0 * w_all[pi.wbase] + wsum_c2));
    b->mc_cost_per_traj.push_back(2.0 * d * w_all[pi.wbase]);
    b->dmax = std::max(b->dmax, d);
    item_bound += (P.kind == QT_KIND_ME) ? 1 : (nt + 31) / 32;
  }
  if ((int64_t)cols.size() >= ((int64_t)1 << 31)) {
    delete b;
    return fail(QT_ENOTIMPL, "packed operators exceed 2^31 stored entries");
  }
  if ((rc = ensure_device())) { delete b; return rc; }
  std::vector<float2> v32(2 * vals.size());
  split_fp32(vals, v32);
  auto up = [&](const void *src, size_t bytes) -> void * {
    void *d = b->alloc(bytes);
    if (d && bytes && src && cudaMemcpy(d, src, bytes, cudaMemcpyHostToDevice) != cudaSuccess)
      return nullptr;
    return d;
  };
  int *w_dev = (int *)up(w_all.data(), w_all.size() * sizeof(int));
  int64_t *off_dev = (int64_t *)up(off_all.data(), off_all.size() * sizeof(int64_t));
  int *off32_dev = (int *)up(off32_all.data(), off32_all.size() * sizeof(int));
  int *col_dev = (int *)up(cols.data(), cols.size() * sizeof(int));
  double2 *v64_dev = (double2 *)up(vals.data(), vals.size() * sizeof(double2));
  float2 *v32_dev = (float2 *)up(v32.data(), v32.size() * sizeof(float2));
  double2 *st_dev = (double2 *)up(states.data(), states.size() * sizeof(double2));
  if (!w_dev || !off_dev || !off32_dev || !col_dev || !v64_dev || !v32_dev || !st_dev) {
    delete b;
    return fail(QT_ENOMEM, "device allocation or upload of the batch failed");
  }
  std::vector<qt::BatchProblem> probs(n_problems);
  for (int p = 0; p < n_problems; ++p) {
    const PInfo &pi = info[p];
    qt::BatchProblem &q = probs[p];
    std::memset(&q, 0, sizeof q);
    q.ops.d = pi.d;
    q.ops.n_ops = pi.n_ops;
    q.ops.w = w_dev + pi.wbase;
    q.ops.off = off_dev + pi.wbase;
    q.ops.col = col_dev;
    q.ops.val64 = v64_dev;
    q.ops.val32 = v32_dev;
    q.ops.val32lo = v32_dev + vals.size();
    q.opoff32 = off32_dev + pi.wbase;
    q.kind = problems[p].kind;
    q.n_c = problems[p].n_c;
    q.n_e = problems[p].n_e;
    q.state_is_ket = problems[p].state_is_ket ? 1 : 0;
    q.ntraj = b->ntraj[p];
    q.seed = problems[p].seed;
    q.state0 = st_dev + pi.sbase;
    q.expect_off = b->expect_base[p];
  }
  b->probs = (qt::BatchProblem *)up(probs.data(), probs.size() * sizeof(qt::BatchProblem));
  b->items_cap = (int)std::max<int64_t>(item_bound, 1);
  b->items = (qt::BatchItem *)b->alloc((size_t)b->items_cap * sizeof(qt::BatchItem));
  b->item_work = (unsigned long long *)b->alloc((size_t)b->items_cap * sizeof(unsigned long long));
  b->ctl = (unsigned long long *)b->alloc(kCtlBytes);
  b->prob_ctl = (unsigned long long *)b->alloc((size_t)std::max(n_problems, 1) * 6 *
                                               sizeof(unsigned long long));
  const int g64 = qt::batch_grid(QT_FP64), g32 = qt::batch_grid(QT_MIXED);
  b->grid = std::max(g64, g32);
  b->ws_stride = qt::batch_ws_stride(b->dmax, QT_FP64);
  if (b->grid <= 0) {
    delete b;
    return fail(QT_ECUDA, "cannot size the batch launch");
  }
  b->ws = b->alloc((size_t)b->grid * b->ws_stride);
  if (!b->probs || !b->items || !b->item_work || !b->ctl || !b->prob_ctl || !b->ws) {
    delete b;
    return fail(QT_ENOMEM, "device allocation of the batch failed");
  }
  if ((rc = build_items(b, 64))) { delete b; return rc; }
  *out = b;
  return QT_OK;
}

int qt_batch_destroy(qt_batch b) {
  if (!b) return QT_OK;
  cudaDeviceSynchronize();
  delete b;
  return QT_OK;
}

int64_t qt_batch_expect_offset(qt_batch b, int p, int n_t) {
  if (!b || p < 0 || p > b->n || n_t < 0) return QT_EINVAL;
  return (p == b->n ? b->expect_units : b->expect_base[p]) * (int64_t)n_t;
}

int qt_batch_solve_dev(qt_batch b, const double *tlist_dev, int n_t, const qt_opts *o,
                       qt_c128 *expect_dev, qt_stats *stats_dev, void *stream) {
  g_err.clear();
  if (!b) return fail(QT_EINVAL, "null batch");
  int rc = check_opts(o);
  if (rc) return rc;
  if (o->me_method == QT_ME_DENSE_TC)
    return fail(QT_ENOTIMPL, "batches solve master equations on the sparse path only");
  if (!tlist_dev || n_t < 1) return fail(QT_EINVAL, "tlist is required");
  if (b->expect_units > 0 && !expect_dev) return fail(QT_EINVAL, "expect_dev is required");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  QT_CK(cudaMemsetAsync(b->ctl, 0, kCtlBytes, st));
  QT_CK(cudaMemsetAsync(b->prob_ctl, 0, (size_t)std::max(b->n, 1) * 6 * sizeof(unsigned long long),
                        st));
  if (b->n_items > 0)
    QT_CK(cudaMemsetAsync(b->item_work, 0, (size_t)b->n_items * sizeof(unsigned long long), st));
  if (b->expect_units > 0)
    QT_CK(cudaMemsetAsync(expect_dev, 0, (size_t)b->expect_units * n_t * sizeof(qt_c128), st));
  qt::BatchArgs a;
  std::memset(&a, 0, sizeof a);
  a.probs = b->probs;
  a.items = b->items;
  a.n_items = b->n_items;
  a.n_problems = b->n;
  a.tlist = tlist_dev;
  a.n_t = n_t;
  a.rtol = o->rtol;
  a.atol = o->atol;
  a.h0 = o->h0;
  a.bisect_tol = o->bisect_tol;
  a.max_steps = o->max_steps;
  a.expect = reinterpret_cast<double2 *>(expect_dev);
  a.item_work = b->item_work;
  a.next_item = b->ctl + 7;
  a.counters = b->ctl;
  a.prob_counters = b->prob_ctl;
  a.n_jumps = b->ctl + 6;
  a.status = reinterpret_cast<int *>(b->ctl + 8);
  a.ws = b->ws;
  a.ws_stride = b->ws_stride;
  a.small_group_dim = b->small_group_dim;
  const int grid = qt::batch_grid(o->precision);
  if (grid <= 0) return fail(QT_ECUDA, "cannot size the batch launch");
  QT_CK(qt::launch_batch(a, o->precision, std::min(grid, b->grid), st));
  QT_CK(qt::launch_batch_finalize(a, st));
  if (stats_dev)
    QT_CK(qt::launch_finalize_stats(a.counters, a.status, a.n_jumps, stats_dev, st));
  return QT_OK;
}

int qt_batch_problem_stats(qt_batch b, qt_stats *stats) {
  g_err.clear();
  if (!b || !stats) return fail(QT_EINVAL, "null batch or output");
  std::vector<unsigned long long> c((size_t)b->n * 6);
  if (b->n > 0)
    QT_CK(cudaMemcpy(c.data(), b->prob_ctl, c.size() * sizeof(unsigned long long),
                     cudaMemcpyDeviceToHost));
  for (int p = 0; p < b->n; ++p) {
    qt_stats &x = stats[p];
    x.accepted = (int64_t)c[6 * (size_t)p + 0];
    x.rejected = (int64_t)c[6 * (size_t)p + 1];
    x.rhs_evals = (int64_t)c[6 * (size_t)p + 2];
    x.bisect_iters = (int64_t)c[6 * (size_t)p + 3];
    x.jumps = (int64_t)c[6 * (size_t)p + 4];
    x.near_miss = (int64_t)c[6 * (size_t)p + 5];
    x.status = 0;
    x.reserved = 0;
  }
  return QT_OK;
}

int qt_batch_tune(qt_batch b, const double *tlist_dev, int n_t, const qt_opts *o,
                  qt_c128 *expect_dev, void *stream) {
  g_err.clear();
  if (!b) return fail(QT_EINVAL, "null batch");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  QT_CK(cudaEventCreate(&e0));
  QT_CK(cudaEventCreate(&e1));
  // two passes: the trajectory groups of small Monte-Carlo problems (whole
  // warps, or half-warps up to dimension 16 or 32) at the default block, then
  // the trajectory block for the best grouping
  int rc = QT_OK;
  float best_ms = 1e30f;
  int best_tb = 64, best_sgd = 0;
  auto timed = [&](int tb, int sgd, float *ms) -> int {
    int r;
    if ((r = build_items(b, tb))) return r;
    b->small_group_dim = sgd;
    if ((r = qt_batch_solve_dev(b, tlist_dev, n_t, o, expect_dev, nullptr, stream))) return r;
    cudaEventRecord(e0, st);
    if ((r = qt_batch_solve_dev(b, tlist_dev, n_t, o, expect_dev, nullptr, stream))) return r;
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess) return fail(QT_ECUDA, "tuning run failed");
    cudaEventElapsedTime(ms, e0, e1);
    return QT_OK;
  };
  for (int sgd : {0, 16, 32}) {
    float ms = 0.f;
    if ((rc = timed(64, sgd, &ms))) break;
    if (ms < best_ms) { best_ms = ms; best_sgd = sgd; }
  }
  if (!rc)
    for (int tb : {32, 128, 256}) {
      float ms = 0.f;
      if ((rc = timed(tb, best_sgd, &ms))) break;
      if (ms < best_ms) { best_ms = ms; best_tb = tb; }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->small_group_dim = best_sgd;
  if (rc) return rc;
  b->tuned_ms = best_ms;
  return build_items(b, best_tb);
}

int qt_batch_set_config(qt_batch b, int traj_block, int small_group_dim) {
  g_err.clear();
  if (!b) return fail(QT_EINVAL, "null batch");
  if (traj_block < 1 || traj_block > (1 << 20))
    return fail(QT_EINVAL, "traj_block must be in 1 .. 2^20");
  if (small_group_dim != 0 && small_group_dim != 16 && small_group_dim != 32)
    return fail(QT_EINVAL, "small_group_dim must be 0, 16 or 32");
  b->small_group_dim = small_group_dim;
  return build_items(b, traj_block);
}

int qt_batch_config(qt_batch b, int *traj_block, int *small_group_dim, double *tuned_ms) {
  g_err.clear();
  if (!b) return fail(QT_EINVAL, "null batch");
  if (traj_block) *traj_block = b->tb;
  if (small_group_dim) *small_group_dim = b->small_group_dim;
  if (tuned_ms) *tuned_ms = b->tuned_ms;
  return QT_OK;
}

// --------------------------------------------------------------- adjoint

}  // extern "C"

struct qt_adjoint_s {
  int d = 0, nk = 0, n_seg = 0, batch = 0, maxs = 0;
  double t_seg = 0.0;
  qt::OpTable ops;
  std::vector<void *> dev;
  double2 *rho0 = nullptr, *ckpt = nullptr, *work = nullptr;
  int *nsteps = nullptr;
  double *hgrid = nullptr, *omega = nullptr, *gamma = nullptr, *loss = nullptr;
  unsigned long long *ctl = nullptr;
  int64_t slots = 0;
  bool have_forward = false;
  ~qt_adjoint_s() {
    for (void *p : dev)
      if (p) cudaFree(p);
  }
  void *alloc(size_t bytes) {
    void *p = nullptr;
    if (cudaMalloc(&p, bytes ? bytes : 16) != cudaSuccess) return nullptr;
    dev.push_back(p);
    return p;
  }
};

namespace {

Csr csr_dagger(const Csr &A) {
  Csr out;
  out.d = A.d;
  std::vector<std::vector<std::pair<int, cplx>>> rows(A.d);
  for (int i = 0; i < A.d; ++i)
    for (int64_t p = A.ptr[i]; p < A.ptr[i + 1]; ++p) rows[A.col[p]].emplace_back(i, std::conj(A.val[p]));
  out.ptr.assign(A.d + 1, 0);
  for (int i = 0; i < A.d; ++i) {
    std::sort(rows[i].begin(), rows[i].end(),
              [](const std::pair<int, cplx> &x, const std::pair<int, cplx> &y) { return x.first < y.first; });
    for (auto &e : rows[i]) { out.col.push_back(e.first); out.val.push_back(e.second); }
    out.ptr[i + 1] = (int64_t)out.col.size();
  }
  return out;
}

// A^dag A, from the effective-Hamiltonian builder: H_eff(0, {A}) = -(i/2) A^dag A.
Csr dagger_product(const Csr &A) {
  Csr zero;
  zero.d = A.d;
  zero.ptr.assign(A.d + 1, 0);
  Csr h = effective_hamiltonian(zero, {A});
  for (auto &v : h.val) v *= cplx(0.0, 2.0);  // (2i)(-(i/2) A^dag A) = A^dag A
  return h;
}

bool hermitian(const Csr &A) {
  Csr ad = csr_dagger(A);
  if (ad.col != A.col || ad.ptr != A.ptr) return false;
  for (size_t q = 0; q < A.val.size(); ++q)
    if (std::abs(A.val[q] - ad.val[q]) > 1e-12 * (1.0 + std::abs(A.val[q]))) return false;
  return true;
}

qt::AdjArgs adj_args(qt_adjoint a) {
  qt::AdjArgs x;
  std::memset(&x, 0, sizeof x);
  x.ops = a->ops;
  x.nk = a->nk;
  x.n_seg = a->n_seg;
  x.batch = a->batch;
  x.maxs = a->maxs;
  x.t_seg = a->t_seg;
  x.rho0 = a->rho0;
  x.nsteps = a->nsteps;
  x.hgrid = a->hgrid;
  x.ckpt = a->ckpt;
  x.work = a->work;
  x.slots = a->slots;
  x.counters = a->ctl;
  x.status = reinterpret_cast<int *>(a->ctl + 8);
  x.max_steps = 1000000;
  return x;
}

}  // namespace

extern "C" {

int qt_adjoint_create(const qt_op *H0, const qt_op *Hd, const qt_op *A, int n_k, const qt_op *P1,
                      const qt_op *P2, const qt_c128 *state0, int state_is_ket, int n_seg,
                      double t_seg, int batch, int max_per_seg, qt_adjoint *out) {
  g_err.clear();
  if (!out) return fail(QT_EINVAL, "null output handle");
  *out = nullptr;
  if (n_k < 0 || n_k > 8 || (n_k > 0 && !A)) return fail(QT_EINVAL, "need 0 <= n_k <= 8");
  if (n_seg < 1 || !(t_seg > 0.0) || batch < 1 || max_per_seg < 1 || !state0)
    return fail(QT_EINVAL, "bad segments, batch, step bound or state");
  int rc;
  Csr h0, hd, p1, p2;
  if ((rc = to_csr(H0, -1, "H0", h0))) return rc;
  const int d = h0.d;
  if (d > 64) return fail(QT_ENOTIMPL, "adjoint for dim %d > 64 is not built", d);
  if ((rc = to_csr(Hd, d, "Hd", hd)) || (rc = to_csr(P1, d, "P1", p1)) ||
      (rc = to_csr(P2, d, "P2", p2)))
    return rc;
  for (const Csr *m : {&h0, &hd, &p1, &p2})
    if (!hermitian(*m)) return fail(QT_ENONHERM, "H0, Hd, P1 and P2 must be Hermitian");
  std::vector<Csr> Ak(n_k);
  for (int k = 0; k < n_k; ++k) {
    char what[32];
    snprintf(what, sizeof what, "A[%d]", k);
    if ((rc = to_csr(&A[k], d, what, Ak[k]))) return rc;
  }
  if ((rc = ensure_device())) return rc;
  qt_adjoint a = new (std::nothrow) qt_adjoint_s();
  if (!a) return fail(QT_ENOMEM, "host allocation");
  a->d = d;
  a->nk = n_k;
  a->n_seg = n_seg;
  a->t_seg = t_seg;
  a->batch = batch;
  a->maxs = max_per_seg;
  std::vector<int> cols, w;
  std::vector<int64_t> off;
  std::vector<double2> vals;
  auto add = [&](const Csr &m) {
    off.push_back((int64_t)cols.size());
    w.push_back(ell_append(m, cols, vals));
  };
  add(h0);
  add(hd);
  for (const Csr &m : Ak) add(m);
  for (const Csr &m : Ak) add(csr_dagger(m));
  for (const Csr &m : Ak) add(dagger_product(m));
  add(p1);
  add(p2);
  // rho0
  std::vector<double2> rho((size_t)d * d);
  if (state_is_ket) {
    double nrm = 0.0;
    for (int i = 0; i < d; ++i) nrm += state0[i].re * state0[i].re + state0[i].im * state0[i].im;
    if (!(nrm > 0.0)) { delete a; return fail(QT_ENORM, "zero initial ket"); }
    for (int i = 0; i < d; ++i)
      for (int j = 0; j < d; ++j) {
        const cplx v = cplx(state0[i].re, state0[i].im) * std::conj(cplx(state0[j].re, state0[j].im)) / nrm;
        rho[(size_t)i * d + j] = make_double2(v.real(), v.imag());
      }
  } else {
    for (size_t q = 0; q < rho.size(); ++q) rho[q] = make_double2(state0[q].re, state0[q].im);
  }
  auto up = [&](const void *src, size_t bytes) -> void * {
    void *p = a->alloc(bytes);
    if (p && src && bytes && cudaMemcpy(p, src, bytes, cudaMemcpyHostToDevice) != cudaSuccess)
      return nullptr;
    return p;
  };
  const int64_t n = (int64_t)d * d;
  a->slots = (int64_t)qt::adjoint_slots(max_per_seg);
  a->ops.d = d;
  a->ops.n_ops = (int)w.size();
  a->ops.w = (int *)up(w.data(), w.size() * sizeof(int));
  a->ops.off = (int64_t *)up(off.data(), off.size() * sizeof(int64_t));
  a->ops.col = (int *)up(cols.data(), cols.size() * sizeof(int));
  a->ops.val64 = (double2 *)up(vals.data(), vals.size() * sizeof(double2));
  a->ops.val32 = nullptr;
  a->ops.val32lo = nullptr;
  a->rho0 = (double2 *)up(rho.data(), rho.size() * sizeof(double2));
  a->nsteps = (int *)a->alloc((size_t)batch * n_seg * sizeof(int));
  a->hgrid = (double *)a->alloc((size_t)batch * n_seg * max_per_seg * sizeof(double));
  a->ckpt = (double2 *)a->alloc((size_t)batch * (n_seg + 1) * n * sizeof(double2));
  a->work = (double2 *)a->alloc((size_t)batch * a->slots * n * sizeof(double2));
  a->omega = (double *)a->alloc((size_t)batch * n_seg * sizeof(double));
  a->gamma = (double *)a->alloc((size_t)batch * std::max(n_k, 1) * sizeof(double));
  a->loss = (double *)a->alloc((size_t)batch * sizeof(double));
  a->ctl = (unsigned long long *)a->alloc(kCtlBytes);
  if (!a->ops.w || !a->ops.off || !a->ops.col || !a->ops.val64 || !a->rho0 || !a->nsteps ||
      !a->hgrid || !a->ckpt || !a->work || !a->omega || !a->gamma || !a->loss || !a->ctl) {
    delete a;
    return fail(QT_ENOMEM, "device allocation of the adjoint workspace failed");
  }
  *out = a;
  return QT_OK;
}

int qt_adjoint_destroy(qt_adjoint a) {
  if (!a) return QT_OK;
  cudaDeviceSynchronize();
  delete a;
  return QT_OK;
}

int qt_adjoint_forward_dev(qt_adjoint a, const double *omega_dev, const double *gamma_dev,
                           const qt_opts *o, double *loss_dev, qt_stats *stats_dev,
                           void *stream) {
  g_err.clear();
  if (!a) return fail(QT_EINVAL, "null adjoint handle");
  int rc = check_opts(o);
  if (rc) return rc;
  if (!omega_dev || (a->nk > 0 && !gamma_dev) || !loss_dev)
    return fail(QT_EINVAL, "omega, gamma and loss are required");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  QT_CK(cudaMemcpyAsync(a->omega, omega_dev, (size_t)a->batch * a->n_seg * sizeof(double),
                        cudaMemcpyDeviceToDevice, st));
  if (a->nk > 0)
    QT_CK(cudaMemcpyAsync(a->gamma, gamma_dev, (size_t)a->batch * a->nk * sizeof(double),
                          cudaMemcpyDeviceToDevice, st));
  QT_CK(cudaMemsetAsync(a->ctl, 0, kCtlBytes, st));
  qt::AdjArgs x = adj_args(a);
  x.omega = a->omega;
  x.gamma = a->gamma;
  x.rtol = o->rtol;
  x.atol = o->atol;
  x.max_steps = o->max_steps;
  x.fixed = 0;
  x.loss = loss_dev;
  QT_CK(qt::launch_adjoint_forward(x, st));
  if (stats_dev)
    QT_CK(qt::launch_finalize_stats(a->ctl, x.status, a->ctl + 6, stats_dev, st));
  a->have_forward = true;
  return QT_OK;
}

int qt_adjoint_loss_fixed_dev(qt_adjoint a, const double *omega_dev, const double *gamma_dev,
                              double *loss_dev, void *stream) {
  g_err.clear();
  if (!a) return fail(QT_EINVAL, "null adjoint handle");
  if (!a->have_forward) return fail(QT_EINVAL, "no forward pass has recorded a grid");
  if (!omega_dev || (a->nk > 0 && !gamma_dev) || !loss_dev)
    return fail(QT_EINVAL, "omega, gamma and loss are required");
  qt::AdjArgs x = adj_args(a);
  x.omega = omega_dev;
  x.gamma = gamma_dev;
  x.fixed = 1;
  x.loss = loss_dev;
  // the fixed-grid pass reuses the workspace but neither the grid nor the
  // checkpoints of the last forward pass
  QT_CK(qt::launch_adjoint_forward(x, reinterpret_cast<cudaStream_t>(stream)));
  return QT_OK;
}

int qt_adjoint_backward_dev(qt_adjoint a, const double *dloss_dev, double *grad_omega_dev,
                            double *grad_gamma_dev, void *stream) {
  g_err.clear();
  if (!a) return fail(QT_EINVAL, "null adjoint handle");
  if (!a->have_forward) return fail(QT_EINVAL, "no forward pass to differentiate");
  if (!grad_omega_dev || (a->nk > 0 && !grad_gamma_dev))
    return fail(QT_EINVAL, "gradient outputs are required");
  qt::AdjArgs x = adj_args(a);
  x.omega = a->omega;
  x.gamma = a->gamma;
  x.dloss = dloss_dev;
  x.g_omega = grad_omega_dev;
  x.g_gamma = grad_gamma_dev;
  QT_CK(qt::launch_adjoint_backward(x, reinterpret_cast<cudaStream_t>(stream)));
  return QT_OK;
}

int qt_adjoint_grid(qt_adjoint a, int b, int32_t *nsteps, double *h) {
  g_err.clear();
  if (!a || b < 0 || b >= a->batch || !nsteps || !h) return fail(QT_EINVAL, "bad arguments");
  QT_CK(cudaDeviceSynchronize());
  QT_CK(cudaMemcpy(nsteps, a->nsteps + (size_t)b * a->n_seg, a->n_seg * sizeof(int),
                   cudaMemcpyDeviceToHost));
  QT_CK(cudaMemcpy(h, a->hgrid + (size_t)b * a->n_seg * a->maxs,
                   (size_t)a->n_seg * a->maxs * sizeof(double), cudaMemcpyDeviceToHost));
  return QT_OK;
}

// ------------------------------------------------------- host-memory calls

struct SystemGuard {
  qt_system s = nullptr;
  ~SystemGuard() {
    if (s) qt_system_destroy(s);
  }
};

int qt_mcsolve(const qt_op *H, const qt_op *c_ops, int n_c, const qt_op *e_ops, int n_e,
               const qt_c128 *psi0, const double *tlist, int n_t, int64_t ntraj, uint64_t seed,
               const qt_opts *o, qt_c128 *expect_out, qt_c128 *traj_expect_out, qt_jump *jumps,
               int64_t jump_cap, int64_t *n_jumps, qt_stats *stats) {
  return qt_mcsolve_td(H, nullptr, c_ops, n_c, e_ops, n_e, psi0, tlist, n_t, ntraj, seed, o,
                       expect_out, traj_expect_out, jumps, jump_cap, n_jumps, stats);
}

int qt_mcsolve_td(const qt_op *H, const qt_td *td, const qt_op *c_ops, int n_c,
                  const qt_op *e_ops, int n_e, const qt_c128 *psi0, const double *tlist,
                  int n_t, int64_t ntraj, uint64_t seed, const qt_opts *o, qt_c128 *expect_out,
                  qt_c128 *traj_expect_out, qt_jump *jumps, int64_t jump_cap, int64_t *n_jumps,
                  qt_stats *stats) {
  g_err.clear();
  int rc = check_opts(o);
  if (rc) return rc;
  if (!psi0) return fail(QT_EINVAL, "null psi0");
  if ((rc = check_tlist_host(tlist, n_t))) return rc;
  if (ntraj < 0) return fail(QT_EINVAL, "negative ntraj");
  if (n_e > 0 && !expect_out) return fail(QT_EINVAL, "null expect_out");
  if (jump_cap < 0 || (jump_cap > 0 && !jumps)) return fail(QT_EINVAL, "bad jump buffer");
  SystemGuard g;
  if ((rc = qt_system_create_td(H, td, c_ops, n_c, e_ops, n_e, &g.s))) return rc;
  const int d = g.s->d;
  const int64_t ntr = (n_c == 0 && ntraj > 0) ? 1 : ntraj;
  StreamGuard sg;
  QT_CK(cudaStreamCreateWithFlags(&sg.s, cudaStreamNonBlocking));
  DevBuf dpsi, dt, dexp, dtraj, djump, dnj, dst;
  const size_t exp_bytes = (size_t)n_t * n_e * sizeof(qt_c128);
  const size_t traj_bytes = traj_expect_out ? (size_t)ntr * n_t * n_e * sizeof(qt_c128) : 0;
  if ((rc = dpsi.alloc((size_t)d * sizeof(qt_c128))) || (rc = dt.alloc((size_t)n_t * sizeof(double))) ||
      (rc = dexp.alloc(exp_bytes)) || (traj_bytes && (rc = dtraj.alloc(traj_bytes))) ||
      (jump_cap > 0 && (rc = djump.alloc((size_t)jump_cap * sizeof(qt_jump)))) ||
      (rc = dnj.alloc(sizeof(int64_t))) || (rc = dst.alloc(sizeof(qt_stats))))
    return rc;
  QT_CK(cudaMemcpyAsync(dpsi.p, psi0, (size_t)d * sizeof(qt_c128), cudaMemcpyHostToDevice, sg.s));
  QT_CK(cudaMemcpyAsync(dt.p, tlist, (size_t)n_t * sizeof(double), cudaMemcpyHostToDevice, sg.s));
  rc = qt_mcsolve_dev(g.s, dpsi.as<qt_c128>(), dt.as<double>(), n_t, 0, ntraj, seed, o,
                      dexp.as<qt_c128>(), traj_bytes ? dtraj.as<qt_c128>() : nullptr,
                      jump_cap > 0 ? djump.as<qt_jump>() : nullptr, jump_cap, dnj.as<int64_t>(),
                      dst.as<qt_stats>(), sg.s);
  if (rc) return rc;
  qt_stats hs;
  int64_t hnj = 0;
  std::vector<qt_c128> sums((size_t)n_t * n_e);
  if (exp_bytes) QT_CK(cudaMemcpyAsync(sums.data(), dexp.p, exp_bytes, cudaMemcpyDeviceToHost, sg.s));
  if (traj_bytes)
    QT_CK(cudaMemcpyAsync(traj_expect_out, dtraj.p, traj_bytes, cudaMemcpyDeviceToHost, sg.s));
  QT_CK(cudaMemcpyAsync(&hnj, dnj.p, sizeof hnj, cudaMemcpyDeviceToHost, sg.s));
  QT_CK(cudaMemcpyAsync(&hs, dst.p, sizeof hs, cudaMemcpyDeviceToHost, sg.s));
  QT_CK(cudaStreamSynchronize(sg.s));
  if (jump_cap > 0 && hnj > 0) {
    const int64_t nc = std::min(hnj, jump_cap);
    QT_CK(cudaMemcpy(jumps, djump.p, (size_t)nc * sizeof(qt_jump), cudaMemcpyDeviceToHost));
  }
  if (stats) *stats = hs;
  if (n_jumps) *n_jumps = hnj;
  if (hs.status != QT_OK) return fail(hs.status, "device solver reported status %d", hs.status);
  const double inv = ntr > 0 ? 1.0 / (double)ntr : 0.0;
  for (size_t q = 0; q < sums.size(); ++q) {
    expect_out[q].re = sums[q].re * inv;
    expect_out[q].im = sums[q].im * inv;
  }
  if (jump_cap > 0 && hnj > jump_cap) return fail(QT_ECAP, "%lld jumps exceed the buffer of %lld", (long long)hnj,
                                  (long long)jump_cap);
  return QT_OK;
}

int qt_mesolve(const qt_op *H, const qt_op *c_ops, int n_c, const qt_op *e_ops, int n_e,
               const qt_c128 *state0, int state_is_ket, const double *tlist, int n_t,
               const qt_opts *o, qt_c128 *expect_out, qt_c128 *states_out, qt_stats *stats) {
  return qt_mesolve_td(H, nullptr, c_ops, n_c, e_ops, n_e, state0, state_is_ket, tlist, n_t, o,
                       expect_out, states_out, stats);
}

int qt_mesolve_td(const qt_op *H, const qt_td *td, const qt_op *c_ops, int n_c,
                  const qt_op *e_ops, int n_e, const qt_c128 *state0, int state_is_ket,
                  const double *tlist, int n_t, const qt_opts *o, qt_c128 *expect_out,
                  qt_c128 *states_out, qt_stats *stats) {
  g_err.clear();
  int rc = check_opts(o);
  if (rc) return rc;
  if (!state0) return fail(QT_EINVAL, "null state0");
  if ((rc = check_tlist_host(tlist, n_t))) return rc;
  if (n_e > 0 && !expect_out) return fail(QT_EINVAL, "null expect_out");
  SystemGuard g;
  if ((rc = qt_system_create_td(H, td, c_ops, n_c, e_ops, n_e, &g.s))) return rc;
  const int d = g.s->d;
  StreamGuard sg;
  QT_CK(cudaStreamCreateWithFlags(&sg.s, cudaStreamNonBlocking));
  const size_t sbytes = (state_is_ket ? (size_t)d : (size_t)d * d) * sizeof(qt_c128);
  const size_t exp_bytes = (size_t)n_t * n_e * sizeof(qt_c128);
  const size_t st_bytes = states_out ? (size_t)n_t * d * d * sizeof(qt_c128) : 0;
  DevBuf ds, dt, dexp, dstates, dst;
  if ((rc = ds.alloc(sbytes)) || (rc = dt.alloc((size_t)n_t * sizeof(double))) ||
      (rc = dexp.alloc(exp_bytes)) || (st_bytes && (rc = dstates.alloc(st_bytes))) ||
      (rc = dst.alloc(sizeof(qt_stats))))
    return rc;
  QT_CK(cudaMemcpyAsync(ds.p, state0, sbytes, cudaMemcpyHostToDevice, sg.s));
  QT_CK(cudaMemcpyAsync(dt.p, tlist, (size_t)n_t * sizeof(double), cudaMemcpyHostToDevice, sg.s));
  rc = qt_mesolve_dev(g.s, ds.as<qt_c128>(), state_is_ket, dt.as<double>(), n_t, o,
                      dexp.as<qt_c128>(), st_bytes ? dstates.as<qt_c128>() : nullptr,
                      dst.as<qt_stats>(), sg.s);
  if (rc) return rc;
  qt_stats hs;
  if (exp_bytes) QT_CK(cudaMemcpyAsync(expect_out, dexp.p, exp_bytes, cudaMemcpyDeviceToHost, sg.s));
  if (st_bytes) QT_CK(cudaMemcpyAsync(states_out, dstates.p, st_bytes, cudaMemcpyDeviceToHost, sg.s));
  QT_CK(cudaMemcpyAsync(&hs, dst.p, sizeof hs, cudaMemcpyDeviceToHost, sg.s));
  QT_CK(cudaStreamSynchronize(sg.s));
  if (stats) *stats = hs;
  if (hs.status != QT_OK) return fail(hs.status, "device solver reported status %d", hs.status);
  return QT_OK;
}

int qt_correlation_2op_2t(const qt_op *H, const qt_td *td, const qt_op *c_ops, int n_c,
                          const qt_op *A, const qt_op *B, const qt_c128 *state0, int state_is_ket,
                          const double *tlist, int n_t, const double *taulist, int n_tau,
                          const qt_opts *o, qt_c128 *corr_out, qt_stats *stats) {
  g_err.clear();
  int rc = check_opts(o);
  if (rc) return rc;
  if (!A || !B || !state0 || !corr_out) return fail(QT_EINVAL, "null argument");
  if ((rc = check_tlist_host(tlist, n_t))) return rc;
  if ((rc = check_tlist_host(taulist, n_tau))) return rc;
  if (taulist[0] != 0.0) return fail(QT_EINVAL, "taulist must start at 0");
  const qt_op eo[2] = {*A, *B};
  SystemGuard g;
  if ((rc = qt_system_create_td(H, td, c_ops, n_c, eo, 2, &g.s))) return rc;
  const int d = g.s->d;
  StreamGuard sg;
  QT_CK(cudaStreamCreateWithFlags(&sg.s, cudaStreamNonBlocking));
  const size_t sbytes = (state_is_ket ? (size_t)d : (size_t)d * d) * sizeof(qt_c128);
  const size_t cbytes = (size_t)n_t * n_tau * 2 * sizeof(qt_c128);
  DevBuf ds, dt, dtau, dc, dst;
  if ((rc = ds.alloc(sbytes)) || (rc = dt.alloc((size_t)n_t * sizeof(double))) ||
      (rc = dtau.alloc((size_t)n_tau * sizeof(double))) || (rc = dc.alloc(cbytes)) ||
      (rc = dst.alloc(sizeof(qt_stats))))
    return rc;
  QT_CK(cudaMemcpyAsync(ds.p, state0, sbytes, cudaMemcpyHostToDevice, sg.s));
  QT_CK(cudaMemcpyAsync(dt.p, tlist, (size_t)n_t * sizeof(double), cudaMemcpyHostToDevice, sg.s));
  QT_CK(cudaMemcpyAsync(dtau.p, taulist, (size_t)n_tau * sizeof(double), cudaMemcpyHostToDevice,
                        sg.s));
  rc = qt_correlation_2op_2t_dev(g.s, ds.as<qt_c128>(), state_is_ket, dt.as<double>(), n_t,
                                 dtau.as<double>(), n_tau, 1, o, dc.as<qt_c128>(),
                                 dst.as<qt_stats>(), sg.s);
  if (rc) return rc;
  std::vector<qt_c128> all((size_t)n_t * n_tau * 2);
  qt_stats hs;
  QT_CK(cudaMemcpyAsync(all.data(), dc.p, cbytes, cudaMemcpyDeviceToHost, sg.s));
  QT_CK(cudaMemcpyAsync(&hs, dst.p, sizeof hs, cudaMemcpyDeviceToHost, sg.s));
  QT_CK(cudaStreamSynchronize(sg.s));
  if (stats) *stats = hs;
  if (hs.status != QT_OK) return fail(hs.status, "device solver reported status %d", hs.status);
  for (size_t q = 0; q < (size_t)n_t * n_tau; ++q) corr_out[q] = all[2 * q];
  return QT_OK;
}

int qt_steadystate(const qt_op *H, const qt_op *c_ops, int n_c, double tol, int64_t max_iter,
                   int krylov_dim, qt_c128 *rho_out, double *info_out, qt_stats *stats) {
  g_err.clear();
  if (!rho_out) return fail(QT_EINVAL, "null rho_out");
  if (!(tol > 0.0) || max_iter < 0) return fail(QT_EINVAL, "tol must be > 0 and max_iter >= 0");
  SystemGuard g;
  int rc = qt_system_create(H, c_ops, n_c, nullptr, 0, &g.s);
  if (rc) return rc;
  const int d = g.s->d;
  StreamGuard sg;
  QT_CK(cudaStreamCreateWithFlags(&sg.s, cudaStreamNonBlocking));
  DevBuf drho, dinfo, dst;
  if ((rc = drho.alloc((size_t)d * d * sizeof(qt_c128))) || (rc = dinfo.alloc(3 * sizeof(double))) ||
      (rc = dst.alloc(sizeof(qt_stats))))
    return rc;
  rc = qt_steadystate_dev(g.s, tol, max_iter, krylov_dim, drho.as<qt_c128>(),
                          dinfo.as<double>(), dst.as<qt_stats>(), sg.s);
  if (rc) return rc;
  qt_stats hs;
  double hinfo[3];
  QT_CK(cudaMemcpyAsync(rho_out, drho.p, (size_t)d * d * sizeof(qt_c128), cudaMemcpyDeviceToHost,
                        sg.s));
  QT_CK(cudaMemcpyAsync(hinfo, dinfo.p, sizeof hinfo, cudaMemcpyDeviceToHost, sg.s));
  QT_CK(cudaMemcpyAsync(&hs, dst.p, sizeof hs, cudaMemcpyDeviceToHost, sg.s));
  QT_CK(cudaStreamSynchronize(sg.s));
  if (stats) *stats = hs;
  if (info_out) std::memcpy(info_out, hinfo, sizeof hinfo);
  if (hs.status == QT_ESTEP)
    return fail(QT_ESTEP, "no convergence in %lld iterations (relative residual %.3g)",
                (long long)max_iter, hinfo[0]);
  if (hs.status != QT_OK) return fail(hs.status, "device solver reported status %d", hs.status);
  return QT_OK;
}

int qt_propagator_steadystate(const qt_op *H, const qt_op *c_ops, int n_c, const qt_c128 *rho0,
                              double period, double tol, int64_t max_periods, const qt_opts *o,
                              qt_c128 *rho_out, double *info_out, qt_stats *stats) {
  g_err.clear();
  if (!rho_out) return fail(QT_EINVAL, "null rho_out");
  int rc = check_opts(o);
  if (rc) return rc;
  if (!(period > 0.0) || !std::isfinite(period) || !(tol > 0.0) || max_periods < 1)
    return fail(QT_EINVAL, "period and tol must be > 0, max_periods >= 1");
  SystemGuard g;
  rc = qt_system_create(H, c_ops, n_c, nullptr, 0, &g.s);
  if (rc) return rc;
  const int d = g.s->d;
  const size_t bytes = (size_t)d * d * sizeof(qt_c128);
  StreamGuard sg;
  QT_CK(cudaStreamCreateWithFlags(&sg.s, cudaStreamNonBlocking));
  DevBuf d0, drho, dst;
  if ((rho0 && (rc = d0.alloc(bytes))) || (rc = drho.alloc(bytes)) ||
      (rc = dst.alloc(sizeof(qt_stats))))
    return rc;
  if (rho0) QT_CK(cudaMemcpyAsync(d0.p, rho0, bytes, cudaMemcpyHostToDevice, sg.s));
  double info[2] = {0.0, 0.0};
  rc = qt_propagator_steadystate_dev(g.s, rho0 ? d0.as<qt_c128>() : nullptr, period, tol,
                                     max_periods, o, drho.as<qt_c128>(), info,
                                     dst.as<qt_stats>(), sg.s);
  if (rc) return rc;
  qt_stats hs;
  QT_CK(cudaMemcpyAsync(rho_out, drho.p, bytes, cudaMemcpyDeviceToHost, sg.s));
  QT_CK(cudaMemcpyAsync(&hs, dst.p, sizeof hs, cudaMemcpyDeviceToHost, sg.s));
  QT_CK(cudaStreamSynchronize(sg.s));
  if (stats) *stats = hs;
  if (info_out) std::memcpy(info_out, info, sizeof info);
  if (hs.status == QT_ESTEP)
    return fail(QT_ESTEP,
                "no convergence to %.3g after %lld periods (last change %.3g; the change stops "
                "falling at the integration error of one period: tighten rtol/atol or loosen tol)",
                tol, (long long)info[1], info[0]);
  if (hs.status != QT_OK) return fail(hs.status, "device solver reported status %d", hs.status);
  return QT_OK;
}

int qt_propagator(const qt_op *H, const qt_td *td, const qt_op *c_ops, int n_c,
                  const double *tlist, int n_t, const qt_opts *o, qt_c128 *U_out,
                  qt_stats *stats) {
  g_err.clear();
  int rc = check_opts(o);
  if (rc) return rc;
  if (!U_out) return fail(QT_EINVAL, "null U_out");
  if ((rc = check_tlist_host(tlist, n_t))) return rc;
  SystemGuard g;
  if ((rc = qt_system_create_td(H, td, c_ops, n_c, nullptr, 0, &g.s))) return rc;
  const int d = g.s->d;
  if (d > qt::kMeSmallDim)
    return fail(QT_ENOTIMPL, "the propagator is built for dim <= %d (dim^4 entries per time)",
                qt::kMeSmallDim);
  const size_t ubytes = (size_t)n_t * d * d * d * d * sizeof(qt_c128);
  StreamGuard sg;
  QT_CK(cudaStreamCreateWithFlags(&sg.s, cudaStreamNonBlocking));
  DevBuf dt, du, dst;
  if ((rc = dt.alloc((size_t)n_t * sizeof(double))) || (rc = du.alloc(ubytes)) ||
      (rc = dst.alloc(sizeof(qt_stats))))
    return rc;
  QT_CK(cudaMemcpyAsync(dt.p, tlist, (size_t)n_t * sizeof(double), cudaMemcpyHostToDevice, sg.s));
  rc = qt_propagator_dev(g.s, dt.as<double>(), n_t, o, du.as<qt_c128>(), dst.as<qt_stats>(), sg.s);
  if (rc) return rc;
  qt_stats hs;
  QT_CK(cudaMemcpyAsync(U_out, du.p, ubytes, cudaMemcpyDeviceToHost, sg.s));
  QT_CK(cudaMemcpyAsync(&hs, dst.p, sizeof hs, cudaMemcpyDeviceToHost, sg.s));
  QT_CK(cudaStreamSynchronize(sg.s));
  if (stats) *stats = hs;
  if (hs.status != QT_OK) return fail(hs.status, "device solver reported status %d", hs.status);
  return QT_OK;
}

int qt_correlation_ss(const qt_op *H, const qt_op *c_ops, int n_c, const qt_op *A,
                      const qt_op *B, const double *taulist, int n_tau, double tol,
                      const qt_opts *o, qt_c128 *corr_out, qt_stats *stats) {
  g_err.clear();
  int rc = check_opts(o);
  if (rc) return rc;
  if (!A || !B || !corr_out) return fail(QT_EINVAL, "null argument");
  if ((rc = check_tlist_host(taulist, n_tau))) return rc;
  if (taulist[0] != 0.0) return fail(QT_EINVAL, "taulist must start at 0");
  if (!(tol > 0.0)) return fail(QT_EINVAL, "tol must be > 0");
  const qt_op eo[2] = {*A, *B};
  SystemGuard g;
  if ((rc = qt_system_create_td(H, nullptr, c_ops, n_c, eo, 2, &g.s))) return rc;
  const int d = g.s->d;
  StreamGuard sg;
  QT_CK(cudaStreamCreateWithFlags(&sg.s, cudaStreamNonBlocking));
  const size_t cbytes = (size_t)n_tau * 2 * sizeof(qt_c128);
  DevBuf drho, dt, dtau, dc, dst;
  if ((rc = drho.alloc((size_t)d * d * sizeof(qt_c128))) || (rc = dt.alloc(sizeof(double))) ||
      (rc = dtau.alloc((size_t)n_tau * sizeof(double))) || (rc = dc.alloc(cbytes)) ||
      (rc = dst.alloc(sizeof(qt_stats))))
    return rc;
  const double t0 = 0.0;
  QT_CK(cudaMemcpyAsync(dt.p, &t0, sizeof t0, cudaMemcpyHostToDevice, sg.s));
  QT_CK(cudaMemcpyAsync(dtau.p, taulist, (size_t)n_tau * sizeof(double), cudaMemcpyHostToDevice,
                        sg.s));
  // the steady state (FP64 GMRES), then <A(tau) B(0)> from it
  if ((rc = qt_steadystate_dev(g.s, tol, 200000, 0, drho.as<qt_c128>(), nullptr,
                               dst.as<qt_stats>(), sg.s)))
    return rc;
  qt_stats hs;
  QT_CK(cudaMemcpyAsync(&hs, dst.p, sizeof hs, cudaMemcpyDeviceToHost, sg.s));
  QT_CK(cudaStreamSynchronize(sg.s));
  if (hs.status != QT_OK) {
    if (stats) *stats = hs;
    return fail(hs.status, "steady state: device solver reported status %d", hs.status);
  }
  rc = qt_correlation_2op_2t_dev(g.s, drho.as<qt_c128>(), 0, dt.as<double>(), 1,
                                 dtau.as<double>(), n_tau, 1, o, dc.as<qt_c128>(),
                                 dst.as<qt_stats>(), sg.s);
  if (rc) return rc;
  std::vector<qt_c128> all((size_t)n_tau * 2);
  QT_CK(cudaMemcpyAsync(all.data(), dc.p, cbytes, cudaMemcpyDeviceToHost, sg.s));
  QT_CK(cudaMemcpyAsync(&hs, dst.p, sizeof hs, cudaMemcpyDeviceToHost, sg.s));
  QT_CK(cudaStreamSynchronize(sg.s));
  if (stats) *stats = hs;
  if (hs.status != QT_OK) return fail(hs.status, "device solver reported status %d", hs.status);
  for (int j = 0; j < n_tau; ++j) corr_out[j] = all[2 * (size_t)j];
  return QT_OK;
}

int qt_expect(const qt_op *O, const qt_c128 *states, int is_ket, int64_t batch, qt_c128 *out) {
  g_err.clear();
  if (!O) return fail(QT_EINVAL, "null operator");
  if (batch < 0 || (batch > 0 && (!states || !out))) return fail(QT_EINVAL, "bad state batch");
  SystemGuard g;
  int rc = qt_system_create(O, nullptr, 0, O, 1, &g.s);
  if (rc) return rc;
  if (batch == 0) return QT_OK;
  const int d = g.s->d;
  const size_t sbytes = (size_t)batch * (is_ket ? (size_t)d : (size_t)d * d) * sizeof(qt_c128);
  DevBuf ds, dout;
  if ((rc = ds.alloc(sbytes)) || (rc = dout.alloc((size_t)batch * sizeof(qt_c128)))) return rc;
  QT_CK(cudaMemcpy(ds.p, states, sbytes, cudaMemcpyHostToDevice));
  if ((rc = qt_expect_dev(g.s, 0, ds.as<qt_c128>(), is_ket, batch, dout.as<qt_c128>(), nullptr)))
    return rc;
  QT_CK(cudaMemcpy(out, dout.p, (size_t)batch * sizeof(qt_c128), cudaMemcpyDeviceToHost));
  return QT_OK;
}

}  // extern "C"
