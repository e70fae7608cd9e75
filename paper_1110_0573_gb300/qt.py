"""Python binding of libqt's C ABI (include/qt.h): argument marshalling only.

Every function here converts numpy / scipy / torch arguments into the plain
pointers and sizes of the C calls of the same name and raises QtError when a
call returns a negative status.  All arithmetic runs in libqt's CUDA kernels;
when libqt.so has not been built this module raises instead of computing
anything itself.

Host-memory calls take numpy arrays.  The *_dev calls take torch CUDA
tensors (complex128 / float64 / int64 as documented in qt.h) and the current
torch stream.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libqt.so")

QT_OK = 0
QT_EINVAL, QT_ENONHERM, QT_ENORM, QT_ENOMEM, QT_ECUDA = -1, -2, -3, -4, -5
QT_ESTEP, QT_EBISECT, QT_ETIMEOUT, QT_ENUMERIC, QT_ECAP = -6, -7, -8, -9, -10
QT_ENOTIMPL, QT_ENODEV = -11, -12
QT_DENSE, QT_CSR = 0, 1
QT_FP64, QT_MIXED = 0, 1
QT_ME_AUTO, QT_ME_SPARSE, QT_ME_DENSE_TC = 0, 1, 2

STATUS_NAMES = {0: "QT_OK", -1: "QT_EINVAL", -2: "QT_ENONHERM", -3: "QT_ENORM",
                -4: "QT_ENOMEM", -5: "QT_ECUDA", -6: "QT_ESTEP", -7: "QT_EBISECT",
                -8: "QT_ETIMEOUT", -9: "QT_ENUMERIC", -10: "QT_ECAP", -11: "QT_ENOTIMPL",
                -12: "QT_ENODEV"}


class QtError(RuntimeError):
    def __init__(self, code, where, msg):
        super().__init__(f"{where}: {STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class qt_op(C.Structure):
    _fields_ = [("dim", C.c_int32), ("fmt", C.c_int32), ("nnz", C.c_int64),
                ("indptr", C.c_void_p), ("indices", C.c_void_p), ("values", C.c_void_p)]


class qt_opts(C.Structure):
    _fields_ = [("rtol", C.c_double), ("atol", C.c_double), ("h0", C.c_double),
                ("max_steps", C.c_int64), ("bisect_tol", C.c_double), ("precision", C.c_int32),
                ("traj_block", C.c_int32), ("me_method", C.c_int32), ("reserved", C.c_int32)]


class qt_stats(C.Structure):
    _fields_ = [("accepted", C.c_int64), ("rejected", C.c_int64), ("rhs_evals", C.c_int64),
                ("bisect_iters", C.c_int64), ("jumps", C.c_int64), ("near_miss", C.c_int64),
                ("status", C.c_int32), ("reserved", C.c_int32)]


JUMP_DTYPE = np.dtype([("traj", np.int64), ("k", np.int64), ("channel", np.int64),
                       ("tau", np.float64), ("degenerate", np.int64)])
STATS_DTYPE = np.dtype([(n, np.int64) for n in ("accepted", "rejected", "rhs_evals",
                                                 "bisect_iters", "jumps", "near_miss")]
                       + [("status", np.int32), ("reserved", np.int32)])

_lock = threading.Lock()
_lib = None

# (name, restype, argtypes) of every exported function, in qt.h order
P, I, I64, U64, D = C.c_void_p, C.c_int, C.c_int64, C.c_uint64, C.c_double
SIGNATURES = [
    ("qt_opts_default", None, [P]),
    ("qt_last_error", C.c_char_p, []),
    ("qt_version", C.c_char_p, []),
    ("qt_mesolve", I, [P, P, I, P, I, P, I, P, I, P, P, P, P]),
    ("qt_mcsolve", I, [P, P, I, P, I, P, P, I, I64, U64, P, P, P, P, I64, P, P]),
    ("qt_expect", I, [P, P, I, I64, P]),
    ("qt_system_create", I, [P, P, I, P, I, P]),
    ("qt_system_destroy", I, [P]),
    ("qt_system_dim", I, [P]),
    ("qt_mcsolve_dev", I, [P, P, P, I, I64, I64, U64, P, P, P, P, I64, P, P, P]),
    ("qt_mesolve_dev", I, [P, P, I, P, I, P, P, P, P, P]),
    ("qt_mesolve_dev_noalloc", I, [P, P, I, P, I, P, P, P, P, P]),
    ("qt_me_rhs_dev", I, [P, C.c_double, P, P, P, P, P]),
    ("qt_system_create_td", I, [P, P, P, I, P, I, P]),
    ("qt_mesolve_td", I, [P, P, P, I, P, I, P, I, P, I, P, P, P, P]),
    ("qt_mcsolve_td", I, [P, P, P, I, P, I, P, P, I, I64, U64, P, P, P, P, I64, P, P]),
    ("qt_expect_dev", I, [P, I, P, I, I64, P, P]),
    ("qt_steadystate", I, [P, P, I, D, I64, I, P, P, P]),
    ("qt_steadystate_dev", I, [P, D, I64, I, P, P, P, P]),
    ("qt_propagator_steadystate", I, [P, P, I, P, D, D, I64, P, P, P, P]),
    ("qt_propagator_steadystate_dev", I, [P, P, D, D, I64, P, P, P, P, P]),
    ("qt_propagator", I, [P, P, P, I, P, I, P, P, P]),
    ("qt_propagator_dev", I, [P, P, I, P, P, P, P]),
    ("qt_correlation_ss", I, [P, P, I, P, P, P, I, D, P, P, P]),
    ("qt_correlation_2op_2t", I, [P, P, P, I, P, P, P, I, P, I, P, I, P, P, P]),
    ("qt_correlation_2op_2t_dev", I, [P, P, I, P, I, P, I, I, P, P, P, P]),
    ("qt_batch_create", I, [P, I, P]),
    ("qt_batch_destroy", I, [P]),
    ("qt_batch_expect_offset", I64, [P, I, I]),
    ("qt_batch_tune", I, [P, P, I, P, P, P]),
    ("qt_batch_solve_dev", I, [P, P, I, P, P, P, P]),
    ("qt_batch_problem_stats", I, [P, P]),
    ("qt_batch_config", I, [P, P, P, P]),
    ("qt_batch_set_config", I, [P, I, I]),
    ("qt_adjoint_create", I, [P, P, P, I, P, P, P, I, I, D, I, I, P]),
    ("qt_adjoint_destroy", I, [P]),
    ("qt_adjoint_forward_dev", I, [P, P, P, P, P, P, P]),
    ("qt_adjoint_loss_fixed_dev", I, [P, P, P, P, P]),
    ("qt_adjoint_backward_dev", I, [P, P, P, P, P]),
    ("qt_adjoint_grid", I, [P, I, P, P]),
    ("qt_fma_peak", I, [I, I64, I, P, P, P, P]),
]
QT_KIND_ME, QT_KIND_MC = 0, 1
QT_PEAK_FP32, QT_PEAK_FP32X2, QT_PEAK_FP64 = 0, 1, 2


class qt_problem(C.Structure):
    _fields_ = [("kind", C.c_int32), ("state_is_ket", C.c_int32), ("H", C.c_void_p),
                ("c_ops", C.c_void_p), ("n_c", C.c_int32), ("n_e", C.c_int32),
                ("e_ops", C.c_void_p), ("state0", C.c_void_p), ("ntraj", C.c_int64),
                ("seed", C.c_uint64)]


def lib():
    """The loaded libqt (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"libqt.so is not built ({LIB_PATH}); run "
                    "`python -m paper_1110_0573_gb300.build` (there is no CPU fallback)")
            L = C.CDLL(LIB_PATH)
            for name, res, args in SIGNATURES:
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def qt_last_error() -> str:
    return lib().qt_last_error().decode()


def qt_version() -> str:
    return lib().qt_version().decode()


def _check(rc, where):
    if rc != QT_OK:
        raise QtError(rc, where, qt_last_error())


def qt_opts_default(**overrides) -> qt_opts:
    o = qt_opts()
    lib().qt_opts_default(C.byref(o))
    for k, v in overrides.items():
        if v is not None:
            setattr(o, k, v)
    return o


def _ptr(a):
    return None if a is None else a.ctypes.data


class _Ops:
    """Holds qt_op structs and the arrays they point to."""

    def __init__(self, ops):
        import scipy.sparse as sp
        self.keep = []
        self.n = len(ops)
        self.arr = (qt_op * max(1, self.n))()
        for i, op in enumerate(ops):
            m = sp.csr_matrix(op, dtype=np.complex128)
            if m.shape[0] != m.shape[1]:
                raise ValueError(f"operator {i} is not square: {m.shape}")
            indptr = np.ascontiguousarray(m.indptr, dtype=np.int64)
            indices = np.ascontiguousarray(m.indices, dtype=np.int32)
            values = np.ascontiguousarray(m.data, dtype=np.complex128)
            self.keep += [indptr, indices, values]
            self.arr[i] = qt_op(m.shape[0], QT_CSR, m.nnz, _ptr(indptr), _ptr(indices),
                                _ptr(values))

    @property
    def ptr(self):
        return C.addressof(self.arr) if self.n else None


def _stats_dict(st: qt_stats) -> dict:
    return {k: int(getattr(st, k)) for k, _ in qt_stats._fields_ if k != "reserved"}


# ------------------------------------------------------------ host memory


class qt_td(C.Structure):
    _fields_ = [("n_terms", C.c_int32), ("H", C.c_void_p), ("n_knots", C.c_void_p),
                ("times", C.c_void_p), ("values", C.c_void_p)]


class _Td:
    """Holds a qt_td for the time-dependent terms [(H_k, knot_times,
    knot_values), ...] of H(t) = H + sum_k f_k(t) H_k."""

    def __init__(self, td):
        td = list(td or [])
        self.n = len(td)
        self.ops = _Ops([h for h, _, _ in td])
        ts = [np.asarray(t, dtype=np.float64).reshape(-1) for _, t, _ in td]
        vs = [np.asarray(v, dtype=np.float64).reshape(-1) for _, _, v in td]
        self.nk = np.ascontiguousarray([len(t) for t in ts] or [0], dtype=np.int64)
        self.t = np.ascontiguousarray(np.concatenate(ts) if ts else np.zeros(1), dtype=np.float64)
        self.v = np.ascontiguousarray(np.concatenate(vs) if vs else np.zeros(1), dtype=np.float64)
        if any(len(t) != len(v) for t, v in zip(ts, vs)):
            raise ValueError("each time-dependent term needs one value per knot")
        self.st = qt_td(self.n, self.ops.ptr, _ptr(self.nk), _ptr(self.t), _ptr(self.v))

    @property
    def ptr(self):
        return C.addressof(self.st) if self.n else None


def qt_mesolve(H, c_ops, e_ops, state0, tlist, opts=None, store_states=False, td=None):
    """Master equation (td: time-dependent terms [(H_k, knot_times,
    knot_values), ...]).  Returns (expect[n_t, n_e], states[n_t, d, d] |
    None, stats dict)."""
    o = opts or qt_opts_default()
    Hs, Cs, Es = _Ops([H]), _Ops(c_ops), _Ops(e_ops)
    T = _Td(td)
    d = Hs.arr[0].dim
    s0 = np.ascontiguousarray(state0, dtype=np.complex128)
    is_ket = 1 if s0.ndim == 1 else 0
    tl = np.ascontiguousarray(tlist, dtype=np.float64)
    nt, ne = len(tl), len(e_ops)
    out = np.zeros((nt, max(ne, 1)), dtype=np.complex128)
    states = np.zeros((nt, d, d), dtype=np.complex128) if store_states else None
    st = qt_stats()
    rc = lib().qt_mesolve_td(Hs.ptr, T.ptr, Cs.ptr, len(c_ops), Es.ptr, ne, _ptr(s0), is_ket,
                             _ptr(tl), nt, C.byref(o), _ptr(out), _ptr(states), C.byref(st))
    _check(rc, "qt_mesolve")
    return out[:, :ne], states, _stats_dict(st)


def qt_mcsolve(H, c_ops, e_ops, psi0, tlist, ntraj, seed=0, opts=None, traj_expect=False,
               jump_cap=None, td=None):
    """Monte-Carlo wave function (td: time-dependent terms).  Returns
    (expect[n_t, n_e] trajectory mean, traj_expect[ntraj, n_t, n_e] | None,
    jumps (JUMP_DTYPE, sorted by trajectory and jump index), stats dict)."""
    o = opts or qt_opts_default()
    Hs, Cs, Es = _Ops([H]), _Ops(c_ops), _Ops(e_ops)
    T = _Td(td)
    psi = np.ascontiguousarray(np.asarray(psi0, dtype=np.complex128).reshape(-1))
    tl = np.ascontiguousarray(tlist, dtype=np.float64)
    nt, ne = len(tl), len(e_ops)
    ntr = 1 if (len(c_ops) == 0 and ntraj > 0) else ntraj
    out = np.zeros((nt, max(ne, 1)), dtype=np.complex128)
    tex = np.zeros((ntr, nt, max(ne, 1)), dtype=np.complex128) if traj_expect else None
    cap = (64 * ntr + 1024) if jump_cap is None else jump_cap
    jumps = np.zeros(max(cap, 1), dtype=JUMP_DTYPE)
    nj = C.c_int64(0)
    st = qt_stats()
    rc = lib().qt_mcsolve_td(Hs.ptr, T.ptr, Cs.ptr, len(c_ops), Es.ptr, ne, _ptr(psi), _ptr(tl),
                             nt, ntraj, seed, C.byref(o), _ptr(out), _ptr(tex), _ptr(jumps), cap,
                             C.byref(nj), C.byref(st))
    if rc == QT_ECAP and jump_cap is None:
        return qt_mcsolve(H, c_ops, e_ops, psi0, tlist, ntraj, seed, opts, traj_expect,
                          jump_cap=int(nj.value), td=td)
    _check(rc, "qt_mcsolve")
    j = jumps[: nj.value].copy()
    j.sort(order=["traj", "k"])
    return out[:, :ne], (tex[:, :, :ne] if tex is not None else None), j, _stats_dict(st)


def qt_correlation_2op_2t(H, c_ops, A, B, state0, tlist, taulist, opts=None, td=None):
    """Two-time correlation <A(t_k + tau_j) B(t_k)> by the quantum regression
    theorem (ODE form).  taulist must start at 0.  Returns (corr[n_t, n_tau],
    stats dict)."""
    o = opts or qt_opts_default()
    Hs, Cs, As, Bs = _Ops([H]), _Ops(c_ops), _Ops([A]), _Ops([B])
    T = _Td(td)
    s0 = np.ascontiguousarray(state0, dtype=np.complex128)
    is_ket = 1 if s0.ndim == 1 else 0
    tl = np.ascontiguousarray(tlist, dtype=np.float64)
    tau = np.ascontiguousarray(taulist, dtype=np.float64)
    out = np.zeros((len(tl), len(tau)), dtype=np.complex128)
    st = qt_stats()
    rc = lib().qt_correlation_2op_2t(Hs.ptr, T.ptr, Cs.ptr, len(c_ops), As.ptr, Bs.ptr, _ptr(s0),
                                     is_ket, _ptr(tl), len(tl), _ptr(tau), len(tau), C.byref(o),
                                     _ptr(out), C.byref(st))
    _check(rc, "qt_correlation_2op_2t")
    return out, _stats_dict(st)


def qt_steadystate(H, c_ops, tol=1e-12, max_iter=20000, krylov_dim=0):
    """Steady state of the master equation (FP64 restarted GMRES on the GPU).
    Returns (rho[d, d], info dict: residual, w, iterations; stats dict)."""
    Hs, Cs = _Ops([H]), _Ops(c_ops)
    d = Hs.arr[0].dim
    rho = np.zeros((d, d), dtype=np.complex128)
    info = np.zeros(3)
    st = qt_stats()
    rc = lib().qt_steadystate(Hs.ptr, Cs.ptr, len(c_ops), float(tol), int(max_iter),
                              int(krylov_dim), _ptr(rho), _ptr(info), C.byref(st))
    _check(rc, "qt_steadystate")
    return rho, {"residual": float(info[0]), "w": float(info[1]),
                 "steps": int(info[2])}, _stats_dict(st)


def qt_propagator_steadystate(H, c_ops, period, tol=1e-10, max_periods=2000, rho0=None,
                              opts=None):
    """Fixed point of the master-equation propagator over one period (the
    paper's propagator_steadystate).  Returns (rho[d, d], info dict: change,
    periods; stats dict)."""
    o = opts or qt_opts_default()
    Hs, Cs = _Ops([H]), _Ops(c_ops)
    d = Hs.arr[0].dim
    r0 = None if rho0 is None else np.ascontiguousarray(rho0, dtype=np.complex128)
    rho = np.zeros((d, d), dtype=np.complex128)
    info = np.zeros(2)
    st = qt_stats()
    rc = lib().qt_propagator_steadystate(Hs.ptr, Cs.ptr, len(c_ops), _ptr(r0), float(period),
                                         float(tol), int(max_periods), C.byref(o), _ptr(rho),
                                         _ptr(info), C.byref(st))
    _check(rc, "qt_propagator_steadystate")
    return rho, {"change": float(info[0]), "periods": int(info[1])}, _stats_dict(st)


def qt_propagator(H, c_ops, tlist, opts=None, td=None):
    """Master-equation propagator: U[k] maps row-major vec(rho(tlist[0])) to
    vec(rho(tlist[k])).  Returns (U[n_t, d^2, d^2], stats dict)."""
    o = opts or qt_opts_default()
    Hs, Cs = _Ops([H]), _Ops(c_ops)
    T = _Td(td)
    d = Hs.arr[0].dim
    tl = np.ascontiguousarray(tlist, dtype=np.float64)
    U = np.zeros((len(tl), d * d, d * d), dtype=np.complex128)
    st = qt_stats()
    rc = lib().qt_propagator(Hs.ptr, T.ptr, Cs.ptr, len(c_ops), _ptr(tl), len(tl), C.byref(o),
                             _ptr(U), C.byref(st))
    _check(rc, "qt_propagator")
    return U, _stats_dict(st)


def qt_correlation_ss(H, c_ops, A, B, taulist, tol=1e-12, opts=None):
    """<A(tau) B(0)> in the steady state.  Returns (corr[n_tau], stats dict)."""
    o = opts or qt_opts_default()
    Hs, Cs, As, Bs = _Ops([H]), _Ops(c_ops), _Ops([A]), _Ops([B])
    tau = np.ascontiguousarray(taulist, dtype=np.float64)
    out = np.zeros(len(tau), dtype=np.complex128)
    st = qt_stats()
    rc = lib().qt_correlation_ss(Hs.ptr, Cs.ptr, len(c_ops), As.ptr, Bs.ptr, _ptr(tau), len(tau),
                                 float(tol), C.byref(o), _ptr(out), C.byref(st))
    _check(rc, "qt_correlation_ss")
    return out, _stats_dict(st)


def qt_expect(O, states, is_ket):
    """<psi|O|psi> per ket or Tr(O rho) per density matrix (batch first)."""
    Os = _Ops([O])
    d = Os.arr[0].dim
    s = np.ascontiguousarray(states, dtype=np.complex128)
    batch = s.size // (d if is_ket else d * d)
    out = np.zeros(batch, dtype=np.complex128)
    _check(lib().qt_expect(Os.ptr, _ptr(s), int(bool(is_ket)), batch, _ptr(out)), "qt_expect")
    return out


def qt_fma_peak(kind, iters, reps=5, stream=None):
    """Measured multiply-add rate of the current device (flop/s), with the
    flops and milliseconds of one launch: {"flop_per_s", "flop_per_launch",
    "ms_per_launch"}."""
    r, f, m = C.c_double(0.0), C.c_double(0.0), C.c_double(0.0)
    _check(lib().qt_fma_peak(int(kind), int(iters), int(reps), C.byref(r), C.byref(f), C.byref(m),
                             _stream(stream)), "qt_fma_peak")
    return {"flop_per_s": r.value, "flop_per_launch": f.value, "ms_per_launch": m.value}


# ---------------------------------------------------------- device resident


def _tptr(t):
    return None if t is None else t.data_ptr()


def _stream(stream):
    if stream is not None:
        return stream
    import torch
    return torch.cuda.current_stream().cuda_stream


class System:
    """A qt_system: operators packed and resident on the current CUDA device."""

    def __init__(self, H, c_ops, e_ops, td=None):
        Hs, Cs, Es = _Ops([H]), _Ops(c_ops), _Ops(e_ops)
        T = _Td(td)
        self.handle = C.c_void_p()
        _check(lib().qt_system_create_td(Hs.ptr, T.ptr, Cs.ptr, len(c_ops), Es.ptr, len(e_ops),
                                         C.byref(self.handle)), "qt_system_create")
        self.dim = lib().qt_system_dim(self.handle)
        self.n_c, self.n_e = len(c_ops), len(e_ops)

    def close(self):
        if self.handle:
            lib().qt_system_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def qt_mcsolve_dev(self, psi0, tlist, ntraj, seed, opts, expect_sum, traj_begin=0,
                       traj_expect=None, jumps=None, n_jumps=None, stats=None, stream=None):
        """Enqueue trajectories traj_begin .. traj_begin+ntraj-1.  Tensors:
        psi0 complex128[d], tlist float64[n_t], expect_sum complex128[n_t, n_e]
        (receives the SUM over trajectories), traj_expect complex128 or None,
        jumps uint8[cap * 40] or None, n_jumps int64[1] or None, stats
        uint8[56] or None."""
        cap = 0 if jumps is None else jumps.numel() * jumps.element_size() // JUMP_DTYPE.itemsize
        rc = lib().qt_mcsolve_dev(self.handle, _tptr(psi0), _tptr(tlist), tlist.numel(),
                                  traj_begin, ntraj, seed, C.byref(opts), _tptr(expect_sum),
                                  _tptr(traj_expect), _tptr(jumps), cap, _tptr(n_jumps),
                                  _tptr(stats), _stream(stream))
        _check(rc, "qt_mcsolve_dev")

    def qt_mesolve_dev(self, state0, tlist, opts, expect, states=None, stats=None, stream=None):
        """Enqueue a master-equation solve.  state0 complex128[d] (ket) or
        [d, d]; expect complex128[n_t, n_e]."""
        is_ket = 1 if state0.dim() == 1 else 0
        rc = lib().qt_mesolve_dev(self.handle, _tptr(state0), is_ket, _tptr(tlist),
                                  tlist.numel(), C.byref(opts), _tptr(expect), _tptr(states),
                                  _tptr(stats), _stream(stream))
        _check(rc, "qt_mesolve_dev")

    def qt_mesolve_dev_noalloc(self, state0, tlist, opts, expect, states=None, stats=None,
                               stream=None):
        """qt_mesolve_dev on the library's preallocated workspace: for callers
        that cannot allocate device memory (see qt.h for the size limit and
        the sharing rules)."""
        is_ket = 1 if state0.dim() == 1 else 0
        rc = lib().qt_mesolve_dev_noalloc(self.handle, _tptr(state0), is_ket, _tptr(tlist),
                                          tlist.numel(), C.byref(opts), _tptr(expect),
                                          _tptr(states), _tptr(stats), _stream(stream))
        _check(rc, "qt_mesolve_dev_noalloc")

    def qt_me_rhs_dev(self, rho, out, opts, stats=None, stream=None, t=0.0):
        """Enqueue one evaluation of d rho/dt at time t: rho, out
        complex128[d, d] on the device; opts selects precision and method."""
        rc = lib().qt_me_rhs_dev(self.handle, float(t), _tptr(rho), _tptr(out), C.byref(opts),
                                 _tptr(stats), _stream(stream))
        _check(rc, "qt_me_rhs_dev")

    def qt_correlation_2op_2t_dev(self, state0, tlist, taulist, b_index, opts, corr, stats=None,
                                  stream=None):
        """Enqueue <O_m(t_k + tau_j) B(t_k)> for every observable O_m, with B
        observable b_index: corr complex128[n_t, n_tau, n_e] on the device."""
        is_ket = 1 if state0.dim() == 1 else 0
        rc = lib().qt_correlation_2op_2t_dev(self.handle, _tptr(state0), is_ket, _tptr(tlist),
                                             tlist.numel(), _tptr(taulist), taulist.numel(),
                                             b_index, C.byref(opts), _tptr(corr), _tptr(stats),
                                             _stream(stream))
        _check(rc, "qt_correlation_2op_2t_dev")

    def qt_steadystate_dev(self, rho, tol=1e-12, max_iter=20000, krylov_dim=0, info=None,
                           stats=None, stream=None):
        """Enqueue the steady-state solve into rho complex128[d, d] (device);
        info: float64[3] on the device (residual, w, Arnoldi steps)."""
        rc = lib().qt_steadystate_dev(self.handle, float(tol), int(max_iter), int(krylov_dim),
                                      _tptr(rho), _tptr(info), _tptr(stats), _stream(stream))
        _check(rc, "qt_steadystate_dev")

    def qt_propagator_dev(self, tlist, opts, U, stats=None, stream=None):
        """Enqueue the propagator into U complex128[n_t, d^2, d^2] (device)."""
        rc = lib().qt_propagator_dev(self.handle, _tptr(tlist), tlist.numel(), C.byref(opts),
                                     _tptr(U), _tptr(stats), _stream(stream))
        _check(rc, "qt_propagator_dev")

    def qt_expect_dev(self, e_index, states, is_ket, out, stream=None):
        batch = out.numel()
        rc = lib().qt_expect_dev(self.handle, e_index, _tptr(states), int(bool(is_ket)), batch,
                                 _tptr(out), _stream(stream))
        _check(rc, "qt_expect_dev")


class Batch:
    """A qt_batch: many problems of uneven dimension for one persistent
    launch.  problems: list of dicts with H, c_ops, e_ops, state0 (ket or
    density matrix), kind ('me' or 'mc'), ntraj and seed (mc)."""

    def __init__(self, problems):
        keep = []
        arr = (qt_problem * len(problems))()
        self.n_e = []
        for i, pr in enumerate(problems):
            Hs, Cs, Es = _Ops([pr["H"]]), _Ops(pr["c_ops"]), _Ops(pr["e_ops"])
            st = np.ascontiguousarray(pr["state0"], dtype=np.complex128)
            keep += [Hs, Cs, Es, st]
            kind = QT_KIND_MC if pr["kind"] == "mc" else QT_KIND_ME
            arr[i] = qt_problem(kind, 1 if st.ndim == 1 else 0, Hs.ptr, Cs.ptr, len(pr["c_ops"]),
                                len(pr["e_ops"]), Es.ptr, _ptr(st), int(pr.get("ntraj", 0)),
                                int(pr.get("seed", 0)))
            self.n_e.append(len(pr["e_ops"]))
        self.handle = C.c_void_p()
        _check(lib().qt_batch_create(C.addressof(arr), len(problems), C.byref(self.handle)),
               "qt_batch_create")
        self.n = len(problems)

    def expect_offset(self, p, n_t):
        return int(lib().qt_batch_expect_offset(self.handle, p, n_t))

    def split(self, expect, n_t):
        """Per-problem [n_t, n_e] views of a flat expect array."""
        out = []
        for p in range(self.n):
            o = self.expect_offset(p, n_t)
            out.append(expect[o:o + n_t * self.n_e[p]].reshape(n_t, self.n_e[p]))
        return out

    def qt_batch_tune(self, tlist, opts, expect, stream=None):
        _check(lib().qt_batch_tune(self.handle, _tptr(tlist), tlist.numel(), C.byref(opts),
                                   _tptr(expect), _stream(stream)), "qt_batch_tune")

    def qt_batch_solve_dev(self, tlist, opts, expect, stats=None, stream=None):
        _check(lib().qt_batch_solve_dev(self.handle, _tptr(tlist), tlist.numel(), C.byref(opts),
                                        _tptr(expect), _tptr(stats), _stream(stream)),
               "qt_batch_solve_dev")

    def config(self):
        """{"traj_block", "small_group_dim", "tuned_ms"} of the batch's launch."""
        tb, sg, ms = C.c_int(0), C.c_int(0), C.c_double(0.0)
        _check(lib().qt_batch_config(self.handle, C.byref(tb), C.byref(sg), C.byref(ms)),
               "qt_batch_config")
        return {"traj_block": tb.value, "small_group_dim": sg.value, "tuned_ms": ms.value}

    def set_config(self, traj_block, small_group_dim):
        _check(lib().qt_batch_set_config(self.handle, int(traj_block), int(small_group_dim)),
               "qt_batch_set_config")

    def problem_stats(self):
        """Per-problem statistics of the last solve: numpy STATS_DTYPE[n]."""
        out = np.zeros(max(self.n, 1), dtype=STATS_DTYPE)
        _check(lib().qt_batch_problem_stats(self.handle, out.ctypes.data),
               "qt_batch_problem_stats")
        return out[:self.n]

    def close(self):
        if self.handle:
            lib().qt_batch_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Adjoint:
    """A qt_adjoint handle: a master equation with piecewise-constant drive
    amplitudes Omega[n_seg] and decay rates gamma[n_k] as parameters, for a
    batch of parameter vectors (see qt.h)."""

    def __init__(self, H0, Hd, A, P1, P2, state0, n_seg, t_seg, batch, max_per_seg=256):
        ops = _Ops([H0, Hd, P1, P2])
        As = _Ops(A)
        st = np.ascontiguousarray(state0, dtype=np.complex128)
        self._keep = (ops, As, st)
        sz = C.sizeof(qt_op)
        base = ops.ptr
        self.handle = C.c_void_p()
        _check(lib().qt_adjoint_create(base, base + sz, As.ptr, len(A), base + 2 * sz,
                                       base + 3 * sz, _ptr(st), 1 if st.ndim == 1 else 0, n_seg,
                                       t_seg, batch, max_per_seg, C.byref(self.handle)),
               "qt_adjoint_create")
        self.n_seg, self.nk, self.batch, self.max_per_seg = n_seg, len(A), batch, max_per_seg

    def forward(self, omega, gamma, opts, loss, stats=None, stream=None):
        _check(lib().qt_adjoint_forward_dev(self.handle, _tptr(omega), _tptr(gamma),
                                            C.byref(opts), _tptr(loss), _tptr(stats),
                                            _stream(stream)), "qt_adjoint_forward_dev")

    def loss_fixed(self, omega, gamma, loss, stream=None):
        _check(lib().qt_adjoint_loss_fixed_dev(self.handle, _tptr(omega), _tptr(gamma),
                                               _tptr(loss), _stream(stream)),
               "qt_adjoint_loss_fixed_dev")

    def backward(self, dloss, grad_omega, grad_gamma, stream=None):
        _check(lib().qt_adjoint_backward_dev(self.handle, _tptr(dloss), _tptr(grad_omega),
                                             _tptr(grad_gamma), _stream(stream)),
               "qt_adjoint_backward_dev")

    def grid(self, b):
        ns = np.zeros(self.n_seg, dtype=np.int32)
        h = np.zeros((self.n_seg, self.max_per_seg))
        _check(lib().qt_adjoint_grid(self.handle, b, _ptr(ns), _ptr(h)), "qt_adjoint_grid")
        return ns, h

    def close(self):
        if self.handle:
            lib().qt_adjoint_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def master_equation_loss(adjoint, omega, gamma, opts):
    """Differentiable losses L_b (one per parameter vector) of an Adjoint
    problem: forward by the adaptive solver, backward by the library's
    adjoint kernel on the forward pass's step grid (segment checkpoints
    recomputed).  omega: float64 CUDA tensor [batch, n_seg]; gamma:
    [batch, n_k]."""
    import torch

    class _MasterEquationLoss(torch.autograd.Function):
        @staticmethod
        def forward(ctx, om, ga):
            om_c, ga_c = om.detach().contiguous(), ga.detach().contiguous()
            loss = torch.empty(adjoint.batch, dtype=torch.float64, device=om.device)
            adjoint.forward(om_c, ga_c, opts, loss)
            return loss

        @staticmethod
        def backward(ctx, gloss):
            g = gloss.detach().to(torch.float64).contiguous()
            go = torch.empty((adjoint.batch, adjoint.n_seg), dtype=torch.float64, device=g.device)
            gg = torch.empty((adjoint.batch, max(adjoint.nk, 1)), dtype=torch.float64,
                             device=g.device)
            adjoint.backward(g, go, gg)
            return go, gg[:, :adjoint.nk]

    return _MasterEquationLoss.apply(omega, gamma)


def stats_from_bytes(t) -> dict:
    """Decode a qt_stats written to a uint8 tensor by a *_dev call."""
    a = np.frombuffer(t.cpu().numpy().tobytes(), dtype=STATS_DTYPE)[0]
    return {k: int(a[k]) for k in STATS_DTYPE.names if k != "reserved"}


def jumps_from_bytes(t, n) -> np.ndarray:
    a = np.frombuffer(t.cpu().numpy().tobytes(), dtype=JUMP_DTYPE)[:n].copy()
    a.sort(order=["traj", "k"])
    return a
