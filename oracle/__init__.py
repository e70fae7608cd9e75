"""FP64 CPU oracle for the QuTiP paper's master-equation and Monte-Carlo
solvers (paper sections 3.1 and 3.2).

TEST INFRASTRUCTURE ONLY: the test-suite, the smoke check and the CPU-baseline
leg of the benchmark use this package to check and time the CUDA library.  It
shares no code with the library and the library never calls it.

The arithmetic lives in ``qt_oracle.c`` (plain C, FP64); this module compiles
it with gcc on first use and marshals numpy arrays through ctypes.
Operators may be given as scipy.sparse matrices or dense numpy arrays; they are
handed to C as CSR with int64 row pointers, int32 columns and complex128
values.

Pinned by ``tests/test_oracle_*.py`` against closed forms, matrix-exponential
brute force, invariants and cuRAND's Philox4x32-10.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np
import scipy.sparse as sp

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qt_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, EINVAL, ENORM, ENOMEM, ESTEP, ENUMERIC, ECAP = 0, -1, -3, -4, -6, -9, -10


class OracleError(RuntimeError):
    def __init__(self, code, where):
        super().__init__(f"oracle {where} failed with status {code}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile qt_oracle.c into oracle/_build/liboracle.so (gcc, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and \
            os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-fopenmp", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _CSR(C.Structure):
    _fields_ = [("d", C.c_int32), ("indptr", C.c_void_p), ("indices", C.c_void_p),
                ("values", C.c_void_p)]


class _Stats(C.Structure):
    _fields_ = [("accepted", C.c_int64), ("rejected", C.c_int64), ("rhs_evals", C.c_int64),
                ("bisect_iters", C.c_int64), ("jumps", C.c_int64)]


JUMP_DTYPE = np.dtype([("traj", np.int64), ("k", np.int64), ("channel", np.int64),
                       ("tau", np.float64), ("degenerate", np.int64)])


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P, I, D, I64, U64 = C.c_void_p, C.c_int, C.c_double, C.c_int64, C.c_uint64
            lib.or_philox4x32_10.argtypes = [P, P, P]
            lib.or_uniform.argtypes = [U64, U64, U64, C.c_uint32]
            lib.or_uniform.restype = D
            lib.or_mesolve.argtypes = [I, P, P, I, P, I, P, P, I, D, D, D, I64, P, P, P, P]
            lib.or_mcsolve.argtypes = [I, P, P, I, P, I, P, P, I, I64, I64, U64, D, D, D, I64,
                                       D, P, P, I64, P, P, I, P]
            lib.or_me_rhs_td.argtypes = [I, P, P, I, P, D, P, P]
            lib.or_mc_rhs_td.argtypes = [I, P, P, I, P, D, P, P]
            lib.or_td_coef.argtypes = [P, I, D]
            lib.or_td_coef.restype = D
            lib.or_expect.argtypes = [P, P, I, I64, P]
            lib.or_mc_dp45_step.argtypes = [I, P, P, I, P, D, P]
            lib.or_mc_rhs.argtypes = [I, P, P, I, P, P]
            lib.or_me_rhs.argtypes = [I, P, P, I, P, P]
            lib.or_dp45_tableau.argtypes = [P, P, P, P]
            lib.or_has_openmp.restype = I
            lib.or_adjoint_forward.argtypes = [I, P, P, P, I, P, P, P, I, D, P, P, D, D, I, P, P, P]
            lib.or_adjoint_loss_fixed.argtypes = [I, P, P, P, I, P, P, P, I, P, P, I, P, P, P]
            lib.or_adjoint_grad.argtypes = [I, P, P, P, I, P, P, P, I, P, P, I, P, P, P, P, P]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


class _OpPack:
    """Keeps CSR arrays alive while C uses them."""

    def __init__(self, ops, d):
        self.keep = []
        self.arr = (_CSR * max(1, len(ops)))()
        for i, op in enumerate(ops):
            m = sp.csr_matrix(op, dtype=np.complex128)
            if m.shape != (d, d):
                raise ValueError(f"operator {i} has shape {m.shape}, expected {(d, d)}")
            m.sort_indices()
            indptr = np.ascontiguousarray(m.indptr, dtype=np.int64)
            indices = np.ascontiguousarray(m.indices, dtype=np.int32)
            values = np.ascontiguousarray(m.data, dtype=np.complex128)
            self.keep += [indptr, indices, values]
            self.arr[i] = _CSR(d, _ptr(indptr), _ptr(indices), _ptr(values))

    @property
    def ptr(self):
        return C.addressof(self.arr)


def _dim(H):
    return int(H.shape[0])


class _TdStruct(C.Structure):
    _fields_ = [("n", C.c_int), ("H", C.c_void_p), ("off", C.c_void_p), ("t", C.c_void_p),
                ("v", C.c_void_p)]


class _Td:
    """Time-dependent terms [(H_k, knot_times, knot_values), ...] of
    H(t) = H + sum_k f_k(t) H_k (piecewise-linear f_k, constant outside the
    knots), kept alive while C uses them."""

    def __init__(self, td, d):
        td = list(td or [])
        self.ops = _OpPack([h for h, _, _ in td], d)
        ts = [np.asarray(t, dtype=np.float64).reshape(-1) for _, t, _ in td]
        vs = [np.asarray(v, dtype=np.float64).reshape(-1) for _, _, v in td]
        for k, (t, v) in enumerate(zip(ts, vs)):
            if len(t) < 1 or len(t) != len(v) or np.any(np.diff(t) <= 0):
                raise ValueError(f"term {k}: knot times must be strictly increasing, one value each")
        self.off = np.ascontiguousarray(np.concatenate([[0], np.cumsum([len(t) for t in ts])]),
                                        dtype=np.int64)
        self.t = np.ascontiguousarray(np.concatenate(ts) if ts else np.zeros(1), dtype=np.float64)
        self.v = np.ascontiguousarray(np.concatenate(vs) if vs else np.zeros(1), dtype=np.float64)
        self.st = _TdStruct(len(td), self.ops.ptr, _ptr(self.off), _ptr(self.t), _ptr(self.v))
        self.n = len(td)

    @property
    def ptr(self):
        return C.addressof(self.st) if self.n else None


def td_coef(td, k, t):
    """f_k(t) of the time-dependent terms td (the oracle's definition)."""
    T = _Td(td, _dim(td[0][0]))
    return _load().or_td_coef(T.ptr, k, float(t))


def _stats(s: _Stats) -> dict:
    return {k: int(getattr(s, k)) for k, _ in _Stats._fields_}


def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 block: 4 x uint32 counter, 2 x uint32 key -> 4 x uint32."""
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.or_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def uniform(seed: int, traj: int, k: int, stream: int) -> float:
    """U(seed, traj, k, stream) in (0, 1): the jump threshold (stream 0) or the
    channel draw (stream 1) of jump k of trajectory traj."""
    return float(_load().or_uniform(seed, traj, k, stream))


def ket_to_dm(psi) -> np.ndarray:
    """rho0 = |psi><psi| / <psi|psi> for a ket initial state (paper section 4.1
    passes a ket to odesolve)."""
    v = np.asarray(psi, dtype=np.complex128).reshape(-1)
    return np.outer(v, v.conj()) / np.vdot(v, v).real


def mesolve(H, c_ops, e_ops, state0, tlist, rtol=1e-8, atol=None, h0=0.0,
            max_steps=10**6, store_states=False, td=None):
    """Lindblad master equation (Eq. (master_equation)) over tlist.

    state0: a ket (d,) or a density matrix (d, d); td: time-dependent terms
    [(H_k, knot_times, knot_values), ...] of H(t) = H + sum_k f_k(t) H_k.
    Returns (expect[nt, ne] complex, states[nt, d, d] or None, stats dict)."""
    lib = _load()
    d = _dim(H)
    atol = rtol * 1e-2 if atol is None else atol
    s0 = np.asarray(state0, dtype=np.complex128)
    rho0 = ket_to_dm(s0) if s0.ndim == 1 or s0.shape == (d, 1) else np.ascontiguousarray(s0)
    tl = np.ascontiguousarray(tlist, dtype=np.float64)
    nt, ne, nc = len(tl), len(e_ops), len(c_ops)
    Hp, Cp, Ep = _OpPack([H], d), _OpPack(c_ops, d), _OpPack(e_ops, d)
    out = np.zeros((nt, max(ne, 1)), dtype=np.complex128)
    states = np.zeros((nt, d, d), dtype=np.complex128) if store_states else None
    st = _Stats()
    T = _Td(td, d)
    rc = lib.or_mesolve(d, Hp.ptr, Cp.ptr, nc, Ep.ptr, ne, _ptr(rho0), _ptr(tl), nt, rtol,
                        atol, h0, max_steps, _ptr(out),
                        _ptr(states) if states is not None else None, C.byref(st), T.ptr)
    if rc != OK:
        raise OracleError(rc, "mesolve")
    return out[:, :ne], states, _stats(st)


def mcsolve(H, c_ops, e_ops, psi0, tlist, ntraj, seed=0, rtol=1e-8, atol=None, h0=0.0,
            max_steps=10**6, bisect_tol=1e-13, traj_begin=0, nthreads=1, jump_cap=None,
            td=None):
    """Monte-Carlo wave-function trajectories traj_begin .. traj_begin+ntraj-1
    (section 3.2, steps I-IV).  With no collapse operators a single trajectory
    is run (the Schrodinger equation, section 4.3).

    Returns (traj_expect[ntraj, nt, ne] complex: normalised per-trajectory
    expectation values, jumps: structured array JUMP_DTYPE, stats dict)."""
    lib = _load()
    d = _dim(H)
    atol = rtol * 1e-2 if atol is None else atol
    if len(c_ops) == 0:
        ntraj = 1
    psi = np.ascontiguousarray(np.asarray(psi0, dtype=np.complex128).reshape(-1))
    tl = np.ascontiguousarray(tlist, dtype=np.float64)
    nt, ne, nc = len(tl), len(e_ops), len(c_ops)
    Hp, Cp, Ep = _OpPack([H], d), _OpPack(c_ops, d), _OpPack(e_ops, d)
    out = np.zeros((ntraj, nt, max(ne, 1)), dtype=np.complex128)
    cap = 64 * ntraj + 1024 if jump_cap is None else jump_cap
    jumps = np.zeros(max(cap, 1), dtype=JUMP_DTYPE)
    nj = C.c_int64(0)
    st = _Stats()
    T = _Td(td, d)
    rc = lib.or_mcsolve(d, Hp.ptr, Cp.ptr, nc, Ep.ptr, ne, _ptr(psi), _ptr(tl), nt,
                        traj_begin, traj_begin + ntraj, seed, rtol, atol, h0, max_steps,
                        bisect_tol, _ptr(out), _ptr(jumps), cap, C.byref(nj), C.byref(st),
                        nthreads, T.ptr)
    if rc == ECAP and jump_cap is None:
        return mcsolve(H, c_ops, e_ops, psi0, tlist, ntraj, seed, rtol, atol, h0, max_steps,
                       bisect_tol, traj_begin, nthreads, jump_cap=int(nj.value), td=td)
    if rc != OK:
        raise OracleError(rc, "mcsolve")
    return out[:, :, :ne], jumps[: nj.value].copy(), _stats(st)


def correlation_2op_2t(H, c_ops, A, B, state0, tlist, taulist, rtol=1e-8, atol=None,
                       h0=0.0, max_steps=10**6, td=None):
    """Two-time correlation <A(t_k + tau_j) B(t_k)> by the quantum regression
    theorem, the ODE form of the paper's correlation functions (section 5,
    function list): rho(t_k) from the master equation over tlist, then the
    matrix X_k = B rho(t_k) evolved by the same Lindblad equation from t_k,
    and C[k, j] = Tr(A X_k(t_k + tau_j)).  taulist starts at 0.  Every solve
    is mesolve above.

    Returns (corr[n_t, n_tau] complex, stats summed over the n_t + 1 solves)."""
    tl = np.asarray(tlist, dtype=np.float64)
    tau = np.asarray(taulist, dtype=np.float64)
    if tau[0] != 0.0:
        raise OracleError(EINVAL, "correlation_2op_2t (taulist must start at 0)")
    _, rho, stats = mesolve(H, c_ops, [], state0, tl, rtol, atol, h0, max_steps,
                            store_states=True, td=td)
    Bd = B.toarray() if sp.issparse(B) else np.asarray(B, dtype=np.complex128)
    out = np.zeros((len(tl), len(tau)), dtype=np.complex128)
    for k in range(len(tl)):
        X = Bd @ rho[k]
        ex, _, st = mesolve(H, c_ops, [A], X, tl[k] + tau, rtol, atol, h0, max_steps, td=td)
        out[k] = ex[:, 0]
        for key in stats:
            stats[key] += st[key]
    return out, stats


def propagator(H, c_ops, tlist, rtol=1e-8, atol=None, h0=0.0, max_steps=10**6, td=None):
    """The master-equation propagator (the paper's propagator, section 5
    function list): U[k] maps rho(tlist[0]) to rho(tlist[k]) as a
    d^2 x d^2 matrix on row-major vec(rho); column a d + b is the solution
    from the matrix unit E_ab (mesolve above, one solve per unit).

    Returns (U[nt, d^2, d^2] complex, stats summed over the d^2 solves)."""
    d = _dim(H)
    tl = np.asarray(tlist, dtype=np.float64)
    U = np.zeros((len(tl), d * d, d * d), dtype=np.complex128)
    stats = None
    E = np.zeros((d, d), dtype=np.complex128)
    for a in range(d):
        for b in range(d):
            E[a, b] = 1.0
            _, states, st = mesolve(H, c_ops, [], E, tl, rtol, atol, h0, max_steps,
                                    store_states=True, td=td)
            E[a, b] = 0.0
            U[:, :, a * d + b] = states.reshape(len(tl), d * d)
            if stats is None:
                stats = dict(st)
            else:
                for key in stats:
                    stats[key] += st[key]
    return U, stats


def correlation_ss(H, c_ops, A, B, taulist, rtol=1e-8, atol=None):
    """<A(tau) B(0)> with the system in its steady state: steadystate below,
    then correlation_2op_2t above from it at the single time 0."""
    rho, _ = steadystate(H, c_ops)
    corr, stats = correlation_2op_2t(H, c_ops, A, B, rho, [0.0], taulist, rtol, atol)
    return corr[0], stats


def liouvillian_matrix(H, c_ops):
    """The master-equation generator as a d^2 x d^2 matrix in row-major vec
    form (column a d + b = me_rhs of the matrix unit E_ab)."""
    d = _dim(H)
    L = np.zeros((d * d, d * d), dtype=np.complex128)
    E = np.zeros((d, d), dtype=np.complex128)
    for a in range(d):
        for b in range(d):
            E[a, b] = 1.0
            L[:, a * d + b] = me_rhs(H, c_ops, E).reshape(-1)
            E[a, b] = 0.0
    return L


def steadystate(H, c_ops):
    """Steady state of the master equation (the paper's steadystate, section 5
    function list): the density matrix rho with L(rho) = 0 and Tr rho = 1,
    taken as the right singular vector of the Liouvillian matrix for its
    smallest singular value, made Hermitian ((X + X^dag) / 2) and scaled to
    unit trace.  Raises when the null space is not one-dimensional (second
    smallest singular value below 1e-10 of the largest).

    Returns (rho[d, d], singular values in increasing order)."""
    d = _dim(H)
    L = liouvillian_matrix(H, c_ops)
    _, sv, vh = np.linalg.svd(L)
    if sv[-2] <= 1e-10 * sv[0]:
        raise OracleError(EINVAL, "steadystate (the stationary state is not unique)")
    X = vh[-1].conj().reshape(d, d)
    X = 0.5 * (X + X.conj().T)
    return X / np.trace(X).real, sv[::-1]


def expect(O, states, is_ket):
    """<psi|O|psi> per ket (not normalised) or Tr(O rho) per density matrix."""
    lib = _load()
    d = _dim(O)
    s = np.ascontiguousarray(states, dtype=np.complex128)
    batch = s.size // (d if is_ket else d * d)
    Op = _OpPack([O], d)
    out = np.zeros(batch, dtype=np.complex128)
    rc = lib.or_expect(Op.ptr, _ptr(s), int(bool(is_ket)), batch, _ptr(out))
    if rc != OK:
        raise OracleError(rc, "expect")
    return out


def me_rhs(H, c_ops, rho, td=None, t=0.0):
    """Right-hand side of Eq. (master_equation) at rho (and time t when the
    Hamiltonian has time-dependent terms td)."""
    lib = _load()
    d = _dim(H)
    r = np.ascontiguousarray(rho, dtype=np.complex128)
    out = np.zeros((d, d), dtype=np.complex128)
    Hp, Cp = _OpPack([H], d), _OpPack(c_ops, d)
    if td:
        T = _Td(td, d)
        lib.or_me_rhs_td(d, Hp.ptr, Cp.ptr, len(c_ops), T.ptr, float(t), _ptr(r), _ptr(out))
    else:
        lib.or_me_rhs(d, Hp.ptr, Cp.ptr, len(c_ops), _ptr(r), _ptr(out))
    return out


def mc_rhs(H, c_ops, psi, td=None, t=0.0):
    """-i H_eff psi with H_eff of Eq. (heff) (at time t with terms td)."""
    lib = _load()
    d = _dim(H)
    v = np.ascontiguousarray(psi, dtype=np.complex128)
    out = np.zeros(d, dtype=np.complex128)
    Hp, Cp = _OpPack([H], d), _OpPack(c_ops, d)
    if td:
        T = _Td(td, d)
        lib.or_mc_rhs_td(d, Hp.ptr, Cp.ptr, len(c_ops), T.ptr, float(t), _ptr(v), _ptr(out))
    else:
        lib.or_mc_rhs(d, Hp.ptr, Cp.ptr, len(c_ops), _ptr(v), _ptr(out))
    return out


def mc_dp45_step(H, c_ops, psi, h):
    """One Dormand-Prince step of length h of d psi/dt = -i H_eff psi."""
    lib = _load()
    d = _dim(H)
    v = np.ascontiguousarray(psi, dtype=np.complex128)
    out = np.zeros(d, dtype=np.complex128)
    Hp, Cp = _OpPack([H], d), _OpPack(c_ops, d)
    rc = lib.or_mc_dp45_step(d, Hp.ptr, Cp.ptr, len(c_ops), _ptr(v), h, _ptr(out))
    if rc != OK:
        raise OracleError(rc, "dp45 step")
    return out


def dp45_tableau():
    """(c[7], A[7, 6], b5[7], b4[7]) as used by the oracle's integrator."""
    lib = _load()
    c = np.zeros(7)
    a = np.zeros((7, 6))
    b5 = np.zeros(7)
    b4 = np.zeros(7)
    lib.or_dp45_tableau(_ptr(c), _ptr(a), _ptr(b5), _ptr(b4))
    return c, a, b5, b4


def openmp_threads() -> int:
    """Maximum OpenMP threads (0 if built without OpenMP)."""
    return int(_load().or_has_openmp())


# ------------------------------------------------- master-equation adjoint


class AdjointProblem:
    """A master equation with piecewise-constant drive and decay rates as
    parameters: F = -i[H0 + Omega_s Hd, .] + sum_k gamma_k D[A_k];
    loss = Re Tr(P1 rho(T)) + int_0^T Re Tr(P2 rho) dt."""

    def __init__(self, H0, Hd, A, P1, P2, state0, n_seg, t_seg, max_per_seg=256):
        self.d = _dim(H0)
        self._H0, self._Hd = _OpPack([H0], self.d), _OpPack([Hd], self.d)
        self._A = _OpPack(A, self.d)
        self._P1, self._P2 = _OpPack([P1], self.d), _OpPack([P2], self.d)
        s0 = np.asarray(state0, dtype=np.complex128)
        self.rho0 = ket_to_dm(s0) if s0.ndim == 1 else np.ascontiguousarray(s0)
        self.nk = len(A)
        self.n_seg, self.t_seg, self.max_per_seg = n_seg, t_seg, max_per_seg

    def _args(self):
        return (self.d, self._H0.ptr, self._Hd.ptr, self._A.ptr, self.nk, self._P1.ptr,
                self._P2.ptr, _ptr(self.rho0), self.n_seg)

    def forward(self, omega, gamma, rtol=1e-8, atol=1e-10):
        """Adaptive solve: (loss, nsteps[n_seg], hgrid[n_seg, max_per_seg])."""
        om = np.ascontiguousarray(omega, dtype=np.float64)
        ga = np.ascontiguousarray(gamma, dtype=np.float64)
        nsteps = np.zeros(self.n_seg, dtype=np.int32)
        hgrid = np.zeros((self.n_seg, self.max_per_seg))
        loss = C.c_double(0.0)
        rc = _load().or_adjoint_forward(*self._args(), self.t_seg, _ptr(om), _ptr(ga), rtol, atol,
                                        self.max_per_seg, _ptr(nsteps), _ptr(hgrid),
                                        C.byref(loss))
        if rc != OK:
            raise OracleError(rc, "adjoint forward")
        return loss.value, nsteps, hgrid

    def loss_fixed(self, omega, gamma, nsteps, hgrid):
        om = np.ascontiguousarray(omega, dtype=np.float64)
        ga = np.ascontiguousarray(gamma, dtype=np.float64)
        ns = np.ascontiguousarray(nsteps, dtype=np.int32)
        hg = np.ascontiguousarray(hgrid, dtype=np.float64)
        loss = C.c_double(0.0)
        rc = _load().or_adjoint_loss_fixed(*self._args(), _ptr(om), _ptr(ga), hg.shape[1],
                                           _ptr(ns), _ptr(hg), C.byref(loss))
        if rc != OK:
            raise OracleError(rc, "adjoint loss")
        return loss.value

    def grad(self, omega, gamma, nsteps, hgrid):
        """(loss, dL/domega[n_seg], dL/dgamma[nk]) on the fixed grid."""
        om = np.ascontiguousarray(omega, dtype=np.float64)
        ga = np.ascontiguousarray(gamma, dtype=np.float64)
        ns = np.ascontiguousarray(nsteps, dtype=np.int32)
        hg = np.ascontiguousarray(hgrid, dtype=np.float64)
        loss = C.c_double(0.0)
        go = np.zeros(self.n_seg)
        gg = np.zeros(self.nk)
        rc = _load().or_adjoint_grad(*self._args(), _ptr(om), _ptr(ga), hg.shape[1], _ptr(ns),
                                     _ptr(hg), C.byref(loss), _ptr(go), _ptr(gg))
        if rc != OK:
            raise OracleError(rc, "adjoint gradient")
        return loss.value, go, gg
