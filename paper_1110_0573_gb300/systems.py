"""Operator library and the synthetic test systems (inputs only).

This module builds the *inputs* of the solvers: Hamiltonians, collapse
operators, observables, initial states and time lists, as scipy.sparse CSR
matrices (complex128) and numpy arrays.  It holds none of the solvers'
arithmetic (no effective Hamiltonian, no right-hand side, no integrator), so
both the CUDA library's callers and the FP64 oracle's tests can take their
inputs from here.

Conventions (paper section 2, operator library of Appendix A):
  * hbar = 1.
  * tensor(A, B, ...) is the Kronecker product with the first factor most
    significant.
  * destroy(N)[n-1, n] = sqrt(n).
  * Two-level systems: basis index 0 is the ground state |g>, index 1 the
    excited state |e>; sigma_- = destroy(2) = |g><e|, sigma_+ = sigma_-^dag,
    sigma_z = sigma_+ sigma_- - sigma_- sigma_+ = diag(-1, +1),
    sigma_x = sigma_+ + sigma_-, sigma_y = -i sigma_+ + i sigma_-.
    (With this sign the Jaynes-Cummings example of section 4.2 is resonant at
    omega_0 = epsilon, as its figure caption states.)
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

TWO_PI = 2.0 * np.pi


def _csr(m) -> sp.csr_matrix:
    out = sp.csr_matrix(m, dtype=np.complex128)
    out.sort_indices()
    out.eliminate_zeros()
    return out


def qeye(n: int) -> sp.csr_matrix:
    return _csr(sp.identity(n, dtype=np.complex128))


def destroy(n: int) -> sp.csr_matrix:
    return _csr(sp.diags(np.sqrt(np.arange(1, n, dtype=np.float64)), 1, shape=(n, n)))


def create(n: int) -> sp.csr_matrix:
    return _csr(destroy(n).conj().T)


def num(n: int) -> sp.csr_matrix:
    return _csr(sp.diags(np.arange(n, dtype=np.float64), 0, shape=(n, n)))


def sigmam() -> sp.csr_matrix:
    return destroy(2)


def sigmap() -> sp.csr_matrix:
    return create(2)


def sigmaz() -> sp.csr_matrix:
    return _csr(sp.diags([-1.0, 1.0]))


def sigmax() -> sp.csr_matrix:
    return _csr(np.array([[0, 1], [1, 0]], dtype=np.complex128))


def sigmay() -> sp.csr_matrix:
    return _csr(np.array([[0, 1j], [-1j, 0]], dtype=np.complex128))


def basis(n: int, k: int) -> np.ndarray:
    v = np.zeros(n, dtype=np.complex128)
    v[k] = 1.0
    return v


fock = basis


def tensor(*ops):
    """Kronecker product, first factor most significant (operators or kets)."""
    if all(isinstance(o, np.ndarray) and o.ndim == 1 for o in ops):
        out = ops[0]
        for o in ops[1:]:
            out = np.kron(out, o)
        return out
    out = sp.csr_matrix(ops[0], dtype=np.complex128)
    for o in ops[1:]:
        out = sp.kron(out, sp.csr_matrix(o, dtype=np.complex128), format="csr")
    return _csr(out)


def dag(a) -> sp.csr_matrix:
    return _csr(sp.csr_matrix(a).conj().T)


def site_op(op, i: int, L: int, local_dim: int = 2) -> sp.csr_matrix:
    """op acting on site i of an L-site chain (site 0 most significant)."""
    factors = [qeye(local_dim)] * L
    factors[i] = op
    return tensor(*factors)


# --------------------------------------------------------------- systems
# Each builder returns a dict with H, c_ops, e_ops, psi0 (ket), tlist and a
# name; sizes are arguments so the tests can run small cases of each shape.


def jaynes_cummings(N=10, wc=TWO_PI, wa=TWO_PI, g=TWO_PI * 0.05, kappa=0.005, gamma=0.05,
                    n0=5, t_end=50.0, nt=201):
    """Dissipative Jaynes-Cummings model (paper Eq. (hamiltonian_jc), section
    4.2): H = wc a^dag a + wa sigma_z / 2 + g (a^dag sigma_- + a sigma_+),
    collapse sqrt(kappa) a and sqrt(gamma) sigma_-, psi0 = |n0> (x) |g>,
    observables <a^dag a> and <sigma_+ sigma_->."""
    a = tensor(destroy(N), qeye(2))
    sm = tensor(qeye(N), sigmam())
    sz = tensor(qeye(N), sigmaz())
    H = wc * dag(a) @ a + 0.5 * wa * sz + g * (dag(a) @ sm + a @ dag(sm))
    c_ops = []
    if kappa > 0:
        c_ops.append(_csr(np.sqrt(kappa) * a))
    if gamma > 0:
        c_ops.append(_csr(np.sqrt(gamma) * sm))
    e_ops = [_csr(dag(a) @ a), _csr(dag(sm) @ sm)]
    psi0 = tensor(basis(N, n0), basis(2, 0))
    return dict(name=f"jaynes_cummings_N{N}", H=_csr(H), c_ops=c_ops, e_ops=e_ops, psi0=psi0,
                tlist=np.linspace(0.0, t_end, nt))


def kerr_cavity(N=64, Delta=0.5, K=0.1, E=1.0, kappa=0.5, nth=0.1, t_end=20.0, nt=401):
    """Driven damped Kerr cavity: H = Delta a^dag a + (K/2) a^dag a^dag a a +
    E (a + a^dag), collapse sqrt(kappa) a and sqrt(kappa nth) a^dag, from the
    vacuum; observables <a^dag a> and <a>."""
    a = destroy(N)
    ad = dag(a)
    H = Delta * ad @ a + 0.5 * K * ad @ ad @ a @ a + E * (a + ad)
    c_ops = [_csr(np.sqrt(kappa) * a)]
    if nth > 0:
        c_ops.append(_csr(np.sqrt(kappa * nth) * ad))
    return dict(name=f"kerr_N{N}", H=_csr(H), c_ops=c_ops, e_ops=[_csr(ad @ a), _csr(a)],
                psi0=basis(N, 0), tlist=np.linspace(0.0, t_end, nt))


def xxz_chain(L=10, J=1.0, Delta=0.5, h=0.3, gamma_deph=0.05, gamma_damp=0.02, t_end=10.0,
              nt=101):
    """Dissipative XXZ chain in the paper's -1/2 convention (Eq. (spinchain)),
    open boundary, with a transverse field:
      H = -1/2 h sum_i sx_i - 1/2 J sum_i (sx_i sx_i+1 + sy_i sy_i+1 + Delta sz_i sz_i+1);
    collapse sqrt(gamma_deph) sz_i and sqrt(gamma_damp) s-_i on every site;
    Neel initial state |e, g, e, g, ...>; observables <sz_i> for every site."""
    sx = [site_op(sigmax(), i, L) for i in range(L)]
    sy = [site_op(sigmay(), i, L) for i in range(L)]
    sz = [site_op(sigmaz(), i, L) for i in range(L)]
    sm = [site_op(sigmam(), i, L) for i in range(L)]
    H = sp.csr_matrix((2**L, 2**L), dtype=np.complex128)
    for i in range(L):
        H = H - 0.5 * h * sx[i]
    for i in range(L - 1):
        H = H - 0.5 * J * (sx[i] @ sx[i + 1] + sy[i] @ sy[i + 1] + Delta * sz[i] @ sz[i + 1])
    c_ops = [_csr(np.sqrt(gamma_deph) * sz[i]) for i in range(L)]
    c_ops += [_csr(np.sqrt(gamma_damp) * sm[i]) for i in range(L)]
    psi0 = tensor(*[basis(2, 1 if i % 2 == 0 else 0) for i in range(L)])
    return dict(name=f"xxz_L{L}", H=_csr(H), c_ops=c_ops, e_ops=[_csr(s) for s in sz],
                psi0=psi0, tlist=np.linspace(0.0, t_end, nt))


def tight_binding_chain(d=300, J=1.0, gamma=0.05, t_end=1.0, nt=11):
    """A particle hopping on an open chain of d sites: H = -J sum_i (|i><i+1| +
    |i+1><i|), one collapse operator sqrt(gamma) sum_i |i><i+1| (a step
    towards site 0), from the middle site; observables the mean position / d
    and the population of the middle site.  H_eff has one off-diagonal value
    and columns i +- 1 (not a fixed set of bit flips, unlike a spin chain)."""
    hop = sp.diags([np.ones(d - 1)], [1], shape=(d, d), format="csr", dtype=np.complex128)
    H = -J * (hop + hop.T)
    pos = sp.diags([np.arange(d) / d], [0], format="csr", dtype=np.complex128)
    mid = np.zeros(d)
    mid[d // 2] = 1.0
    return dict(name=f"tight_binding_{d}", H=_csr(H), c_ops=[_csr(np.sqrt(gamma) * hop)],
                e_ops=[_csr(pos), _csr(sp.diags([mid], [0], dtype=np.complex128))],
                psi0=basis(d, d // 2), tlist=np.linspace(0.0, t_end, nt))


def cavity_thermal_decay(N=5, kappa=1.0 / 0.129, nth=0.063, n0=1, t_end=0.6, nt=100):
    """Single-photon cavity decay in a thermal bath (paper section 3.2.1,
    Eq. (heffth)): H = a^dag a, collapse sqrt(kappa (1 + nth)) a and
    sqrt(kappa nth) a^dag, psi0 = |n0>, observable <a^dag a>."""
    a = destroy(N)
    c_ops = [_csr(np.sqrt(kappa * (1 + nth)) * a)]
    if nth > 0:
        c_ops.append(_csr(np.sqrt(kappa * nth) * dag(a)))
    return dict(name=f"cavity_decay_N{N}", H=_csr(dag(a) @ a), c_ops=c_ops,
                e_ops=[_csr(dag(a) @ a)], psi0=basis(N, n0), tlist=np.linspace(0.0, t_end, nt))


def driven_tls(Delta=0.3, Omega=1.0, gamma=0.5, t_end=40.0, nt=81):
    """Driven damped two-level system: H = Delta sigma_+ sigma_- +
    (Omega / 2) sigma_x, collapse sqrt(gamma) sigma_-, from |g>; observable
    sigma_+ sigma_-."""
    sm = sigmam()
    H = Delta * dag(sm) @ sm + 0.5 * Omega * sigmax()
    return dict(name="driven_tls", H=_csr(H), c_ops=[_csr(np.sqrt(gamma) * sm)],
                e_ops=[_csr(dag(sm) @ sm)], psi0=basis(2, 0), tlist=np.linspace(0.0, t_end, nt))


def iswap_pair(g=TWO_PI, nt=100):
    """Two qubits under H = g (sx (x) sx + sy (x) sy) for T = pi / (4 g)
    (paper Eq. (hamiltonian_iswap), section 4.1), closed system, from
    |e> (x) |g>."""
    H = g * (tensor(sigmax(), sigmax()) + tensor(sigmay(), sigmay()))
    T = np.pi / (4 * g)
    psi0 = tensor(basis(2, 1), basis(2, 0))
    e_ops = [tensor(dag(sigmam()) @ sigmam(), qeye(2)), tensor(qeye(2), dag(sigmam()) @ sigmam())]
    return dict(name="iswap", H=_csr(H), c_ops=[], e_ops=[_csr(e) for e in e_ops], psi0=psi0,
                tlist=np.linspace(0.0, T, nt))


def random_system(d, n_c, n_e, seed, density=0.3, nt=11, t_end=1.0):
    """Random sparse Hermitian H, random sparse collapse operators and
    Hermitian observables, a random ket; for parity tests over many shapes.
    Generated with numpy's Philox bit generator."""
    rng = np.random.Generator(np.random.Philox(seed))

    def rand_sparse(herm):
        mask = rng.random((d, d)) < density
        m = (rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))) * mask
        if herm:
            m = 0.5 * (m + m.conj().T)
        return m

    H = rand_sparse(True) + np.diag(rng.standard_normal(d))
    c_ops = [_csr(0.3 * rand_sparse(False)) for _ in range(n_c)]
    e_ops = [_csr(rand_sparse(True)) for _ in range(n_e)]
    psi0 = rng.standard_normal(d) + 1j * rng.standard_normal(d)
    psi0 /= np.linalg.norm(psi0)
    return dict(name=f"random_d{d}_c{n_c}_s{seed}", H=_csr(H), c_ops=c_ops, e_ops=e_ops,
                psi0=psi0, tlist=np.linspace(0.0, t_end, nt))


def landau_zener(delta=TWO_PI * 0.5, v=TWO_PI * 2.0, t0=-10.0, t1=10.0, nt=201, gamma=0.0):
    """Landau-Zener sweep (paper section 4.3, Eq. (lz-hamiltonian)):
    H(t) = (delta/2) sigma_x + (v t/2) sigma_z, written as H0 + f(t) H1 with
    H0 = (delta/2) sigma_x, H1 = (v/2) sigma_z and f(t) = t (two knots, exact
    on [t0, t1]); psi0 = basis 0; observables sigma_+ sigma_-, sigma_x,
    sigma_y, sigma_z; optional decay sqrt(gamma) sigma_-."""
    H0 = (delta / 2.0) * sigmax()
    H1 = (v / 2.0) * sigmaz()
    sm = sigmam()
    c_ops = [np.sqrt(gamma) * sm] if gamma > 0 else []
    return dict(name="landau_zener", H=_csr(H0), td=[(_csr(H1), np.array([t0, t1]), np.array([t0, t1]))],
                c_ops=c_ops, e_ops=[_csr(sm.T.conj() @ sm), sigmax(), sigmay(), sigmaz()],
                psi0=basis(2, 0), tlist=np.linspace(t0, t1, nt), delta=delta, v=v)


def coherent(n: int, alpha: complex) -> np.ndarray:
    """Truncated coherent state |alpha> (Fock amplitudes e^{-|a|^2/2} a^k /
    sqrt(k!)), renormalised after the truncation."""
    k = np.arange(n)
    logfact = np.concatenate([[0.0], np.cumsum(np.log(np.arange(1, n)))])
    amp = np.exp(-abs(alpha) ** 2 / 2 + k * np.log(abs(alpha) + 1e-300) - logfact / 2)
    v = amp * np.exp(1j * np.angle(alpha) * k)
    return v / np.linalg.norm(v)


def trilinear(N=17, K=1.0, g=(0.1, 0.4, 0.1), alpha=np.sqrt(10.0), t_end=4.0, nt=201):
    """Trilinear Hamiltonian of paper section 4.3 (Eq. (trilinear)): pump a,
    signal b, idler c, H = i K (a b^dag c^dag - a^dag b c), collapse
    sqrt(2 g_i) on each mode's lowering operator, pump coherent with
    |alpha|^2 = 10, signal and idler in vacuum; observables the three
    occupation numbers; dim N^3 (4913 at N = 17)."""
    a = tensor(destroy(N), qeye(N), qeye(N))
    b = tensor(qeye(N), destroy(N), qeye(N))
    c = tensor(qeye(N), qeye(N), destroy(N))
    H = 1j * K * (a @ b.T.conj() @ c.T.conj() - a.T.conj() @ b @ c)
    c_ops = [np.sqrt(2.0 * gi) * op for gi, op in zip(g, (a, b, c))]
    e_ops = [op.T.conj() @ op for op in (a, b, c)]
    psi0 = np.kron(np.kron(coherent(N, alpha), basis(N, 0)), basis(N, 0))
    return dict(name=f"trilinear_N{N}", H=_csr(H), c_ops=[_csr(x) for x in c_ops],
                e_ops=[_csr(x) for x in e_ops], psi0=psi0, tlist=np.linspace(0.0, t_end, nt))


def dense_random_hamiltonian(d=1024, seed=3, gamma=0.1, t_end=0.5, nt=6):
    """A system whose Hamiltonian is a dense matrix (every entry nonzero): a
    random Hermitian H (complex Gaussian entries scaled by 1/sqrt(d), so that
    its spectrum spans about [-2, 2]) on a d-level ladder with decay
    sqrt(gamma) a and dephasing sqrt(gamma) n/d; from the ladder's top state,
    observables n/d and the ground-state projector.  numpy Philox generator."""
    rng = np.random.Generator(np.random.Philox(seed))
    X = (rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))) / np.sqrt(2.0 * d)
    H = 0.5 * (X + X.conj().T)
    a = destroy(d)
    n = num(d)
    P0 = _csr(np.diag(np.eye(d)[0]))
    return dict(name=f"dense_random_d{d}", H=_csr(H), c_ops=[np.sqrt(gamma) * a, np.sqrt(gamma) * n / d],
                e_ops=[n / d, P0], psi0=basis(d, d - 1), tlist=np.linspace(0.0, t_end, nt))


def dense_collapse_system(d=1024, n_c=2, seed=4, t_end=0.1, nt=3):
    """Dense Hamiltonian and dense collapse operators: a random Hermitian H
    (complex Gaussian entries scaled by 1/sqrt(2d)) and n_c random complex
    collapse operators with entries of scale 0.3/sqrt(2d), from a random ket;
    observables n/d on the basis index and the ground-state projector.  numpy
    Philox generator."""
    rng = np.random.Generator(np.random.Philox(seed))
    X = (rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))) / np.sqrt(2.0 * d)
    H = 0.5 * (X + X.conj().T)
    c_ops = [_csr(0.3 * (rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))) /
                  np.sqrt(2.0 * d)) for _ in range(n_c)]
    psi = rng.standard_normal(d) + 1j * rng.standard_normal(d)
    return dict(name=f"dense_collapse_d{d}_c{n_c}", H=_csr(H), c_ops=c_ops,
                e_ops=[num(d) / d, _csr(np.diag(np.eye(d)[0]))], psi0=psi / np.linalg.norm(psi),
                tlist=np.linspace(0.0, t_end, nt))


def cavity_qubit_sweep(n_instances=4096, seed=1, g=0.3, ntraj=256, t_end=30.0, nt=121,
                       cutoff=(4, 32)):
    """A parameter sweep of driven damped cavity + qubit systems of uneven
    dimension: per instance a cavity cutoff N_c uniform in cutoff (dim 2 N_c),
    detuning delta ~ U[-1, 1], drive E ~ U[0, 2], decay kappa ~ U[0.01, 0.5];
    H = delta (a^dag a + sigma_+ sigma_-) + g (a^dag sigma_- + a sigma_+)
        + E (a + a^dag), collapse sqrt(kappa) a, from |0, g>, observables
    <a^dag a> and <sigma_+ sigma_->.  Even instances are master-equation
    problems, odd ones Monte-Carlo problems with ntraj trajectories (seed =
    instance index).  Parameters from numpy's Philox generator."""
    rng = np.random.Generator(np.random.Philox(seed))
    problems = []
    cache = {}
    for i in range(n_instances):
        nc = int(rng.integers(cutoff[0], cutoff[1] + 1))
        delta = float(rng.uniform(-1.0, 1.0))
        E = float(rng.uniform(0.0, 2.0))
        kappa = float(rng.uniform(0.01, 0.5))
        if nc not in cache:
            a = tensor(destroy(nc), qeye(2))
            sm = tensor(qeye(nc), sigmam())
            cache[nc] = (a, sm, dag(a) @ a + dag(sm) @ sm, dag(a) @ sm + a @ dag(sm),
                         a + dag(a), [_csr(dag(a) @ a), _csr(dag(sm) @ sm)],
                         tensor(basis(nc, 0), basis(2, 0)))
        a, sm, nsum, coup, drive, e_ops, psi0 = cache[nc]
        H = _csr(delta * nsum + g * coup + E * drive)
        problems.append(dict(H=H, c_ops=[_csr(np.sqrt(kappa) * a)], e_ops=e_ops, state0=psi0,
                             kind="me" if i % 2 == 0 else "mc", ntraj=ntraj, seed=i,
                             dim=2 * nc))
    return problems, np.linspace(0.0, t_end, nt)


def transmon_cavity(N=20, chi=TWO_PI * 0.002, alpha=-TWO_PI * 0.2, T1=20.0, T2=15.0,
                    kappa=0.001, n_seg=64, t_seg=1.0):
    """Driven transmon (3 levels) (x) cavity (N levels) in the rotating frame:
    H0 = (alpha / 2) b^dag b^dag b b + chi a^dag a b^dag b, drive operator
    Hd = b + b^dag with amplitude Omega_s on segment s (length t_seg);
    collapse shapes b, b^dag b, a with rates 1/T1, 2 gamma_phi
    (gamma_phi = 1/T2 - 1/(2 T1)) and kappa; from |g, 0>; loss operators
    P1 = |1><1| (transmon, final population) and P2 = |2><2| (leakage,
    integrated over time)."""
    b = tensor(destroy(3), qeye(N))
    a = tensor(qeye(3), destroy(N))
    bd, ad = dag(b), dag(a)
    H0 = 0.5 * alpha * bd @ bd @ b @ b + chi * (ad @ a) @ (bd @ b)
    gphi = 1.0 / T2 - 1.0 / (2.0 * T1)
    proj = lambda k: tensor(_csr(np.diag(np.eye(3)[k])), qeye(N))
    return dict(name=f"transmon_cavity_N{N}", H0=_csr(H0), Hd=_csr(b + bd),
                A=[_csr(b), _csr(bd @ b), _csr(a)],
                gamma=np.array([1.0 / T1, 2.0 * gphi, kappa]), P1=proj(1), P2=proj(2),
                psi0=tensor(basis(3, 0), basis(N, 0)), n_seg=n_seg, t_seg=t_seg)


def drive_vectors(batch=256, n_seg=64, amp=0.05, seed=2):
    """Piecewise-constant drive amplitudes Omega ~ U[-amp, amp] (numpy Philox)."""
    rng = np.random.Generator(np.random.Philox(seed))
    return rng.uniform(-amp, amp, size=(batch, n_seg))
