"""Pins of the oracle's master-equation solver (paper section 3.1).

* The right-hand side against the Kronecker-product Liouvillian.
* The solution against expm(L t) on tiny random systems.
* Closed forms: cavity decay at zero and finite temperature (the system of
  the paper's section 3.2.1), the steady state of a driven damped two-level
  system, resonant Jaynes-Cummings Rabi oscillation, the i-SWAP gate of
  section 4.1 in its closed-system limit.
* Invariants: unit trace, Hermiticity and positivity of rho(t).
"""
import numpy as np
import pytest
import scipy.linalg as sl

import oracle
from paper_1110_0573_gb300 import systems as S


def dense(m):
    return np.asarray(m.todense()) if hasattr(m, "todense") else np.asarray(m)


def liouvillian(H, c_ops):
    """Row-major vec: vec(A X B) = (A kron B^T) vec(X)."""
    H = dense(H)
    d = H.shape[0]
    I = np.eye(d)
    L = -1j * (np.kron(H, I) - np.kron(I, H.T))
    for c in c_ops:
        Cm = dense(c)
        CdC = Cm.conj().T @ Cm
        L += np.kron(Cm, Cm.conj()) - 0.5 * np.kron(CdC, I) - 0.5 * np.kron(I, CdC.T)
    return L


def test_rhs_matches_liouvillian():
    s = S.random_system(5, 3, 1, seed=11)
    rng = np.random.default_rng(0)
    X = rng.standard_normal((5, 5)) + 1j * rng.standard_normal((5, 5))
    rho = X @ X.conj().T
    rho /= np.trace(rho)
    got = oracle.me_rhs(s["H"], s["c_ops"], rho)
    want = (liouvillian(s["H"], s["c_ops"]) @ rho.reshape(-1)).reshape(5, 5)
    assert np.allclose(got, want, atol=1e-13)
    # trace preserving
    assert abs(np.trace(got)) < 1e-13


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_mesolve_vs_expm(seed):
    d = 4 + seed % 3
    s = S.random_system(d, 2, 2, seed=seed, nt=6, t_end=2.0)
    L = liouvillian(s["H"], s["c_ops"])
    rho0 = np.outer(s["psi0"], s["psi0"].conj())
    ex, states, _ = oracle.mesolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"],
                                   rtol=1e-11, atol=1e-13, store_states=True)
    for k, t in enumerate(s["tlist"]):
        rho_t = (sl.expm(L * t) @ rho0.reshape(-1)).reshape(d, d)
        assert np.abs(states[k] - rho_t).max() < 1e-9
        for m, e in enumerate(s["e_ops"]):
            assert abs(ex[k, m] - np.trace(dense(e) @ rho_t)) < 1e-9


def test_cavity_decay_zero_temperature():
    s = S.cavity_thermal_decay(N=6, kappa=0.7, nth=0.0, n0=3, t_end=5.0, nt=26)
    ex, _, _ = oracle.mesolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"],
                              rtol=1e-11, atol=1e-13)
    assert np.abs(ex[:, 0] - 3 * np.exp(-0.7 * s["tlist"])).max() < 1e-9


def test_cavity_decay_thermal_paper_parameters():
    # kappa = 1/0.129, n_th = 0.063 (paper section 3.2.1); truncated at N = 30
    kappa, nth = 1 / 0.129, 0.063
    s = S.cavity_thermal_decay(N=30, kappa=kappa, nth=nth, n0=1, t_end=0.6, nt=100)
    ex, _, _ = oracle.mesolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"],
                              rtol=1e-10, atol=1e-12)
    exact = nth + (1 - nth) * np.exp(-kappa * s["tlist"])
    assert np.abs(ex[:, 0].real - exact).max() < 1e-8
    # thermal steady state at long times
    s2 = S.cavity_thermal_decay(N=30, kappa=kappa, nth=nth, n0=1, t_end=5.0, nt=3)
    ex2, _, _ = oracle.mesolve(s2["H"], s2["c_ops"], s2["e_ops"], s2["psi0"], s2["tlist"],
                               rtol=1e-10, atol=1e-12)
    assert abs(ex2[-1, 0].real - nth) < 1e-8


def test_driven_tls_steady_state():
    Delta, Omega, gamma = 0.3, 1.0, 0.5
    s = S.driven_tls(Delta=Delta, Omega=Omega, gamma=gamma, t_end=150.0, nt=4)
    ex, _, _ = oracle.mesolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"],
                              rtol=1e-11, atol=1e-13)
    ree = (Omega**2 / 4) / (Delta**2 + gamma**2 / 4 + Omega**2 / 2)
    assert abs(ex[-1, 0].real - ree) < 1e-8


def test_jc_vacuum_rabi_closed_form():
    g = 2 * np.pi * 0.05
    s = S.jaynes_cummings(N=7, g=g, kappa=0.0, gamma=0.0, n0=5, t_end=20.0, nt=41)
    P = np.zeros((14, 14))
    P[5 * 2 + 0, 5 * 2 + 0] = 1.0
    ex, _, _ = oracle.mesolve(s["H"], [], [P], s["psi0"], s["tlist"], rtol=1e-11, atol=1e-13)
    assert np.abs(ex[:, 0].real - np.cos(np.sqrt(5) * g * s["tlist"]) ** 2).max() < 1e-9


def test_iswap_closed_limit():
    s = S.iswap_pair()
    _, states, _ = oracle.mesolve(s["H"], [], [], s["psi0"], s["tlist"], rtol=1e-11,
                                  atol=1e-13, store_states=True)
    ideal = -1j * S.tensor(S.basis(2, 0), S.basis(2, 1))  # |e,g> -> -i |g,e>
    fid = np.vdot(ideal, states[-1] @ ideal).real
    assert abs(fid - 1.0) < 1e-9


def test_invariants_and_ket_dm_equivalence():
    s = S.jaynes_cummings(N=4, n0=2, t_end=10.0, nt=21, kappa=0.2, gamma=0.3)
    rtol = 1e-8
    ex, states, _ = oracle.mesolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"],
                                   rtol=rtol, store_states=True)
    for rho in states:
        assert abs(np.trace(rho) - 1) < 10 * rtol
        assert np.abs(rho - rho.conj().T).max() < 10 * rtol
        assert np.linalg.eigvalsh(0.5 * (rho + rho.conj().T)).min() > -10 * rtol
    rho0 = np.outer(s["psi0"], s["psi0"].conj())
    ex2, _, _ = oracle.mesolve(s["H"], s["c_ops"], s["e_ops"], rho0, s["tlist"], rtol=rtol)
    assert np.array_equal(ex, ex2)


def test_expect_definitions():
    s = S.random_system(5, 1, 2, seed=5)
    O = s["e_ops"][0]
    psi = np.stack([s["psi0"], 2 * s["psi0"]])
    got = oracle.expect(O, psi, is_ket=True)
    ref = np.vdot(s["psi0"], dense(O) @ s["psi0"])
    assert np.allclose(got, [ref, 4 * ref])  # not normalised
    rho = np.outer(s["psi0"], s["psi0"].conj())[None]
    assert np.allclose(oracle.expect(O, rho, is_ket=False), [ref])


def test_step_limit_is_an_error():
    s = S.jaynes_cummings(N=4, n0=2, t_end=10.0, nt=3)
    with pytest.raises(oracle.OracleError) as ei:
        oracle.mesolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"], rtol=1e-8,
                       max_steps=3)
    assert ei.value.code == oracle.ESTEP
