"""Pins of the oracle's two-time correlation functions <A(t + tau) B(t)>
(the ODE form of the paper's correlation functions, section 5 function list;
the quantum regression theorem: C(t, tau) = Tr[A V(t + tau, t) (B rho(t))]).

* a closed form: the damped cavity H = omega a^dag a with collapse operators
  sqrt(kappa (1 + n_th)) a and sqrt(kappa n_th) a^dag has
  <a^dag(t + tau) a(t)> = n(t) exp((i omega - kappa/2) tau) and
  <a(t + tau) a^dag(t)> = (n(t) + 1) exp((-i omega - kappa/2) tau) with
  n(t) = n_th + (n(0) - n_th) exp(-kappa t) -- a swapped operator order,
  a wrong sign of the generator or tau measured from 0 instead of t fails it;
* brute force: Liouvillian matrix exponentials for a random system with
  non-Hermitian A and B;
* brute force for a time-dependent Hamiltonian: time-ordered products of
  Liouvillian exponentials (midpoint rule, error O(dt^2)), which fixes that
  the tau evolution sees H(t + tau).
"""
import math

import numpy as np
import pytest
import scipy.linalg as sl
import scipy.sparse as sp

import oracle
from paper_1110_0573_gb300 import systems as S


def liouvillian(H, c_ops):
    """Row-major vec: vec(X Y Z) = (X kron Z^T) vec(Y)."""
    d = H.shape[0]
    I = np.eye(d)
    L = -1j * (np.kron(H, I) - np.kron(I, H.T))
    for c in c_ops:
        cdc = c.conj().T @ c
        L += np.kron(c, c.conj()) - 0.5 * np.kron(cdc, I) - 0.5 * np.kron(I, cdc.T)
    return L


def dense(op):
    return op.toarray() if sp.issparse(op) else np.asarray(op, dtype=complex)


@pytest.mark.parametrize("n_th", [0.0, 0.3])
def test_damped_cavity_closed_form(n_th):
    N, omega, kappa, alpha = 26, 1.1, 0.5, 1.2
    a = S.destroy(N)
    ad = a.T.conj()
    c_ops = [np.sqrt(kappa * (1 + n_th)) * a]
    if n_th:
        c_ops.append(np.sqrt(kappa * n_th) * ad)
    psi0 = np.array([np.exp(-alpha ** 2 / 2) * alpha ** k / math.sqrt(math.factorial(k))
                     for k in range(N)], dtype=complex)
    tlist = np.array([0.0, 0.8, 2.0])
    taulist = np.linspace(0.0, 3.0, 13)
    H = omega * (ad @ a)
    c1, _ = oracle.correlation_2op_2t(H, c_ops, ad, a, psi0, tlist, taulist, rtol=1e-11,
                                      atol=1e-13)
    c2, _ = oracle.correlation_2op_2t(H, c_ops, a, ad, psi0, tlist, taulist, rtol=1e-11,
                                      atol=1e-13)
    for k, t in enumerate(tlist):
        n_t = n_th + (alpha ** 2 - n_th) * np.exp(-kappa * t)
        want1 = n_t * np.exp((1j * omega - kappa / 2) * taulist)
        want2 = (n_t + 1) * np.exp((-1j * omega - kappa / 2) * taulist)
        assert np.abs(c1[k] - want1).max() < 1e-8, (t, np.abs(c1[k] - want1).max())
        assert np.abs(c2[k] - want2).max() < 1e-8, (t, np.abs(c2[k] - want2).max())


def test_liouvillian_brute_force():
    rng = np.random.default_rng(11)
    d = 5
    X = rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))
    H = 0.5 * (X + X.conj().T)
    c_ops = [0.6 * (rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))) / np.sqrt(d)
             for _ in range(2)]
    A = rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))
    B = rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))
    Y = rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))
    rho0 = Y @ Y.conj().T
    rho0 /= np.trace(rho0)
    tlist = np.array([0.0, 0.3, 1.1])
    taulist = np.array([0.0, 0.2, 0.7, 1.5])
    corr, st = oracle.correlation_2op_2t(H, c_ops, A, B, rho0, tlist, taulist, rtol=1e-11,
                                         atol=1e-13)
    L = liouvillian(H, c_ops)
    for k, t in enumerate(tlist):
        rho_t = (sl.expm(L * t) @ rho0.reshape(-1)).reshape(d, d)
        X0 = (B @ rho_t).reshape(-1)
        for j, tau in enumerate(taulist):
            Xt = (sl.expm(L * tau) @ X0).reshape(d, d)
            want = np.trace(A @ Xt)
            assert abs(corr[k, j] - want) < 1e-8 * max(1.0, abs(want)), (t, tau)
    assert st["accepted"] > 0


def test_time_dependent_brute_force():
    rng = np.random.default_rng(5)
    d = 4
    X = rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))
    H0 = 0.5 * (X + X.conj().T)
    X1 = rng.standard_normal((d, d))
    H1 = 0.5 * (X1 + X1.T).astype(complex)
    c_ops = [0.5 * np.diag(np.arange(1, d, dtype=complex) ** 0.5, 1)]
    A = rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))
    B = rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))
    tk = np.array([0.0, 0.5, 1.25, 2.0])
    vk = np.array([0.0, 1.5, -1.0, 0.5])
    td = [(H1, tk, vk)]
    psi0 = np.zeros(d, dtype=complex)
    psi0[1] = 1.0
    tlist = np.array([0.0, 0.5, 1.0])
    taulist = np.array([0.0, 0.25, 0.5, 1.0])
    corr, _ = oracle.correlation_2op_2t(H0, c_ops, A, B, psi0, tlist, taulist, rtol=1e-11,
                                        atol=1e-13, td=td)
    L0, L1 = liouvillian(H0, c_ops), liouvillian(H1, []) * 1.0

    h = 1.0 / 1024  # every knot and output time is a multiple of h

    def step(t):
        return sl.expm((L0 + np.interp(t + 0.5 * h, tk, vk) * L1) * h)

    def propagate(v, t0, t1):
        n = int(round((t1 - t0) / h))
        for q in range(n):
            v = step(t0 + q * h) @ v
        return v

    v = np.outer(psi0, psi0.conj()).reshape(-1)
    t = 0.0
    for k, tk_ in enumerate(tlist):
        v = propagate(v, t, tk_)
        t = tk_
        x = (B @ v.reshape(d, d)).reshape(-1)
        s = tk_
        for j, tau in enumerate(taulist):
            x = propagate(x, s, tk_ + tau)
            s = tk_ + tau
            want = np.trace(A @ x.reshape(d, d))
            assert abs(corr[k, j] - want) < 1e-5, (tk_, tau, corr[k, j], want)
    # and it differs from the evolution that restarts the clock at tau = 0
    wrong, _ = oracle.correlation_2op_2t(H0, c_ops, A, B, psi0, tlist, taulist, rtol=1e-11,
                                         atol=1e-13, td=[(H1, tk - 0.5, vk)])
    assert np.abs(wrong - corr).max() > 1e-2


def test_rejects_nonzero_first_tau():
    a = S.destroy(4)
    with pytest.raises(oracle.OracleError):
        oracle.correlation_2op_2t(a.T.conj() @ a, [a], a.T.conj(), a, np.eye(4)[0],
                                  [0.0, 1.0], [0.1, 0.2])


def test_steady_state_closed_form():
    # thermal cavity in its steady state: <a^dag(tau) a(0)> = n_th exp((i w - k/2) tau)
    N, omega, kappa, n_th = 16, 0.9, 0.6, 0.3
    a = S.destroy(N)
    ad = a.T.conj()
    c_ops = [np.sqrt(kappa * (1 + n_th)) * a, np.sqrt(kappa * n_th) * ad]
    taulist = np.linspace(0.0, 4.0, 9)
    corr, _ = oracle.correlation_ss(omega * (ad @ a), c_ops, ad, a, taulist, rtol=1e-11,
                                    atol=1e-13)
    want = n_th * np.exp((1j * omega - kappa / 2) * taulist)
    assert np.abs(corr - want).max() < 1e-8

