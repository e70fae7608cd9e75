"""Pins of the oracle's master-equation adjoint.

* The discrete adjoint equals central finite differences of the same
  discrete map (frozen step grid, h = 1e-6) for every drive amplitude and
  decay rate.
* The adaptive forward loss equals the fixed-grid loss on its own grid.
* The loss itself against the exact solution: rho(T) and the integral of
  Tr(P2 rho) from the matrix exponential of the Liouvillian augmented by one
  row for the integral, segment by segment (scipy.linalg.expm); and the
  gradient against finite differences of that exact loss.
"""
import numpy as np
import pytest
import scipy.linalg as sl

import oracle
from paper_1110_0573_gb300 import systems as S


def dense(m):
    return np.asarray(m.todense()) if hasattr(m, "todense") else np.asarray(m)


def problem(N=4, n_seg=6):
    s = S.transmon_cavity(N=N, n_seg=n_seg)
    pr = oracle.AdjointProblem(s["H0"], s["Hd"], s["A"], s["P1"], s["P2"], s["psi0"], n_seg,
                               s["t_seg"])
    return s, pr


def exact_loss(s, omega, gamma):
    """Re Tr(P1 rho(T)) + Re int Tr(P2 rho) from expm of [[L, 0], [p2^T, 0]]."""
    H0, Hd = dense(s["H0"]), dense(s["Hd"])
    A = [dense(a) for a in s["A"]]
    d = H0.shape[0]
    I = np.eye(d)
    P1, P2 = dense(s["P1"]), dense(s["P2"])
    rho = np.outer(s["psi0"], s["psi0"].conj()).reshape(-1)
    # row-major vec: vec(A X B) = (A kron B^T) vec(X); Tr(P X) = vec(P^T) . vec(X)
    p2 = P2.T.reshape(-1)
    z = np.concatenate([rho, [0.0]])
    for w in omega:
        H = H0 + w * Hd
        L = -1j * (np.kron(H, I) - np.kron(I, H.T))
        for g, a in zip(gamma, A):
            n = a.conj().T @ a
            L += g * (np.kron(a, a.conj()) - 0.5 * np.kron(n, I) - 0.5 * np.kron(I, n.T))
        M = np.zeros((d * d + 1, d * d + 1), dtype=complex)
        M[:d * d, :d * d] = L
        M[d * d, :d * d] = p2
        z = sl.expm(M * s["t_seg"]) @ z
    rho_T = z[:d * d].reshape(d, d)
    return (np.trace(P1 @ rho_T) + z[d * d]).real


def test_discrete_adjoint_matches_finite_differences():
    s, pr = problem()
    rng = np.random.default_rng(0)
    omega = rng.uniform(-0.3, 0.3, s["n_seg"])
    gamma = s["gamma"] * np.array([3.0, 2.0, 50.0])  # make every rate matter
    _, ns, hg = pr.forward(omega, gamma, rtol=1e-8, atol=1e-10)
    loss, go, gg = pr.grad(omega, gamma, ns, hg)
    h = 1e-6
    for i in range(s["n_seg"]):
        e = np.zeros_like(omega)
        e[i] = h
        fd = (pr.loss_fixed(omega + e, gamma, ns, hg) - pr.loss_fixed(omega - e, gamma, ns, hg)) / (2 * h)
        assert abs(fd - go[i]) <= 1e-6 * max(abs(go[i]), 1e-3), (i, fd, go[i])
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        fd = (pr.loss_fixed(omega, gamma + e, ns, hg) - pr.loss_fixed(omega, gamma - e, ns, hg)) / (2 * h)
        assert abs(fd - gg[k]) <= 1e-6 * max(abs(gg[k]), 1e-3), (k, fd, gg[k])
    assert loss == pr.loss_fixed(omega, gamma, ns, hg)


def test_forward_loss_and_gradient_against_exact_solution():
    s, pr = problem(N=3, n_seg=4)
    omega = np.array([0.2, -0.15, 0.3, 0.05])
    gamma = s["gamma"] * np.array([2.0, 1.0, 30.0])
    loss, ns, hg = pr.forward(omega, gamma, rtol=1e-11, atol=1e-13)
    assert abs(loss - exact_loss(s, omega, gamma)) < 1e-9
    _, go, gg = pr.grad(omega, gamma, ns, hg)
    h = 1e-5
    for i in range(len(omega)):
        e = np.zeros_like(omega)
        e[i] = h
        fd = (exact_loss(s, omega + e, gamma) - exact_loss(s, omega - e, gamma)) / (2 * h)
        assert abs(fd - go[i]) < 1e-7, (i, fd, go[i])
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        fd = (exact_loss(s, omega, gamma + e) - exact_loss(s, omega, gamma - e)) / (2 * h)
        assert abs(fd - gg[k]) < 1e-7, (k, fd, gg[k])


def test_undriven_closed_system_has_no_drive_gradient_at_zero():
    # from the ground state, the first-order effect of a drive on populations
    # vanishes at Omega = 0 (the populations are even in Omega)
    s, pr = problem(N=3, n_seg=3)
    omega = np.zeros(3)
    gamma = np.zeros(3)
    _, ns, hg = pr.forward(omega, gamma)
    _, go, _ = pr.grad(omega, gamma, ns, hg)
    assert np.abs(go).max() < 1e-12
