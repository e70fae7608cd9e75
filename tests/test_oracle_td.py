"""Pins of the oracle's time-dependent Hamiltonians H(t) = H + sum_k f_k(t) H_k
(paper section 4.3; f_k piecewise linear between knots, constant outside).

* the coefficient definition on hand-computed values;
* a closed form: for H(t) = (omega + f(t)) a^dag a and collapse sqrt(kappa) a,
  d<a>/dt = -i (omega + f(t)) <a> - kappa/2 <a> exactly, so
  <a>(t) = <a>(0) exp(-kappa t / 2 - i (omega t + F(t))), F = int f (exact
  trapezoid sums for piecewise-linear f) -- wrong stage times would show up as
  an O(h f') error;
* brute force: the Landau-Zener sweep against a product of many 2 x 2 matrix
  exponentials at midpoint times (error O(dt^2));
* the Landau-Zener formula P = 1 - exp(-pi Delta^2 / 2v) (asymptotic; finite
  sweeps deviate by ~1e-2);
* Monte-Carlo with a time-dependent H against the master equation (5 sigma).
"""
import math

import numpy as np
import pytest
import scipy.linalg as sl

import oracle
from paper_1110_0573_gb300 import systems as S


def test_coefficient_definition():
    H1 = S.sigmaz()
    td = [(H1, [0.0, 1.0, 3.0], [2.0, 4.0, 0.0])]
    cases = {-5.0: 2.0, 0.0: 2.0, 0.5: 3.0, 1.0: 4.0, 2.0: 2.0, 3.0: 0.0, 7.0: 0.0, 2.5: 1.0}
    for t, want in cases.items():
        assert oracle.td_coef(td, 0, t) == pytest.approx(want, abs=1e-15), t


def pwl_integral(tk, vk, t):
    """int_0^t of the piecewise-linear coefficient (t >= 0, knots from 0)."""
    ts = np.concatenate([[0.0], tk[(tk > 0) & (tk < t)], [t]])
    f = np.interp(ts, tk, vk)
    return np.sum(0.5 * (f[1:] + f[:-1]) * np.diff(ts))


@pytest.mark.parametrize("kappa", [0.0, 0.4])
def test_closed_form_cavity_with_ramp(kappa):
    N, omega, alpha = 24, 1.3, 1.0
    a = S.destroy(N)
    n = a.T.conj() @ a
    tk = np.array([0.0, 0.7, 1.5, 3.0])
    vk = np.array([0.0, 2.0, -1.0, 0.5])
    td = [(n, tk, vk)]
    # truncated coherent state
    psi0 = np.array([np.exp(-alpha ** 2 / 2) * alpha ** k / np.sqrt(float(math.factorial(k)))
                     for k in range(N)], dtype=complex)
    tlist = np.linspace(0.0, 4.0, 21)
    ex, _, _ = oracle.mesolve(omega * n, [np.sqrt(kappa) * a] if kappa else [], [a], psi0, tlist,
                              rtol=1e-11, atol=1e-13, td=td)
    a0 = np.vdot(psi0, a @ psi0)
    for k, t in enumerate(tlist):
        want = a0 * np.exp(-kappa * t / 2 - 1j * (omega * t + pwl_integral(tk, vk, t)))
        assert abs(ex[k, 0] - want) < 1e-8, (t, ex[k, 0], want)
    if kappa == 0.0:
        # one Schrodinger trajectory: the same closed form
        te, _, _ = oracle.mcsolve(omega * n, [], [a], psi0, tlist, 1, rtol=1e-11, atol=1e-13, td=td)
        for k, t in enumerate(tlist):
            want = a0 * np.exp(-1j * (omega * t + pwl_integral(tk, vk, t)))
            assert abs(te[0, k, 0] - want) < 1e-8


def lz_bruteforce(s, t_end, steps):
    H0 = s["H"].toarray()
    H1, tk, vk = s["td"][0]
    H1 = H1.toarray()
    t0 = s["tlist"][0]
    dt = (t_end - t0) / steps
    psi = s["psi0"].astype(complex)
    for q in range(steps):
        tm = t0 + (q + 0.5) * dt
        psi = sl.expm(-1j * dt * (H0 + np.interp(tm, tk, vk) * H1)) @ psi
    return psi


def test_landau_zener_against_fine_exponential_products():
    s = S.landau_zener(t0=-3.0, t1=3.0, nt=7)
    ex, states, _ = oracle.mesolve(s["H"], [], s["e_ops"], s["psi0"], s["tlist"], rtol=1e-11,
                                   atol=1e-13, store_states=True, td=s["td"])
    psi = lz_bruteforce(s, 3.0, 20000)
    rho = np.outer(psi, psi.conj())
    assert np.abs(states[-1] - rho).max() < 1e-6
    # Richardson: halving dt moves the brute force by ~3/4 of its error
    psi2 = lz_bruteforce(s, 3.0, 40000)
    assert np.abs(np.outer(psi2, psi2.conj()) - states[-1]).max() < np.abs(rho - states[-1]).max()


def test_landau_zener_formula():
    s = S.landau_zener()
    ex, _, _ = oracle.mesolve(s["H"], [], s["e_ops"], s["psi0"], s["tlist"], rtol=1e-9,
                              atol=1e-11, td=s["td"])
    P = 1.0 - np.exp(-np.pi * s["delta"] ** 2 / (2.0 * s["v"]))
    assert abs(ex[-1, 0].real - P) < 2e-2
    # a trace-preserving, populations in [0, 1]
    assert np.all(ex[:, 0].real > -1e-9) and np.all(ex[:, 0].real < 1 + 1e-9)


def test_mc_mean_matches_master_equation_with_time_dependence():
    s = S.landau_zener(t0=-4.0, t1=4.0, nt=41, gamma=0.3)
    me, _, _ = oracle.mesolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"], rtol=1e-9,
                              atol=1e-11, td=s["td"])
    ntraj = 600
    te, jumps, _ = oracle.mcsolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"], ntraj,
                                  seed=11, rtol=1e-8, atol=1e-10, nthreads=8, td=s["td"])
    assert len(jumps) > 50
    mean = te.mean(axis=0)
    sem = te.std(axis=0, ddof=1) / np.sqrt(ntraj)
    assert np.all(np.abs(mean - me) <= 5 * np.maximum(sem, 1e-3))
