"""Pins of the oracle's steady state (the paper's steadystate, section 5
function list: rho with L(rho) = 0, Tr rho = 1).

* closed forms: the truncated thermal cavity, p_k proportional to
  (n/(1+n))^k (exact in the truncated space: detailed balance holds level by
  level), and the driven damped two-level system, rho_ee =
  (Omega^2/4) / (Delta^2 + gamma^2/4 + Omega^2/2) with the coherence
  <sigma_-> = i (Omega/2) <sigma_z> / (i Delta + gamma/2);
* the residual of the Kronecker-product Liouvillian (built independently of
  the oracle's right-hand side);
* the long-time limit of the oracle's master-equation solve (another
  route: time integration);
* a non-unique stationary state is refused.
"""
import numpy as np
import pytest

import oracle
from paper_1110_0573_gb300 import systems as S
from tests.test_oracle_corr import liouvillian


def test_thermal_cavity():
    N, kappa, n = 12, 0.7, 0.4
    s = S.cavity_thermal_decay(N=N, kappa=kappa, nth=n)
    rho, sv = oracle.steadystate(s["H"], s["c_ops"])
    r = n / (1 + n)
    p = r ** np.arange(N)
    p /= p.sum()
    assert np.abs(rho - np.diag(p)).max() < 1e-12
    assert sv[0] < 1e-12 * sv[-1]


def test_driven_tls():
    Delta, Omega, gamma = 0.3, 1.0, 0.5
    s = S.driven_tls(Delta=Delta, Omega=Omega, gamma=gamma)
    rho, _ = oracle.steadystate(s["H"], s["c_ops"])
    ree = (Omega ** 2 / 4) / (Delta ** 2 + gamma ** 2 / 4 + Omega ** 2 / 2)
    # index 0 = ground, 1 = excited
    assert abs(rho[1, 1].real - ree) < 1e-12
    sz = 2 * ree - 1
    sm = 1j * (Omega / 2) * sz / (1j * Delta + gamma / 2)
    assert abs(rho[1, 0] - sm) < 1e-12  # <sigma_-> = <e|rho|g>


def test_random_residual_and_long_time_limit():
    s = S.random_system(6, 2, 1, seed=4, density=0.8)
    rho, _ = oracle.steadystate(s["H"], s["c_ops"])
    H = s["H"].toarray()
    C = [c.toarray() for c in s["c_ops"]]
    L = liouvillian(H, C)
    assert np.abs(L @ rho.reshape(-1)).max() < 1e-12
    assert abs(np.trace(rho) - 1) < 1e-14 and np.abs(rho - rho.conj().T).max() < 1e-15
    assert np.linalg.eigvalsh(rho).min() > -1e-12
    # time integration to t = 400 (the slowest decay rate here is ~0.1)
    ev = np.linalg.eigvals(L)
    gap = np.sort(-ev.real)[1]
    T = 40.0 / gap
    _, states, _ = oracle.mesolve(s["H"], s["c_ops"], [], s["psi0"], [0.0, T], rtol=1e-11,
                                  atol=1e-13, store_states=True)
    assert np.abs(states[-1] - rho).max() < 1e-8


def test_non_unique_refused():
    # no dissipation: every diagonal state in the energy basis is stationary
    with pytest.raises(oracle.OracleError):
        oracle.steadystate(S.num(4), [])
