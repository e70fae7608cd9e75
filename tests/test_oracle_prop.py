"""Pins of the oracle's propagator (the paper's propagator, section 5
function list: U(t) with vec(rho(t)) = U(t) vec(rho(t0))).

* matrix-exponential brute force: U(t) = expm(L (t - t0)) with the
  Kronecker-product Liouvillian built independently of the oracle;
* composition: U(t2) = U(t2, t1) U(t1) (the solve restarted at t1);
* without collapse operators, U(t) = V kron conj(V) with V = expm(-i H t);
* trace preservation: vec(I)^dag U(t) = vec(I)^dag.
"""
import numpy as np
import scipy.linalg as sl

import oracle
from paper_1110_0573_gb300 import systems as S
from tests.test_oracle_corr import liouvillian


def test_expm_brute_force_and_trace():
    s = S.random_system(4, 2, 1, seed=8, density=0.8)
    tlist = np.array([0.0, 0.4, 1.3])
    U, st = oracle.propagator(s["H"], s["c_ops"], tlist, rtol=1e-11, atol=1e-13)
    L = liouvillian(s["H"].toarray(), [c.toarray() for c in s["c_ops"]])
    for k, t in enumerate(tlist):
        assert np.abs(U[k] - sl.expm(L * t)).max() < 1e-9
    tr = np.eye(4).reshape(-1)
    assert np.abs(tr @ U[-1] - tr).max() < 1e-9
    assert st["accepted"] > 0


def test_composition():
    s = S.random_system(3, 1, 1, seed=2, density=1.0)
    U, _ = oracle.propagator(s["H"], s["c_ops"], [0.0, 0.5, 1.2], rtol=1e-11, atol=1e-13)
    U2, _ = oracle.propagator(s["H"], s["c_ops"], [0.5, 1.2], rtol=1e-11, atol=1e-13)
    assert np.abs(U[2] - U2[1] @ U[1]).max() < 1e-9


def test_unitary_limit():
    s = S.random_system(3, 0, 1, seed=5, density=1.0)
    t = 0.9
    U, _ = oracle.propagator(s["H"], [], [0.0, t], rtol=1e-11, atol=1e-13)
    V = sl.expm(-1j * s["H"].toarray() * t)
    assert np.abs(U[1] - np.kron(V, V.conj())).max() < 1e-9
