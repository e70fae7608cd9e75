"""Pins of the oracle's Dormand-Prince 5(4) integrator.

* The Butcher tableau satisfies every Runge-Kutta order condition (rooted
  trees, Butcher's theory) up to order 5 for the propagated weights and up to
  order 4 for the embedded ones, and fails order 5 for the embedded weights
  (otherwise the error estimate would be empty).
* One step of d psi/dt = -i H_eff psi shows local error O(h^6) against the
  exact matrix exponential (scipy.linalg.expm).
"""
import itertools

import numpy as np
import scipy.linalg as sl

import oracle
from paper_1110_0573_gb300 import systems as S


def rooted_trees(order):
    """All rooted trees with `order` vertices as nested sorted tuples."""
    if order == 1:
        return [()]
    out = set()
    # a tree is a multiset of subtrees whose orders sum to order - 1
    def partitions(n, maxpart):
        if n == 0:
            yield []
            return
        for p in range(min(n, maxpart), 0, -1):
            for rest in partitions(n - p, p):
                yield [p] + rest
    for parts in partitions(order - 1, order - 1):
        for combo in itertools.product(*[rooted_trees(p) for p in parts]):
            out.add(tuple(sorted(combo)))
    return sorted(out)


def tree_order(t):
    return 1 + sum(tree_order(s) for s in t)


def gamma(t):
    g = tree_order(t)
    for s in t:
        g *= gamma(s)
    return g


def phi_stage(t, A):
    """Vector over stages i of prod_k sum_j a_ij Phi_j(subtree k)."""
    v = np.ones(A.shape[0])
    for s in t:
        v = v * (A @ phi_stage(s, A))
    return v


def test_tree_counts():
    # number of rooted trees of order 1..5 is 1, 1, 2, 4, 9
    assert [len(rooted_trees(n)) for n in range(1, 6)] == [1, 1, 2, 4, 9]


def test_order_conditions():
    c, a, b5, b4 = oracle.dp45_tableau()
    A = np.zeros((7, 7))
    A[:, :6] = a
    assert np.allclose(A.sum(axis=1), c, atol=1e-15)  # row-sum condition
    assert np.allclose(A[6, :6], b5[:6]) and b5[6] == 0  # first same as last
    for order in range(1, 6):
        for t in rooted_trees(order):
            want = 1.0 / gamma(t)
            assert abs(b5 @ phi_stage(t, A) - want) < 1e-14, (order, t)
            if order <= 4:
                assert abs(b4 @ phi_stage(t, A) - want) < 1e-14, (order, t)
    worst = max(abs(b4 @ phi_stage(t, A) - 1 / gamma(t)) for t in rooted_trees(5))
    assert worst > 1e-5


def test_local_error_order():
    s = S.jaynes_cummings(N=4, n0=2)
    H = np.asarray(s["H"].todense())
    Heff = H - 0.5j * sum(np.asarray((c.conj().T @ c).todense()) for c in s["c_ops"])
    psi = s["psi0"] + 0.3 * S.tensor(S.basis(4, 1), S.basis(2, 1))
    psi = psi / np.linalg.norm(psi)
    errs = []
    for h in (0.04, 0.02, 0.01):
        got = oracle.mc_dp45_step(s["H"], s["c_ops"], psi, h)
        exact = sl.expm(-1j * Heff * h) @ psi
        errs.append(np.linalg.norm(got - exact))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 50 < r1 < 80 and 50 < r2 < 80, errs  # 2^6 = 64


def test_mc_rhs_is_minus_i_heff():
    s = S.random_system(6, 2, 1, seed=3)
    H = np.asarray(s["H"].todense())
    Cs = [np.asarray(c.todense()) for c in s["c_ops"]]
    psi = s["psi0"]
    got = oracle.mc_rhs(s["H"], s["c_ops"], psi)
    # the norm decays at the rate sum_n ||C_n psi||^2 (Eq. (jump)):
    # d<psi|psi>/dt = 2 Re <psi|dpsi> = -sum_n ||C_n psi||^2
    rate = 2 * np.vdot(psi, got).real
    assert np.isclose(rate, -sum(np.linalg.norm(Cm @ psi) ** 2 for Cm in Cs))
    # and with no collapse operators it is the Schrodinger equation
    got0 = oracle.mc_rhs(s["H"], [], psi)
    assert np.allclose(got0, -1j * H @ psi)
