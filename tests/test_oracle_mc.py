"""Pins of the oracle's Monte-Carlo wave-function solver (paper section 3.2).

* Jump times: tau solves <psi(tau)|psi(tau)> = r with psi(tau) the exact
  non-Hermitian evolution expm(-i H_eff (tau - t)) psi (root found here with
  scipy's brentq), for the first and the following jumps.
* Collapse choice: the recorded channel satisfies the cumulative rule of
  Eq. (mc3) with the channel weights of Eq. (pcn) recomputed from the exact
  state.
* Ensemble: the trajectory mean converges to the master equation within
  5 standard errors (paper section 3.2.1, the 904-trajectory cavity decay of
  its Fig. 4), and to the closed form n_th + (n0 - n_th) e^{-kappa t}.
* No collapse operators: one trajectory equal to the Schrodinger equation.
* Any split of the trajectory range gives identical records.
"""
import numpy as np
import pytest
import scipy.linalg as sl
from scipy.optimize import brentq

import oracle
from paper_1110_0573_gb300 import systems as S


def dense(m):
    return np.asarray(m.todense()) if hasattr(m, "todense") else np.asarray(m)


def heff(s):
    H = dense(s["H"])
    return H - 0.5j * sum(dense(c).conj().T @ dense(c) for c in s["c_ops"])


def exact_jump_sequence(s, seed, j, njumps):
    """Reconstructs the first njumps (tau, channel) of trajectory j from the
    exact evolution, using the oracle's recorded channels only to continue."""
    He = heff(s)
    Cs = [dense(c) for c in s["c_ops"]]
    psi = s["psi0"] / np.linalg.norm(s["psi0"])
    t0 = 0.0
    out = []
    for k in range(njumps):
        r = oracle.uniform(seed, j, k, 0)

        def f(tau):
            v = sl.expm(-1j * He * (tau - t0)) @ psi
            return np.vdot(v, v).real - r
        hi = t0 + 1.0
        while f(hi) > 0:
            hi = t0 + 2 * (hi - t0)
        tau = brentq(f, t0, hi, xtol=1e-14, rtol=1e-15)
        v = sl.expm(-1j * He * (tau - t0)) @ psi
        p = np.array([np.linalg.norm(Cm @ v) ** 2 for Cm in Cs])
        r2 = oracle.uniform(seed, j, k, 1)
        n = int(np.argmax(np.cumsum(p) >= r2 * p.sum()))
        out.append((tau, n))
        w = Cs[n] @ v
        psi = w / np.linalg.norm(w)
        t0 = tau
    return out


@pytest.mark.parametrize("system", ["cavity", "jc"])
def test_jump_times_and_channels_match_exact_evolution(system):
    if system == "cavity":
        s = S.cavity_thermal_decay(N=5, kappa=1.3, nth=0.2, n0=2, t_end=3.0, nt=7)
    else:
        s = S.jaynes_cummings(N=3, n0=1, kappa=0.4, gamma=0.6, g=0.5, t_end=6.0, nt=7)
    seed = 42
    _, jumps, _ = oracle.mcsolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"], 6,
                                 seed=seed, rtol=1e-12, atol=1e-14)
    checked = 0
    for j in range(6):
        rec = jumps[jumps["traj"] == j]
        if len(rec) == 0:
            continue
        exact = exact_jump_sequence(s, seed, j, min(len(rec), 3))
        for (tau, n), row in zip(exact, rec):
            assert abs(row["tau"] - tau) < 1e-10, (j, row, tau)
            assert row["channel"] == n
            checked += 1
        assert list(rec["k"]) == list(range(len(rec)))
    assert checked >= 4


def test_no_jump_before_first_crossing():
    # a trajectory whose threshold is never reached has no record and a norm
    # decay matching the exact evolution at the end time
    s = S.cavity_thermal_decay(N=4, kappa=0.05, nth=0.0, n0=1, t_end=1.0, nt=3)
    seed = 3
    for j in range(20):
        r = oracle.uniform(seed, j, 0, 0)
        v = sl.expm(-1j * heff(s) * 1.0) @ s["psi0"]
        if np.vdot(v, v).real > r:
            _, jumps, _ = oracle.mcsolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"],
                                         1, seed=seed, traj_begin=j, rtol=1e-10)
            assert len(jumps) == 0
            return
    pytest.fail("no non-jumping trajectory found")


def test_cavity_decay_ensemble_904_trajectories():
    # paper section 3.2.1: N = 5, kappa = 1/0.129, n_th = 0.063, 904 trajectories
    kappa, nth = 1 / 0.129, 0.063
    s = S.cavity_thermal_decay(N=5, kappa=kappa, nth=nth, n0=1, t_end=0.6, nt=100)
    te, _, _ = oracle.mcsolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"], 904,
                              seed=7, rtol=1e-8, nthreads=4)
    vals = te[:, :, 0].real
    mean, sd = vals.mean(axis=0), vals.std(axis=0, ddof=1)
    me, _, _ = oracle.mesolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"], rtol=1e-10)
    sem = np.maximum(sd / np.sqrt(904), 1e-3)
    assert np.all(np.abs(mean - me[:, 0].real) <= 5 * sem)
    closed = nth + (1 - nth) * np.exp(-kappa * s["tlist"])
    # truncation at N = 5 is negligible here
    assert np.all(np.abs(mean - closed) <= 5 * sem + 1e-4)


def test_jc_ensemble_matches_master_equation():
    s = S.jaynes_cummings(N=4, n0=2, kappa=0.3, gamma=0.5, t_end=8.0, nt=17)
    ntraj = 400
    te, _, _ = oracle.mcsolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"], ntraj,
                              seed=11, rtol=1e-8, nthreads=4)
    me, _, _ = oracle.mesolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"], rtol=1e-10)
    for m in range(2):
        vals = te[:, :, m].real
        sem = np.maximum(vals.std(axis=0, ddof=1) / np.sqrt(ntraj), 1e-3)
        assert np.all(np.abs(vals.mean(axis=0) - me[:, m].real) <= 5 * sem)


def test_no_collapse_is_schrodinger():
    s = S.iswap_pair(nt=9)
    te, jumps, st = oracle.mcsolve(s["H"], [], s["e_ops"], s["psi0"], s["tlist"], 50,
                                   rtol=1e-11, atol=1e-13)
    assert te.shape[0] == 1 and len(jumps) == 0
    H = dense(s["H"])
    for k, t in enumerate(s["tlist"]):
        v = sl.expm(-1j * H * t) @ s["psi0"]
        for m, e in enumerate(s["e_ops"]):
            assert abs(te[0, k, m] - np.vdot(v, dense(e) @ v)) < 1e-9


def test_trajectory_split_and_threads_are_invariant():
    s = S.jaynes_cummings(N=3, n0=1, kappa=0.4, gamma=0.6, g=0.5, t_end=6.0, nt=13)
    args = (s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"])
    full, jf, _ = oracle.mcsolve(*args, 10, seed=5, rtol=1e-8)
    a, ja, _ = oracle.mcsolve(*args, 4, seed=5, rtol=1e-8, traj_begin=0)
    b, jb, _ = oracle.mcsolve(*args, 6, seed=5, rtol=1e-8, traj_begin=4, nthreads=3)
    assert np.array_equal(full, np.concatenate([a, b]))
    assert np.array_equal(jf, np.concatenate([ja, jb]))


def test_expectations_are_normalised():
    s = S.cavity_thermal_decay(N=4, kappa=0.5, nth=0.0, n0=2, t_end=2.0, nt=5)
    ident = S.qeye(4)
    te, _, _ = oracle.mcsolve(s["H"], s["c_ops"], [ident], s["psi0"], s["tlist"], 5, seed=1)
    assert np.allclose(te[:, :, 0], 1.0, atol=1e-14)


def test_step_limit_is_an_error():
    s = S.jaynes_cummings(N=3, n0=1, t_end=10.0, nt=3)
    with pytest.raises(oracle.OracleError) as ei:
        oracle.mcsolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"], 2, max_steps=3)
    assert ei.value.code == oracle.ESTEP


def _decaying_level(channels):
    # H = 0 on a two-level system, excited start, collapse operators
    # sqrt(g_n) sigma_-: <psi|psi> = exp(-t sum g_n), so the first jump of a
    # trajectory with threshold r is at tau = -ln(r) / sum g_n, and channel n
    # carries weight g_n / sum g_n
    sm = np.array([[0.0, 1.0], [0.0, 0.0]])
    H = np.zeros((2, 2))
    c_ops = [np.sqrt(g) * sm for g in channels]
    return H, c_ops, [np.diag([0.0, 1.0])], np.array([0.0, 1.0])


def test_jump_near_an_output_time_is_flagged():
    # bit 1 of a record: tau within 4e-6 max(1, |tau|) of an output time
    H, c_ops, e_ops, psi0 = _decaying_level([0.7])
    seed = 3
    for j in range(4):
        tau = -np.log(oracle.uniform(seed, j, 0, 0)) / 0.7
        w = 4e-6 * max(1.0, tau)
        for offset, flagged in ((0.5 * w, True), (-0.5 * w, True), (2.0 * w, False),
                                (-2.0 * w, False)):
            tl = np.array([0.0, tau + offset, tau + 1.0])
            _, jumps, _ = oracle.mcsolve(H, c_ops, e_ops, psi0, tl, 1, seed=seed, traj_begin=j,
                                         rtol=1e-11, atol=1e-13)
            assert len(jumps) == 1
            assert abs(jumps["tau"][0] - tau) < 1e-9
            assert bool(jumps["degenerate"][0] & 2) == flagged, (j, offset)
            assert not jumps["degenerate"][0] & 1


@pytest.mark.parametrize("weights,boundary", [([1.0, 1.0], 0.5), ([1.0, 3.0], 0.25)])
def test_channel_draw_near_a_boundary_is_flagged(weights, boundary):
    # bit 0: the fresh uniform r2 of Eq. (mc3) within 1e-5 of a cumulative
    # boundary of the weights; the channel is the first whose cumulative
    # weight reaches r2 sum p
    H, c_ops, e_ops, psi0 = _decaying_level(weights)
    seed = 11
    r2 = np.array([oracle.uniform(seed, j, 0, 1) for j in range(200000)])
    near = np.flatnonzero(np.abs(r2 - boundary) < 0.6e-5)
    clear = np.flatnonzero((np.abs(r2 - boundary) > 1.5e-5) & (np.abs(r2 - boundary) < 1e-3))
    assert len(near) >= 1 and len(clear) >= 2
    tl = np.array([0.0, 50.0])
    for j, flagged in [(near[0], True), (clear[0], False), (clear[1], False)]:
        _, jumps, _ = oracle.mcsolve(H, c_ops, e_ops, psi0, tl, 1, seed=seed, traj_begin=int(j))
        assert len(jumps) == 1
        assert bool(jumps["degenerate"][0] & 1) == flagged, (j, r2[j])
        assert jumps["channel"][0] == (0 if r2[j] <= boundary else 1)
