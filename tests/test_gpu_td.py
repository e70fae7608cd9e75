"""GPU parity of time-dependent Hamiltonians H(t) = H + sum_k f_k(t) H_k
(paper section 4.3; piecewise-linear coefficients) against the FP64 oracle,
through the C ABI: every master-equation solver (one CTA for small systems,
the general and the Hermitian cooperative solvers) and the Monte-Carlo
kernels (warp groups of 1, 2 and 4 rows per lane, CTA-wide groups).

FP64: identical jump records, jump times within 1e-10, expectation values
within 1e-8.  Mixed: the stated tolerances of the time-independent tests."""
import os

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from paper_1110_0573_gb300 import systems as S
from tests.parity import (compare_jump_records, integration_slack, kept_samples,
                          max_traj_expect_diff)

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

NCPU = os.cpu_count() or 1


@pytest.fixture(scope="module")
def qt():
    from paper_1110_0573_gb300 import build
    build.build()
    from paper_1110_0573_gb300 import qt as q
    return q


def drive_system(d, seed, n_terms=2, kinks_on_outputs=True):
    """A random sparse system with n_terms time-dependent Hermitian terms.
    The coefficients have knots outside [0, 2] and, inside it, on output times
    (tlist = 0, 0.25, ..., 2), where every solver ends a step, so that no step
    straddles a kink; with kinks_on_outputs=False the inner knots are random."""
    s = S.random_system(d, 2, 2, seed=seed, density=min(1.0, 6.0 / d), nt=9, t_end=2.0)
    rng = np.random.default_rng(seed + 100)
    td = []
    for k in range(n_terms):
        X = sp.random(d, d, density=min(1.0, 4.0 / d), random_state=seed + k, dtype=float)
        Hk = sp.csr_matrix(0.5 * (X + X.T), dtype=np.complex128)
        if kinks_on_outputs:
            inner = np.sort(rng.choice(s["tlist"][1:-1], 3, replace=False))
        else:
            inner = np.sort(rng.uniform(0.1, 1.9, 3))
        tk = np.concatenate([[-0.5], inner, [2.5]])
        vk = rng.uniform(-1.5, 1.5, 5)
        td.append((Hk, tk, vk))
    s["td"] = td
    return s


@pytest.mark.parametrize("d,method", [(2, "auto"), (30, "auto"), (100, "auto"),
                                      (100, "sparse")])
def test_fp64_master_equation(qt, d, method):
    s = S.landau_zener(t0=-3.0, t1=3.0, nt=13, gamma=0.2) if d == 2 else drive_system(d, d)
    m = qt.QT_ME_AUTO if method == "auto" else qt.QT_ME_SPARSE
    o = qt.qt_opts_default(rtol=1e-10, atol=1e-12, me_method=m)
    ex, _, st = qt.qt_mesolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"], opts=o,
                              td=s["td"])
    ref, _, _ = oracle.mesolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"],
                               rtol=1e-10, atol=1e-12, td=s["td"])
    assert st["status"] == 0
    assert np.abs(ex - ref).max() < 1e-8


@pytest.mark.parametrize("d", [30, 100])
def test_mixed_master_equation(qt, d):
    s = drive_system(d, d + 7)
    o = qt.qt_opts_default(rtol=1e-6, atol=1e-8, precision=qt.QT_MIXED)
    ex, _, st = qt.qt_mesolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"], opts=o,
                              td=s["td"])
    ref, _, _ = oracle.mesolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"],
                               rtol=1e-10, atol=1e-12, td=s["td"])
    assert st["status"] == 0
    assert np.abs(ex - ref).max() < 2e-5


def test_landau_zener_full_sweep(qt):
    # the paper's sweep, t in [-10, 10]: FP64 against the oracle, and the
    # Landau-Zener formula as the paper states it (asymptotic, ~1e-2)
    s = S.landau_zener()
    o = qt.qt_opts_default(rtol=1e-9, atol=1e-11)
    ex, _, st = qt.qt_mesolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"], opts=o,
                              td=s["td"])
    ref, _, _ = oracle.mesolve(s["H"], [], s["e_ops"], s["psi0"], s["tlist"], rtol=1e-9,
                               atol=1e-11, td=s["td"])
    assert np.abs(ex - ref).max() < 1e-8
    P = 1.0 - np.exp(-np.pi * s["delta"] ** 2 / (2.0 * s["v"]))
    assert abs(ex[-1, 0].real - P) < 2e-2
    # no collapse operators: mcsolve runs one Schrodinger trajectory
    mean, _, _, st2 = qt.qt_mcsolve(s["H"], [], s["e_ops"], s["psi0"], s["tlist"], 10, opts=o,
                                    td=s["td"])
    assert st2["status"] == 0 and np.abs(mean - ref).max() < 1e-7


@pytest.mark.parametrize("d", [2, 40, 100, 200])
def test_fp64_trajectories(qt, d):
    # d = 2, 40, 100: warp groups with 1, 2, 4 rows per lane; 200: CTA-wide
    s = S.landau_zener(t0=-3.0, t1=3.0, nt=13, gamma=0.5) if d == 2 else drive_system(d, d + 3)
    ntraj, seed = 24, d
    o = qt.qt_opts_default(rtol=1e-9, atol=1e-11)
    mean, tex, jumps, st = qt.qt_mcsolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"],
                                         ntraj, seed=seed, opts=o, traj_expect=True, td=s["td"])
    otex, ojumps, ost = oracle.mcsolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"],
                                       ntraj, seed=seed, rtol=1e-9, atol=1e-11, nthreads=NCPU,
                                       td=s["td"])
    assert st["accepted"] == ost["accepted"] and st["rejected"] == ost["rejected"]
    assert st["status"] == 0
    n, degen = compare_jump_records(jumps, ojumps, range(ntraj), 1e-10, False)
    assert n == len(ojumps) and not degen and len(ojumps) > 0
    assert np.abs(tex - otex).max() < 1e-8


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_tridiagonal_drive_ramp(qt, precision):
    # a Kerr cavity (dim 40) with its drive E (a + a^dag) ramped: H_eff and the
    # drive term have 3 entries per row (the exact-width instance)
    s = S.kerr_cavity(N=40, E=0.0, t_end=4.0, nt=17)
    a = S.destroy(40)
    td = [((a + a.T.conj()).tocsr(), np.array([-1.0, 0.5, 2.0, 5.0]),
           np.array([0.0, 0.0, 1.2, 1.2]))]
    fp64 = precision == "fp64"
    rtol, atol = (1e-9, 1e-11) if fp64 else (1e-6, 1e-8)
    o = qt.qt_opts_default(rtol=rtol, atol=atol, precision=qt.QT_FP64 if fp64 else qt.QT_MIXED)
    _, tex, jumps, st = qt.qt_mcsolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"], 24,
                                      seed=5, opts=o, traj_expect=True, td=td)
    otex, ojumps, _ = oracle.mcsolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"], 24,
                                     seed=5, rtol=rtol, atol=atol, nthreads=NCPU, td=td)
    assert st["status"] == 0
    if fp64:
        n, degen = compare_jump_records(jumps, ojumps, range(24), 1e-10, False)
        assert n == len(ojumps) > 0 and not degen
        assert np.abs(tex - otex).max() < 1e-8
    else:
        _, div = compare_jump_records(jumps, ojumps, range(24), 1e-5, True)
        assert max_traj_expect_diff(tex, otex, s["tlist"], div, range(24), jumps, ojumps,
                                    1e-5) < 1e-5


def test_fp64_trajectories_with_kinks_inside_steps(qt):
    # a coefficient kink inside a step makes the step control reject near
    # err = 1, where rounding-level differences of the two sides (the kernels
    # contract products into FMAs) can flip a decision: the records stay the
    # same and the values agree to the integration tolerance, not bit for bit
    s = drive_system(40, 43, kinks_on_outputs=False)
    o = qt.qt_opts_default(rtol=1e-9, atol=1e-11)
    _, tex, jumps, st = qt.qt_mcsolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"], 24,
                                      seed=43, opts=o, traj_expect=True, td=s["td"])
    otex, ojumps, _ = oracle.mcsolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"], 24,
                                     seed=43, rtol=1e-9, atol=1e-11, nthreads=NCPU, td=s["td"])
    n, _ = compare_jump_records(jumps, ojumps, range(24), 1e-8, False)
    assert n == len(ojumps) > 0
    assert np.abs(tex - otex).max() < 1e-6


@pytest.mark.parametrize("d", [2, 40])
def test_mixed_trajectories(qt, d):
    s = S.landau_zener(t0=-3.0, t1=3.0, nt=13, gamma=0.5) if d == 2 else drive_system(d, d + 5)
    ntraj, seed = 48, d + 1
    o = qt.qt_opts_default(rtol=1e-6, atol=1e-8, precision=qt.QT_MIXED)
    mean, tex, jumps, st = qt.qt_mcsolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"],
                                         ntraj, seed=seed, opts=o, traj_expect=True, td=s["td"])
    otex, ojumps, _ = oracle.mcsolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"], ntraj,
                                     seed=seed, rtol=1e-6, atol=1e-8, nthreads=NCPU, td=s["td"])
    assert st["status"] == 0
    # the oracle's own integration error at these tolerances (against a
    # converged run) is the slack beyond 1e-5 that the comparison allows: the
    # Landau-Zener trajectories cross their thresholds while the excited
    # population, hence the norm's decay, is small, and their jump times move
    # by up to 1e-3 between rtol 1e-6 and convergence in FP64 alike
    ctex, cjumps, _ = oracle.mcsolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"],
                                     ntraj, seed=seed, rtol=1e-11, atol=1e-13, nthreads=NCPU,
                                     td=s["td"])
    slack_e, slack_tau = integration_slack(otex, ctex, ojumps, cjumps)
    assert len(jumps) == len(ojumps) > 0
    assert np.array_equal(jumps["channel"], ojumps["channel"])
    assert np.all(np.abs(jumps["tau"] - ojumps["tau"]) <=
                  1e-5 * np.maximum(1.0, np.abs(ojumps["tau"])) + 2 * slack_tau)
    keep = kept_samples(ntraj, range(ntraj), s["tlist"], {}, jumps, ojumps, 1e-5)
    excess = (np.abs(tex - otex) - 2 * slack_e)[keep]
    assert excess.max() < 1e-5, excess.max()


def test_rhs_at_a_given_time(qt):
    s = drive_system(100, 9)
    rng = np.random.default_rng(3)
    X = rng.standard_normal((100, 100)) + 1j * rng.standard_normal((100, 100))
    rho = X @ X.conj().T
    rho /= np.trace(rho)
    sysm = qt.System(s["H"], s["c_ops"], s["e_ops"], td=s["td"])
    r = torch.tensor(rho, dtype=torch.complex128, device="cuda")
    out = torch.zeros_like(r)
    for t in (-1.0, 0.37, 1.9, 4.0):
        for m in (qt.QT_ME_AUTO, qt.QT_ME_SPARSE):
            sysm.qt_me_rhs_dev(r, out, qt.qt_opts_default(me_method=m), t=t)
            torch.cuda.synchronize()
            ref = oracle.me_rhs(s["H"], s["c_ops"], rho, td=s["td"], t=t)
            assert np.abs(out.cpu().numpy() - ref).max() < 1e-12 * max(1.0, np.abs(ref).max())
    sysm.close()


def test_unsupported_combinations(qt):
    s = drive_system(30, 1)
    o = qt.qt_opts_default(precision=qt.QT_MIXED, me_method=qt.QT_ME_DENSE_TC)
    with pytest.raises(qt.QtError) as e:
        qt.qt_mesolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"], opts=o, td=s["td"])
    assert e.value.code == qt.QT_ENOTIMPL
    with pytest.raises(qt.QtError) as e:  # knot times must increase
        qt.qt_mesolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"],
                      td=[(s["td"][0][0], [1.0, 0.0], [0.0, 1.0])])
    assert e.value.code == qt.QT_EINVAL
