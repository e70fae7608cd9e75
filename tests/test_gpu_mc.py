"""GPU parity of qt_mcsolve (paper section 3.2) against the FP64 oracle,
through the C ABI.

FP64 mode: identical jump records (count, index, channel), jump times within
1e-10, expectation values within 1e-8 absolute.
Mixed mode (complex FP32 state, FP64 jump logic): identical records up to
threshold-degenerate events, which both sides flag; per-trajectory
expectations and trajectory means within the stated tolerances below.
"""
import os

import numpy as np
import pytest
import scipy.linalg as sl

import oracle
from paper_1110_0573_gb300 import systems as S
from tests.parity import compare_jump_records, kept_samples, max_mean_diff, max_traj_expect_diff

pytestmark = pytest.mark.gpu

NCPU = os.cpu_count() or 1
FP64_EXPECT_TOL = 1e-8
FP64_TAU_TOL = 1e-10
# Mixed mode against the oracle at the same tolerances: per-trajectory values
# and trajectory means within 1e-5 absolute, jump records identical.  Output
# samples within 1e-5 max(1, |tau|) of a jump time of either side are not
# compared (the jump may fall on the other side of the sample in the other
# precision), nor anything after a channel draw that parted ways at a flagged
# boundary.  Measured on 2048 Kerr trajectories (dim 64, t in [0, 20]):
# jump times agree to 1e-6 max(1, |tau|), per-trajectory values to 6e-6.
MIXED_TRAJ_TOL = 1e-5
MIXED_MEAN_TOL = 1e-5
MIXED_TAU_TOL = 1e-5
SKIP_WINDOW = 1e-5


@pytest.fixture(scope="module")
def qt():
    from paper_1110_0573_gb300 import build
    build.build()
    from paper_1110_0573_gb300 import qt as q
    return q


def run_both(qt, s, ntraj, seed, rtol, atol, precision, traj_begin=0, oracle_trajs=None):
    o = qt.qt_opts_default(rtol=rtol, atol=atol, precision=precision)
    mean, tex, jumps, st = qt.qt_mcsolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"],
                                         ntraj, seed=seed, opts=o, traj_expect=True)
    assert st["status"] == 0
    return mean, tex, jumps, st


def test_fp64_jaynes_cummings_full_config(qt):
    # dim 20, 500 trajectories, t in [0, 50] at 201 points, rtol 1e-8, seed 0
    s = S.jaynes_cummings()
    rtol, atol = 1e-8, 1e-10
    mean, tex, jumps, st = run_both(qt, s, 500, 0, rtol, atol, qt.QT_FP64)
    otex, ojumps, ost = oracle.mcsolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"], 500,
                                       seed=0, rtol=rtol, atol=atol, nthreads=NCPU)
    n, degen = compare_jump_records(jumps, ojumps, range(500), FP64_TAU_TOL, False)
    assert n == len(ojumps) and not degen
    assert len(jumps) == len(ojumps) > 50
    assert np.abs(tex - otex).max() < FP64_EXPECT_TOL
    assert np.abs(mean - otex.mean(axis=0)).max() < FP64_EXPECT_TOL
    assert st["accepted"] == ost["accepted"] and st["jumps"] == ost["jumps"]


@pytest.mark.parametrize("d,density,seed", [(5, 0.6, 1), (13, 0.4, 2), (33, 0.2, 3),
                                            (70, 0.1, 4), (24, 0.9, 5)])
def test_fp64_random_systems(qt, d, density, seed):
    s = S.random_system(d, 2, 2, seed=seed, density=density, nt=9, t_end=2.0)
    mean, tex, jumps, _ = run_both(qt, s, 24, seed, 1e-9, 1e-11, qt.QT_FP64)
    otex, ojumps, _ = oracle.mcsolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"], 24,
                                     seed=seed, rtol=1e-9, atol=1e-11, nthreads=NCPU)
    n, degen = compare_jump_records(jumps, ojumps, range(24), FP64_TAU_TOL, False)
    assert n == len(ojumps) and not degen
    assert np.abs(tex - otex).max() < FP64_EXPECT_TOL


def test_fp64_tridiagonal_instance(qt):
    # the Kerr cavity's H_eff has 3 entries per row: the exact-width instance
    s = S.kerr_cavity(N=40, t_end=4.0, nt=41)
    mean, tex, jumps, st = run_both(qt, s, 24, 7, 1e-9, 1e-11, qt.QT_FP64)
    otex, ojumps, ost = oracle.mcsolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"], 24,
                                       seed=7, rtol=1e-9, atol=1e-11, nthreads=NCPU)
    n, degen = compare_jump_records(jumps, ojumps, range(24), FP64_TAU_TOL, False)
    assert n == len(ojumps) > 0 and not degen
    assert np.abs(tex - otex).max() < FP64_EXPECT_TOL
    assert st["accepted"] == ost["accepted"]


def test_mixed_kerr_trajectories(qt):
    # at rtol 1e-7 the integration error of either side stays below 4e-6 on
    # every trajectory (at 1e-6 the oracle itself is 4e-4 off its converged
    # values on rare trajectories with bursts of jumps), so the comparison
    # measures the precision of the mixed kernel
    s = S.kerr_cavity(t_end=20.0, nt=401)
    ntraj, seed = 48, 3
    rtol, atol = 1e-7, 1e-9
    mean, tex, jumps, st = run_both(qt, s, ntraj, seed, rtol, atol, qt.QT_MIXED)
    otex, ojumps, _ = oracle.mcsolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"], ntraj,
                                     seed=seed, rtol=rtol, atol=atol, nthreads=NCPU)
    n, div = compare_jump_records(jumps, ojumps, range(ntraj), MIXED_TAU_TOL)
    assert n == len(ojumps) == len(jumps) > 100 and not div
    worst = max_traj_expect_diff(tex, otex, s["tlist"], div, range(ntraj), jumps, ojumps,
                                 SKIP_WINDOW)
    keep = kept_samples(ntraj, range(ntraj), s["tlist"], div, jumps, ojumps, SKIP_WINDOW)
    mean_err = max_mean_diff(tex, otex, keep)
    print(f"mixed kerr: {n} records, worst traj diff {worst:.2e}, mean diff {mean_err:.2e}, "
          f"{(~keep).sum()} samples skipped")
    assert worst < MIXED_TRAJ_TOL
    assert mean_err < MIXED_MEAN_TOL
    assert (~keep).sum() <= 0.01 * keep.size


def test_mixed_full_size_kerr_sampled(qt):
    # the benchmark configuration: dim 64, 16384 trajectories, t in [0, 20] at
    # 401 points; the oracle recomputes a sample of trajectories one by one
    s = S.kerr_cavity()
    ntraj, seed = 16384, 0
    rtol, atol = 1e-7, 1e-9
    mean, tex, jumps, st = run_both(qt, s, ntraj, seed, rtol, atol, qt.QT_MIXED)
    sample = [0, 1, 777, 4096, 9999, 16383]
    worst = 0.0
    for j in sample:
        otex, ojumps, _ = oracle.mcsolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"], 1,
                                         seed=seed, rtol=rtol, atol=atol, traj_begin=j)
        _, div = compare_jump_records(jumps, ojumps, [j], MIXED_TAU_TOL)
        worst = max(worst, max_traj_expect_diff(tex[j:j + 1], otex, s["tlist"], div, [j],
                                                jumps, ojumps, SKIP_WINDOW))
    assert worst < MIXED_TRAJ_TOL
    # the trajectory mean agrees with the oracle's master equation within 5
    # standard errors (paper section 3.2: the ensemble average is the ME)
    me, _, _ = oracle.mesolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"], rtol=1e-8)
    for m in range(2):
        sem = tex[:, :, m].std(axis=0, ddof=1) / np.sqrt(ntraj)
        dev = np.abs(mean[:, m] - me[:, m])
        assert np.all(dev <= 5 * np.maximum(sem, 1e-6)), dev.max()
    assert st["jumps"] == len(jumps)


def test_no_collapse_is_one_schrodinger_trajectory(qt):
    s = S.iswap_pair(nt=9)
    o = qt.qt_opts_default(rtol=1e-11, atol=1e-13)
    mean, tex, jumps, st = qt.qt_mcsolve(s["H"], [], s["e_ops"], s["psi0"], s["tlist"], 100,
                                         opts=o, traj_expect=True)
    assert tex.shape[0] == 1 and len(jumps) == 0
    H = np.asarray(s["H"].todense())
    for k, t in enumerate(s["tlist"]):
        v = sl.expm(-1j * H * t) @ s["psi0"]
        for m, e in enumerate(s["e_ops"]):
            assert abs(mean[k, m] - np.vdot(v, e @ v)) < 1e-9


def test_trajectory_ranges_on_device(qt):
    torch = pytest.importorskip("torch")
    s = S.jaynes_cummings(N=4, n0=2, kappa=0.3, gamma=0.5, t_end=8.0, nt=17)
    sysm = qt.System(s["H"], s["c_ops"], s["e_ops"])
    dev = torch.device("cuda")
    psi0 = torch.tensor(s["psi0"], dtype=torch.complex128, device=dev)
    tl = torch.tensor(s["tlist"], dtype=torch.float64, device=dev)
    o = qt.qt_opts_default()
    cap = 4096

    def run(begin, n):
        es = torch.zeros((17, 2), dtype=torch.complex128, device=dev)
        jb = torch.zeros(cap * 40, dtype=torch.uint8, device=dev)
        nj = torch.zeros(1, dtype=torch.int64, device=dev)
        stb = torch.zeros(56, dtype=torch.uint8, device=dev)
        sysm.qt_mcsolve_dev(psi0, tl, n, 9, o, es, traj_begin=begin, jumps=jb, n_jumps=nj,
                            stats=stb)
        torch.cuda.synchronize()
        return es.cpu().numpy(), qt.jumps_from_bytes(jb, int(nj.item())), qt.stats_from_bytes(stb)

    full, jf, sf = run(0, 40)
    a, ja, _ = run(0, 17)
    b, jb_, _ = run(17, 23)
    assert sf["status"] == 0
    assert np.abs(full - (a + b)).max() < 1e-12
    both = np.concatenate([ja, jb_])
    both.sort(order=["traj", "k"])
    assert np.array_equal(jf[["traj", "k", "channel"]], both[["traj", "k", "channel"]])
    assert np.array_equal(jf["tau"], both["tau"])
    otex, ojumps, _ = oracle.mcsolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"], 40,
                                     seed=9, rtol=o.rtol, atol=o.atol)
    assert np.abs(full / 40 - otex.mean(axis=0)).max() < FP64_EXPECT_TOL
    sysm.close()


def test_error_statuses(qt):
    s = S.jaynes_cummings(N=3, n0=1, t_end=10.0, nt=3)
    with pytest.raises(qt.QtError) as e:
        qt.qt_mcsolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"], 8,
                      opts=qt.qt_opts_default(max_steps=3))
    assert e.value.code == qt.QT_ESTEP
    with pytest.raises(qt.QtError) as e:
        qt.qt_mcsolve(s["H"], s["c_ops"], s["e_ops"], np.zeros(6), s["tlist"], 8)
    assert e.value.code == qt.QT_ENORM


def test_degenerate_sizes(qt):
    s = S.jaynes_cummings(N=3, n0=1, t_end=2.0, nt=5)
    mean, tex, jumps, st = qt.qt_mcsolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"], 0,
                                         traj_expect=True)
    assert st["accepted"] == 0 and len(jumps) == 0 and tex.shape[0] == 0
    one = np.array([0.0])
    mean, tex, jumps, st = qt.qt_mcsolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], one, 5,
                                         traj_expect=True)
    ref = oracle.mcsolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], one, 5)[0]
    assert np.abs(tex - ref).max() < 1e-14 and st["accepted"] == 0
    # dimension 1: a single decaying level
    H1 = np.array([[0.5]])
    C1 = [np.array([[0.7]])]
    mean, tex, jumps, st = qt.qt_mcsolve(H1, C1, [np.eye(1)], np.array([1.0]),
                                         np.linspace(0, 3, 4), 20, traj_expect=True)
    o1, oj, _ = oracle.mcsolve(H1, C1, [np.eye(1)], np.array([1.0]), np.linspace(0, 3, 4), 20)
    n, degen = compare_jump_records(jumps, oj, range(20), FP64_TAU_TOL, False)
    assert n == len(oj) and not degen


@pytest.mark.parametrize("L,precision", [(8, "fp64"), (10, "fp64"), (8, "mixed"), (9, "mixed"),
                                         (10, "mixed"), (11, "mixed")])
def test_xxz_chain_cta_wide_groups(qt, L, precision):
    # dimensions 256, 512, 1024 and 2048 run one trajectory per CTA; in mixed
    # precision up to dim 1024 with the dictionary H_eff in shared memory
    # (entries grouped by value: the chain has two off-diagonal values)
    s = S.xxz_chain(L=L, t_end=1.0, nt=11)
    ntraj = 12 if L < 11 else 4
    if precision == "fp64":
        rtol, atol, prec = 1e-8, 1e-10, qt.QT_FP64
    else:
        rtol, atol, prec = 1e-6, 1e-8, qt.QT_MIXED
    o = qt.qt_opts_default(rtol=rtol, atol=atol, precision=prec)
    mean, tex, jumps, st = qt.qt_mcsolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"],
                                         ntraj, seed=2, opts=o, traj_expect=True)
    assert st["status"] == 0
    otex, ojumps, _ = oracle.mcsolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"], ntraj,
                                     seed=2, rtol=rtol, atol=atol, nthreads=NCPU)
    if precision == "fp64":
        n, degen = compare_jump_records(jumps, ojumps, range(ntraj), FP64_TAU_TOL, False)
        assert n == len(ojumps)
        assert np.abs(tex - otex).max() < FP64_EXPECT_TOL
    else:
        n, div = compare_jump_records(jumps, ojumps, range(ntraj), MIXED_TAU_TOL)
        worst = max_traj_expect_diff(tex, otex, s["tlist"], div, range(ntraj), jumps, ojumps,
                                     SKIP_WINDOW)
        assert worst < MIXED_TRAJ_TOL, worst
    assert len(ojumps) > 0


@pytest.mark.parametrize("name", ["tight_binding_300", "kerr_200"])
def test_dictionary_forms_cta_wide(qt, name):
    # H_eff in shared memory as a dictionary beyond the spin chains above: a
    # tight-binding chain, one coupling value at columns i +- 1 (entries
    # grouped by value), and a Kerr cavity at dim 200, whose 200 distinct
    # ladder values take plain (column, value index) codes
    if name == "tight_binding_300":
        s = S.tight_binding_chain(d=300, gamma=1.0, t_end=2.0, nt=11)
    else:
        s = S.kerr_cavity(N=200, t_end=2.0, nt=11)
    ntraj, rtol, atol = 12, 1e-6, 1e-8
    mean, tex, jumps, st = run_both(qt, s, ntraj, 4, rtol, atol, qt.QT_MIXED)
    otex, ojumps, _ = oracle.mcsolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"], ntraj,
                                     seed=4, rtol=rtol, atol=atol, nthreads=NCPU)
    n, div = compare_jump_records(jumps, ojumps, range(ntraj), MIXED_TAU_TOL)
    assert n == len(ojumps) > 0
    worst = max_traj_expect_diff(tex, otex, s["tlist"], div, range(ntraj), jumps, ojumps,
                                 SKIP_WINDOW)
    assert worst < MIXED_TRAJ_TOL, worst


@pytest.mark.parametrize("N,ntraj", [(14, 12), (17, 8)])
def test_large_dimension_trilinear_fp64(qt, N, ntraj):
    # the paper's trilinear example (section 4.3), dim 2744 and 4913: one CTA
    # per trajectory with its stage vectors in global memory
    s = S.trilinear(N=N, t_end=1.0, nt=11)
    rtol, atol = 1e-8, 1e-10
    mean, tex, jumps, st = run_both(qt, s, ntraj, 5, rtol, atol, qt.QT_FP64)
    otex, ojumps, ost = oracle.mcsolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"],
                                       ntraj, seed=5, rtol=rtol, atol=atol, nthreads=NCPU)
    n, degen = compare_jump_records(jumps, ojumps, range(ntraj), FP64_TAU_TOL, False)
    assert n == len(ojumps) > 0 and not degen
    assert np.abs(tex - otex).max() < FP64_EXPECT_TOL
    assert st["accepted"] == ost["accepted"]


def test_large_dimension_mixed(qt):
    # a ragged dimension (2500 of the 5120 rows a CTA holds), mixed precision
    s = S.random_system(2500, 2, 2, seed=8, density=3.0 / 2500, nt=6, t_end=1.0)
    ntraj = 16
    mean, tex, jumps, st = run_both(qt, s, ntraj, 9, 1e-6, 1e-8, qt.QT_MIXED)
    otex, ojumps, _ = oracle.mcsolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"], ntraj,
                                     seed=9, rtol=1e-6, atol=1e-8, nthreads=NCPU)
    _, div = compare_jump_records(jumps, ojumps, range(ntraj), MIXED_TAU_TOL, True)
    assert max_traj_expect_diff(tex, otex, s["tlist"], div, range(ntraj), jumps, ojumps,
                                SKIP_WINDOW) < MIXED_TRAJ_TOL
