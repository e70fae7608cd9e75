"""GPU parity of the batched persistent launch (qt_batch_*): problems of
uneven dimension, master-equation and Monte-Carlo, in one launch, against
the FP64 oracle problem by problem; tuning and CUDA-graph replay keep the
results."""
import os

import numpy as np
import pytest

import oracle
from paper_1110_0573_gb300 import systems as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
NCPU = os.cpu_count() or 1


@pytest.fixture(scope="module")
def qt():
    from paper_1110_0573_gb300 import build
    build.build()
    from paper_1110_0573_gb300 import qt as q
    return q


def run_batch(qt, problems, tlist, opts, tune=False, graph=False, config=None):
    dev = torch.device("cuda")
    b = qt.Batch(problems)
    if config is not None:
        b.set_config(*config)
    tl = torch.tensor(tlist, dtype=torch.float64, device=dev)
    n = b.expect_offset(b.n, len(tlist))
    ex = torch.zeros(n, dtype=torch.complex128, device=dev)
    stb = torch.zeros(56, dtype=torch.uint8, device=dev)
    if tune:
        b.qt_batch_tune(tl, opts, ex)
    if graph:
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            b.qt_batch_solve_dev(tl, opts, ex, stats=stb, stream=s.cuda_stream)  # warm-up
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            b.qt_batch_solve_dev(tl, opts, ex, stats=stb,
                                 stream=torch.cuda.current_stream().cuda_stream)
        ex.zero_()
        g.replay()
        g.replay()
    else:
        b.qt_batch_solve_dev(tl, opts, ex, stats=stb)
    torch.cuda.synchronize()
    st = qt.stats_from_bytes(stb)
    out = [x.copy() for x in b.split(ex.cpu().numpy(), len(tlist))]
    b.close()
    return out, st


def oracle_results(problems, tlist, rtol, atol):
    ref = []
    for p in problems:
        if p["kind"] == "me":
            ex, _, _ = oracle.mesolve(p["H"], p["c_ops"], p["e_ops"], p["state0"], tlist,
                                      rtol=rtol, atol=atol)
        else:
            te, _, _ = oracle.mcsolve(p["H"], p["c_ops"], p["e_ops"], p["state0"], tlist,
                                      p["ntraj"], seed=p["seed"], rtol=rtol, atol=atol,
                                      nthreads=NCPU)
            ex = te.mean(axis=0)
        ref.append(ex)
    return ref


def small_sweep(n=12, ntraj=16):
    problems, _ = S.cavity_qubit_sweep(n, seed=3, ntraj=ntraj, cutoff=(2, 10))
    return problems, np.linspace(0.0, 5.0, 11)


def test_fp64_batch_matches_oracle_problem_by_problem(qt):
    problems, tlist = small_sweep()
    o = qt.qt_opts_default(rtol=1e-8, atol=1e-10)
    got, st = run_batch(qt, problems, tlist, o)
    assert st["status"] == 0
    ref = oracle_results(problems, tlist, 1e-8, 1e-10)
    for p, (g, r) in enumerate(zip(got, ref)):
        assert np.abs(g - r).max() < 1e-8, (p, problems[p]["kind"], np.abs(g - r).max())


def test_tuned_and_graph_replayed_batch_give_the_same_results(qt):
    problems, tlist = small_sweep(10, ntraj=40)
    o = qt.qt_opts_default(rtol=1e-8, atol=1e-10)
    plain, _ = run_batch(qt, problems, tlist, o)
    tuned, _ = run_batch(qt, problems, tlist, o, tune=True)
    graphed, st = run_batch(qt, problems, tlist, o, graph=True)
    assert st["status"] == 0
    for a, b, c in zip(plain, tuned, graphed):
        assert np.abs(a - b).max() < 1e-12 and np.abs(a - c).max() < 1e-12


def test_mixed_batch(qt):
    problems, _ = S.cavity_qubit_sweep(8, seed=5, ntraj=256, cutoff=(3, 12))
    tlist = np.linspace(0.0, 10.0, 21)
    o = qt.qt_opts_default(rtol=1e-6, atol=1e-8, precision=qt.QT_MIXED)
    got, st = run_batch(qt, problems, tlist, o)
    assert st["status"] == 0
    for p, g in zip(problems, got):
        me, _, _ = oracle.mesolve(p["H"], p["c_ops"], p["e_ops"], p["state0"], tlist,
                                  rtol=1e-6 if p["kind"] == "me" else 1e-8, atol=1e-8)
        if p["kind"] == "me":
            assert np.abs(g - me).max() < 1e-5
        else:
            # trajectory mean vs the master equation: within 5 standard errors
            # (a standard error of an observable bounded by the cutoff)
            te, _, _ = oracle.mcsolve(p["H"], p["c_ops"], p["e_ops"], p["state0"], tlist, 256,
                                      seed=p["seed"], rtol=1e-6, atol=1e-8, nthreads=NCPU)
            sem = te.std(axis=0, ddof=1) / np.sqrt(256)
            assert np.all(np.abs(g - me) <= 5 * np.maximum(sem, 1e-4) + 1e-4)


def test_batch_rejects_large_dimension(qt):
    s = S.kerr_cavity(N=80)
    with pytest.raises(qt.QtError) as e:
        qt.Batch([dict(H=s["H"], c_ops=s["c_ops"], e_ops=s["e_ops"], state0=s["psi0"],
                       kind="me")])
    assert e.value.code == qt.QT_ENOTIMPL


def full_size_sweep(ntraj=16):
    # the largest items of the parameter sweep: cavity cutoffs 28..32 (dim
    # 56..64), the register-resident MC instance and the widest ME items
    problems, _ = S.cavity_qubit_sweep(8, seed=9, ntraj=ntraj, cutoff=(28, 32))
    assert max(p["dim"] for p in problems) >= 62 and min(p["dim"] for p in problems) >= 56
    return problems, np.linspace(0.0, 5.0, 11)


def test_fp64_full_size_items_match_oracle(qt):
    problems, tlist = full_size_sweep()
    o = qt.qt_opts_default(rtol=1e-8, atol=1e-10)
    got, st = run_batch(qt, problems, tlist, o)
    assert st["status"] == 0
    ref = oracle_results(problems, tlist, 1e-8, 1e-10)
    for p, (g, r) in enumerate(zip(got, ref)):
        assert np.abs(g - r).max() < 1e-8, (p, problems[p]["kind"], np.abs(g - r).max())


def test_mixed_full_size_items_match_oracle(qt):
    # mixed precision against the oracle at the same tolerances: the master
    # equation within 1e-5; the Monte-Carlo problems' trajectory means (the
    # same trajectories on both sides) within 1e-5
    problems, tlist = full_size_sweep()
    o = qt.qt_opts_default(rtol=1e-7, atol=1e-9, precision=qt.QT_MIXED)
    got, st = run_batch(qt, problems, tlist, o)
    assert st["status"] == 0
    ref = oracle_results(problems, tlist, 1e-7, 1e-9)
    for p, (g, r) in enumerate(zip(got, ref)):
        assert np.abs(g - r).max() < 1e-5, (p, problems[p]["kind"], np.abs(g - r).max())


def test_per_problem_statistics_add_up(qt):
    problems, tlist = small_sweep(6, ntraj=8)
    dev = torch.device("cuda")
    b = qt.Batch(problems)
    tl = torch.tensor(tlist, dtype=torch.float64, device=dev)
    ex = torch.zeros(b.expect_offset(b.n, len(tlist)), dtype=torch.complex128, device=dev)
    stb = torch.zeros(56, dtype=torch.uint8, device=dev)
    b.qt_batch_solve_dev(tl, qt.qt_opts_default(rtol=1e-8, atol=1e-10), ex, stats=stb)
    torch.cuda.synchronize()
    st = qt.stats_from_bytes(stb)
    per = b.problem_stats()
    b.close()
    for k in ("accepted", "rejected", "rhs_evals", "jumps"):
        assert int(per[k].sum()) == st[k]
    assert np.all(per["accepted"] > 0)
    # per problem the same counts as a solve of that problem alone
    p = problems[1]
    _, jumps, ost = oracle.mcsolve(p["H"], p["c_ops"], p["e_ops"], p["state0"], tlist, p["ntraj"],
                                   seed=p["seed"], rtol=1e-8, atol=1e-10)
    assert int(per["accepted"][1]) == ost["accepted"] and int(per["jumps"][1]) == len(jumps)


@pytest.mark.parametrize("config", [(16, 16), (48, 32), (8, 0)])
def test_trajectory_groupings_match_oracle(qt, config):
    # Monte-Carlo problems on half-warp groups (dimensions up to 16 or 32) or
    # whole warps, with several work-item sizes: every configuration gives the
    # oracle's trajectory means in FP64
    problems, _ = S.cavity_qubit_sweep(10, seed=13, ntraj=20, cutoff=(4, 16))
    tlist = np.linspace(0.0, 4.0, 9)
    o = qt.qt_opts_default(rtol=1e-8, atol=1e-10)
    got, st = run_batch(qt, problems, tlist, o, config=config)
    assert st["status"] == 0
    ref = oracle_results(problems, tlist, 1e-8, 1e-10)
    for p, (g, r) in enumerate(zip(got, ref)):
        assert np.abs(g - r).max() < 1e-8, (p, problems[p]["dim"], np.abs(g - r).max())


def test_mixed_half_warp_groups(qt):
    problems, _ = S.cavity_qubit_sweep(8, seed=17, ntraj=32, cutoff=(4, 16))
    tlist = np.linspace(0.0, 4.0, 9)
    o = qt.qt_opts_default(rtol=1e-7, atol=1e-9, precision=qt.QT_MIXED)
    got, st = run_batch(qt, problems, tlist, o, config=(16, 32))
    assert st["status"] == 0
    ref = oracle_results(problems, tlist, 1e-7, 1e-9)
    for p, (g, r) in enumerate(zip(got, ref)):
        assert np.abs(g - r).max() < 1e-5, (p, problems[p]["dim"], np.abs(g - r).max())


def test_config_is_reported_and_checked(qt):
    problems, tlist = small_sweep(4, ntraj=4)
    b = qt.Batch(problems)
    assert b.config() == {"traj_block": 64, "small_group_dim": 0, "tuned_ms": 0.0}
    b.set_config(32, 16)
    assert b.config()["traj_block"] == 32 and b.config()["small_group_dim"] == 16
    with pytest.raises(qt.QtError):
        b.set_config(32, 20)
    b.close()
