"""The multi-process path on CPU: two gloo ranks each integrate their share of
the trajectories (the FP64 oracle stands in for the per-rank GPU solve) and
sum the partial expectation sums; the result equals the single-process run."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1110_0573_gb300 import shard  # noqa: E402
from paper_1110_0573_gb300 import systems as S  # noqa: E402


def test_traj_range_partitions():
    for ntraj in (0, 1, 7, 100, 16384):
        for world in (1, 2, 3, 8):
            got = [shard.traj_range(r, world, ntraj) for r in range(world)]
            assert sum(n for _, n in got) == ntraj
            assert got[0][0] == 0
            for (b0, n0), (b1, _) in zip(got, got[1:]):
                assert b0 + n0 == b1


def _system():
    return S.jaynes_cummings(N=3, n0=1, kappa=0.4, gamma=0.6, g=0.5, t_end=4.0, nt=9)


def _oracle_range(begin, n):
    import oracle
    s = _system()
    tex, jumps, _ = oracle.mcsolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"], n,
                                   seed=4, rtol=1e-8, traj_begin=begin)
    return tex.sum(axis=0), jumps


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    jumps_local = []

    def solve(begin, n):
        s, j = _oracle_range(begin, n)
        jumps_local.append(j)
        return s
    mean = shard.mcsolve_sharded(solve, 11, rank, world)
    np.save(os.path.join(out, f"mean{rank}.npy"), mean)
    np.save(os.path.join(out, f"jumps{rank}.npy"), jumps_local[0])
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_reproduce_one_process(tmp_path):
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    full_sum, full_jumps = _oracle_range(0, 11)
    ref = full_sum / 11
    for r in range(world):
        mean = np.load(tmp_path / f"mean{r}.npy")
        assert np.abs(mean - ref).max() < 1e-14
    both = np.concatenate([np.load(tmp_path / f"jumps{r}.npy") for r in range(world)])
    assert np.array_equal(both, full_jumps)


def test_cost_split_balances_and_covers():
    costs = [9.0, 1.0, 4.0, 4.0, 7.0, 2.0, 3.0, 8.0]
    for world in (1, 2, 3):
        parts = shard.cost_split(costs, world)
        assert sorted(i for p in parts for i in p) == list(range(len(costs)))
        loads = [sum(costs[i] for i in p) for p in parts]
        # greedy longest-first: no rank above the mean by more than the largest item
        assert max(loads) <= sum(costs) / world + max(costs)
    assert shard.cost_split(costs, 2) == shard.cost_split(list(costs), 2)  # deterministic


def test_problem_cost_orders_by_dimension():
    problems, _ = S.cavity_qubit_sweep(6, seed=3, ntraj=4, cutoff=(2, 8))
    small = [p for p in problems if p["dim"] == min(q["dim"] for q in problems)][0]
    big = [p for p in problems if p["dim"] == max(q["dim"] for q in problems)][0]
    for kind in ("me", "mc"):
        assert shard.problem_cost(dict(small, kind=kind)) < shard.problem_cost(dict(big, kind=kind))


def _batch_problems():
    problems, tlist = S.cavity_qubit_sweep(6, seed=3, ntraj=5, cutoff=(2, 6))
    return problems, np.linspace(0.0, 2.0, 5)


def _oracle_problems(problems):
    # the FP64 oracle stands in for one rank's batched GPU launch
    import oracle
    _, tlist = _batch_problems()
    out = []
    for p in problems:
        if p["kind"] == "me":
            ex, _, _ = oracle.mesolve(p["H"], p["c_ops"], p["e_ops"], p["state0"], tlist,
                                      rtol=1e-8, atol=1e-10)
        else:
            te, _, _ = oracle.mcsolve(p["H"], p["c_ops"], p["e_ops"], p["state0"], tlist,
                                      p["ntraj"], seed=p["seed"], rtol=1e-8, atol=1e-10)
            ex = te.mean(axis=0)
        out.append(ex)
    return out


def _adjoint():
    import oracle
    s = S.transmon_cavity(N=3, n_seg=4, t_seg=0.5)
    prob = oracle.AdjointProblem(s["H0"], s["Hd"], s["A"], s["P1"], s["P2"], s["psi0"],
                                 s["n_seg"], s["t_seg"])
    omega = S.drive_vectors(5, s["n_seg"], seed=2)
    return prob, omega, s["gamma"]


def _adjoint_range(begin, n):
    prob, omega, gamma = _adjoint()
    loss, go, gg = np.zeros(n), np.zeros((n, omega.shape[1])), np.zeros((n, len(gamma)))
    for i in range(n):
        _, ns, hg = prob.forward(omega[begin + i], gamma)
        loss[i], go[i], gg[i] = prob.grad(omega[begin + i], gamma, ns, hg)
    return loss, go, gg


def _batch_worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    problems, tlist = _batch_problems()
    res = shard.batch_sharded(problems, _oracle_problems, rank, world, len(tlist))
    np.save(os.path.join(out, f"batch{rank}.npy"), np.concatenate([r.reshape(-1) for r in res]))
    loss, go, gg = shard.vectors_sharded(5, _adjoint_range, rank, world)
    np.save(os.path.join(out, f"adj{rank}.npy"), np.concatenate([loss, go.reshape(-1),
                                                                  gg.reshape(-1)]))
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_batches_and_drive_vectors(tmp_path):
    # batched problems split by cost and adjoint drive vectors split by range
    # over two ranks give, on every rank, exactly the single-process results
    world = 2
    mp.spawn(_batch_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    problems, _ = _batch_problems()
    ref = np.concatenate([r.reshape(-1) for r in _oracle_problems(problems)])
    loss, go, gg = _adjoint_range(0, 5)
    ref_adj = np.concatenate([loss, go.reshape(-1), gg.reshape(-1)])
    for r in range(world):
        assert np.array_equal(np.load(tmp_path / f"batch{r}.npy"), ref)
        assert np.array_equal(np.load(tmp_path / f"adj{r}.npy"), ref_adj)
    # both ranks had work
    parts = shard.cost_split([shard.problem_cost(p) for p in problems], world)
    assert all(parts)


@pytest.mark.gpu
def test_gpu_solve_range_on_one_rank():
    # the GPU solve behind mcsolve_sharded, on one rank: the mean over two
    # ranges equals the one-range solve and the FP64 oracle
    import oracle
    from paper_1110_0573_gb300 import build
    build.build()
    from paper_1110_0573_gb300 import qt
    s = _system()
    sysm = qt.System(s["H"], s["c_ops"], s["e_ops"])
    opts = qt.qt_opts_default(rtol=1e-8, atol=1e-10)
    run = shard.gpu_solve_range(sysm, s["psi0"], s["tlist"], 4, opts)
    mean = shard.mcsolve_sharded(run, 11, 0, 1)
    split = (run(0, 6) + run(6, 5)) / 11
    ref = _oracle_range(0, 11)[0] / 11
    sysm.close()
    assert np.abs(mean - split).max() < 1e-14
    assert np.abs(mean - ref).max() < 1e-8
