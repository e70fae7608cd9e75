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
