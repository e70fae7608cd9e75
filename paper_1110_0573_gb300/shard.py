"""Trajectory sharding across processes (one GPU per process).

Monte-Carlo trajectories are independent and their random streams depend only
on the global trajectory index (Philox counter = (trajectory, jump index,
stream, 0)), so any split of the index range reproduces the single-process
trajectories exactly.  Each rank integrates a contiguous range; the only
exchange is one sum of the FP64 expectation sums (n_t x n_e complex values)
over ranks.
"""
from __future__ import annotations

import numpy as np


def traj_range(rank: int, world: int, ntraj: int) -> tuple[int, int]:
    """(first global index, count) of rank's contiguous share of ntraj."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    base, extra = divmod(ntraj, world)
    begin = rank * base + min(rank, extra)
    return begin, base + (1 if rank < extra else 0)


def allreduce_sum(x: np.ndarray) -> np.ndarray:
    """Sum a complex128 / float64 array over all ranks of the default
    torch.distributed group (identity without an initialised group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    real = np.ascontiguousarray(x).view(np.float64) if np.iscomplexobj(x) else x
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.from_numpy(np.array(real, dtype=np.float64)).to(dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    out = t.cpu().numpy()
    return out.view(np.complex128).reshape(x.shape) if np.iscomplexobj(x) else out.reshape(x.shape)


def mcsolve_sharded(solve_range, ntraj: int, rank: int, world: int):
    """Runs this rank's share and returns the trajectory mean over all ranks.

    solve_range(begin, n) -> (sum over its trajectories of the normalised
    expectation values, complex128[n_t, n_e]).  The sum of the partial sums
    is divided by ntraj."""
    begin, n = traj_range(rank, world, ntraj)
    local = np.asarray(solve_range(begin, n), dtype=np.complex128)
    return allreduce_sum(local) / ntraj


def gpu_solve_range(system, psi0, tlist, seed, opts):
    """A solve_range for the CUDA library: qt_mcsolve_dev on the current device."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    p = torch.as_tensor(np.asarray(psi0, dtype=np.complex128), device=dev)
    t = torch.as_tensor(np.asarray(tlist, dtype=np.float64), device=dev)

    def run(begin, n):
        es = torch.zeros((len(tlist), system.n_e), dtype=torch.complex128, device=dev)
        system.qt_mcsolve_dev(p, t, n, seed, opts, es, traj_begin=begin)
        torch.cuda.synchronize()
        return es.cpu().numpy()
    return run
