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


# ------------------------------------------------------------------ batches
# Independent problems (the batched parameter sweep, the drive vectors of the
# adjoint) are split over ranks by an estimated cost; each rank solves its
# own problems in one launch and the per-problem results are summed over
# ranks into the full result (every other rank contributes zeros there), the
# only exchange.


def problem_cost(problem) -> float:
    """Estimated work of one problem per unit time: a master-equation problem
    d^2 (2 w_H + sum_n w_C^2), a Monte-Carlo problem ntraj 2 d w_H, with w the
    widest row of H_eff (H and the C^dag C terms) and of each C_n: the cost
    per right-hand side, with the same number of steps assumed for every
    problem."""
    import scipy.sparse as sp
    H = sp.csr_matrix(problem["H"])
    d = H.shape[0]
    cs = [sp.csr_matrix(c) for c in problem["c_ops"]]
    heff = H.copy()
    for c in cs:
        heff = heff + c.conj().T @ c
    w_h = int(np.diff(heff.tocsr().indptr).max(initial=0))
    if problem.get("kind", "me") == "mc":
        return float(problem.get("ntraj", 1)) * 2.0 * d * w_h
    w_c = sum(int(np.diff(c.indptr).max(initial=0)) ** 2 for c in cs)
    return float(d * d) * (2.0 * w_h + w_c)


def cost_split(costs, world: int) -> list[list[int]]:
    """Greedy longest-first assignment of items with the given costs to world
    ranks (each item to the rank with the least load so far, ties to the
    lowest rank); returns the item indices of each rank in ascending order."""
    if world < 1:
        raise ValueError("bad world")
    load = [0.0] * world
    parts = [[] for _ in range(world)]
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += float(costs[i])
    return [sorted(p) for p in parts]


def batch_sharded(problems, solve_problems, rank: int, world: int, n_t: int):
    """Solves this rank's share of the problems and returns every problem's
    [n_t, n_e] result on every rank.  solve_problems(list of problems) ->
    list of complex128[n_t, n_e] arrays (one batched launch on this rank's
    GPU)."""
    mine = cost_split([problem_cost(p) for p in problems], world)[rank]
    sizes = [n_t * len(p["e_ops"]) for p in problems]
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(int)
    flat = np.zeros(int(offs[-1]), dtype=np.complex128)
    if mine:
        for i, r in zip(mine, solve_problems([problems[i] for i in mine])):
            flat[offs[i]:offs[i + 1]] = np.asarray(r, dtype=np.complex128).reshape(-1)
    flat = allreduce_sum(flat)
    return [flat[offs[i]:offs[i + 1]].reshape(n_t, len(p["e_ops"]))
            for i, p in enumerate(problems)]


def vectors_sharded(n_vectors: int, run_range, rank: int, world: int):
    """Drive vectors of the adjoint (all of the same cost): rank runs the
    contiguous range traj_range(rank, world, n_vectors) with run_range(begin,
    n) -> tuple of arrays whose first axis is the n vectors (loss, gradients;
    also for n = 0); returns the full arrays (first axis n_vectors) on every
    rank."""
    begin, n = traj_range(rank, world, n_vectors)
    local = run_range(begin, n)
    out = []
    for a in local:
        a = np.asarray(a)
        full = np.zeros((n_vectors,) + a.shape[1:], dtype=a.dtype)
        full[begin:begin + n] = a
        out.append(allreduce_sum(full))
    return tuple(out)
