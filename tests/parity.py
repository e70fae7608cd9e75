"""Helpers shared by the GPU parity tests (comparison logic only)."""
import numpy as np


def per_traj(rec, j):
    return rec[rec["traj"] == j]


def compare_jump_records(gpu, ora, trajs, tau_tol, honour_degenerate=True):
    """Compares jump records trajectory by trajectory.

    Counts, jump indices and channels must agree exactly and jump times
    within tau_tol.  With honour_degenerate (mixed precision), a trajectory
    is compared only up to the first record that either side flags as
    threshold-degenerate and is reported; without it (FP64) every record
    must agree.  Returns (n_records_compared, {traj: first degenerate
    time})."""
    compared = 0
    degenerate = {}
    for j in trajs:
        g, o = per_traj(gpu, j), per_traj(ora, j)
        n = max(len(g), len(o))
        for k in range(n):
            gk = g[k] if k < len(g) else None
            ok = o[k] if k < len(o) else None
            flagged = (gk is not None and gk["degenerate"]) or (ok is not None and ok["degenerate"])
            if flagged and honour_degenerate:
                degenerate[j] = float((gk if gk is not None else ok)["tau"])
                break
            assert gk is not None and ok is not None, \
                f"trajectory {j}: jump count differs (gpu {len(g)}, oracle {len(o)})"
            assert gk["k"] == ok["k"] == k
            assert gk["channel"] == ok["channel"], f"trajectory {j} jump {k}: channel differs"
            assert abs(gk["tau"] - ok["tau"]) <= tau_tol, \
                f"trajectory {j} jump {k}: tau {gk['tau']!r} vs {ok['tau']!r}"
            compared += 1
    return compared, degenerate


def max_traj_expect_diff(gpu_tex, ora_tex, tlist, degenerate, traj_ids):
    """Largest |gpu - oracle| over per-trajectory expectation values, skipping
    output times at or after a trajectory's first degenerate event."""
    worst = 0.0
    for row, j in enumerate(traj_ids):
        lim = len(tlist)
        if j in degenerate:
            lim = int(np.searchsorted(tlist, degenerate[j] - 1e-9))
        if lim == 0:
            continue
        diff = np.abs(gpu_tex[row, :lim] - ora_tex[row, :lim]).max()
        worst = max(worst, float(diff))
    return worst
