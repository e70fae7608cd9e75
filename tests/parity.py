"""Helpers shared by the GPU parity tests (comparison logic only)."""
import numpy as np


def per_traj(rec, j):
    return rec[rec["traj"] == j]


def compare_jump_records(gpu, ora, trajs, tau_tol, honour_degenerate=True):
    """Compares jump records trajectory by trajectory.

    Counts, jump indices and channels must agree exactly and jump times
    within tau_tol.  With honour_degenerate (mixed precision), a trajectory
    whose records part ways at a jump that either side flags as a
    channel-draw boundary case (bit 0) is compared up to that jump only, and
    the jump's time is reported as the trajectory's divergence time; a
    flagged jump with the same channel on both sides is compared like any
    other.  Without it (FP64) every record must agree.  Returns
    (n_records_compared, {traj: divergence time})."""
    compared = 0
    diverged = {}
    for j in trajs:
        g, o = per_traj(gpu, j), per_traj(ora, j)
        n = max(len(g), len(o))
        for k in range(n):
            gk = g[k] if k < len(g) else None
            ok = o[k] if k < len(o) else None
            same = gk is not None and ok is not None and gk["channel"] == ok["channel"]
            chan_flag = (gk is not None and gk["degenerate"] & 1) or \
                (ok is not None and ok["degenerate"] & 1)
            if honour_degenerate and chan_flag and not same:
                diverged[j] = float((gk if gk is not None else ok)["tau"])
                break
            assert gk is not None and ok is not None, \
                f"trajectory {j}: jump count differs (gpu {len(g)}, oracle {len(o)})"
            assert gk["k"] == ok["k"] == k
            assert same, f"trajectory {j} jump {k}: channel differs"
            assert abs(gk["tau"] - ok["tau"]) <= tau_tol, \
                f"trajectory {j} jump {k}: tau {gk['tau']!r} vs {ok['tau']!r}"
            compared += 1
    return compared, diverged


def near_jump_mask(tlist, taus, window):
    """Output samples that lie within window * max(1, |tau|) of one of the
    jump times taus: the jump may fall on either side of such a sample in
    another precision, so the sample is not compared."""
    tl = np.asarray(tlist, dtype=float)
    mask = np.zeros(len(tl), dtype=bool)
    for tau in np.asarray(taus, dtype=float).reshape(-1):
        mask |= np.abs(tl - tau) < window * max(1.0, abs(tau))
    return mask


def max_traj_expect_diff(gpu_tex, ora_tex, tlist, diverged, traj_ids, gpu_jumps=None,
                         ora_jumps=None, window=1e-5):
    """Largest |gpu - oracle| over per-trajectory expectation values.  Skips
    the output times at or after a trajectory's divergence time and, when the
    jump records are given, the output samples within window of a jump of
    that trajectory on either side (near_jump_mask)."""
    worst = 0.0
    tl = np.asarray(tlist, dtype=float)
    for row, j in enumerate(traj_ids):
        keep = np.ones(len(tl), dtype=bool)
        if j in diverged:
            keep[int(np.searchsorted(tl, diverged[j] - 1e-9)):] = False
        for rec in (gpu_jumps, ora_jumps):
            if rec is not None:
                keep &= ~near_jump_mask(tl, per_traj(rec, j)["tau"], window)
        if not keep.any():
            continue
        diff = np.abs(gpu_tex[row][keep] - ora_tex[row][keep]).max()
        worst = max(worst, float(diff))
    return worst


def kept_samples(n_traj_rows, traj_ids, tlist, diverged, gpu_jumps=None, ora_jumps=None,
                 window=1e-5):
    """Boolean [rows, n_t] of the per-trajectory samples that max_traj_expect_diff
    compares."""
    tl = np.asarray(tlist, dtype=float)
    keep = np.ones((n_traj_rows, len(tl)), dtype=bool)
    for row, j in enumerate(traj_ids):
        if j in diverged:
            keep[row, int(np.searchsorted(tl, diverged[j] - 1e-9)):] = False
        for rec in (gpu_jumps, ora_jumps):
            if rec is not None:
                keep[row] &= ~near_jump_mask(tl, per_traj(rec, j)["tau"], window)
    return keep


def max_mean_diff(gpu_tex, ora_tex, keep):
    """Largest |mean_gpu - mean_oracle| over output times and observables, each
    mean taken over the trajectories whose sample is kept (both sides alike)."""
    k = keep[:, :, None].astype(float)
    n = np.maximum(k.sum(axis=0), 1.0)
    mg = (gpu_tex * k).sum(axis=0) / n
    mo = (ora_tex * k).sum(axis=0) / n
    return float(np.abs(mg - mo).max())


def integration_slack(ora_tex, ora_tex_converged, ora_jumps, ora_jumps_converged):
    """What the FP64 oracle's own integration tolerance allows: per sample
    |oracle - converged oracle| and per jump |tau - converged tau| (records
    must agree).  A mixed-precision result is compared with the oracle at the
    same tolerances within 1e-5 plus twice this slack, so that an
    ill-conditioned jump time (a threshold crossed while the norm barely
    decays) is not charged to the precision."""
    assert len(ora_jumps) == len(ora_jumps_converged)
    assert np.array_equal(ora_jumps["channel"], ora_jumps_converged["channel"])
    return (np.abs(ora_tex - ora_tex_converged),
            np.abs(ora_jumps["tau"] - ora_jumps_converged["tau"]))
