"""Benchmark: Monte-Carlo trajectory steps per second on one GB300.

Workload (one "step"): a complete qt_mcsolve_dev of the driven damped Kerr
cavity, dim 64 (Delta 0.5, K 0.1, E 1, collapse sqrt(0.5) a and
sqrt(0.05) a^dag), 16384 trajectories from the vacuum, t in [0, 20] with 401
output times, observables <a^dag a> and <a>, complex FP32 state with FP64
jump logic (rtol 1e-7, atol 1e-9).  The metric counts accepted
Dormand-Prince steps summed over trajectories.  A secondary line item
reports master-equation right-hand-side evaluations per second.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 it runs under torch.distributed (one rank per GPU); each rank
integrates its own 16384 trajectories (global indices rank * 16384 + j, so
the random streams never overlap) with no collective on the data path
("weak" scaling).  --impl reference times the FP64 CPU oracle on a bounded
sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NTRAJ = 16384
SEED = 0
RTOL, ATOL = 1e-7, 1e-9
L2_FLUSH_BYTES = 512 << 20  # larger than the 129 MB L2


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


# DRAM traffic of the MC kernel per launch of this workload (dram__bytes_read
# plus dram__bytes_write of one ncu capture of the headline launch); reported
# only while the kernel source is the one that was captured.
MC_TRAFFIC = {"source_sha256_16": "0e435eb287b8dada", "bytes_per_launch": 159232}


def mc_traffic():
    import hashlib
    src = os.path.join(ROOT, "paper_1110_0573_gb300", "csrc", "qt_mc_impl.cuh")
    with open(src, "rb") as f:
        h = hashlib.sha256(f.read()).hexdigest()[:16]
    return MC_TRAFFIC["bytes_per_launch"] if h == MC_TRAFFIC["source_sha256_16"] else None


# Arithmetic roofs, measured at the start of each run by qt_fma_peak (FP32,
# packed FP32x2 and FP64 multiply-add throughput of this GPU); the unit-count
# figures below are used only when no measurement could be taken.
NOMINAL_PEAKS = {"fp32": 152 * 128 * 2 * 2.07e9 / 1e12, "fp64": 1.25}
PEAKS = {}


def measure_peaks(qt, index):
    """FP32 / FP32x2 / FP64 multiply-add rates (TFLOP/s) with the SM clock
    sampled while they run; fills PEAKS."""
    out = {}
    with Clocks(index) as clk:
        for name, kind, iters in (("fp32", qt.QT_PEAK_FP32, 4000),
                                  ("fp32x2", qt.QT_PEAK_FP32X2, 2000),
                                  ("fp64", qt.QT_PEAK_FP64, 100)):
            r = qt.qt_fma_peak(kind, iters, reps=2)
            it = max(1, int(iters * 30.0 / max(r["ms_per_launch"], 1e-3)))  # ~30 ms launches
            r = qt.qt_fma_peak(kind, it, reps=8)
            out[name] = r["flop_per_s"] / 1e12
    out["clocks"] = clk.summary()
    out["how"] = ("qt_fma_peak: independent multiply-add chains on every SM at the occupancy "
                  "limit, 8 launches of ~30 ms timed with CUDA events")
    PEAKS.update(out)
    return out


def peak(name):
    """(TFLOP/s, source) of a measured roof, else the nominal figure."""
    if name in PEAKS:
        return PEAKS[name], "measured (qt_fma_peak)"
    if name.startswith("bf16"):
        p = peaks()
        key = "bf16_tflops_sustained" if name == "bf16_sustained" else "bf16_tflops"
        if key in p:
            return p[key], f"measured (MEASURED_PEAKS.json {key})"
        return 1900.0 if name == "bf16" else 1700.0, "fallback"
    return NOMINAL_PEAKS[name], "nominal (no measurement)"


def roof(flops, seconds, name, bound="alu", **extra):
    """Roofline entry of a line: algorithmic flops / time against a roof."""
    p, src = peak(name)
    achieved = flops / seconds / 1e12
    r = {"bound": bound, "achieved": achieved, "peak": p, "unit": "TFLOP/s",
         "frac": achieved / p, "peak_source": f"{name} {src}"}
    r.update(extra)
    return r


def mc_flops_per_traj_step(d, nnz_heff):
    """Algorithmic flops of one accepted Dormand-Prince step of one trajectory
    as the hot-path table counts them: 6 right-hand sides of 8 flops per stored
    H_eff entry, and 30 complex multiply-adds (8 flops) per state element for
    the stage combinations, the error estimate and the norm (this counts a
    real coefficient times a complex entry as a full complex multiply-add; the
    tighter count, 2 flops per real multiply-add, is 130 flops per element)."""
    return 6 * 8 * nnz_heff + 30 * 8 * d


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_init(n_gpus):
    rank, world = 0, 1
    if n_gpus > 1 or "WORLD_SIZE" in os.environ:
        import torch.distributed as dist
        world = int(os.environ.get("WORLD_SIZE", "1"))
        rank = int(os.environ.get("RANK", "0"))
        if world > 1:
            backend = "nccl" if os.environ.get("QT_BENCH_BACKEND", "nccl") == "nccl" else "gloo"
            dist.init_process_group(backend=backend)
    return rank, world


def dist_max(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_sum(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def time_oracle_sample(s, budget_s=10.0, seed=SEED, traj_begin=0):
    """Times the FP64 oracle (all host cores) on a bounded number of
    trajectories of the workload; returns (traj-steps/s, cores, sample text,
    per-trajectory expectations, jumps, n)."""
    import oracle
    cores = os.cpu_count() or 1
    pilot = max(cores, 8)
    t0 = time.perf_counter()
    oracle.mcsolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"], pilot, seed=seed,
                   rtol=RTOL, atol=ATOL, nthreads=cores, traj_begin=traj_begin)
    dt = time.perf_counter() - t0
    n = int(min(NTRAJ, max(pilot, pilot * budget_s / max(dt, 1e-3))))
    n = max(cores, (n // cores) * cores)
    t0 = time.perf_counter()
    tex, jumps, st = oracle.mcsolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"], n,
                                    seed=seed, rtol=RTOL, atol=ATOL, nthreads=cores,
                                    traj_begin=traj_begin)
    dt = time.perf_counter() - t0
    rate = st["accepted"] / dt
    sample = (f"trajectories {traj_begin}..{traj_begin + n - 1} of {NTRAJ} ({n} of the workload), "
              f"{st['accepted']} accepted steps in {dt:.1f} s on {cores} OpenMP threads")
    return rate, cores, sample, tex, jumps, n


def time_oracle_one_core(s, budget_s=3.0, seed=SEED):
    """The FP64 oracle on one host core (one OpenMP thread) on the first few
    trajectories of the workload: (traj-steps/s, sample text)."""
    import oracle
    pilot = 2
    t0 = time.perf_counter()
    oracle.mcsolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"], pilot, seed=seed,
                   rtol=RTOL, atol=ATOL, nthreads=1)
    dt = time.perf_counter() - t0
    n = int(min(NTRAJ, max(pilot, pilot * budget_s / max(dt, 1e-3))))
    t0 = time.perf_counter()
    _, _, st = oracle.mcsolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"], n,
                              seed=seed, rtol=RTOL, atol=ATOL, nthreads=1)
    dt = time.perf_counter() - t0
    return st["accepted"] / dt, (f"trajectories 0..{n - 1} of {NTRAJ}, {st['accepted']} "
                                 f"accepted steps in {dt:.1f} s on 1 thread")


def time_oracle_me(s, rtol, atol, n_rhs=0):
    """The FP64 oracle's master equation (the literal Lindblad form with CSR
    loops) on one host core: right-hand-side evaluations per second of the
    whole solve, or, with n_rhs > 0, of that many evaluations at the initial
    state (where a whole solve would take minutes)."""
    import numpy as np
    import oracle
    t0 = time.perf_counter()
    if n_rhs > 0:
        psi = np.asarray(s["psi0"], dtype=np.complex128)
        rho = np.outer(psi, psi.conj()) / np.vdot(psi, psi).real
        for _ in range(n_rhs):
            oracle.me_rhs(s["H"], s["c_ops"], rho)
        n, what = n_rhs, f"{n_rhs} right-hand sides at the initial state"
    else:
        _, _, st = oracle.mesolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"],
                                  rtol=rtol, atol=atol)
        n, what = st["rhs_evals"], f"the whole solve ({st['rhs_evals']} right-hand sides)"
    dt = time.perf_counter() - t0
    return {"rhs_evals_per_s": n / dt, "cores": 1, "kind": "oracle",
            "sample": f"{what} in {dt:.2f} s"}


def run_reference(args, s, config):
    rank, world = dist_init(args.gpus)
    if rank != 0:
        return
    times, rates = [], []
    for i in range(args.warmup + args.steps):
        rate, cores, sample, _, _, n = time_oracle_sample(s, budget_s=5.0)
        if i >= args.warmup:
            rates.append(rate)
    value = statistics.median(rates)
    line = {"impl": "reference", "metric": "MC traj-steps/s", "value": value,
            "unit": "traj-steps/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config,
            "cpu_baseline": {"value": value, "unit": "traj-steps/s", "cores": cores,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "traj-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-me", action="store_true")
    ap.add_argument("--profile-case", choices=["mc", "mc_fp64", "mc_xxz", "me", "me_fp64", "me_tc",
                                               "ss", "corr"],
                    default=None,
                    help="run one small launch of a kernel for an ncu capture and exit")
    ap.add_argument("--profile-ntraj", type=int, default=2048)
    args = ap.parse_args()
    if args.profile_case:
        return profile_case(args)

    from paper_1110_0573_gb300 import systems as S
    s = S.kerr_cavity()
    config = {"workload": "Kerr cavity dim 64, 16384 MC trajectories, t in [0,20] at 401 points, "
                          "rtol 1e-7 atol 1e-9, seed 0",
              "dim": 64, "ntraj_per_gpu": NTRAJ, "n_t": 401, "precision": "mixed (c64 state, "
              "f64 jump logic and accumulation)",
              "l2": "512 MiB buffer written between timed steps (state is on chip; "
                    "operators are KB-sized)"}
    if args.impl == "reference":
        return run_reference(args, s, config)

    import torch
    rank, world = dist_init(args.gpus)
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1110_0573_gb300 import build as B
    if rank == 0 or world == 1:
        B.build()
    barrier(world)
    from paper_1110_0573_gb300 import qt

    sysm = qt.System(s["H"], s["c_ops"], s["e_ops"])
    nnz_heff = int((s["H"] - 0.5j * sum((c.conj().T @ c) for c in s["c_ops"])).nnz)
    flops_step = mc_flops_per_traj_step(64, nnz_heff)
    psi0 = torch.tensor(s["psi0"], dtype=torch.complex128, device=dev)
    tl = torch.tensor(s["tlist"], dtype=torch.float64, device=dev)
    nt, ne = len(s["tlist"]), len(s["e_ops"])
    es = torch.zeros((nt, ne), dtype=torch.complex128, device=dev)
    stb = torch.zeros(56, dtype=torch.uint8, device=dev)
    o = qt.qt_opts_default(rtol=RTOL, atol=ATOL, precision=qt.QT_MIXED)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    begin = rank * NTRAJ

    def one_step():
        sysm.qt_mcsolve_dev(psi0, tl, NTRAJ, SEED, o, es, traj_begin=begin, stats=stb,
                            stream=stream.cuda_stream)

    for _ in range(args.warmup):
        flush.fill_(1)
        one_step()
    torch.cuda.synchronize()
    st0 = qt.stats_from_bytes(stb)
    assert st0["status"] == 0, st0

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    accepted = 0
    barrier(world)
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        wall0 = time.perf_counter()
        for i in range(args.steps):
            flush.fill_(i & 0xFF)
            ev[i][0].record(stream)
            one_step()
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
        barrier(world)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    st = qt.stats_from_bytes(stb)
    assert st["status"] == 0, st
    accepted = st["accepted"] * args.steps  # deterministic per step
    t_dev = sum(step_ms) / 1e3
    t_max = dist_max(t_dev, world)
    total_steps = dist_sum(float(accepted), world)
    value = total_steps / t_max
    ms_per_step = t_max * 1e3 / args.steps

    # end to end through the host-memory C call (packing, copies, solve, read-back)
    e2e = None
    if rank == 0:
        import scipy.sparse as sp
        h2d = 0
        for op in [s["H"], *s["c_ops"], *s["e_ops"]]:
            m = sp.csr_matrix(op)
            h2d += m.indptr.size * 8 + m.indices.size * 4 + m.data.size * 16
        h2d += s["psi0"].size * 16 + s["tlist"].size * 8
        d2h = nt * ne * 16 + 8 + 56
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        reps = max(1, min(args.steps, 3))
        acc_e2e = 0
        for _ in range(reps):
            _, _, _, st_h = qt.qt_mcsolve(s["H"], s["c_ops"], s["e_ops"], s["psi0"], s["tlist"],
                                          NTRAJ, seed=SEED, opts=o, jump_cap=0)
            acc_e2e += st_h["accepted"]
        e2e_t = time.perf_counter() - t0
        e2e = {"value": acc_e2e / e2e_t, "unit": "traj-steps/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h)}

    line = None
    if rank == 0:
        measure_peaks(qt, local)
        kernel_s = statistics.mean(step_ms) / 1e3
        line = {
            "metric": "MC traj-steps/s", "value": value, "unit": "traj-steps/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c64+f64", "data": "synthetic", "config": config,
            "gpu_launches": 3 * args.steps,
            "stats_per_step": {k: st[k] for k in ("accepted", "rejected", "rhs_evals",
                                                  "bisect_iters", "jumps", "near_miss")},
            "roofline": roof(flops_step * st["accepted"], kernel_s, "fp32",
                             traffic=mc_traffic(), kernel="mc_kernel<float,32,2,3>",
                             flops_per_traj_step=flops_step),
            "clocks": clk.summary(),
            "peaks_measured": dict(PEAKS),
            "e2e": e2e,
            "wall_s": wall,
        }
    barrier(world)

    if rank == 0:
        # the plain FP64 kernel on a share of the same workload, same tolerances
        n64 = 2048
        o64 = qt.qt_opts_default(rtol=RTOL, atol=ATOL, precision=qt.QT_FP64)
        es64 = torch.zeros((nt, ne), dtype=torch.complex128, device=dev)
        stb64 = torch.zeros(56, dtype=torch.uint8, device=dev)
        sysm.qt_mcsolve_dev(psi0, tl, n64, SEED, o64, es64, stats=stb64)
        torch.cuda.synchronize()
        a64, b64 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a64.record(stream)
        sysm.qt_mcsolve_dev(psi0, tl, n64, SEED, o64, es64, stats=stb64,
                            stream=stream.cuda_stream)
        b64.record(stream)
        torch.cuda.synchronize()
        st64 = qt.stats_from_bytes(stb64)
        v64 = st64["accepted"] / (a64.elapsed_time(b64) / 1e3)
        line["fp64_kernel_same_workload"] = {
            "value": v64, "unit": "traj-steps/s", "trajectories": n64,
            "mixed_speedup": value / v64,
            "note": "mc_kernel<double> on trajectories 0..2047 of the same workload"}
    if rank == 0 and not args.no_me:
        line["mc_jc_dim20_fp64"] = bench_mc_jc(qt, S, dev)
        line["mc_xxz_dim1024"] = bench_mc_xxz(qt, S, dev)
        line["mc_kerr_time_dependent_drive"] = bench_mc_kerr_td(qt, S, dev)
        line["mc_trilinear_dim4913"] = bench_mc_trilinear(qt, S, dev)
        line["batch_sweep_4096"] = bench_batch(qt, S, dev)
        line["adjoint_transmon_256"] = bench_adjoint(qt, S, dev)
        line["mesolve"] = bench_me(qt, S, dev, oracle_timing=not args.no_cpu_baseline)
        line["correlation"] = bench_corr(qt, S, dev)
        line["steadystate"] = bench_ss(qt, S, dev)
    if rank == 0 and not args.no_cpu_baseline:
        rate, cores, sample, otex, ojumps, n = time_oracle_sample(s)
        line["cpu_baseline"] = {"value": rate, "unit": "traj-steps/s", "cores": cores,
                                "kind": "oracle", "sample": sample}
        rate1, sample1 = time_oracle_one_core(s)
        line["cpu_baseline"]["one_core"] = {"value": rate1, "unit": "traj-steps/s",
                                            "sample": sample1}
        # error of this precision against the FP64 oracle on the sampled trajectories
        line["error_vs_fp64_oracle"] = error_vs_oracle(qt, sysm, s, psi0, tl, o, dev, n, otex,
                                                       ojumps)
        if BATCH_OUT and "batch_sweep_4096" in line:
            line["batch_sweep_4096"]["error_vs_fp64_oracle"] = batch_error_vs_oracle()
    if rank == 0:
        print(json.dumps(line))
    sysm.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def error_vs_oracle(qt, sysm, s, psi0, tl, o, dev, n, otex, ojumps):
    """The mixed kernel's per-trajectory values and means on trajectories
    0..n-1 against the FP64 oracle's at the same tolerances.  Output samples
    within 1e-5 max(1, |tau|) of a jump time of either side are set aside (the
    jump may fall on the other side of the sample in the other precision) and
    counted; records must agree, which the line reports."""
    import torch
    from tests.parity import compare_jump_records, kept_samples, max_mean_diff
    nt, ne = len(s["tlist"]), len(s["e_ops"])
    tex = torch.zeros((n, nt, ne), dtype=torch.complex128, device=dev)
    es2 = torch.zeros((nt, ne), dtype=torch.complex128, device=dev)
    cap = 64 * n
    jb = torch.zeros(cap * 40, dtype=torch.uint8, device=dev)
    nj = torch.zeros(1, dtype=torch.int64, device=dev)
    sysm.qt_mcsolve_dev(psi0, tl, n, SEED, o, es2, traj_begin=0, traj_expect=tex, jumps=jb,
                        n_jumps=nj)
    torch.cuda.synchronize()
    gj = qt.jumps_from_bytes(jb, min(int(nj.item()), cap))
    gj.sort(order=["traj", "k"])
    gtex = tex.cpu().numpy()
    try:
        n_rec, div = compare_jump_records(gj, ojumps, range(n), 1e-3)
        records = "identical" if not div else f"{len(div)} trajectories part at a flagged channel draw"
    except AssertionError as e:
        return {"records": f"differ: {e}"}
    keep = kept_samples(n, range(n), s["tlist"], div, gj, ojumps, 1e-5)
    diff = np.abs(gtex - otex)
    per_traj = np.where(keep[:, :, None], diff, 0.0).max(axis=(1, 2))
    tau_rel = np.abs(gj["tau"] - ojumps["tau"]) / np.maximum(1.0, np.abs(ojumps["tau"]))
    sem = float((otex.std(axis=0, ddof=1) / np.sqrt(n)).max())
    return {
        "trajectories": n, "jump_records": records, "jumps_compared": n_rec,
        "max_abs_traj_expect": float(per_traj.max()),
        "median_abs_traj_expect": float(np.median(per_traj)),
        "max_abs_mean_expect": max_mean_diff(gtex, otex, keep),
        "max_standard_error_of_mean": sem,
        "samples_set_aside": int((~keep).sum()), "samples": int(keep.size),
        "max_abs_mean_expect_all_samples": float(np.abs(gtex.mean(axis=0) -
                                                        otex.mean(axis=0)).max()),
        "jump_time_rel_err_max": float(tau_rel.max()),
        "jump_time_rel_err_median": float(np.median(tau_rel)),
        "flagged_jumps_gpu": int((gj["degenerate"] != 0).sum()),
        "note": "<a^dag a>, <a> at all 401 times against the FP64 oracle at the same tolerances; "
                "samples within 1e-5 max(1,|tau|) of a jump of either side set aside and "
                "counted; the all-samples mean includes them (a sample on the other side of a "
                "jump moves the mean by the jump's size / n)"}


def batch_error_vs_oracle():
    """The batch's results for its largest problems against the FP64 oracle at
    the same tolerances: master equation per value, Monte Carlo per trajectory
    mean (the same trajectories on both sides)."""
    import oracle
    tl = BATCH_OUT["tlist"]
    err = {}
    for i, p, g in zip(BATCH_OUT["index"], BATCH_OUT["problems"], BATCH_OUT["results"]):
        if p["kind"] == "me":
            r, _, _ = oracle.mesolve(p["H"], p["c_ops"], p["e_ops"], p["state0"], tl,
                                     rtol=BATCH_RTOL, atol=BATCH_ATOL)
        else:
            te, _, _ = oracle.mcsolve(p["H"], p["c_ops"], p["e_ops"], p["state0"], tl, p["ntraj"],
                                      seed=p["seed"], rtol=BATCH_RTOL, atol=BATCH_ATOL,
                                      nthreads=os.cpu_count() or 1)
            r = te.mean(axis=0)
        err[f"problem_{i}_{p['kind']}_dim{p['dim']}"] = float(np.abs(g - r).max())
    return {"max_abs": max(err.values()), "per_problem": err,
            "note": "largest-dimension problems of the sweep against the FP64 oracle at "
                    "rtol 1e-6, atol 1e-8; Monte Carlo: means over the same 256 trajectories"}


def profile_case(args):
    """One warm-up and one measured launch of a small case, for ncu: the MC
    kernel on args.profile_ntraj Kerr trajectories, or the ME kernel on the
    XXZ chain (dim 1024, t in [0, 0.05]; me_tc: the tensor-core path)."""
    import torch
    from paper_1110_0573_gb300 import build as B
    from paper_1110_0573_gb300 import qt
    from paper_1110_0573_gb300 import systems as S
    B.build()
    dev = torch.device("cuda", 0)
    if args.profile_case == "ss":
        # the GMRES steady state of the Kerr cavity (dim 64), twice
        s = S.kerr_cavity()
        sysm = qt.System(s["H"], s["c_ops"], [])
        rho = torch.zeros((64, 64), dtype=torch.complex128, device=dev)
        stb = torch.zeros(56, dtype=torch.uint8, device=dev)
        for _ in range(2):
            sysm.qt_steadystate_dev(rho, max_iter=60000, stats=stb)
        torch.cuda.synchronize()
        print(json.dumps({"case": "ss", "stats": qt.stats_from_bytes(stb)}))
        sysm.close()
        return
    if args.profile_case == "corr":
        # <a^dag(t + tau) a(t)> of the Jaynes-Cummings model (dim 20, mixed):
        # 304 times x 151 delays, one CTA per time, twice
        import numpy as np
        s = S.jaynes_cummings()
        a = S.tensor(S.destroy(10), S.qeye(2))
        sysm = qt.System(s["H"], s["c_ops"], [S.dag(a), a])
        psi0 = torch.tensor(s["psi0"], dtype=torch.complex128, device=dev)
        tl = torch.tensor(np.linspace(0.0, 30.0, 304), dtype=torch.float64, device=dev)
        tau = torch.tensor(np.linspace(0.0, 30.0, 151), dtype=torch.float64, device=dev)
        out = torch.zeros((304, 151, 2), dtype=torch.complex128, device=dev)
        stb = torch.zeros(56, dtype=torch.uint8, device=dev)
        o = qt.qt_opts_default(rtol=1e-6, atol=1e-8, precision=qt.QT_MIXED)
        for _ in range(2):
            sysm.qt_correlation_2op_2t_dev(psi0, tl, tau, 1, o, out, stats=stb)
        torch.cuda.synchronize()
        print(json.dumps({"case": "corr", "stats": qt.stats_from_bytes(stb)}))
        sysm.close()
        return
    if args.profile_case == "mc_xxz":
        # the CTA-wide MC kernel on the XXZ chain (dim 1024): 304 trajectories
        # (two per CTA), t in [0, 10] at 101 points, mixed precision, twice
        s = S.xxz_chain()
        sysm = qt.System(s["H"], s["c_ops"], s["e_ops"])
        psi0 = torch.tensor(s["psi0"], dtype=torch.complex128, device=dev)
        tl = torch.tensor(s["tlist"], dtype=torch.float64, device=dev)
        es = torch.zeros((len(s["tlist"]), len(s["e_ops"])), dtype=torch.complex128, device=dev)
        stb = torch.zeros(56, dtype=torch.uint8, device=dev)
        o = qt.qt_opts_default(rtol=RTOL, atol=ATOL, precision=qt.QT_MIXED)
        for _ in range(2):
            sysm.qt_mcsolve_dev(psi0, tl, args.profile_ntraj, SEED, o, es, stats=stb)
        torch.cuda.synchronize()
        print(json.dumps({"case": args.profile_case, "stats": qt.stats_from_bytes(stb)}))
    elif args.profile_case.startswith("mc"):
        s = S.kerr_cavity()
        prec = qt.QT_MIXED if args.profile_case == "mc" else qt.QT_FP64
        sysm = qt.System(s["H"], s["c_ops"], s["e_ops"])
        psi0 = torch.tensor(s["psi0"], dtype=torch.complex128, device=dev)
        tl = torch.tensor(s["tlist"], dtype=torch.float64, device=dev)
        es = torch.zeros((len(s["tlist"]), 2), dtype=torch.complex128, device=dev)
        stb = torch.zeros(56, dtype=torch.uint8, device=dev)
        o = qt.qt_opts_default(rtol=RTOL, atol=ATOL, precision=prec)
        for _ in range(2):
            sysm.qt_mcsolve_dev(psi0, tl, args.profile_ntraj, SEED, o, es, stats=stb)
        torch.cuda.synchronize()
        print(json.dumps({"case": args.profile_case, "stats": qt.stats_from_bytes(stb)}))
    else:
        s = S.xxz_chain(t_end=0.05, nt=2)
        prec = qt.QT_FP64 if args.profile_case == "me_fp64" else qt.QT_MIXED
        method = qt.QT_ME_DENSE_TC if args.profile_case == "me_tc" else qt.QT_ME_AUTO
        sysm = qt.System(s["H"], s["c_ops"], s["e_ops"])
        psi0 = torch.tensor(s["psi0"], dtype=torch.complex128, device=dev)
        tl = torch.tensor(s["tlist"], dtype=torch.float64, device=dev)
        ex = torch.zeros((2, len(s["e_ops"])), dtype=torch.complex128, device=dev)
        stb = torch.zeros(56, dtype=torch.uint8, device=dev)
        o = qt.qt_opts_default(rtol=1e-6 if prec == qt.QT_MIXED else 1e-8,
                               atol=1e-8 if prec == qt.QT_MIXED else 1e-10, precision=prec,
                               me_method=method)
        for _ in range(2):
            sysm.qt_mesolve_dev(psi0, tl, o, ex, stats=stb)
        torch.cuda.synchronize()
        print(json.dumps({"case": args.profile_case, "stats": qt.stats_from_bytes(stb)}))
    sysm.close()


def bench_mc_xxz(qt, S, dev):
    """MC on the dissipative XXZ chain, dim 1024 (one trajectory per CTA):
    4096 trajectories, t in [0, 10] at 101 points, mixed precision."""
    import torch
    s = S.xxz_chain()
    sysm = qt.System(s["H"], s["c_ops"], s["e_ops"])
    psi0 = torch.tensor(s["psi0"], dtype=torch.complex128, device=dev)
    tl = torch.tensor(s["tlist"], dtype=torch.float64, device=dev)
    es = torch.zeros((len(s["tlist"]), len(s["e_ops"])), dtype=torch.complex128, device=dev)
    stb = torch.zeros(56, dtype=torch.uint8, device=dev)
    o = qt.qt_opts_default(rtol=RTOL, atol=ATOL, precision=qt.QT_MIXED)
    sysm.qt_mcsolve_dev(psi0, tl, 256, SEED, o, es, stats=stb)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    sysm.qt_mcsolve_dev(psi0, tl, 4096, SEED, o, es, stats=stb)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    st = qt.stats_from_bytes(stb)
    nnz = int((s["H"] - 0.5j * sum((c.conj().T @ c) for c in s["c_ops"])).nnz)
    flops = mc_flops_per_traj_step(1024, nnz) * st["accepted"]
    sysm.close()
    return {"traj_steps_per_s": st["accepted"] / (ms / 1e3), "ms": ms, "trajectories": 4096,
            "accepted": st["accepted"], "jumps": st["jumps"], "status": st["status"],
            "roofline": roof(flops, ms / 1e3, "fp32", kernel="mc_kernel<float,512,2,-2,CTA-wide>",
                             flops_per_traj_step=mc_flops_per_traj_step(1024, nnz))}


def bench_mc_kerr_td(qt, S, dev):
    """MC with a time-dependent Hamiltonian: the Kerr workload with its drive
    switched on by a piecewise-linear coefficient, H(t) = H_Kerr(E=0) +
    f(t) (a + a^dag), f rising from 0 to E = 1 on [0, 5] (paper section 4.3
    in the form of the library); 16384 trajectories, t in [0, 20] at 401
    points, mixed precision -- beside the time-independent workload above."""
    import numpy as np
    import torch
    s = S.kerr_cavity(E=0.0)
    a = S.destroy(64)
    td = [((a + a.T.conj()).tocsr(), np.array([0.0, 5.0]), np.array([0.0, 1.0]))]
    sysm = qt.System(s["H"], s["c_ops"], s["e_ops"], td=td)
    psi0 = torch.tensor(s["psi0"], dtype=torch.complex128, device=dev)
    tl = torch.tensor(s["tlist"], dtype=torch.float64, device=dev)
    es = torch.zeros((len(s["tlist"]), len(s["e_ops"])), dtype=torch.complex128, device=dev)
    stb = torch.zeros(56, dtype=torch.uint8, device=dev)
    o = qt.qt_opts_default(rtol=RTOL, atol=ATOL, precision=qt.QT_MIXED)
    sysm.qt_mcsolve_dev(psi0, tl, 2048, SEED, o, es, stats=stb)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    sysm.qt_mcsolve_dev(psi0, tl, NTRAJ, SEED, o, es, stats=stb)
    ev1.record()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    st = qt.stats_from_bytes(stb)
    sysm.close()
    heff = s["H"] - 0.5j * sum((c.conj().T @ c) for c in s["c_ops"])
    nnz = int(heff.tocsr().nnz) + int(td[0][0].nnz)  # H_eff and the drive term per RHS
    fl = mc_flops_per_traj_step(64, nnz)
    return {"traj_steps_per_s": st["accepted"] / (ms / 1e3), "ms": ms, "trajectories": NTRAJ,
            "accepted": st["accepted"], "jumps": st["jumps"], "status": st["status"],
            "roofline": roof(fl * st["accepted"], ms / 1e3, "fp32",
                             kernel="mc_kernel<float,32,2,3,time-dependent>",
                             flops_per_traj_step=fl)}


def bench_mc_jc(qt, S, dev):
    """The Jaynes-Cummings Monte-Carlo workload in FP64 (cavity N = 10 x
    qubit, dim 20): 500 trajectories, t in [0, 50] at 201 points, rtol 1e-8,
    seed 0 (paper section 4.2), beside its master-equation solve."""
    import torch
    s = S.jaynes_cummings()
    sysm = qt.System(s["H"], s["c_ops"], s["e_ops"])
    psi0 = torch.tensor(s["psi0"], dtype=torch.complex128, device=dev)
    tl = torch.tensor(s["tlist"], dtype=torch.float64, device=dev)
    es = torch.zeros((len(s["tlist"]), len(s["e_ops"])), dtype=torch.complex128, device=dev)
    stb = torch.zeros(56, dtype=torch.uint8, device=dev)
    o = qt.qt_opts_default(rtol=1e-8, atol=1e-10, precision=qt.QT_FP64)
    sysm.qt_mcsolve_dev(psi0, tl, 500, 0, o, es, stats=stb)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    sysm.qt_mcsolve_dev(psi0, tl, 500, 0, o, es, stats=stb)
    ev1.record()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    st = qt.stats_from_bytes(stb)
    sysm.close()
    heff = s["H"] - 0.5j * sum((c.conj().T @ c) for c in s["c_ops"])
    fl = mc_flops_per_traj_step(20, int(heff.tocsr().nnz))
    return {"traj_steps_per_s": st["accepted"] / (ms / 1e3), "ms": ms, "trajectories": 500,
            "accepted": st["accepted"], "jumps": st["jumps"], "status": st["status"],
            "roofline": roof(fl * st["accepted"], ms / 1e3, "fp64",
                             kernel="mc_kernel<double,32,1,4>", flops_per_traj_step=fl,
                             note="500 trajectories fill 500 of the GPU's 4864 warp slots")}


def bench_mc_trilinear(qt, S, dev):
    """The paper's trilinear Monte-Carlo example (section 4.3): three modes of
    17 levels (dim 4913), 1000 trajectories, t in [0, 4] at 201 points, mixed
    precision; one CTA per trajectory with the stage vectors in global
    memory."""
    import torch
    s = S.trilinear()
    sysm = qt.System(s["H"], s["c_ops"], s["e_ops"])
    psi0 = torch.tensor(s["psi0"], dtype=torch.complex128, device=dev)
    tl = torch.tensor(s["tlist"], dtype=torch.float64, device=dev)
    es = torch.zeros((len(s["tlist"]), len(s["e_ops"])), dtype=torch.complex128, device=dev)
    stb = torch.zeros(56, dtype=torch.uint8, device=dev)
    o = qt.qt_opts_default(rtol=RTOL, atol=ATOL, precision=qt.QT_MIXED)
    sysm.qt_mcsolve_dev(psi0, tl, 152, SEED, o, es, stats=stb)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    sysm.qt_mcsolve_dev(psi0, tl, 1000, SEED, o, es, stats=stb)
    ev1.record()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    st = qt.stats_from_bytes(stb)
    means = (es[-1] / 1000).real.cpu().tolist()
    sysm.close()
    heff = s["H"] - 0.5j * sum((c.conj().T @ c) for c in s["c_ops"])
    d = s["H"].shape[0]
    fl = mc_flops_per_traj_step(d, int(heff.tocsr().nnz))
    return {"traj_steps_per_s": st["accepted"] / (ms / 1e3), "ms": ms, "trajectories": 1000,
            "accepted": st["accepted"], "jumps": st["jumps"], "status": st["status"],
            "final_occupations": means,
            "roofline": roof(fl * st["accepted"], ms / 1e3, "fp32",
                             kernel="mc_kernel<float,512,10,0,CTA-wide,stages in global memory>",
                             flops_per_traj_step=fl,
                             note="bound by the latency of the stage vectors' L2 traffic")}


BATCH_RTOL, BATCH_ATOL = 1e-6, 1e-8
BATCH_OUT = {}


def bench_batch(qt, S, dev, n_instances=4096):
    """The uneven parameter sweep in one persistent launch: 4096 cavity+qubit
    instances (dim 8..64), half master equation, half Monte Carlo with 256
    trajectories, t in [0, 30] at 121 points, mixed precision at rtol 1e-6;
    launch configuration autotuned, the solve captured in a CUDA graph and
    replayed.  The results of the largest problems are kept for the error
    check against the oracle (cpu_baseline leg)."""
    import torch
    problems, tlist = S.cavity_qubit_sweep(n_instances, seed=1)
    b = qt.Batch(problems)
    tl = torch.tensor(tlist, dtype=torch.float64, device=dev)
    ex = torch.zeros(b.expect_offset(b.n, len(tlist)), dtype=torch.complex128, device=dev)
    stb = torch.zeros(56, dtype=torch.uint8, device=dev)
    o = qt.qt_opts_default(rtol=BATCH_RTOL, atol=BATCH_ATOL, precision=qt.QT_MIXED)
    t0 = time.perf_counter()
    b.qt_batch_tune(tl, o, ex)
    tune_s = time.perf_counter() - t0
    tuned = b.config()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        b.qt_batch_solve_dev(tl, o, ex, stats=stb, stream=side.cuda_stream)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        b.qt_batch_solve_dev(tl, o, ex, stats=stb, stream=torch.cuda.current_stream().cuda_stream)
    g.replay()
    torch.cuda.synchronize()
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a0.record()
    g.replay()
    a1.record()
    torch.cuda.synchronize()
    ms = a0.elapsed_time(a1)
    st = qt.stats_from_bytes(stb)
    per = b.problem_stats()
    out = b.split(ex.cpu().numpy(), len(tlist))
    n_mc = sum(1 for p in problems if p["kind"] == "mc")
    # two master-equation and two Monte-Carlo problems of the largest dimension
    sample = [i for k in ("me", "mc")
              for i in sorted((i for i, p in enumerate(problems) if p["kind"] == k),
                              key=lambda i: (-problems[i]["dim"], i))[:2]]
    BATCH_OUT.update(problems=[problems[i] for i in sample], results=[out[i] for i in sample],
                     tlist=tlist, index=sample)
    # algorithmic flops from each problem's own counts: Monte-Carlo accepted
    # trajectory steps x mc_flops_per_traj_step, master-equation right-hand
    # sides x me_sparse_flops_per_rhs
    flops, mc_steps = 0.0, 0
    for pr, ps in zip(problems, per):
        if pr["kind"] == "mc":
            heff = pr["H"] - 0.5j * sum((c.conj().T @ c) for c in pr["c_ops"])
            flops += mc_flops_per_traj_step(pr["dim"], int(heff.tocsr().nnz)) * int(ps["accepted"])
            mc_steps += int(ps["accepted"])
        else:
            flops += me_sparse_flops_per_rhs(pr) * int(ps["rhs_evals"])
    b.close()
    return {"ms": ms, "instances": n_instances, "me_instances": n_instances - n_mc,
            "mc_instances": n_mc, "trajectories": n_mc * 256,
            "accepted_steps": st["accepted"], "mc_traj_steps": mc_steps,
            "rhs_evals": st["rhs_evals"],
            "accepted_steps_per_s": st["accepted"] / (ms / 1e3),
            "rhs_evals_per_s": st["rhs_evals"] / (ms / 1e3), "status": st["status"],
            "tune_s": tune_s, "tuned": tuned, "graph": True,
            "roofline": roof(flops, ms / 1e3, "fp32", kernel="batch_kernel<float>")}


def bench_adjoint(qt, S, dev, batch=256):
    """Gradients of the transmon-cavity loss (dim 60, 64 drive segments,
    three decay rates) for 256 random drive vectors: adaptive forward pass
    with segment checkpoints plus the adjoint backward pass, FP64."""
    import torch
    s = S.transmon_cavity()
    adj = qt.Adjoint(s["H0"], s["Hd"], s["A"], s["P1"], s["P2"], s["psi0"], s["n_seg"],
                     s["t_seg"], batch)
    omega = torch.tensor(S.drive_vectors(batch, s["n_seg"], seed=2), dtype=torch.float64,
                         device=dev)
    gamma = torch.tensor(np.tile(s["gamma"], (batch, 1)), dtype=torch.float64, device=dev)
    o = qt.qt_opts_default(rtol=1e-8, atol=1e-10)
    loss = torch.zeros(batch, dtype=torch.float64, device=dev)
    go = torch.zeros((batch, s["n_seg"]), dtype=torch.float64, device=dev)
    gg = torch.zeros((batch, 3), dtype=torch.float64, device=dev)
    stb = torch.zeros(56, dtype=torch.uint8, device=dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    ev[0].record()
    adj.forward(omega, gamma, o, loss, stats=stb)
    ev[1].record()
    adj.backward(None, go, gg)
    ev[2].record()
    torch.cuda.synchronize()
    st = qt.stats_from_bytes(stb)
    fwd, bwd = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
    adj.close()
    # algorithmic work: 6 right-hand sides per accepted step forward, and per
    # step backward 6 recomputed ones plus 6 adjoint ones of the same cost
    frhs = me_sparse_flops_per_rhs({"H": s["H0"] + s["Hd"], "c_ops": s["A"]})
    fl = 18 * frhs * st["accepted"]
    return {"forward_ms": fwd, "backward_ms": bwd, "batch": batch,
            "gradients_per_s": batch / ((fwd + bwd) / 1e3),
            "accepted_steps": st["accepted"], "status": st["status"],
            "mean_loss": float(loss.mean().item()),
            "roofline": roof(fl, (fwd + bwd) / 1e3, "fp64",
                             kernel="adjoint_forward_kernel + adjoint_backward_kernel",
                             flops_per_rhs=frhs,
                             note="18 right-hand sides of algorithmic work per accepted step")}


def me_tc_flops_per_rhs(d, n_dense_c=0):
    """Tensor-core flops of one dense right-hand side: the real GEMM
    (dp x 2dp) = (dp x 2dp)(2dp x 2dp)^T, dp = d rounded up to 128, three
    BF16 products (hi*hi, hi*lo, lo*hi): 3 * 2 * dp * 2dp * 2dp; with dense
    collapse operators also T = [C_1; ...] y (n_c such GEMMs) and W = T [C
    ...]^dag (K = 2 n_c dp): 24 dp^3 (1 + 2 n_c)."""
    dp = (d + 127) // 128 * 128
    return 24.0 * dp ** 3 * (1 + 2 * n_dense_c)


def me_sparse_flops_per_rhs(s, hermitian=False):
    """Algorithmic flops of one sparse right-hand side: 8 flops per complex
    multiply-add; H_eff rho and rho H_eff^dag take nnz(H_eff) * d each, the
    collapse terms sum_n (row nnz of C_n)^2 * d^2 (for C with one entry per
    row: d^2 each).  For a Hermitian state (hermitian=True) the work the
    right-hand side needs is half of that: rho H_eff^dag = (H_eff rho)^dag and
    C rho C^dag is Hermitian, so one product and one triangle of the collapse
    terms determine it."""
    import numpy as np
    H = s["H"].tocsr()
    d = H.shape[0]
    heff = H.copy()
    for c in s["c_ops"]:
        heff = heff - 0.5j * (c.conj().T @ c)
    nnz = heff.tocsr().nnz
    csum = sum(float(np.sum(np.diff(c.tocsr().indptr) ** 2)) * d for c in s["c_ops"])
    return 8.0 * (2 * nnz * d + csum) * (0.5 if hermitian else 1.0)


def run_me(qt, s, dev, prec, rtol, atol, method):
    import torch
    sysm = qt.System(s["H"], s["c_ops"], s["e_ops"])
    psi0 = torch.tensor(s["psi0"], dtype=torch.complex128, device=dev)
    tl = torch.tensor(s["tlist"], dtype=torch.float64, device=dev)
    ex = torch.zeros((len(s["tlist"]), len(s["e_ops"])), dtype=torch.complex128, device=dev)
    stb = torch.zeros(56, dtype=torch.uint8, device=dev)
    o = qt.qt_opts_default(rtol=rtol, atol=atol, precision=prec, me_method=method)
    sysm.qt_mesolve_dev(psi0, tl, o, ex, stats=stb)  # warm-up (allocates the workspace)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    sysm.qt_mesolve_dev(psi0, tl, o, ex, stats=stb)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    st = qt.stats_from_bytes(stb)
    sysm.close()
    return ex.cpu().numpy(), ms, st


def me_line(qt, s, d, ex, ms, st, prec, method, ref):
    """One master-equation line: right-hand sides per second, the roofline of
    its kernel (sparse: algorithmic flops against the FP64 or FP32 roof;
    tensor cores: the dense GEMM flops against the measured BF16 roof, with
    the sparse algorithmic rate beside it) and the error against ref."""
    import numpy as np
    sec = ms / 1e3
    r = {"rhs_evals_per_s": st["rhs_evals"] / sec, "ms": ms, "rhs_evals": st["rhs_evals"],
         "accepted": st["accepted"], "status": st["status"]}
    sparse = me_sparse_flops_per_rhs(s, hermitian=True) * st["rhs_evals"]
    if method == qt.QT_ME_DENSE_TC:
        wide = any(np.diff(c.tocsr().indptr).max(initial=0) >= 32 for c in s["c_ops"])
        nd = len(s["c_ops"]) if wide else 0
        r["roofline"] = roof(me_tc_flops_per_rhs(d, nd) * st["rhs_evals"], sec, "bf16",
                             bound="tensor", kernel="me_tc_kernel",
                             sparse_algorithmic_tflops=sparse / sec / 1e12)
    else:
        r["roofline"] = roof(sparse, sec, "fp64" if prec == qt.QT_FP64 else "fp32",
                             kernel="me_kernel / me_block_kernel")
    if ref is not None:
        r["max_err_vs_fp64"] = float(np.abs(ex - ref).max())
    return r


def bench_me(qt, S, dev, oracle_timing=True):
    """mesolve right-hand-side evaluations per second: the Jaynes-Cummings
    model (dim 20, FP64, t in [0, 50]) and the XXZ chain (dim 1024, t in
    [0, 10] at 101 points) on the sparse FP64, sparse mixed and dense
    tensor-core paths, with each result's error against the sparse FP64 one
    (the FP64 solvers agree with the FP64 oracle within 1e-8 in the parity
    tests, on the full-size XXZ chain over t in [0, 0.02]); with
    oracle_timing, the FP64 oracle's rate on one host core beside the FP64
    lines."""
    import numpy as np
    out = {}
    s = S.jaynes_cummings()
    ex, ms, st = run_me(qt, s, dev, qt.QT_FP64, 1e-8, 1e-10, qt.QT_ME_AUTO)
    out["jc_dim20_fp64"] = me_line(qt, s, 20, ex, ms, st, qt.QT_FP64, qt.QT_ME_AUTO, None)
    if oracle_timing:
        out["jc_dim20_fp64"]["cpu_oracle"] = time_oracle_me(s, 1e-8, 1e-10)
    s = S.xxz_chain()
    d = s["H"].shape[0]
    ref = None
    for name, prec, rtol, atol, method in [
            ("xxz_dim1024_fp64_sparse", qt.QT_FP64, 1e-8, 1e-10, qt.QT_ME_AUTO),
            ("xxz_dim1024_mixed_sparse", qt.QT_MIXED, 1e-6, 1e-8, qt.QT_ME_AUTO),
            ("xxz_dim1024_mixed_dense_tc", qt.QT_MIXED, 1e-6, 1e-8, qt.QT_ME_DENSE_TC)]:
        ex, ms, st = run_me(qt, s, dev, prec, rtol, atol, method)
        out[name] = me_line(qt, s, d, ex, ms, st, prec, method, ref)
        ref = ex if ref is None else ref
    if oracle_timing:
        out["xxz_dim1024_fp64_sparse"]["cpu_oracle"] = time_oracle_me(s, 1e-8, 1e-10, n_rhs=2)
    # a dense Hamiltonian (every entry nonzero), where the tensor-core product
    # does the algorithmic work: dim 1024, t in [0, 0.5]
    s = S.dense_random_hamiltonian()
    ref = None
    for name, prec, rtol, atol, method in [
            ("dense_h_dim1024_fp64_sparse", qt.QT_FP64, 1e-8, 1e-10, qt.QT_ME_AUTO),
            ("dense_h_dim1024_mixed_sparse", qt.QT_MIXED, 1e-6, 1e-8, qt.QT_ME_AUTO),
            ("dense_h_dim1024_mixed_dense_tc", qt.QT_MIXED, 1e-6, 1e-8, qt.QT_ME_DENSE_TC)]:
        ex, ms, st = run_me(qt, s, dev, prec, rtol, atol, method)
        out[name] = me_line(qt, s, d, ex, ms, st, prec, method, ref)
        ref = ex if ref is None else ref
    # dense collapse operators as well (every collapse term on the tensor
    # cores), dim 1024, t in [0, 0.1]
    s = S.dense_collapse_system()
    ex, ms, st = run_me(qt, s, dev, qt.QT_MIXED, 1e-6, 1e-8, qt.QT_ME_DENSE_TC)
    out["dense_h_dense_c_dim1024_mixed_dense_tc"] = me_line(qt, s, 1024, ex, ms, st, qt.QT_MIXED,
                                                            qt.QT_ME_DENSE_TC, None)
    return out


def run_corr(qt, s, A, B, dev, prec, rtol, atol, tlist, taulist):
    import torch
    sysm = qt.System(s["H"], s["c_ops"], [A, B])
    psi0 = torch.tensor(s["psi0"], dtype=torch.complex128, device=dev)
    tl = torch.tensor(tlist, dtype=torch.float64, device=dev)
    tau = torch.tensor(taulist, dtype=torch.float64, device=dev)
    out = torch.zeros((len(tlist), len(taulist), 2), dtype=torch.complex128, device=dev)
    stb = torch.zeros(56, dtype=torch.uint8, device=dev)
    o = qt.qt_opts_default(rtol=rtol, atol=atol, precision=prec)
    sysm.qt_correlation_2op_2t_dev(psi0, tl, tau, 1, o, out, stats=stb)  # allocates the store
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    sysm.qt_correlation_2op_2t_dev(psi0, tl, tau, 1, o, out, stats=stb)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    st = qt.stats_from_bytes(stb)
    sysm.close()
    return out[:, :, 0].cpu().numpy(), ms, st


def bench_corr(qt, S, dev):
    """Two-time correlation functions <a^dag(t + tau) a(t)> (quantum
    regression theorem): the Jaynes-Cummings model (dim 20; 304 times t_k in
    [0, 30], 151 delays tau in [0, 30]; every X_k = a rho(t_k) on its own CTA)
    in FP64 and mixed precision, and the XXZ chain (dim 1024, mixed; 4 times,
    21 delays in [0, 2]; one cooperative launch per t_k) with <S^+_0(t + tau)
    S^-_0(t)>.  Values: correlation entries and right-hand sides per second,
    the mixed results' error against the FP64 run."""
    import numpy as np
    out = {}
    s = S.jaynes_cummings()
    N = 10
    a = S.tensor(S.destroy(N), S.qeye(2))
    tlist, taulist = np.linspace(0.0, 30.0, 304), np.linspace(0.0, 30.0, 151)
    ref = None
    for name, prec, rtol, atol in [("jc_dim20_fp64", qt.QT_FP64, 1e-8, 1e-10),
                                   ("jc_dim20_mixed", qt.QT_MIXED, 1e-6, 1e-8)]:
        c, ms, st = run_corr(qt, s, S.dag(a), a, dev, prec, rtol, atol, tlist, taulist)
        r = {"corr_entries_per_s": c.size / (ms / 1e3), "rhs_evals_per_s":
             st["rhs_evals"] / (ms / 1e3), "ms": ms, "rhs_evals": st["rhs_evals"],
             "n_t": len(tlist), "n_tau": len(taulist), "status": st["status"],
             "roofline": roof(me_sparse_flops_per_rhs(s) * st["rhs_evals"], ms / 1e3,
                              "fp64" if prec == qt.QT_FP64 else "fp32",
                              kernel="corr_block_kernel")}
        if ref is None:
            ref = c
        else:
            r["max_err_vs_fp64"] = float(np.abs(c - ref).max())
            r["max_abs_corr"] = float(np.abs(ref).max())
        out[name] = r
    s = S.xxz_chain()
    L = 10
    sp_ = S.site_op(S.sigmap(), 0, L)
    c, ms, st = run_corr(qt, s, sp_, S.dag(sp_), dev, qt.QT_MIXED, 1e-6, 1e-8,
                         np.array([0.0, 0.5, 1.0, 1.5]), np.linspace(0.0, 2.0, 21))
    out["xxz_dim1024_mixed"] = {"corr_entries_per_s": c.size / (ms / 1e3),
                                "rhs_evals_per_s": st["rhs_evals"] / (ms / 1e3), "ms": ms,
                                "rhs_evals": st["rhs_evals"], "status": st["status"],
                                "roofline": roof(me_sparse_flops_per_rhs(s) * st["rhs_evals"],
                                                 ms / 1e3, "fp32", kernel="me_kernel<float>")}
    return out


def bench_ss(qt, S, dev):
    """Steady states: the Kerr cavity (dim 64) by the GMRES solve and by the
    propagator method (FP64 and mixed), and a random sparse system (dim 100)
    by GMRES; each result's residual ||L(rho)||_F and its distance to the
    FP64 GMRES state of the same system."""
    import numpy as np
    import torch
    out = {}

    def timed(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = fn()
        torch.cuda.synchronize()
        return r, (time.perf_counter() - t0) * 1e3

    for name, s in [("kerr_dim64", S.kerr_cavity()),
                    ("random_dim100", S.random_system(100, 2, 1, seed=100, density=0.06))]:
        qt.qt_steadystate(s["H"], s["c_ops"], max_iter=60000)  # warm-up
        (rho, info, st), ms = timed(lambda: qt.qt_steadystate(s["H"], s["c_ops"], max_iter=60000))
        out[name + "_gmres_fp64"] = {"ms": ms, "arnoldi_steps": info["steps"],
                                     "rhs_evals": st["rhs_evals"],
                                     "relative_residual": info["residual"], "status": st["status"]}
        if name == "kerr_dim64":
            ref = rho
            for pname, prec, rtol, atol, tol in [("fp64", qt.QT_FP64, 1e-11, 1e-13, 1e-10),
                                                 ("mixed", qt.QT_MIXED, 1e-7, 1e-9, 1e-5)]:
                o = qt.qt_opts_default(rtol=rtol, atol=atol, precision=prec)
                (rp, pi, pst), ms = timed(lambda: qt.qt_propagator_steadystate(
                    s["H"], s["c_ops"], period=20.0, tol=tol, opts=o))
                out[name + "_propagator_" + pname] = {
                    "ms": ms, "periods": pi["periods"], "rhs_evals": pst["rhs_evals"],
                    "last_change": pi["change"], "max_diff_vs_gmres": float(np.abs(rp - ref).max()),
                    "status": pst["status"]}
    return out


if __name__ == "__main__":
    main()
