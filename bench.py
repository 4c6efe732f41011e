"""Cosm throughput bench: edge-replica updates/s and time-to-target.

Default workload: the 20,000-spin 2D +-1 toroidal glass (100 x 200, 40,000
edges, J uniform in {-1,+1} from seed 0, regular 4-colour partition), FP32
phases resident in shared memory, 1,024 replicas, 10^5 sweeps per trial,
alpha_0 = 14 deg, DWT ratio 0.5 every 3 sweeps, 100 bisectors. One step is
one full trial of every replica (init, all sweeps, DWT, schedule, readout
with exact cuts and best-state tracking).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--storage f32|f16|q16|bf16] [--workload torus20k|torus10k|...]

Prints one JSON line (rank 0). Beside the headline it carries, on the
default workload: the end-to-end rate through the host-buffer call, the
rooflines (the method's shared-memory byte count and 6 FP32 operations per
update against measured peaks, and ncu-measured traffic), time-to-target
with Wilson intervals at 10^5 and 10^6 sweeps per trial, the 2-byte storage
forms, and the ragged batch in three forms. ``--impl reference`` times the
FP64 CPU oracle on the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import instances  # noqa: E402

L2_BYTES = 129 * 1024 * 1024

HEADLINE_METRIC = "edge-replica updates/s (20k-spin 2D +-1 glass, plain FP32 Cosm)"


def metric_name(workload: str) -> str:
    """The metric string of a single-instance workload's JSON line."""
    return {
        "torus10k": "edge-replica updates/s (10k-spin 2D +-1 glass, plain FP32 Cosm)",
        "reg3_20k": "edge-replica updates/s (20k-spin random 3-regular +-1 graph, plain FP32 Cosm)",
        "reg4_20k": "edge-replica updates/s (20k-spin random 4-regular +-1 graph, plain FP32 Cosm)",
        "torus16": "edge-replica updates/s (256-spin 2D +-1 glass, plain FP32 Cosm)",
        "fields2d": "edge+field replica updates/s (planted 2D lattice with local fields)",
        "readout": "edge-replica updates/s with the optimal bisector and tracking every 1000 sweeps",
    }.get(workload, HEADLINE_METRIC)

WORKLOADS = {
    # name: (builder, replicas, sweeps, params, description)
    "torus20k": (lambda: instances.torus2d(100, 200, 0), 1024, 100_000,
                 dict(alpha0_deg=14.0, dwt_ratio=0.5, dwt_period=3),
                 "2D +-1 torus 100x200 (N=20000, E=40000), 4-colour, 1024 replicas, 1e5 sweeps"),
    "torus10k": (lambda: instances.torus2d(100, 100, 0), 1024, 100_000,
                 dict(alpha0_deg=14.0, dwt_ratio=0.5, dwt_period=3),
                 "2D +-1 torus 100x100 (N=10000, E=20000), 4-colour, 1024 replicas, 1e5 sweeps"),
    "reg3_20k": (lambda: instances.random_regular(20000, 3, 0), 2048, 10_000,
                 dict(alpha0_deg=14.0, dwt_ratio=1.0, dwt_period=3),
                 "random 3-regular N=20000, Misra-Gries colouring, 2048 replicas, 1e4 sweeps"),
    "reg4_20k": (lambda: instances.random_regular(20000, 4, 0), 2048, 10_000,
                 dict(alpha0_deg=14.0, dwt_ratio=1.0, dwt_period=3),
                 "random 4-regular N=20000, Misra-Gries colouring, 2048 replicas, 1e4 sweeps"),
    "batch512": (None, None, 2000, dict(alpha0_deg=14.0, dwt_ratio=1.0, dwt_period=3),
                 "ragged batch: 512 instances, N log-uniform in [800, 20000], half 2D +-1 tori, "
                 "half G(n, m) with average degree 4-6 and weights in [-3,3]\\{0}, 64-256 replicas "
                 "each, 2000 sweeps per trial, one graph-captured run"),
    "serve": (None, 32, 2000, dict(alpha0_deg=25.0, dwt_ratio=1.0, dwt_period=3),
              "serving: Poisson arrivals (50 requests/s for 10 s) of frustrated-loop planted "
              "instances on 2D/3D periodic lattices (N in [1000, 50000], loop density 0.2-1.0), "
              "32 replicas x 2000 sweeps per trial, up to 4 trials, target = planted optimum, "
              "FP16 phase storage"),
    "ablation": (lambda: g70_like(0), 512, 20_000, dict(alpha0_deg=14.0, dwt_ratio=1.0, dwt_period=6),
                 "ablation of Table VII on a G70-like graph (G(n, m) with n = 10000, m = 9999, unit "
                 "weights, greedy colouring): Cosm, without SCS, without DWT, neither; 512 trials x "
                 "2e4 sweeps each"),
    "fields2d": (lambda: instances.frustrated_loop_planted((100, 100), 0.6, 11), 1024, 2_000,
                 dict(alpha0_deg=25.0, dwt_ratio=1.0, dwt_period=3, flags=4),
                 "local fields (eq. (1)): frustrated-loop planted 100x100 torus (loop density 0.6) "
                 "with unit fields h = tau (along the planted state) on a random 10% of the "
                 "vertices, drawn twist direction, 1024 replicas, 2e3 sweeps; success = planted "
                 "ground energy"),
    "readout": (lambda: instances.torus2d(100, 200, 0), 1024, 100_000,
                dict(alpha0_deg=14.0, dwt_ratio=0.5, dwt_period=3),
                "readouts on the default torus workload: 100 bisectors at the last sweep "
                "against the optimal bisector plus mid-anneal tracking every 1000 sweeps, on the "
                "same trajectories (same seeds)"),
    "torus16": (lambda: instances.torus2d(16, 16, 0), 64, 1000,
                dict(alpha0_deg=14.0, dwt_ratio=0.5, dwt_period=3),
                "2D +-1 torus 16x16 (N=256), 64 replicas, 1000 sweeps"),
}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def g70_like(seed: int):
    """Stand-in for Gset G70 (Table III: 10,000 vertices, 9,999 edges,
    unweighted, bounded degree): a uniform G(n, m) with unit Max-Cut weights."""
    g = instances.sparse_gnm(10000, 9999, seed, wmax=1)
    g.w = np.ones_like(g.w)
    g.meta["family"] = "g70_like"
    return g


def rank_seed(base: int, rank: int) -> int:
    """Seed of one rank's replicas. The seed keys Philox, so ranks with
    different seeds run disjoint, independent trials (replicas shard across
    ranks with no exchange on the data path)."""
    return int(base) + (int(rank) << 32)


def max_over_ranks(x: float, device: str = "cpu") -> float:
    """The largest x over all ranks (the slowest rank's time); x itself on
    one process."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def global_best(cut: int, spins, device: str = "cpu"):
    """The one exchange of a sharded run, after the timed region: the best
    cut over all ranks (ties -> the lowest rank), its owner, and the owner's
    spins broadcast to every rank. Returns (cut, owner, spins)."""
    import torch
    import torch.distributed as dist
    s = torch.as_tensor(np.asarray(spins, dtype=np.int8)).to(device)
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return int(cut), 0, s.cpu().numpy()
    rank = dist.get_rank()
    # one int64 max-reduce of (cut, -rank) packed as cut * 2^20 + (2^20 - 1 - rank)
    key = torch.tensor([int(cut) * (1 << 20) + ((1 << 20) - 1 - rank)], dtype=torch.int64, device=device)
    dist.all_reduce(key, op=dist.ReduceOp.MAX)
    k = int(key.item())
    best, owner = k >> 20, (1 << 20) - 1 - (k & ((1 << 20) - 1))
    dist.broadcast(s, src=owner)
    return best, owner, s.cpu().numpy()


def spins_cut(inst, spins) -> int:
    """Cut of a spin vector (sum of w over edges whose ends differ), a host
    check of the exchanged spins."""
    sp = np.asarray(spins)
    return int(np.asarray(inst.w, dtype=np.int64)[sp[inst.src] != sp[inst.dst]].sum())


def whole_job_rate(units_per_rank: float, world: int, t_max: float) -> float:
    """Whole-job throughput: every rank processed units_per_rank units; the
    job took the slowest rank's time."""
    return units_per_rank * world / t_max


def _colour(inst, name):
    import paper_2605_30355_gb300 as cosm
    if inst.dims:
        return None, 0  # the library applies the regular lattice pattern
    col, C = cosm.color_misra_gries(inst.n, inst.src, inst.dst)
    return col, C


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def _r99(ps):
    if ps >= 1.0:
        return 1.0
    if ps <= 0.0:
        return math.inf
    return math.log(0.01) / math.log(1.0 - ps)


def _targets():
    path = os.path.join(ROOT, "tests", "golden", "targets.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f)
    return {}


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f)
    return {}


# ---------------------------------------------------------------------- ours

def wilson(k, n, z=1.96):
    """95 % Wilson score interval of a success probability from k of n."""
    if n <= 0:
        return [0.0, 1.0]
    p = k / n
    d = 1.0 + z * z / n
    c = (p + z * z / (2 * n)) / d
    h = z * math.sqrt(p * (1 - p) / n + z * z / (4 * n * n)) / d
    return [max(0.0, c - h), min(1.0, c + h)]


def success_stats(cuts, target, t_step, R):
    """P_s with its 95 % Wilson interval, R99 and TTT = t_trial R99
    (Appendix A) at the target cut and two slightly lower ones, with t_trial
    the step time over the replicas."""
    allc = np.concatenate(cuts) if isinstance(cuts, list) else np.asarray(cuts)
    out = {"trials": int(allc.size), "best_cut": int(allc.max()), "mean_cut": float(allc.mean()),
           "t_trial_s": t_step / R, "levels": []}
    for tgt in (target, target - 2, target - 4):
        k = int((allc >= tgt).sum())
        ps = k / allc.size
        r = _r99(ps)
        out["levels"].append({"cut": int(tgt), "hits": k, "P_s": ps, "P_s_ci95": wilson(k, allc.size),
                              "R99": r if math.isfinite(r) else None,
                              "TTT_s": t_step / R * r if math.isfinite(r) else None})
    return out


def measure_single(cosm, inst, col, C, prm, storage, R, S, steps, warmup, seed, local, stream, flush,
                   h=None, keep=False):
    """Times `steps` full trials of R replicas (one cosm_run each) with CUDA
    events on the launching stream, L2 flushed between steps."""
    import torch
    solver = cosm.Solver.from_instance(inst, color=col, n_colors=C, storage=storage, h=h, **prm)
    for _ in range(warmup):
        solver.run(S, R, seed, stream)
        solver.sync()
    sampler = ClockSampler(local)
    times, cuts, energies = [], [], []
    torch.cuda.synchronize()
    sampler.start()
    for k in range(steps):
        flush.zero_()  # L2 flush between timed steps (not timed)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        solver.run(S, R, seed + 1000 * (k + 1), stream)
        e1.record(stream)
        e1.synchronize()
        solver.sync()
        times.append(e0.elapsed_time(e1) / 1000.0)
        cuts.append(solver.replica_cuts()[0])
        energies.append(solver.replica_energies())
    torch.cuda.synchronize()
    clocks = sampler.stop()
    layout = solver.layout()
    out = {"t_step": sum(times) / len(times), "cuts": cuts, "energies": energies, "clocks": clocks,
           "layout": layout}
    if keep:
        out["solver"] = solver
    else:
        solver.close()
    return out


def circ_rad(a, b):
    d = np.mod(np.asarray(a, dtype=np.float64) - np.asarray(b, dtype=np.float64), 1.0)
    return 2 * math.pi * np.minimum(d, 1.0 - d)


def cut_distribution(cuts):
    c = np.concatenate(cuts) if isinstance(cuts, list) else np.asarray(cuts)
    q = np.percentile(c, [1, 10, 50, 90, 99])
    return {"trials": int(c.size), "mean": float(c.mean()), "std": float(c.std()),
            "sem": float(c.std() / math.sqrt(c.size)), "min": int(c.min()), "max": int(c.max()),
            "p1_p10_p50_p90_p99": [float(v) for v in q]}


def measure_precision(cosm, inst, col, C, prm, R, S, steps, seed, local, stream, flush, f32_cuts):
    """Binary16 storage against binary32 on a bounded-degree graph: the
    final-cut distributions of both over the same trials (seeds), and the
    per-sweep phase difference of one sweep from an identical state (the
    FP16 trial's own state before sweeps 1, 10, 100 and 1000), binary16
    storage against binary32 phases. (The FP64 oracle's side of the same
    comparison is a GPU test.)"""
    f = measure_single(cosm, inst, col, C, prm, cosm.F16, R, S, steps, 1, seed, local, stream, flush)
    d32, d16 = cut_distribution(f32_cuts), cut_distribution(f["cuts"])
    diff = d16["mean"] - d32["mean"]
    se = math.sqrt(d16["sem"] ** 2 + d32["sem"] ** 2)
    per_sweep = {}
    Rs = 16
    h16 = cosm.Solver.from_instance(inst, color=col, n_colors=C, storage=cosm.F16, **prm)
    h32 = cosm.Solver.from_instance(inst, color=col, n_colors=C, storage=cosm.F32, **prm)
    init = cosm.Solver.from_instance(inst, color=col, n_colors=C, storage=cosm.F16,
                                     **dict(prm, alpha0_deg=0.0))
    init.run_range(S, 1, 1, Rs, seed)  # alpha 0, no twist at sweep 1: the initial phases
    a0 = prm["alpha0_deg"] / 360.0
    for sw in (1, 10, 100, 1000):
        if sw == 1:
            x0 = init.get_state()
        else:
            h16.run_range(S, 1, sw - 1, Rs, seed)
            x0 = h16.get_state()
        alpha = float(np.float32(a0 * (S - sw) / (S - 1)))
        h16.set_state(x0, seed=seed)
        h16.step(sw, alpha)
        h32.set_state(x0, seed=seed)
        h32.step(sw, alpha)
        e = circ_rad(h16.get_state(), h32.get_state())
        per_sweep[str(sw)] = {"max_rad": float(e.max()), "p99_rad": float(np.percentile(e, 99)),
                              "median_rad": float(np.median(e)),
                              "frac_above_2e-3_rad": float((e > 2e-3).mean())}
    for h_ in (h16, h32, init):
        h_.close()
    return {"f32": d32, "f16": d16, "mean_difference_f16_minus_f32": diff,
            "mean_difference_ci95": [diff - 1.96 * se, diff + 1.96 * se],
            "f16_updates_per_s": inst.m * S * R / f["t_step"],
            "per_sweep_f16_vs_f32": per_sweep,
            "per_sweep_note": f"one sweep of {Rs} replicas from the binary16 trial's own state before "
                              "that sweep, binary16 storage against binary32 phases, circular "
                              "difference in rad over all phases"}


def measure_long_ttt(cosm, args, inst, col, C, prm, R, seed, local, stream, flush, storage=None):
    """Time-to-target at the oracle's best cut with a longer anneal (Appendix
    A: TTT = t_trial R99; Table X runs 1-2 x 10^6 sweeps per trial on the
    20,000-spin torus): R replicas x args.ttt_sweeps sweeps per step, FP32
    phases unless another storage is given."""
    tgt = _targets().get(args.workload)
    if tgt is None:
        return None
    S = args.ttt_sweeps
    m = measure_single(cosm, inst, col, C, prm, cosm.F32 if storage is None else storage, R, S, args.ttt_steps,
                       0, seed + 555, local, stream, flush)
    st_ = success_stats(m["cuts"], tgt["cut"], m["t_step"], R)
    top = st_["levels"][0]
    return {"sweeps_per_trial": S, "replicas_per_step": R, "steps": args.ttt_steps,
            "target_cut": tgt["cut"], "target_source": tgt["source"], "trials": st_["trials"],
            "hits": top["hits"], "P_s": top["P_s"], "P_s_ci95": top["P_s_ci95"], "R99": top["R99"],
            "t_trial_s": st_["t_trial_s"], "TTT_s": top["TTT_s"],
            "TTT_s_ci95": [m["t_step"] / R * _r99(p) if 0.0 < p < 1.0 else None
                           for p in reversed(top["P_s_ci95"])],
            "best_cut": st_["best_cut"], "mean_cut": st_["mean_cut"], "levels": st_["levels"],
            "updates_per_s": inst.m * S * R / m["t_step"], "clocks": m["clocks"]}


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_2605_30355_gb300 as cosm

    ws, rank, local = _dist()
    if ws > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    builder, R, S, prm, desc = WORKLOADS[args.workload]
    if args.replicas:
        R = args.replicas
    if args.sweeps:
        S = args.sweeps
    storage = {"f32": cosm.F32, "f16": cosm.F16, "q16": cosm.Q16, "bf16": cosm.BF16}[args.storage]
    inst = builder()
    col, C = _colour(inst, args.workload)
    seed = rank_seed(1, rank)  # every rank runs its own independent replicas
    stream = torch.cuda.Stream()
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    if ws > 1:
        dist.barrier()
    m = measure_single(cosm, inst, col, C, prm, storage, R, S, args.steps, args.warmup, seed, local,
                       stream, flush)
    if ws > 1:
        dist.barrier()
    t_step, layout, clocks = m["t_step"], m["layout"], m["clocks"]
    t_max = max_over_ranks(t_step, "cuda")
    updates = inst.m * S * R  # edge-replica updates per step per rank
    value = whole_job_rate(updates, ws, t_max)

    # ---- end to end through the one-shot host-buffer call (cosm_solve)
    e2e_times = []
    h2d = inst.src.nbytes + inst.dst.nbytes + inst.w.nbytes + (col.nbytes if col is not None else 0)
    d2h = inst.n + 16 + 8 * R
    for k in range(args.e2e_steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        cosm.solve(inst.n, inst.src, inst.dst, inst.w, S, R, seed + 77 * (k + 1), color=col,
                   n_colors=C, dims=inst.dims, storage=storage, replica_cuts=True, **prm)
        e2e_times.append(time.perf_counter() - t0)
    e2e_t = sum(e2e_times) / len(e2e_times) if e2e_times else None
    if e2e_t is not None:
        e2e_t = max_over_ranks(e2e_t, "cuda")

    # ---- the other phase-storage forms and the ragged batch ("batched")
    forms = {}
    default_shape = args.workload == "torus20k" and not args.replicas and not args.sweeps
    if args.forms and default_shape:
        # at least 10 steps (10,240 trials) per form for its success rate
        for name, st in (("f16", cosm.F16), ("q16", cosm.Q16), ("bf16", cosm.BF16)):
            if st == storage:
                continue
            f = measure_single(cosm, inst, col, C, prm, st, R, S, max(10, args.steps // 2), 1, seed,
                               local, stream, flush)
            forms[name] = {"value": whole_job_rate(updates, ws, max_over_ranks(f["t_step"], "cuda")),
                           "unit": "updates/s", "ms_per_step": f["t_step"] * 1000.0,
                           "replicas_per_cta": f["layout"]["K"],
                           "roofline": roofline(cosm, inst, prm, st, f["layout"], updates, f["t_step"],
                                                f["clocks"], args.workload, R, S),
                           "clocks": f["clocks"]}
            tgt = _targets().get(args.workload)
            if tgt is not None:
                forms[name]["success"] = success_stats(f["cuts"], tgt["cut"], f["t_step"], R)
            forms[name]["speedup_vs_f32_plain"] = t_step / f["t_step"]
    batched = None
    if args.forms and default_shape:
        # the ragged batch in each 2-byte form beside binary32
        batched = {}
        for name, st in (("f32", cosm.F32), ("f16", cosm.F16), ("q16", cosm.Q16)):
            batched[name] = measure_batch(cosm, args, rank, ws, local, stream, flush, steps=2, warmup=1,
                                          e2e=True, storage=st)
        f32v = batched["f32"]["value"]
        for name in ("f16", "q16"):
            batched[name]["speedup_vs_f32_batch"] = batched[name]["value"] / f32v
    precision = None
    if args.forms and args.workload in ("reg3_20k", "reg4_20k") and not args.replicas and not args.sweeps:
        precision = measure_precision(cosm, inst, col, C, prm, R, S, args.steps, seed, local, stream, flush,
                                      m["cuts"])
    long_ttt = None
    if args.ttt_steps and default_shape:
        long_ttt = measure_long_ttt(cosm, args, inst, col, C, prm, R, seed, local, stream, flush)
        if long_ttt is not None and args.forms:
            # the 2-byte forms on the same long anneal (same seeds)
            long_ttt["forms"] = {}
            for name, st in (("f16", cosm.F16), ("q16", cosm.Q16)):
                f = measure_long_ttt(cosm, args, inst, col, C, prm, R, seed, local, stream, flush, storage=st)
                f.pop("levels", None)
                f["TTT_speedup_vs_f32"] = (long_ttt["TTT_s"] / f["TTT_s"]
                                           if f["TTT_s"] and long_ttt["TTT_s"] else None)
                long_ttt["forms"][name] = f

    # ---- the best state over all ranks (untimed): one max-reduce, one broadcast
    solver = cosm.Solver.from_instance(inst, color=col, n_colors=C, storage=storage, **prm)
    solver.run(min(S, 1000), min(R, 256), seed + 7, stream)
    b_cut, _, _, b_spins = solver.best()
    solver.close()
    g_cut, g_owner, g_spins = global_best(b_cut, b_spins, "cuda" if ws > 1 else "cpu")

    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return None

    # ---- time to target (P_s over this run's replicas)
    tgt = _targets().get(args.workload)
    ttt = None
    if tgt is not None:
        st_ = success_stats(m["cuts"], tgt["cut"], t_step, R)
        top = st_["levels"][0]
        ttt = {"target_cut": tgt["cut"], "target_source": tgt["source"], "P_s": top["P_s"],
               "P_s_ci95": top["P_s_ci95"], "trials": st_["trials"], "R99": top["R99"],
               "t_trial_s": st_["t_trial_s"],
               "TTT_s": top["TTT_s"], "best_cut": st_["best_cut"], "mean_cut": st_["mean_cut"],
               "levels": st_["levels"]}

    # ---- roofline of the sweep kernel: shared memory and FP32 issue
    roof = roofline(cosm, inst, prm, storage, layout, updates, t_step, clocks, args.workload, R, S)

    line = {
        "metric": metric_name(args.workload),
        "value": value, "unit": "updates/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max * 1000.0, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {cosm.F32: "f32", cosm.F16: "f16-storage/f32-compute", cosm.Q16: "u16-fixed-point",
                  cosm.BF16: "bf16-storage/f32-compute"}[storage],
        "data": "synthetic (seeded instance generator; no Gset files)",
        "config": {"workload": args.workload, "description": desc, "n": inst.n, "edges": inst.m,
                   "replicas_per_gpu": R, "sweeps_per_trial": S, "colors": layout["colors"],
                   "replicas_per_cta": layout["K"], "threads_per_cta": layout["threads"],
                   "ctas": layout["grid"], "l2": "flushed between timed steps (256 MB write)",
                   "parallelism": f"replicas sharded over {ws} GPU(s), no collective on the data path"},
        "global_best": {"cut": g_cut, "owner_rank": g_owner, "spins_cut": spins_cut(inst, g_spins),
                        "run": "after the timed region: min(S, 1000) sweeps x min(R, 256) replicas per "
                               "rank, an int64 max-reduce of (cut, rank), a broadcast of the owner's spins"},
        "e2e": None if e2e_t is None else {
            "value": whole_job_rate(updates, ws, e2e_t), "unit": "updates/s", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "api": "cosm_solve (host buffers)"},
        "gpu_launches": 2 * args.steps,
        "clocks": clocks,
        "roofline": roof,
        "time_to_target": ttt,
        "time_to_target_long": long_ttt,
        "precision": precision,
        "forms": forms or None,
        "batched": batched,
        "paper_context": {"updates_per_s": 1.41e10, "hardware": "2x Xeon Gold 6544Y, 64 threads, FP32",
                          "source": "derived from Section III-A and Table II (G72/G77/G81)"},
    }
    if args.cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args, inst, col, C, prm)
    print(json.dumps(line))
    if ws > 1:
        dist.destroy_process_group()
    return line


# ncu records of the sweep kernel's memory traffic on the bench's workloads,
# each taken at the kernel source whose hash it names (the first 12 hex
# digits of the SHA-256 of cosm_kernels.cu): reported only while that source
# is unchanged, else null. Keys: (workload, storage). Values: shared-memory
# bytes per edge-replica update (shared wavefronts x 128 B / updates, from a
# small capture of the same kernel and layout), and DRAM bytes (read +
# write) of one full-size launch with its (replicas, sweeps) -- DRAM traffic
# follows the state, not the sweeps, so it is not scaled from a small case.
NCU_TRAFFIC = {
    ("torus20k", "f32"): (8.60, (83.37e6, 1024, 100_000), "1bcbe8654a3b"),
    ("torus20k", "f16"): (4.43, None, "1bcbe8654a3b"),
    ("torus20k", "q16"): (4.39, None, "1bcbe8654a3b"),
    ("reg3_20k", "f32"): (22.5, None, "1bcbe8654a3b"),
}

# Algorithmic cost of one edge-replica update of eq. (6): FP32 operations
# (the difference, the biased sign, two phase updates, two wraps) and, per
# phase byte b, the shared-memory bytes 4b of two reads and two writes.
ALU_OPS_PER_UPDATE = 6


def kernel_source_hash():
    import hashlib
    path = os.path.join(ROOT, "paper_2605_30355_gb300", "csrc", "cosm_kernels.cu")
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:12]


_PROBES = {}


def probes(cosm):
    """Measured shared-memory bandwidth (bytes per SM clock) and FP32 issue
    rates (operations per SM clock, scalar and packed f32x2), once per run."""
    if not _PROBES:
        bpc, _ = cosm.probe_smem(4096)
        sc, pk = cosm.probe_fp32(2048)
        _PROBES.update(smem_bpc=bpc, fp32_scalar=sc, fp32_packed=pk)
    return _PROBES


def algorithmic_bytes(inst, prm, storage_bytes, lattice, K):
    """Shared-memory bytes of one edge-replica update by the method's own
    count: 4b (two phase reads and two writes) + 2b n / (m P_dwt) (the twist
    reads and writes every phase once per period) + e / K (one edge record
    of e bytes serves the K replicas of a tile; the implicit-index lattice
    needs one weight bit per edge)."""
    b = storage_bytes
    dwt = (2.0 * b * inst.n) / (inst.m * prm["dwt_period"]) if prm.get("dwt_period", 0) > 0 else 0.0
    e = 0.125 if lattice == 2 else 5.0
    return 4.0 * b + dwt + e / max(1, K)


def roofline(cosm, inst, prm, storage, layout, updates, t_step, clocks, workload=None, replicas=0, sweeps=0):
    """Rooflines of the sweep kernel, which is the whole timed step but for a
    finaliser of microseconds, so the step time is its launch duration:
    - smem (the bound of the method's own count): algorithmic shared-memory
      bytes per update against the measured shared-memory bandwidth;
    - alu: 6 FP32 operations per update against the measured FP32 issue rate
      (the larger of scalar and packed f32x2 fused multiply-adds);
    - smem_measured: the kernel's own shared-memory traffic from ncu, where a
      record for the current kernel source exists (the lattice kernel applies
      two colours per load and store of a phase, so it moves fewer bytes than
      the method's count)."""
    import torch
    pr = probes(cosm)
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    sms = props.multi_processor_count
    mhz = clocks.get("sm_mhz") or 2070.0
    b = 4 if storage == cosm.F32 else 2
    K = layout["K"]
    per_update = algorithmic_bytes(inst, prm, b, layout["lattice"], K)
    smem_peak = pr["smem_bpc"] * sms * mhz * 1e6 / 1e9
    rate = updates / t_step
    smem = {"bound": "smem", "achieved": per_update * rate / 1e9, "peak": smem_peak, "unit": "GB/s",
            "frac": per_update * rate / 1e9 / smem_peak, "bytes_per_update": per_update,
            "peak_source": f"measured shared-memory read bandwidth ({pr['smem_bpc']:.1f} B/clk/SM) x {sms} "
                           f"SMs x {mhz:.0f} MHz (median sampled SM clock), of measured"}
    ops_clk = max(pr["fp32_scalar"], pr["fp32_packed"])
    alu_peak = ops_clk * sms * mhz * 1e6 / 1e12
    smem["alu"] = {"bound": "alu", "achieved": ALU_OPS_PER_UPDATE * rate / 1e12, "peak": alu_peak,
                   "unit": "Tops/s", "frac": ALU_OPS_PER_UPDATE * rate / 1e12 / alu_peak,
                   "ops_per_update": ALU_OPS_PER_UPDATE,
                   "peak_source": f"measured FP32 issue rate: {pr['fp32_scalar']:.1f} ops/clk/SM scalar fma, "
                                  f"{pr['fp32_packed']:.1f} packed f32x2 fma; x {sms} SMs x {mhz:.0f} MHz, "
                                  "of measured"}
    key = (workload, {cosm.F32: "f32", cosm.F16: "f16", cosm.Q16: "q16", cosm.BF16: "bf16"}[storage])
    rec = NCU_TRAFFIC.get(key)
    src = kernel_source_hash()
    smem["traffic"] = None
    smem["smem_measured"] = None
    if rec is not None and rec[2] == src:
        smem["smem_measured"] = {"bytes_per_update": rec[0], "achieved": rec[0] * rate / 1e9,
                                 "frac": rec[0] * rate / 1e9 / smem_peak,
                                 "source": "ncu shared wavefronts x 128 B per update, kernel source " + rec[2]}
        if rec[1] is not None and rec[1][1:] == (replicas, sweeps):
            smem["traffic"] = rec[1][0]
            smem["traffic_source"] = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one full-size "
                                      "launch; kernel source " + rec[2])
    return smem


# ---------------------------------------------------------------------- batch

def measure_batch(cosm, args, rank, ws, local, stream, flush, steps, warmup, e2e=True, storage=None):
    """The ragged batch: every step is one cosm_batch_run over all instances."""
    import torch
    _, _, S, prm, desc = WORKLOADS["batch512"]
    if args.workload == "batch512" and args.sweeps:
        S = args.sweeps
    if storage is None:
        storage = {"f32": cosm.F32, "f16": cosm.F16, "q16": cosm.Q16, "bf16": cosm.BF16}[args.storage]
    insts, reps = instances.ragged_batch(512, seed=0)
    seeds = np.arange(len(insts), dtype=np.uint64) + np.uint64(rank_seed(1, rank))
    t0 = time.perf_counter()
    batch = cosm.Batch(insts, storage=storage, **prm)
    create_s = time.perf_counter() - t0
    if not args.no_tune:
        batch.tune(reps, probe_sweeps=200, stream=stream)
    for _ in range(warmup):
        batch.run(S, reps, seeds, stream)
        batch.sync()
    sampler = ClockSampler(local)
    times = []
    torch.cuda.synchronize()
    sampler.start()
    for k in range(steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        batch.run(S, reps, seeds + np.uint64(7919 * (k + 1)), stream)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1000.0)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    t_step = sum(times) / len(times)
    t_max = max_over_ranks(t_step, "cuda")
    updates = sum(int(i.m) * S * r for i, r in zip(insts, reps))
    info = batch.info()
    lays = [batch.layout(i) for i in range(len(insts))]
    batch.close()
    e2e_t = None
    h2d = sum(i.src.nbytes + i.dst.nbytes + i.w.nbytes for i in insts)
    d2h = sum(i.n + 24 for i in insts)
    if e2e:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b2 = cosm.Batch(insts, storage=storage, **prm)
        b2.run(S, reps, seeds + np.uint64(1), stream)
        for i in range(len(insts)):
            b2.best(i)
        b2.close()
        e2e_t = max_over_ranks(time.perf_counter() - t0, "cuda")
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    mhz = clocks.get("sm_mhz") or 2070.0
    pr = probes(cosm)
    sms = props.multi_processor_count
    b = 4 if storage == cosm.F32 else 2
    algo = sum(int(i.m) * S * r * algorithmic_bytes(i, prm, b, lay["lattice"], lay["K"])
               for i, r, lay in zip(insts, reps, lays)) / updates
    smem_peak = pr["smem_bpc"] * sms * mhz * 1e6 / 1e9
    ops_clk = max(pr["fp32_scalar"], pr["fp32_packed"])
    alu_peak = ops_clk * sms * mhz * 1e6 / 1e12
    rate = updates / t_step
    sname = {cosm.F32: "f32", cosm.F16: "f16", cosm.Q16: "q16", cosm.BF16: "bf16"}[storage]
    return {
        "value": whole_job_rate(updates, ws, t_max), "unit": "updates/s", "ms_per_step": t_max * 1000.0,
        "storage": sname,
        "description": desc, "instances": len(insts), "replicas_total": int(sum(reps)),
        "sweeps_per_trial": S, "edges_total": int(sum(i.m for i in insts)), "batch": info,
        "create_s": create_s, "steps": steps, "warmup": warmup, "clocks": clocks,
        "e2e": None if e2e_t is None else {
            "value": whole_job_rate(updates, ws, e2e_t), "unit": "updates/s", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "api": "cosm_batch_create + cosm_batch_run + get_best (host buffers)"},
        "roofline": {"bound": "smem", "achieved": algo * rate / 1e9, "peak": smem_peak, "unit": "GB/s",
                     "frac": algo * rate / 1e9 / smem_peak, "traffic": None, "bytes_per_update": algo,
                     "peak_source": f"measured shared-memory bandwidth ({pr['smem_bpc']:.1f} B/clk/SM) x "
                                    f"{sms} SMs x {mhz:.0f} MHz, of measured; bytes per update by the "
                                    "method's count with each instance's tile width",
                     "alu": {"bound": "alu", "achieved": ALU_OPS_PER_UPDATE * rate / 1e12, "peak": alu_peak,
                             "unit": "Tops/s", "frac": ALU_OPS_PER_UPDATE * rate / 1e12 / alu_peak,
                             "ops_per_update": ALU_OPS_PER_UPDATE}},
    }


def run_batch(args):
    import torch
    import torch.distributed as dist

    import paper_2605_30355_gb300 as cosm

    ws, rank, local = _dist()
    if ws > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    b = measure_batch(cosm, args, rank, ws, local, stream, flush, args.steps, args.warmup,
                      e2e=bool(args.e2e_steps))
    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return None
    line = {
        "metric": "edge-replica updates/s (ragged batch, one graph-captured run)",
        "value": b["value"], "unit": "updates/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": b["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"f32": "f32", "f16": "f16-storage/f32-compute", "q16": "u16-fixed-point",
                  "bf16": "bf16-storage/f32-compute"}[b["storage"]],
        "data": "synthetic (seeded instance generator; no Gset files)",
        "config": {"workload": "batch512", "description": b["description"], "instances": b["instances"],
                   "replicas_total": b["replicas_total"], "sweeps_per_trial": b["sweeps_per_trial"],
                   "edges_total": b["edges_total"], "batch": b["batch"], "create_s": b["create_s"],
                   "l2": "flushed between timed steps (256 MB write)",
                   "parallelism": f"all instances on each of {ws} GPU(s), no collective"},
        "e2e": b["e2e"], "gpu_launches": int(b["batch"]["launches"]) * args.steps,
        "clocks": b["clocks"], "roofline": b["roofline"],
    }
    print(json.dumps(line))
    if ws > 1:
        dist.destroy_process_group()
    return line


# ---------------------------------------------------------------------- ablation

def _base_line(metric, value, unit, args, t_step, desc, inst, R, S, **extra):
    line = {"metric": metric, "value": value, "unit": unit, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_step * 1000.0, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded instance generator)",
            "config": {"workload": args.workload, "description": desc, "n": inst.n, "edges": inst.m,
                       "replicas_per_gpu": R, "sweeps_per_trial": S,
                       "l2": "flushed between timed steps (256 MB write)"}}
    line.update(extra)
    return line


def run_fields(args):
    """Local fields (eq. (1)) on a planted lattice: throughput and the rate
    of reaching the planted ground energy."""
    import torch

    import paper_2605_30355_gb300 as cosm

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if rank != 0:
        return None
    builder, R, S, prm, desc = WORKLOADS[args.workload]
    R = args.replicas or R
    S = args.sweeps or S
    inst = builder()
    h = instances.aligned_fields(inst, 1, 0.1)
    ground = inst.meta["ground_energy"] - int(np.abs(h).sum())
    stream = torch.cuda.Stream()
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    col, C = _colour(inst, args.workload)
    m = measure_single(cosm, inst, col, C, prm, cosm.F32, R, S, args.steps, args.warmup, 1, local,
                       stream, flush, h=h)
    en = np.concatenate(m["energies"])
    ps = float((en <= ground).mean())
    r = _r99(ps)
    updates = (inst.m + inst.n) * S * R  # edge and field updates
    line = _base_line("edge+field replica updates/s (planted 2D lattice with local fields)",
                      updates / m["t_step"], "updates/s", args, m["t_step"], desc, inst, R, S,
                      gpu_launches=2 * args.steps, clocks=m["clocks"],
                      layout=m["layout"],
                      success={"ground_energy": int(ground), "trials": int(en.size),
                               "best_energy": int(en.min()), "mean_energy": float(en.mean()),
                               "P_s": ps, "R99": r if math.isfinite(r) else None,
                               "t_trial_s": m["t_step"] / R,
                               "TTT_s": m["t_step"] / R * r if math.isfinite(r) else None})
    print(json.dumps(line))
    return line


def run_readout(args):
    """Readout quality and cost on the same trajectories: the final readout
    with 100 equally spaced bisectors, against the optimal bisector plus
    mid-anneal tracking every 1000 sweeps (tracking does not change the
    dynamics, so replica r follows the same path in both runs)."""
    import torch

    import paper_2605_30355_gb300 as cosm

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if rank != 0:
        return None
    builder, R, S, prm, desc = WORKLOADS[args.workload]
    R = args.replicas or R
    S = args.sweeps or S
    inst = builder()
    stream = torch.cuda.Stream()
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    T = min(1000, S)
    plain = measure_single(cosm, inst, None, 0, prm, cosm.F32, R, S, args.steps, args.warmup, 1, local,
                           stream, flush)
    rich = measure_single(cosm, inst, None, 0, dict(prm, flags=cosm.OPT_BISECTOR, track_period=T),
                          cosm.F32, R, S, args.steps, args.warmup, 1, local, stream, flush, keep=True)
    # the optimal-bisector readout alone: readouts of the final state
    s = rich.pop("solver")
    times = []
    for k in range(3):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.readout(stream)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1000.0)
    s.close()
    p0 = cosm.Solver.from_instance(inst, **prm)
    p0.run(10, R, 1)
    t_p = []
    for k in range(3):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        p0.readout(stream)
        e1.record(stream)
        e1.synchronize()
        t_p.append(e0.elapsed_time(e1) / 1000.0)
    p0.close()
    a = np.concatenate(plain["cuts"])
    b = np.concatenate(rich["cuts"])
    updates = inst.m * S * R
    # a short anneal, where the phases have not settled into two antipodal
    # groups when the schedule ends
    S2 = 1000
    short = {}
    for name, extra in (("bisectors_100", {}), ("optimal", dict(flags=cosm.OPT_BISECTOR)),
                        ("optimal_and_tracking", dict(flags=cosm.OPT_BISECTOR, track_period=100))):
        sv = cosm.Solver.from_instance(inst, **dict(prm, **extra))
        sv.run(S2, R, 7)
        c = sv.replica_cuts()[0]
        sv.close()
        short[name] = {"mean_cut": float(c.mean()), "best_cut": int(c.max())}
    tgt = _targets().get("torus20k") if inst.n == 20000 else None
    line = _base_line("edge-replica updates/s with the optimal bisector and tracking every 1000 sweeps",
                      updates / rich["t_step"], "updates/s", args, rich["t_step"], desc, inst, R, S,
                      gpu_launches=3 * args.steps, clocks=rich["clocks"],
                      readout={"bisectors_100": {"updates_per_s": updates / plain["t_step"],
                                                 "mean_cut": float(a.mean()), "best_cut": int(a.max())},
                               "optimal_and_tracking": {"updates_per_s": updates / rich["t_step"],
                                                        "mean_cut": float(b.mean()), "best_cut": int(b.max())},
                               "replicas_improved": float((b > a).mean()),
                               "replicas_worse": float((b < a).mean()),
                               "readout_ms": {"bisectors_100": 1000 * min(t_p),
                                              "optimal": 1000 * min(times)},
                               "track_period": T,
                               "short_anneal": dict(short, sweeps=S2, track_period=100)})
    if tgt is not None:
        line["readout"]["success"] = {
            "bisectors_100": success_stats(plain["cuts"], tgt["cut"], plain["t_step"], R)["levels"],
            "optimal_and_tracking": success_stats(rich["cuts"], tgt["cut"], rich["t_step"], R)["levels"]}
    print(json.dumps(line))
    return line


def run_ablation(args):
    """Table VII's four variants on the same graph, replicas and seeds."""
    import torch

    import paper_2605_30355_gb300 as cosm

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if rank != 0:
        return None
    builder, R, S, prm, desc = WORKLOADS[args.workload]
    if args.sweeps:
        S = args.sweeps
    inst = builder()
    rows = {}
    t0 = time.perf_counter()
    for name, flags in (("cosm", 0), ("without_scs", cosm.NO_SCS), ("without_dwt", cosm.NO_DWT),
                        ("neither", cosm.NO_SCS | cosm.NO_DWT)):
        s = cosm.Solver.from_instance(inst, flags=flags, **prm)
        s.run(S, R, 1)
        cuts, _ = s.replica_cuts()
        rows[name] = {"highest_cut": int(cuts.max()), "average_cut": float(cuts.mean()),
                      "P_highest_of_all": None}
        rows[name]["_cuts"] = cuts
        s.close()
    top = max(r["highest_cut"] for r in rows.values())
    for r in rows.values():
        r["P_highest_of_all"] = float((r.pop("_cuts") >= top).mean())
    line = {"metric": "ablation: highest / average cut per variant (Table VII shape)",
            "value": rows["cosm"]["average_cut"], "unit": "cut", "n_gpus": 1, "steps": 1, "warmup": 0,
            "ms_per_step": (time.perf_counter() - t0) * 1000.0, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic G70-like graph (seeded)",
            "config": {"workload": "ablation", "description": desc, "n": inst.n, "edges": inst.m,
                       "replicas": R, "sweeps_per_trial": S},
            "ablation": rows,
            "paper_context": {"G70_1.5M_sweeps": {"cosm": [9595, 9593.39], "without_scs": [9551, 9528.00],
                                                  "without_dwt": [9544, 9501.40], "neither": [9481, 9432.81]},
                              "source": "Table VII (highest, average cut)"}}
    print(json.dumps(line))
    return line


# ---------------------------------------------------------------------- serving

def serve_pool(count=10, seed=0):
    """Planted instances spread over N in [1000, 50000] (2D and 3D, even
    sides) and loop densities 0.2..1.0."""
    st = instances.Stream(seed, tag=9)
    us = (st.u64(count) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    pool = []
    for k in range(count):
        n = 1000 + us[k] * 49000
        rho = [0.2, 0.4, 0.6, 0.8, 1.0][k % 5]
        if k % 2 == 0:
            L = max(4, 2 * int(round(np.sqrt(n) / 2)))
            pool.append(instances.frustrated_loop_planted((L, L), rho, 1000 + k))
        else:
            L = max(4, 2 * int(round(n ** (1 / 3) / 2)))
            pool.append(instances.frustrated_loop_planted((L, L, L), rho, 1000 + k))
    return pool


def run_serve(args):
    import torch

    import paper_2605_30355_gb300 as cosm

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if rank != 0:
        return None
    _, R, S, prm, desc = WORKLOADS[args.workload]
    # the serving workload stores phases in binary16 unless --storage names another form
    sname = args.storage if args.storage_given else "f16"
    storage = {"f32": cosm.F32, "f16": cosm.F16, "q16": cosm.Q16, "bf16": cosm.BF16}[sname]
    desc = desc.replace("FP16 phase storage", {"f32": "FP32 phases", "f16": "FP16 phase storage",
                                              "q16": "u16 fixed-point phases",
                                              "bf16": "bfloat16 phase storage"}[sname])
    pool = serve_pool()
    rate, window, max_trials = 50.0, args.serve_seconds, args.serve_trials
    R = args.replicas or R
    S = args.sweeps or S
    def req_sweeps(inst):
        # with --serve-scale, anneals lengthen with the instance: S sweeps per
        # 10,000 spins, at least S
        return max(S, int(round(S * inst.n / 10000))) if args.serve_scale else S

    desc = desc.replace("32 replicas x 2000 sweeps per trial, up to 4 trials",
                        f"{R} replicas x {S} sweeps per trial" +
                        (" per 10,000 spins (at least 2000)" if args.serve_scale else "") +
                        f", up to {max_trials} trials")
    arr = instances.Stream(77, tag=10)
    gaps = -np.log(1.0 - (arr.u64(100000) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53) / rate
    t_arr = np.cumsum(gaps)
    t_arr = t_arr[t_arr < window]
    picks = arr.below(len(pool), len(t_arr))
    srv = cosm.Server(memory_budget=48 << 30, max_active=256, chunk_sweeps=500)
    # warm-up: one request per pool instance size class
    for inst in pool[:2]:
        srv.wait(srv.submit(inst, S, R, 1, inst.meta["opt_cut"], max_trials=1, storage=storage, **prm), 600)
    sampler = ClockSampler(local)
    sampler.start()
    ids = []
    t0 = time.perf_counter()
    for k, ta in enumerate(t_arr):
        delay = t0 + ta - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        inst = pool[int(picks[k])]
        ids.append(srv.submit(inst, req_sweeps(inst), R, 1000 + k, inst.meta["opt_cut"], max_trials=max_trials,
                              storage=storage, **prm))
    res = [srv.wait(r, 3600) for r in ids]
    t_total = time.perf_counter() - t0
    clocks = sampler.stop()
    st = srv.stats()
    srv.close()
    reached = [r for r in res if r["status"] == cosm.REACHED]
    by_inst = []
    for k, inst in enumerate(pool):
        mine = [r for r, pk in zip(res, picks) if int(pk) == k]
        by_inst.append({"n": int(inst.n), "dims": list(inst.dims), "loop_density": inst.meta.get("rho"),
                        "sweeps": req_sweeps(inst),
                        "requests": len(mine), "reached": sum(r["status"] == cosm.REACHED for r in mine),
                        "mean_trials": float(np.mean([r["trials"] for r in mine])) if mine else None})
    # percentiles over all requests: one that used up its trials without
    # reaching the planted optimum has no time-to-target (infinite)
    ttt_all = np.array([r["ttt"] if r["status"] == cosm.REACHED else np.inf for r in res])
    updates = sum(int(r["updates"]) for r in res)

    def pct(q):
        v = float(np.percentile(ttt_all, q, method="higher")) if len(ttt_all) else math.inf
        return v if math.isfinite(v) else None
    line = {
        "metric": "serving: requests/s and time-to-target p50/p99 (planted instances)",
        "value": len(res) / t_total, "unit": "requests/s", "n_gpus": 1, "steps": 1, "warmup": 1,
        "ms_per_step": t_total * 1000.0, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {cosm.F32: "f32", cosm.F16: "f16-storage/f32-compute", cosm.Q16: "u16-fixed-point",
                  cosm.BF16: "bf16-storage/f32-compute"}[storage],
        "data": "synthetic (seeded frustrated-loop planted instances)",
        "config": {"workload": "serve", "description": desc, "pool": [(i.n, i.m, len(i.dims)) for i in pool],
                   "requests": len(res), "arrival_rate": rate, "window_s": window,
                   "server": {"memory_budget": 48 << 30, "max_active": 256, "chunk_sweeps": 500}},
        "serving": {"requests": len(res), "reached": len(reached), "exhausted": len(res) - len(reached),
                    "reached_fraction": len(reached) / max(1, len(res)),
                    "ttt_p50_s": pct(50), "ttt_p99_s": pct(99),
                    "percentiles_over": "all requests; one that used up its trials without reaching the "
                                        "planted optimum counts as never reached (null: the percentile "
                                        "falls among those)",
                    "ttt_p50_s_reached_only": float(np.percentile(ttt_all[np.isfinite(ttt_all)], 50))
                    if len(reached) else None,
                    "updates_per_s": updates / t_total, "stats": st, "by_instance": by_inst},
        "clocks": clocks,
    }
    print(json.dumps(line))
    return line


# ---------------------------------------------------------------------- oracle

def _oracle_extras(args, inst, prm):
    """Local fields, flags and tracking of the workload, for the oracle."""
    h = instances.aligned_fields(inst, 1, 0.1) if args.workload == "fields2d" else None
    flags = int(prm.get("flags", 0))
    track = 0
    if args.workload == "readout":
        flags |= 8  # the optimal bisector
        track = 1000
    return h, flags, track


def _oracle_sample(args, inst, col, C, prm):
    import oracle
    oracle.build()
    if col is None:
        col, C = oracle.color_instance(inst)
    g = oracle.ColouredGraph(inst.n, inst.src, inst.dst, inst.w, col, C)
    h, flags, track = _oracle_extras(args, inst, prm)
    per_sweep = inst.m + (inst.n if h is not None else 0)
    cores = os.cpu_count() or 1
    reps = cores
    sweeps = max(10, int(args.cpu_updates / (per_sweep * reps)))
    t0 = time.perf_counter()
    if h is None and not flags and not track:
        cuts, _, _, used = oracle.trials(g, sweeps, reps, alpha0=prm["alpha0_deg"] / 360.0,
                                         dwt_period=prm["dwt_period"], dwt_ratio=prm["dwt_ratio"],
                                         seed=1, threads=cores)
    else:
        _, _, _, _ = oracle.trials_ex(g, sweeps, reps, alpha0=prm["alpha0_deg"] / 360.0,
                                      dwt_period=prm["dwt_period"], dwt_ratio=prm["dwt_ratio"], seed=1,
                                      threads=cores, h=h, flags=flags, track=min(track, sweeps))
        used = min(cores, reps)
    dt = time.perf_counter() - t0
    return per_sweep * sweeps * reps / dt, used, f"{reps} replicas x {sweeps} sweeps of the same instance", dt


def cpu_baseline(args, inst, col, C, prm):
    v, used, sample, _ = _oracle_sample(args, inst, col, C, prm)
    return {"value": v, "unit": "updates/s", "cores": used, "kind": "oracle", "sample": sample}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return None
    builder, R, S, prm, desc = WORKLOADS[args.workload]
    # the ragged batch is sampled through its largest torus instance, the
    # serving workload through its first pool instance
    if builder is not None:
        inst = builder()
    elif args.workload == "serve":
        inst = serve_pool()[0]
    else:
        inst = max((i for i in instances.ragged_batch(512, seed=0)[0] if i.dims), key=lambda i: i.m)
    import oracle
    oracle.build()
    col, C = (None, 0)
    times, vals = [], []
    for _ in range(args.warmup):
        _oracle_sample(args, inst, col, C, prm)
    for _ in range(args.steps):
        v, used, sample, dt = _oracle_sample(args, inst, col, C, prm)
        vals.append(v)
        times.append(dt)
    v = sum(vals) / len(vals)
    metric = metric_name(args.workload)
    line = {"impl": "reference", "metric": metric,
            "value": v, "unit": "updates/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * sum(times) / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded instance generator; no Gset files)",
            "config": {"workload": args.workload, "description": desc, "n": inst.n, "edges": inst.m},
            "cpu_baseline": {"value": v, "unit": "updates/s", "cores": used, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return line


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="torus20k")
    ap.add_argument("--storage", choices=["f32", "f16", "q16", "bf16"], default="f32")
    ap.add_argument("--replicas", type=int, default=0)
    ap.add_argument("--sweeps", type=int, default=0)
    ap.add_argument("--e2e-steps", type=int, default=1, help="0 skips the end-to-end leg")
    ap.add_argument("--cpu-updates", type=float, default=6e9,
                    help="edge-replica updates in the bounded oracle sample")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--no-tune", action="store_true", help="batch: skip the autotuner")
    ap.add_argument("--no-forms", dest="forms", action="store_false",
                    help="default workload: skip the FP16 / fixed-point forms and the ragged batch")
    ap.add_argument("--serve-seconds", type=float, default=10.0, help="serving: arrival window")
    ap.add_argument("--serve-trials", type=int, default=4, help="serving: trials per request at most")
    ap.add_argument("--serve-scale", action="store_true",
                    help="serving: sweeps per trial grow with the instance (S per 10,000 spins)")
    ap.add_argument("--ttt-steps", type=int, default=2,
                    help="default workload: steps of the long-anneal time-to-target leg (0 skips it)")
    ap.add_argument("--ttt-sweeps", type=int, default=1_000_000,
                    help="sweeps per trial of the long-anneal time-to-target leg")
    args = ap.parse_args(argv)
    argl = sys.argv[1:] if argv is None else list(argv)
    args.storage_given = any(a == "--storage" or a.startswith("--storage=") for a in argl)
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch512":
        run_batch(args)
    elif args.workload == "serve":
        run_serve(args)
    elif args.workload == "ablation":
        run_ablation(args)
    elif args.workload == "fields2d":
        run_fields(args)
    elif args.workload == "readout":
        run_readout(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
