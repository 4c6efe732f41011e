"""Cosm throughput bench: edge-replica updates/s and time-to-target.

Default workload: the 20,000-spin 2D +-1 toroidal glass (100 x 200, 40,000
edges, J uniform in {-1,+1} from seed 0, regular 4-colour partition), FP32
phases resident in shared memory, 1,024 replicas, 10^5 sweeps per trial,
alpha_0 = 14 deg, DWT ratio 0.5 every 3 sweeps, 100 bisectors. One step is
one full trial of every replica (init, all sweeps, DWT, schedule, readout
with exact cuts and best-state tracking).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--storage f32|f16] [--workload torus20k|torus10k|...]

Prints one JSON line (rank 0). ``--impl reference`` times the FP64 CPU
oracle on the host cores on a bounded sample of the same workload.
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
    "torus16": (lambda: instances.torus2d(16, 16, 0), 64, 1000,
                dict(alpha0_deg=14.0, dwt_ratio=0.5, dwt_period=3),
                "2D +-1 torus 16x16 (N=256), 64 replicas, 1000 sweeps"),
}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


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
    storage = cosm.F16 if args.storage == "f16" else cosm.F32
    inst = builder()
    col, C = _colour(inst, args.workload)
    seed = 1 + rank  # every rank runs its own independent replicas
    solver = cosm.Solver.from_instance(inst, color=col, n_colors=C, storage=storage, **prm)
    stream = torch.cuda.Stream()
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")

    for _ in range(args.warmup):
        solver.run(S, R, seed, stream)
        solver.sync()
    layout = solver.layout()

    sampler = ClockSampler(local)
    times = []
    step_cuts = []
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    for k in range(args.steps):
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
        step_cuts.append(solver.replica_cuts()[0])
    torch.cuda.synchronize()
    clocks = sampler.stop()
    if ws > 1:
        dist.barrier()
    t_step = sum(times) / len(times)
    t_max = t_step
    if ws > 1:
        tt = torch.tensor([t_step], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_max = float(tt.item())
    updates = inst.m * S * R  # edge-replica updates per step per rank
    value = updates * ws / t_max

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
    if ws > 1 and e2e_t is not None:
        tt = torch.tensor([e2e_t], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e2e_t = float(tt.item())

    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return None

    # ---- time to target (P_s over this run's replicas)
    tgt = _targets().get(args.workload)
    ttt = None
    if tgt is not None:
        allc = np.concatenate(step_cuts)
        ps = float((allc >= tgt["cut"]).mean())
        t_trial = t_step / R
        r = _r99(ps)
        ttt = {"target_cut": tgt["cut"], "target_source": tgt["source"], "P_s": ps,
               "trials": int(allc.size), "R99": r if math.isfinite(r) else None,
               "t_trial_s": t_trial, "TTT_s": t_trial * r if math.isfinite(r) else None,
               "best_cut": int(allc.max())}

    # ---- roofline of the sweep kernel: shared memory and FP32 issue
    roof = roofline(cosm, inst, prm, storage, layout, updates, t_step, clocks)

    line = {
        "metric": "edge-replica updates/s (20k-spin 2D +-1 glass, plain FP32 Cosm)",
        "value": value, "unit": "updates/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max * 1000.0, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if storage == cosm.F32 else "f16-storage/f32-compute",
        "data": "synthetic (seeded instance generator; no Gset files)",
        "config": {"workload": args.workload, "description": desc, "n": inst.n, "edges": inst.m,
                   "replicas_per_gpu": R, "sweeps_per_trial": S, "colors": layout["colors"],
                   "replicas_per_cta": layout["K"], "threads_per_cta": layout["threads"],
                   "ctas": layout["grid"], "l2": "flushed between timed steps (256 MB write)",
                   "parallelism": f"replicas sharded over {ws} GPU(s), no collective on the data path"},
        "e2e": None if e2e_t is None else {
            "value": updates * ws / e2e_t, "unit": "updates/s", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "api": "cosm_solve (host buffers)"},
        "gpu_launches": 2 * args.steps,
        "clocks": clocks,
        "roofline": roof,
        "time_to_target": ttt,
        "paper_context": {"updates_per_s": 1.41e10, "hardware": "2x Xeon Gold 6544Y, 64 threads, FP32",
                          "source": "derived from Section III-A and Table II (G72/G77/G81)"},
    }
    if args.cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args, inst, col, C, prm)
    print(json.dumps(line))
    if ws > 1:
        dist.destroy_process_group()
    return line


# Algorithmic FP32 operations of one edge-replica update (eq. (6) on the
# minimum angular difference): difference, rounding to the nearest turn,
# subtraction, sign select, two phase updates, two wraps (round + subtract).
ALU_OPS_PER_UPDATE = 10
FP32_LANES_PER_SM = 128


def roofline(cosm, inst, prm, storage, layout, updates, t_step, clocks):
    """Shared-memory and FP32-issue rooflines of the sweep kernel.

    Shared-memory bytes per update: the implicit-index lattice kernel loads
    and stores each phase once per 2x2 block, i.e. 2 phases moved per edge
    (2b bytes, b = bytes per phase, DWT fused); the edge-list kernel loads
    and stores both endpoints per edge (4b) plus a DWT pass over all phases
    every dwt_period sweeps (2b n / (m dwt_period)). The kernel that
    dominates the step is the sweep kernel (one launch per step; the
    finaliser is microseconds), so the step time is its launch duration."""
    import torch
    bpc, smem_gbps = cosm.probe_smem(4096)
    b = 4 if storage == cosm.F32 else 2
    if layout["lattice"] == 2:
        per_update = 2.0 * b
    else:
        per_update = 4.0 * b + (2.0 * b * inst.n) / (inst.m * max(1, prm["dwt_period"]))
    smem_ach = per_update * updates / t_step / 1e9
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    mhz = clocks.get("sm_mhz") or 2070.0
    alu_peak = FP32_LANES_PER_SM * props.multi_processor_count * mhz * 1e6 / 1e12
    alu_ach = ALU_OPS_PER_UPDATE * updates / t_step / 1e12
    smem = {"bound": "smem", "achieved": smem_ach, "peak": smem_gbps, "unit": "GB/s",
            "frac": smem_ach / smem_gbps, "traffic": None, "bytes_per_update": per_update,
            "peak_source": f"measured shared-memory read bandwidth ({bpc:.1f} B/clk/SM)"}
    alu = {"bound": "alu", "achieved": alu_ach, "peak": alu_peak, "unit": "Tops/s",
           "frac": alu_ach / alu_peak, "traffic": None, "ops_per_update": ALU_OPS_PER_UPDATE,
           "peak_source": f"{FP32_LANES_PER_SM} FP32 lanes/SM x {props.multi_processor_count} SMs "
                          f"x {mhz:.0f} MHz (median sampled SM clock)"}
    main, other = (alu, smem) if alu["frac"] >= smem["frac"] else (smem, alu)
    main = dict(main)
    main["other"] = other
    return main


# ---------------------------------------------------------------------- oracle

def _oracle_sample(args, inst, col, C, prm):
    import oracle
    oracle.build()
    if col is None:
        col, C = oracle.color_instance(inst)
    g = oracle.ColouredGraph(inst.n, inst.src, inst.dst, inst.w, col, C)
    cores = os.cpu_count() or 1
    reps = cores
    sweeps = max(10, int(args.cpu_updates / (inst.m * reps)))
    t0 = time.perf_counter()
    cuts, _, _, used = oracle.trials(g, sweeps, reps, alpha0=prm["alpha0_deg"] / 360.0,
                                     dwt_period=prm["dwt_period"], dwt_ratio=prm["dwt_ratio"],
                                     seed=1, threads=cores)
    dt = time.perf_counter() - t0
    return inst.m * sweeps * reps / dt, used, f"{reps} replicas x {sweeps} sweeps of the same instance", dt


def cpu_baseline(args, inst, col, C, prm):
    v, used, sample, _ = _oracle_sample(args, inst, col, C, prm)
    return {"value": v, "unit": "updates/s", "cores": used, "kind": "oracle", "sample": sample}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return None
    builder, R, S, prm, desc = WORKLOADS[args.workload]
    inst = builder()
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
    line = {"impl": "reference", "metric": "edge-replica updates/s (20k-spin 2D +-1 glass, plain FP32 Cosm)",
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
    ap.add_argument("--storage", choices=["f32", "f16"], default="f32")
    ap.add_argument("--replicas", type=int, default=0)
    ap.add_argument("--sweeps", type=int, default=0)
    ap.add_argument("--e2e-steps", type=int, default=1, help="0 skips the end-to-end leg")
    ap.add_argument("--cpu-updates", type=float, default=6e9,
                    help="edge-replica updates in the bounded oracle sample")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    args = ap.parse_args(argv)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
