"""Writes tests/golden/targets.json: target cuts for time-to-target.

The target of a workload is the best cut the FP64 oracle finds in its
longest run here (all host cores, replicas x sweeps as recorded). Only the
oracle and the seeded instance generators are used.

  python tests/golden/make_targets.py [workload replicas sweeps]
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import instances  # noqa: E402
import oracle  # noqa: E402

WORKLOADS = {
    "torus20k": (lambda: instances.torus2d(100, 200, 0), dict(alpha0=14 / 360, dwt_ratio=0.5, dwt_period=3)),
    "torus10k": (lambda: instances.torus2d(100, 100, 0), dict(alpha0=14 / 360, dwt_ratio=0.5, dwt_period=3)),
}


def main(argv):
    name = argv[0] if argv else "torus20k"
    reps = int(argv[1]) if len(argv) > 1 else 32
    sweeps = int(argv[2]) if len(argv) > 2 else 300_000
    make, prm = WORKLOADS[name]
    inst = make()
    col, C = oracle.color_instance(inst)
    g = oracle.ColouredGraph(inst.n, inst.src, inst.dst, inst.w, col, C)
    t0 = time.time()
    cuts, _, _, used = oracle.trials(g, sweeps, reps, seed=424242, threads=os.cpu_count(), **prm)
    dt = time.time() - t0
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "targets.json")
    data = json.load(open(path)) if os.path.exists(path) else {}
    data[name] = {"cut": int(cuts.max()), "energy": int(inst.total_weight() - 2 * int(cuts.max())),
                  "source": f"FP64 oracle, {reps} replicas x {sweeps} sweeps, seed 424242, "
                            f"{used} threads, {dt:.0f} s",
                  "cut_histogram": {str(int(c)): int((cuts == c).sum()) for c in sorted(set(cuts.tolist()))}}
    with open(path, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    print(name, data[name])


if __name__ == "__main__":
    main(sys.argv[1:])
