"""Bounded-degree non-lattice graphs (random 3- and 4-regular, N = 10,000
and 20,000, +-1 weights, Misra-Gries colouring): one sweep from an
identical state against the FP64 oracle for FP32 phases (1e-5 rad) and
binary16-stored phases (2e-3 rad against the oracle's binary16 mode); the
per-sweep error of binary16 storage against the pure FP64 sweep on the
trial's own states at sweeps 1, 10, 100 and 1000; and the final-cut
distributions over 100 seeds (1,000 vertices) and over 100 seeds x 2,048
replicas (10,000 vertices) against the oracle's."""
import math

import numpy as np
import pytest

import instances
from parity_util import TOL_F16, TOL_F32, circ_rad, f16_exact_turns, one_sweep_error

pytestmark = pytest.mark.gpu

A14 = 14.0 / 360.0


@pytest.fixture(scope="module")
def cosm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2605_30355_gb300 import build
    build.build()
    import paper_2605_30355_gb300 as cosm
    return cosm


GRAPHS = [(10000, 3), (10000, 4), (20000, 3), (20000, 4)]


@pytest.mark.parametrize("n,d", GRAPHS, ids=[f"reg{d}_{n}" for n, d in GRAPHS])
@pytest.mark.parametrize("storage", [0, 1])
def test_one_sweep_regular(cosm, orc, n, d, storage):
    inst = instances.random_regular(n, d, 0)
    col, C = cosm.color_misra_gries(inst.n, inst.src, inst.dst)
    assert C <= d + 1
    s = cosm.Solver(inst.n, inst.src, inst.dst, inst.w, color=col, n_colors=C, storage=storage,
                    dwt_ratio=1.0)
    g = orc.ColouredGraph(inst.n, inst.src, inst.dst, inst.w, col, C)
    R = 4
    x0 = np.stack([orc.init_phases(inst.n, 11, r) for r in range(R)])
    if storage == 1:
        x0 = f16_exact_turns(x0)
    for sweep in (1, 10, 100, 1000):
        s.set_state(x0, seed=11)
        alpha = float(np.float32(orc.alpha(sweep, 1000, A14)))
        s.step(sweep, alpha)
        x1 = s.get_state()
        for r in range(R):
            err, ties = one_sweep_error(orc, g, x0[r], x1[r], alpha, sweep, seed=11, replica=r,
                                        dwt_ratio=1.0, storage=orc.STORE_F16 if storage else 0)
            assert err < (TOL_F16 if storage else TOL_F32), (sweep, r, err, ties)


@pytest.mark.parametrize("d", [3, 4])
def test_final_cut_distribution_over_100_seeds(cosm, orc, d):
    # 100 seeds x 8 replicas of a 1,000-vertex regular graph, 300 sweeps:
    # the GPU's FP32 and binary16-storage final cuts against the oracle's
    # FP64 trials of the same seeds; means within 4 standard errors
    inst = instances.random_regular(1000, d, 2)
    col, C = cosm.color_misra_gries(inst.n, inst.src, inst.dst)
    g = orc.ColouredGraph(inst.n, inst.src, inst.dst, inst.w, col, C)
    S, R, seeds = 300, 8, range(100)
    orc_cuts = np.concatenate([orc.trials(g, S, R, dwt_ratio=1.0, seed=sd)[0] for sd in seeds])
    for storage in (0, 1):
        s = cosm.Solver(inst.n, inst.src, inst.dst, inst.w, color=col, n_colors=C, storage=storage,
                        dwt_ratio=1.0)
        gpu = []
        for sd in seeds:
            s.run(S, R, sd)
            gpu.append(s.replica_cuts()[0])
        gpu = np.concatenate(gpu)
        se = math.sqrt(gpu.var() / gpu.size + orc_cuts.var() / orc_cuts.size)
        assert abs(gpu.mean() - orc_cuts.mean()) < 4 * se + 1e-9, (storage, gpu.mean(), orc_cuts.mean(), se)
        # the spread is that of the same dynamics too
        assert 0.5 < gpu.std() / max(orc_cuts.std(), 1e-9) < 2.0


@pytest.mark.parametrize("n,d", GRAPHS, ids=[f"reg{d}_{n}" for n, d in GRAPHS])
def test_per_sweep_f16_error_against_fp64_on_trial_states(cosm, orc, n, d):
    # the binary16 trial's own state before sweep s (s = 1, 10, 100, 1000 of
    # a 10^4-sweep trial), one more GPU sweep against the oracle's pure FP64
    # sweep from that state: most phases within a few binary16 quanta (a
    # rounding can flip a sign decision near a tie and move a phase by a whole
    # step, so this is a distribution bound), and within 2e-3 rad of the
    # oracle's binary16-storage mode, near-ties either branch
    inst = instances.random_regular(n, d, 0)
    col, C = cosm.color_misra_gries(inst.n, inst.src, inst.dst)
    g = orc.ColouredGraph(inst.n, inst.src, inst.dst, inst.w, col, C)
    S, R, seed = 10000, 3, 17
    s = cosm.Solver(inst.n, inst.src, inst.dst, inst.w, color=col, n_colors=C, storage=1, dwt_ratio=1.0)
    q = 2 * math.pi * 2 ** -12  # the binary16 quantum near 1/2 turn, in rad
    report = {}
    for sweep in (1, 10, 100, 1000):
        if sweep == 1:
            x0 = f16_exact_turns(np.stack([orc.init_phases(inst.n, seed, r) for r in range(R)]))
        else:
            s.run_range(S, 1, sweep - 1, R, seed)
            x0 = s.get_state()
        alpha = float(np.float32(orc.alpha(sweep, S, A14)))
        s.set_state(x0, seed=seed)
        s.step(sweep, alpha)
        x1 = s.get_state()
        errs = []
        for r in range(R):
            xf, _ = orc.sweep(g, x0[r], alpha, sweep, seed=seed, replica=r, dwt_ratio=1.0)
            e = circ_rad(xf, x1[r])
            errs.append(e)
            err16, _ = one_sweep_error(orc, g, x0[r], x1[r], alpha, sweep, seed=seed, replica=r,
                                       dwt_ratio=1.0, storage=orc.STORE_F16)
            assert err16 < TOL_F16, (sweep, r, err16)
        e = np.concatenate(errs)
        report[sweep] = (float(np.median(e)), float(np.percentile(e, 99)), float(e.max()))
        assert np.median(e) <= q and (e > 8 * q).mean() < 0.02, (sweep, report[sweep])
    print(f"reg{d}_{n} binary16 vs FP64 per-sweep error (median, p99, max rad):", report)


@pytest.mark.parametrize("d", [3, 4])
def test_final_cut_distribution_at_ten_thousand(cosm, orc, d):
    # 100 seeds x 2,048 replicas of a 10,000-vertex regular graph, 1,000
    # sweeps, FP32 and binary16 storage, against 64 FP64 oracle trials of
    # the same graph: means within 4 standard errors, the same spread; the
    # binary16-minus-FP32 mean difference is reported with its error
    inst = instances.random_regular(10000, d, 3)
    col, C = cosm.color_misra_gries(inst.n, inst.src, inst.dst)
    g = orc.ColouredGraph(inst.n, inst.src, inst.dst, inst.w, col, C)
    S, R = 1000, 2048
    orc_cuts = orc.trials(g, S, 64, dwt_ratio=1.0, seed=12345)[0]
    means = {}
    for storage in (0, 1):
        s = cosm.Solver(inst.n, inst.src, inst.dst, inst.w, color=col, n_colors=C, storage=storage,
                        dwt_ratio=1.0)
        gpu = []
        for sd in range(100):
            s.run(S, R, sd)
            gpu.append(s.replica_cuts()[0])
        gpu = np.concatenate(gpu)
        se = math.sqrt(gpu.var() / gpu.size + orc_cuts.var() / orc_cuts.size)
        assert abs(gpu.mean() - orc_cuts.mean()) < 4 * se, (storage, gpu.mean(), orc_cuts.mean(), se)
        assert 0.5 < gpu.std() / max(orc_cuts.std(), 1e-9) < 2.0
        means[storage] = (gpu.mean(), gpu.std() / math.sqrt(gpu.size))
    diff = means[1][0] - means[0][0]
    print(f"reg{d}_10000: FP32 mean {means[0][0]:.3f}, binary16 mean {means[1][0]:.3f}, "
          f"difference {diff:.3f} +- {1.96 * math.hypot(means[0][1], means[1][1]):.3f}; "
          f"oracle mean {orc_cuts.mean():.3f} over {orc_cuts.size} trials")
