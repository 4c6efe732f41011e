"""Bounded-degree non-lattice graphs (random 3- and 4-regular, N = 10,000
and 20,000, +-1 weights, Misra-Gries colouring): one sweep from an
identical state against the FP64 oracle for FP32 phases (1e-5 rad) and
binary16-stored phases (2e-3 rad against the oracle's binary16 mode), and
the final-cut distribution over 100 seeds against the oracle's."""
import math

import numpy as np
import pytest

import instances
from parity_util import TOL_F16, TOL_F32, f16_exact_turns, one_sweep_error

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
