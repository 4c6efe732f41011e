"""Fixed-point phases (COSM_Q16): every operation is exact integer
arithmetic on the 2^-16-turn grid, so whole trials -- initial state, every
sweep, the twist, the step schedule and the readout -- are bit-identical to
the oracle's fixed-point mode, on the lattice kernel and the edge-list
kernel alike."""
import numpy as np
import pytest

import instances

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


CASES = [
    ("torus16_lattice", lambda: instances.torus2d(16, 16, 0), True, 0.5),
    ("torus_rect_lattice", lambda: instances.torus2d(12, 20, 3), True, 1.5),
    ("torus16_general", lambda: instances.torus2d(16, 16, 0), False, 0.5),
    ("reg3", lambda: instances.random_regular(600, 3, 1), False, 1.0),
    ("gnm_w3", lambda: instances.sparse_gnm(500, 1500, 2), False, 1.0),
    ("torus3d", lambda: instances.torus3d(4, 6, 8, 5), True, 1.0),
    ("planted", lambda: instances.frustrated_loop_planted((12, 12), 0.6, 4), True, 1.0),
]


@pytest.mark.parametrize("name,make,dims,ratio", CASES, ids=[c[0] for c in CASES])
def test_whole_trials_bit_exact(cosm, orc, name, make, dims, ratio):
    inst = make()
    col, C = orc.color_instance(inst)
    s = cosm.Solver.from_instance(inst, color=col, n_colors=C, use_dims=dims, storage=cosm.Q16,
                                  dwt_ratio=ratio)
    if name.endswith("lattice"):
        assert s.layout()["lattice"] == 2
    S, R, seed = 150, 6, 31
    s.run(S, R, seed)
    x = s.get_state()
    cuts, bps = s.replica_cuts()
    g = orc.ColouredGraph(inst.n, inst.src, inst.dst, inst.w, col, C)
    for r in range(R):
        best, xo, spins, bp = orc.trial(g, S, alpha0=A14, dwt_ratio=ratio, seed=seed, replica=r,
                                        storage=orc.STORE_Q16)
        assert np.array_equal(x[r], xo), (name, r)
        assert cuts[r] == best and bps[r] == bp
    cut, energy, rep, spins = s.best()
    assert orc.cut(inst.src, inst.dst, inst.w, spins) == cut == cuts.max()


@pytest.mark.parametrize("flags", [0, 1, 2, 3])
def test_one_sweep_flags_bit_exact(cosm, orc, flags):
    inst = instances.random_regular(400, 4, 8)
    col, C = orc.color_greedy(inst.n, inst.src, inst.dst)
    s = cosm.Solver(inst.n, inst.src, inst.dst, inst.w, color=col, n_colors=C, storage=cosm.Q16,
                    flags=flags, dwt_ratio=1.0)
    g = orc.ColouredGraph(inst.n, inst.src, inst.dst, inst.w, col, C)
    R = 5
    x0 = np.stack([orc.q16_grid(orc.init_phases(inst.n, 2, r)) for r in range(R)])
    for sweep in (1, 3):
        s.set_state(x0, seed=2)
        alpha = float(np.float32(0.0211))
        s.step(sweep, alpha)
        x1 = s.get_state()
        for r in range(R):
            xo, _ = orc.sweep(g, x0[r], alpha, sweep, seed=2, replica=r, dwt_ratio=1.0, flags=flags,
                              storage=orc.STORE_Q16)
            assert np.array_equal(x1[r], xo), (flags, sweep, r)


def test_q16_batch_and_layouts_bit_exact(cosm, orc):
    import os
    insts = [instances.torus2d(16, 16, 2), instances.sparse_gnm(700, 2000, 3)]
    b = cosm.Batch(insts, storage=cosm.Q16, dwt_ratio=1.0)
    b.run([120, 90], [9, 5], [4, 5])
    for i, inst in enumerate(insts):
        for K in (2, 4, 8):
            os.environ["COSM_K"] = str(K)
            try:
                s = cosm.Solver.from_instance(inst, storage=cosm.Q16, dwt_ratio=1.0)
                s.run([120, 90][i], [9, 5][i], [4, 5][i])
                assert np.array_equal(s.get_state(), b.get_state(i))
            finally:
                del os.environ["COSM_K"]


@pytest.mark.parametrize("K", [2, 4, 8])
@pytest.mark.parametrize("name", ["torus_rect_lattice", "torus16_lattice", "gnm_w3"])
def test_whole_trials_bit_exact_per_tile_width(cosm, orc, K, name):
    # the fixed-point passes keep two replicas per 32-bit word: tiles of 2, 4
    # and 8 replicas hold 1, 2 and 4 words per slot; each against the oracle
    import os
    _, make, dims, ratio = next(c for c in CASES if c[0] == name)
    inst = make()
    col, C = orc.color_instance(inst)
    os.environ["COSM_K"] = str(K)
    try:
        s = cosm.Solver.from_instance(inst, color=col, n_colors=C, use_dims=dims, storage=cosm.Q16,
                                      dwt_ratio=ratio)
        S, R, seed = 120, 2 * K + 1, 17
        s.run(S, R, seed)
    finally:
        del os.environ["COSM_K"]
    assert s.layout()["K"] == K and (s.layout()["lattice"] == 2) == dims
    x = s.get_state()
    cuts, bps = s.replica_cuts()
    g = orc.ColouredGraph(inst.n, inst.src, inst.dst, inst.w, col, C)
    for r in range(R):
        best, xo, _, bp = orc.trial(g, S, alpha0=A14, dwt_ratio=ratio, seed=seed, replica=r,
                                    storage=orc.STORE_Q16)
        assert np.array_equal(x[r], xo), (name, K, r)
        assert cuts[r] == best and bps[r] == bp


def test_full_size_fixed_point_sampled(cosm, orc):
    # the 20k-spin torus in u16 fixed point at the forms' launch configuration
    # (four replicas per CTA, 1,024 replicas): sampled replicas' whole trials
    # bit-exact with the oracle's
    inst = instances.torus2d(100, 200, 0)
    col, C = orc.color_instance(inst)
    s = cosm.Solver.from_instance(inst, color=col, n_colors=C, storage=cosm.Q16, dwt_ratio=0.5)
    S, seed = 45, 23
    s.run(S, 1024, seed)
    assert s.layout()["lattice"] == 2 and s.layout()["K"] == 4
    x = s.get_state()
    cuts, bps = s.replica_cuts()
    g = orc.ColouredGraph(inst.n, inst.src, inst.dst, inst.w, col, C)
    for r in (0, 3, 514, 1023):
        best, xo, _, bp = orc.trial(g, S, alpha0=A14, dwt_ratio=0.5, seed=seed, replica=r,
                                    storage=orc.STORE_Q16)
        assert np.array_equal(x[r], xo), r
        assert cuts[r] == best and bps[r] == bp
