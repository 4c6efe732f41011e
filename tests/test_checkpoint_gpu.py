"""Run control through the C ABI: the success count of cosm_run's target
(Appendix A's P_s), trials split into sweep ranges and resumed from an
exported checkpoint (bit-identical to one uninterrupted run, and for fixed
point to the oracle's whole trial), and the bounded wait between work
segments running out on an injected host-side fault (no device fault: the
waiting CTA gives up, the handle reports COSM_ERR_TIMEOUT and stays usable).
"""
import os

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


def _graph(orc, inst):
    col, C = orc.color_instance(inst)
    return col, C, orc.ColouredGraph(inst.n, inst.src, inst.dst, inst.w, col, C)


@pytest.mark.parametrize("storage", [0, 1, 2])
def test_success_count_matches_oracle_readout(cosm, orc, storage):
    inst = instances.torus2d(16, 16, 0)
    col, C, g = _graph(orc, inst)
    s = cosm.Solver.from_instance(inst, color=col, n_colors=C, storage=storage)
    R = 40
    s.run(300, R, seed=9)
    x = s.get_state()
    ocuts = np.array([orc.binarize(g, x[r])[0] for r in range(R)])
    for target in (int(ocuts.min()), int(np.median(ocuts)), int(ocuts.max()), int(ocuts.max()) + 1):
        s.run(300, R, seed=9, target=target)
        assert s.success() == int((ocuts >= target).sum()), target
    s.run(300, R, seed=9)  # no target: every replica counts
    assert s.success() == R


CASES = [
    ("lattice_f32", lambda: instances.torus2d(16, 20, 1), True, 0),
    ("edges_f32", lambda: instances.sparse_gnm(500, 1400, 3), False, 0),
    ("lattice_f16", lambda: instances.torus2d(16, 16, 2), True, 1),
    ("edges_q16", lambda: instances.random_regular(400, 3, 5), False, 2),
    ("lattice_q16", lambda: instances.torus2d(12, 16, 6), True, 2),
]


@pytest.mark.parametrize("name,make,dims,storage", CASES, ids=[c[0] for c in CASES])
def test_ranges_and_checkpoint_resume_bit_identical(cosm, orc, name, make, dims, storage):
    inst = make()
    col, C, g = _graph(orc, inst)
    S, R, seed = 240, 7, 21

    def solver():
        return cosm.Solver.from_instance(inst, color=col, n_colors=C, use_dims=dims, storage=storage,
                                         dwt_ratio=1.0)

    ref = solver()
    ref.run(S, R, seed)
    ref_cuts, ref_bp = ref.replica_cuts()
    ref_x, ref_idx = ref.export_state()
    assert ref_idx == S
    # three ranges on one handle (the middle one of a single sweep)
    a = solver()
    a.run_range(S, 1, 100, R, seed)
    a.run_range(S, 101, 101, R, seed)
    a.run_range(S, 102, S, R, seed)
    assert np.array_equal(a.replica_cuts()[0], ref_cuts)
    assert np.array_equal(a.export_state()[0], ref_x)
    # checkpoint after sweep 77, resumed on a fresh handle
    b = solver()
    b.run_range(S, 1, 77, R, seed)
    ck, idx = b.export_state()
    assert idx == 77
    b.close()
    c = solver()
    c.import_state(ck, R, seed, idx)
    c.run_range(S, 78, S, R, seed)
    cuts, bp = c.replica_cuts()
    assert np.array_equal(cuts, ref_cuts) and np.array_equal(bp, ref_bp)
    assert np.array_equal(c.export_state()[0], ref_x)
    if storage == cosm.Q16:
        # the resumed fixed-point trial is the oracle's whole trial
        x = c.get_state()
        for r in range(R):
            best, xo, _, bpo = orc.trial(g, S, alpha0=A14, dwt_ratio=1.0, seed=seed, replica=r,
                                         storage=orc.STORE_Q16)
            assert np.array_equal(x[r], xo) and cuts[r] == best and bp[r] == bpo, r


def test_range_misuse_rejected(cosm):
    inst = instances.torus2d(8, 8, 1)
    s = cosm.Solver.from_instance(inst)
    with pytest.raises(cosm.CosmError) as e:
        s.run_range(100, 50, 60, 4, 1)  # no state at sweep 49
    assert e.value.code == cosm.ERR_STATE
    s.run_range(100, 1, 49, 4, 1)
    with pytest.raises(cosm.CosmError) as e:
        s.run_range(100, 50, 60, 4, 2)  # another seed
    assert e.value.code == cosm.ERR_INVALID_ARG
    with pytest.raises(cosm.CosmError) as e:
        s.run_range(100, 60, 50, 4, 1)
    assert e.value.code == cosm.ERR_INVALID_ARG
    with pytest.raises(cosm.CosmError) as e:
        s.success()  # mid-trial: no readout yet
    assert e.value.code == cosm.ERR_STATE


def test_bounded_wait_times_out_on_dropped_signal(cosm, orc):
    # more tiles than resident CTAs: tiles are split between two CTAs and
    # the tail waits for the head's ready flag; the injected fault drops the
    # flags, so every tail gives up after the 50 ms limit
    inst = instances.random_regular(500, 3, 2)
    col, C = orc.color_greedy(inst.n, inst.src, inst.dst)
    os.environ["COSM_GRID_CAP"] = "7"
    try:
        s = cosm.Solver(inst.n, inst.src, inst.dst, inst.w, color=col, n_colors=C, dwt_ratio=1.0)
        s.set_wait_limit(0.05)
        s.inject_fault(cosm.FAULT_DROP_SIGNAL)
        s.run(401, 37, seed=4)
        with pytest.raises(cosm.CosmError) as e:
            s.sync()
        assert e.value.code == cosm.ERR_TIMEOUT
        # the context and the handle stay usable; the next run is normal
        s.run(401, 37, seed=4)
        s.sync()
        cuts = s.replica_cuts()[0]
        x = s.get_state()
    finally:
        os.environ.pop("COSM_GRID_CAP", None)
    assert s.layout()["grid"] == 7
    ref = cosm.Solver(inst.n, inst.src, inst.dst, inst.w, color=col, n_colors=C, dwt_ratio=1.0)
    ref.run(401, 37, seed=4)
    assert np.array_equal(ref.replica_cuts()[0], cuts)
    assert np.array_equal(ref.get_state(), x)


@pytest.mark.parametrize("storage", [0, 2])
def test_tracked_trial_split_into_ranges_on_one_handle(cosm, orc, storage):
    # mid-anneal tracking (Fig. 10) across ranges of one handle: the readouts
    # every T sweeps, the kept readout and its spins equal the uninterrupted
    # tracked trial's (the tracking state stays on the handle)
    inst = instances.torus2d(12, 16, 4)
    S, R, seed, T = 180, 5, 33, 25

    def solver():
        return cosm.Solver.from_instance(inst, storage=storage, track_period=T, dwt_ratio=1.0)

    ref = solver()
    ref.run(S, R, seed)
    a = solver()
    a.run_range(S, 1, 60, R, seed)
    a.run_range(S, 61, 133, R, seed)
    a.run_range(S, 134, S, R, seed)
    assert np.array_equal(a.trace(), ref.trace())
    assert np.array_equal(a.replica_cuts()[0], ref.replica_cuts()[0])
    assert np.array_equal(a.replica_energies(), ref.replica_energies())
    ra, rr = a.best(), ref.best()
    assert ra[:3] == rr[:3] and np.array_equal(ra[3], rr[3])
