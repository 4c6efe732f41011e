"""Ragged batch (many instances of uneven size in one graph-captured run):
every instance's per-replica cuts and best bisectors are bit-exact with the
oracle's readout of the batch's own final phases; fixed-point batches equal
the oracle's whole trials for every replica of every instance; and every
instance's results equal a separate single-instance run with the same
arguments, bit for bit, also after the autotuner changes the layout and
across graph replays with new seeds."""
import numpy as np
import pytest

import instances

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cosm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2605_30355_gb300 import build
    build.build()
    import paper_2605_30355_gb300 as cosm
    return cosm


def _insts():
    return [instances.torus2d(16, 16, 0), instances.sparse_gnm(300, 900, 1),
            instances.torus2d(12, 20, 2), instances.random_regular(500, 3, 3),
            instances.sparse_gnm(1200, 3000, 4), instances.torus2d(20, 20, 5),
            instances.gauge_planted(instances.torus2d(8, 8, 6), 7)]


def _check_against_solo(cosm, b, insts, sweeps, replicas, seeds, storage=0, **kw):
    for i, inst in enumerate(insts):
        solo = cosm.Solver.from_instance(inst, storage=storage, **kw)
        solo.run(sweeps[i], replicas[i], seeds[i])
        c1, p1 = solo.replica_cuts()
        c2, p2 = b.replica_cuts(i)
        assert np.array_equal(c1, c2), i
        assert np.array_equal(p1, p2), i
        assert solo.best()[:3] == b.best(i)[:3]
        assert np.array_equal(solo.best()[3], b.best(i)[3])
        assert np.array_equal(solo.get_state(), b.get_state(i))


@pytest.mark.parametrize("storage", [0, 1])
def test_batch_matches_single_instance_runs(cosm, storage):
    insts = _insts()
    sweeps = [200, 150, 300, 100, 250, 120, 400]
    replicas = [10, 7, 33, 5, 12, 64, 3]
    b = cosm.Batch(insts, storage=storage, dwt_ratio=1.0)
    b.run(sweeps, replicas, [11, 12, 13, 14, 15, 16, 17])
    info = b.info()
    assert info["instances"] == 7 and info["classes"] >= 2 and info["graphs_built"] == 1
    _check_against_solo(cosm, b, insts, sweeps, replicas, [11, 12, 13, 14, 15, 16, 17], storage,
                        dwt_ratio=1.0)
    # replay of the captured graph with other seeds
    b.run(sweeps, replicas, [21, 22, 23, 24, 25, 26, 27])
    assert b.info()["graphs_built"] == 1
    _check_against_solo(cosm, b, insts, sweeps, replicas, [21, 22, 23, 24, 25, 26, 27], storage,
                        dwt_ratio=1.0)


@pytest.mark.parametrize("storage", [0, 1, 2, 3])
def test_batch_cuts_bit_exact_with_oracle_readout(cosm, orc, storage):
    insts = _insts()
    sweeps = [200, 150, 300, 100, 250, 120, 400]
    replicas = [10, 7, 33, 5, 12, 64, 3]
    seeds = [31, 32, 33, 34, 35, 36, 37]
    b = cosm.Batch(insts, storage=storage, dwt_ratio=1.0)
    b.run(sweeps, replicas, seeds)
    for i, inst in enumerate(insts):
        g = orc.coloured(inst)
        x = b.get_state(i)
        cuts, bps = b.replica_cuts(i)
        for r in range(replicas[i]):
            best, bp, _, _ = orc.binarize(g, x[r])
            assert cuts[r] == best and bps[r] == bp, (i, r)
        cut, energy, rep, spins = b.best(i)
        assert cut == cuts.max() and rep == int(np.argmax(cuts))
        assert orc.cut(inst.src, inst.dst, inst.w, spins) == cut
        assert energy == int(np.sum(inst.w)) - 2 * cut


def test_fixed_point_batch_equals_oracle_trials(cosm, orc):
    # fixed point is exact: every replica of every instance is the oracle's
    # whole trial (init, sweeps, twists, schedule, readout) bit for bit
    insts = _insts()
    sweeps = [120, 90, 150, 60, 110, 80, 200]
    replicas = [6, 5, 9, 4, 7, 10, 3]
    seeds = [41, 42, 43, 44, 45, 46, 47]
    b = cosm.Batch(insts, storage=cosm.Q16, dwt_ratio=1.0)
    b.run(sweeps, replicas, seeds)
    for i, inst in enumerate(insts):
        g = orc.coloured(inst)
        x = b.get_state(i)
        cuts, bps = b.replica_cuts(i)
        for r in range(replicas[i]):
            best, xo, _, bp = orc.trial(g, sweeps[i], dwt_ratio=1.0, seed=seeds[i], replica=r,
                                        storage=orc.STORE_Q16)
            assert np.array_equal(x[r], xo), (i, r)
            assert cuts[r] == best and bps[r] == bp, (i, r)


def test_batch_autotuner_keeps_results(cosm, tmp_path, monkeypatch):
    insts = _insts()
    sweeps = [90] * len(insts)
    replicas = [9, 17, 40, 6, 21, 8, 5]
    b = cosm.Batch(insts, dwt_ratio=1.0)
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("COSM_TUNE_CACHE", str(cache))
    b.tune(replicas, probe_sweeps=5)
    choice = (b.info()["policy"], b.info()["threads"])
    assert cache.read_text().strip()
    b.run(sweeps, replicas, [3] * len(insts))
    _check_against_solo(cosm, b, insts, sweeps, replicas, [3] * len(insts), dwt_ratio=1.0)
    # a second batch of the same shape takes the cached choice
    b2 = cosm.Batch(insts, dwt_ratio=1.0)
    b2.tune(replicas, probe_sweeps=5)
    assert (b2.info()["policy"], b2.info()["threads"]) == choice


def test_batch_planted_optimum(cosm):
    inst = instances.gauge_planted(instances.torus2d(24, 24, 1), 2)
    other = instances.sparse_gnm(2000, 5000, 3)
    b = cosm.Batch([inst, other])
    b.run([1500, 50], [48, 10], [1, 2])
    cut, energy, rep, spins = b.best(0)
    assert cut == inst.meta["opt_cut"] and energy == inst.meta["ground_energy"]
