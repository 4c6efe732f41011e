"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Bars: cuts, best bisectors and spins bit-exact on replayed states; initial
phases bit-exact; one sweep from an identical state within 1e-5 rad (FP32
storage) or 2e-3 rad (FP16 storage, against the oracle's binary16-storage
mode), with near-ties allowed either branch.
"""
import os

import numpy as np
import pytest

import instances
from parity_util import TOL_BF16, TOL_F16, TOL_F32, bf16_exact_turns, circ_rad, f16_exact_turns, one_sweep_error

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


def _solver(cosm, orc, inst, storage=0, use_dims=True, color=None, C=0, **kw):
    if color is None:
        color, C = orc.color_instance(inst)
    s = cosm.Solver.from_instance(inst, color=color, n_colors=C, use_dims=use_dims,
                                  storage=storage, **kw)
    g = orc.ColouredGraph(inst.n, inst.src, inst.dst, inst.w, color, C)
    return s, g


def _params_kw(s):
    p = s.params
    return dict(dwt_period=p.dwt_period, dwt_ratio=p.dwt_ratio, window=p.window_deg / 360.0,
                flags=p.flags)


CASES = [
    ("torus16", lambda: instances.torus2d(16, 16, 0), True),
    ("torus16_general", lambda: instances.torus2d(16, 16, 0), False),
    ("torus_rect", lambda: instances.torus2d(12, 20, 3), True),
    ("reg3", lambda: instances.random_regular(1000, 3, 1), False),
    ("gnm_w3", lambda: instances.sparse_gnm(777, 2300, 2), False),
    # weights up to 20: a sweep could carry a phase out of (-2, 2), so the
    # binary32 edge-list kernel wraps after every update here
    ("gnm_w20", lambda: instances.sparse_gnm(600, 1800, 4, wmax=20), False),
    ("torus3d", lambda: instances.torus3d(4, 6, 8, 5), True),
]


@pytest.mark.parametrize("name,make,dims", CASES, ids=[c[0] for c in CASES])
def test_initial_phases_bit_exact(cosm, orc, name, make, dims):
    inst = make()
    s, g = _solver(cosm, orc, inst, use_dims=dims, alpha0_deg=0.0)
    s.run(1, 9, seed=1234)
    x = s.get_state()
    for r in range(9):
        assert np.array_equal(x[r], orc.init_phases(inst.n, 1234, r)), r


def test_initial_phases_f16_rounded(cosm, orc):
    inst = instances.torus2d(16, 16, 0)
    s, g = _solver(cosm, orc, inst, storage=1, alpha0_deg=0.0)
    s.run(1, 6, seed=77)
    x = s.get_state()
    for r in range(6):
        assert np.array_equal(x[r], f16_exact_turns(orc.init_phases(inst.n, 77, r)))


def test_initial_phases_bf16_rounded(cosm, orc):
    inst = instances.torus2d(16, 16, 0)
    s, g = _solver(cosm, orc, inst, storage=3, alpha0_deg=0.0)
    s.run(1, 6, seed=77)
    x = s.get_state()
    for r in range(6):
        assert np.array_equal(x[r], bf16_exact_turns(orc.init_phases(inst.n, 77, r)))


@pytest.mark.parametrize("dims", [True, False])
@pytest.mark.parametrize("sweep", [2, 3, 500])
def test_one_sweep_bf16_storage(cosm, orc, dims, sweep):
    # bfloat16 storage: bounded by one bfloat16 quantum against the oracle's
    # bfloat16-storage mode; against pure FP64 only reported (a distribution
    # bound, as for binary16)
    inst = instances.torus2d(16, 16, 1)
    s, g = _solver(cosm, orc, inst, storage=3, use_dims=dims)
    R = 8
    x0 = np.stack([bf16_exact_turns(orc.init_phases(inst.n, 3, r)) for r in range(R)])
    s.set_state(x0, seed=3)
    alpha = float(np.float32(orc.alpha(sweep, 1000, A14)))
    s.step(sweep, alpha)
    x1 = s.get_state()
    far = []
    # the lattice kernel stores (and rounds) once per pass of two colours,
    # the edge-list kernel at every update
    mode = orc.STORE_BF16_PASS if s.layout()["lattice"] == 2 else orc.STORE_BF16
    assert (s.layout()["lattice"] == 2) == dims
    for r in range(R):
        err, _ = one_sweep_error(orc, g, x0[r], x1[r], alpha, sweep, seed=3, replica=r,
                                 storage=mode, **_params_kw(s))
        assert err <= TOL_BF16, (r, err)
        xf, _ = orc.sweep(g, x0[r], alpha, sweep, seed=3, replica=r, **_params_kw(s))
        far.append(float((circ_rad(xf, x1[r]) > 8 * 2 * np.pi * 2 ** -9).mean()))
    assert np.mean(far) < 0.05


@pytest.mark.parametrize("name,make,dims", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("sweep", [1, 3, 500, 999])
def test_one_sweep_f32(cosm, orc, name, make, dims, sweep):
    inst = make()
    kw = {"dwt_ratio": 1.0} if name in ("reg3", "gnm_w3") else {}
    s, g = _solver(cosm, orc, inst, use_dims=dims, **kw)
    R = 13
    x0 = np.stack([orc.init_phases(inst.n, 5, r) for r in range(R)])
    s.set_state(x0, seed=5)
    alpha = float(np.float32(orc.alpha(sweep, 1000, A14)))
    s.step(sweep, alpha)
    x1 = s.get_state()
    total_ties = 0
    for r in range(R):
        err, nt = one_sweep_error(orc, g, x0[r], x1[r], alpha, sweep, seed=5, replica=r,
                                  **_params_kw(s))
        total_ties += nt
        assert err <= TOL_F32, (r, err)
    assert total_ties <= 0.001 * g.m * R


@pytest.mark.parametrize("alpha0_deg", [25.0, 40.0])
@pytest.mark.parametrize("sweep", [1, 3])
def test_one_sweep_lattice_large_steps(cosm, orc, alpha0_deg, sweep):
    # larger steps (alpha0 of the planted runs, and beyond) keep phases
    # further from their wrapped range inside a sweep
    inst = instances.torus2d(12, 20, 9)
    s, g = _solver(cosm, orc, inst, alpha0_deg=alpha0_deg, dwt_ratio=1.5)
    assert s.layout()["lattice"] == 2
    R = 9
    x0 = np.stack([orc.init_phases(inst.n, 6, r) for r in range(R)])
    s.set_state(x0, seed=6)
    alpha = float(np.float32(alpha0_deg / 360.0))
    s.step(sweep, alpha)
    x1 = s.get_state()
    for r in range(R):
        err, _ = one_sweep_error(orc, g, x0[r], x1[r], alpha, sweep, seed=6, replica=r,
                                 **_params_kw(s))
        assert err <= TOL_F32, (r, err)


@pytest.mark.parametrize("flags", [1, 2, 3])
def test_one_sweep_ablation_flags(cosm, orc, flags):
    inst = instances.random_regular(600, 4, 8)
    s, g = _solver(cosm, orc, inst, use_dims=False, flags=flags, dwt_ratio=1.0)
    R = 6
    x0 = np.stack([orc.init_phases(inst.n, 9, r) for r in range(R)])
    s.set_state(x0, seed=9)
    alpha = float(np.float32(0.021))
    for sweep in (2, 3):
        s.set_state(x0, seed=9)
        s.step(sweep, alpha)
        x1 = s.get_state()
        for r in range(R):
            # eq. (8) sums per-vertex forces in FP32 in a different order than
            # the oracle: a few ulps of the step
            tol = TOL_F32 if not (flags & 2) else 1e-5
            err, _ = one_sweep_error(orc, g, x0[r], x1[r], alpha, sweep, seed=9, replica=r,
                                     **_params_kw(s))
            assert err <= tol, (flags, sweep, r, err)


@pytest.mark.parametrize("dims", [True, False])
@pytest.mark.parametrize("sweep", [2, 3, 6])
def test_one_sweep_f16_storage(cosm, orc, dims, sweep):
    inst = instances.torus2d(16, 16, 1)
    s, g = _solver(cosm, orc, inst, storage=1, use_dims=dims)
    R = 8
    x0 = np.stack([f16_exact_turns(orc.init_phases(inst.n, 3, r)) for r in range(R)])
    s.set_state(x0, seed=3)
    alpha = float(np.float32(orc.alpha(sweep, 100, A14)))
    s.step(sweep, alpha)
    x1 = s.get_state()
    far = []
    # the lattice kernel stores (and rounds) once per pass of two colours,
    # the edge-list kernel at every update
    mode = orc.STORE_F16_PASS if s.layout()["lattice"] == 2 else orc.STORE_F16
    assert (s.layout()["lattice"] == 2) == dims
    for r in range(R):
        err, _ = one_sweep_error(orc, g, x0[r], x1[r], alpha, sweep, seed=3, replica=r,
                                 storage=mode, **_params_kw(s))
        assert err <= TOL_F16, (r, err)
        # against pure FP64 (no storage rounding) most phases stay within a few
        # binary16 quanta; a rounding can flip a sign decision near a tie, which
        # moves a few phases by a whole step, so this is a distribution bound
        xf, _ = orc.sweep(g, x0[r], alpha, sweep, seed=3, replica=r, **_params_kw(s))
        far.append(float((circ_rad(xf, x1[r]) > 8 * 2 * np.pi * 2 ** -12).mean()))
    assert np.mean(far) < 0.02


@pytest.mark.parametrize("name,make,dims", CASES, ids=[c[0] for c in CASES])
def test_readout_bit_exact_on_replayed_state(cosm, orc, name, make, dims):
    inst = make()
    s, g = _solver(cosm, orc, inst, use_dims=dims)
    R = 11
    rng = np.random.default_rng(4)
    # random states, and clustered ones where bisectors matter
    x = rng.integers(0, 2 ** 24, size=(R, inst.n)) / 2 ** 24
    x[5:] = np.mod(np.round((0.3 + 0.5 * (rng.random((R - 5, inst.n)) < 0.5)
                             + rng.normal(0, 0.01, (R - 5, inst.n))) * 2 ** 24) / 2 ** 24, 1.0)
    s.set_state(x, seed=1)
    s.readout()
    cuts, bps = s.replica_cuts()
    for r in range(R):
        best, bp, allcuts, spins = orc.binarize(g, x[r])
        assert cuts[r] == best and bps[r] == bp, r
    cut, energy, rep, spins = s.best()
    assert cut == cuts.max() and rep == int(np.argmax(cuts))
    assert energy == inst.total_weight() - 2 * cut
    _, _, _, ospins = orc.binarize(g, x[rep])
    assert np.array_equal(spins, ospins)
    assert orc.cut(inst.src, inst.dst, inst.w, spins) == cut


@pytest.mark.parametrize("storage", [0, 1, 3])
def test_full_trial_cuts_bit_exact_on_final_state(cosm, orc, storage):
    inst = instances.torus2d(16, 16, 0)
    s, g = _solver(cosm, orc, inst, storage=storage)
    s.run(1000, 64, seed=11)
    cuts, bps = s.replica_cuts()
    x = s.get_state()
    for r in range(64):
        best, bp, _, _ = orc.binarize(g, x[r])
        assert cuts[r] == best and bps[r] == bp
    cut, energy, rep, spins = s.best()
    assert orc.cut(inst.src, inst.dst, inst.w, spins) == cut == cuts.max()
    assert energy == orc.energy(inst.src, inst.dst, inst.w, spins)


def test_solution_quality_matches_oracle_distribution(cosm, orc):
    # distributional parity: FP32 GPU and FP64 oracle reach the same best cut
    inst = instances.torus2d(16, 16, 0)
    s, g = _solver(cosm, orc, inst)
    s.run(1000, 64, seed=2)
    gcuts, _ = s.replica_cuts()
    ocuts, *_ = orc.trials(g, 1000, 64, seed=2)
    assert gcuts.max() == ocuts.max()
    assert abs(gcuts.mean() - ocuts.mean()) < 3.0


def test_planted_optimum_reached(cosm, orc):
    inst = instances.gauge_planted(instances.torus2d(32, 32, 3), 4)
    s, g = _solver(cosm, orc, inst)
    s.run(2000, 64, seed=3)
    cut, energy, rep, spins = s.best()
    assert cut == inst.meta["opt_cut"]
    assert energy == inst.meta["ground_energy"]


def test_layouts_agree_bit_exact(cosm, orc):
    # replicas per CTA (K) never change a trial: within each kernel variant
    # (implicit-index lattice blocks, general edge lists) results are
    # bit-identical across K. The lattice kernel wraps a phase once per 2x2
    # block instead of after every update, so the two variants agree to
    # rounding per sweep (checked by the one-sweep parity tests), not bitwise.
    # The binary32 edge-list kernel pairs two replicas (K = 2, 4) or two edges
    # (K = 1) in its f32x2 lanes; with weights up to 20 it wraps after every
    # update instead of once per sweep.
    torus = instances.torus2d(16, 16, 6)
    heavy = instances.sparse_gnm(500, 1500, 7, wmax=20)
    for inst, dims, Ks, kind in ((torus, True, (1, 2, 4), 2), (torus, False, (1, 2, 4), 0),
                                 (heavy, False, (1, 2, 4), 0)):
        col, C = orc.color_instance(inst)
        res = []
        for K in Ks:
            os.environ["COSM_K"] = str(K)
            try:
                s, _ = _solver(cosm, orc, inst, use_dims=dims, color=col, C=C)
                s.run(300, 10, seed=8)
                assert s.layout()["lattice"] == kind and s.layout()["K"] == K
                res.append((s.replica_cuts()[0], s.get_state()))
            finally:
                del os.environ["COSM_K"]
        for cuts, x in res[1:]:
            assert np.array_equal(cuts, res[0][0])
            assert np.array_equal(x, res[0][1])


def test_lattice_kernel_needs_the_regular_pattern(cosm, orc):
    inst = instances.torus2d(16, 16, 6)
    col, C = orc.color_instance(inst)
    s, _ = _solver(cosm, orc, inst, color=col, C=C)
    assert s.layout()["lattice"] == 2
    # the same partition with colours renumbered runs colours in another
    # order, so it must take the general kernel
    s2, _ = _solver(cosm, orc, inst, color=(col + 1) % 4, C=4)
    assert s2.layout()["lattice"] == 1
    # weights beyond +-1 also take the general kernel
    w3 = instances.Instance(inst.n, inst.src, inst.dst, inst.w * 3, inst.dims)
    s3, _ = _solver(cosm, orc, w3, color=col, C=C)
    assert s3.layout()["lattice"] == 1


def test_chunked_schedule_matches_single_segment(cosm, orc):
    # more tiles than resident CTAs: the wrap-around schedule splits trials
    # across CTAs through global memory, which must not change any result
    inst = instances.random_regular(500, 3, 2)
    col, C = orc.color_greedy(inst.n, inst.src, inst.dst)
    ref = None
    for cap in (0, 7):
        if cap:
            os.environ["COSM_GRID_CAP"] = str(cap)
        try:
            s, _ = _solver(cosm, orc, inst, use_dims=False, color=col, C=C, dwt_ratio=1.0)
            s.run(401, 37, seed=4)
            out = (s.replica_cuts()[0], s.get_state(), s.layout())
        finally:
            os.environ.pop("COSM_GRID_CAP", None)
        if ref is None:
            ref = out
        else:
            assert out[2]["grid"] == 7
            assert np.array_equal(out[0], ref[0])
            assert np.array_equal(out[1], ref[1])


@pytest.mark.parametrize("K", [1, 2, 4])
@pytest.mark.parametrize("make,ratio", [(lambda: instances.sparse_gnm(900, 2600, 3), 1.0),
                                        (lambda: instances.sparse_gnm(600, 1800, 4, wmax=20), 1.0),
                                        (lambda: instances.random_regular(1000, 3, 1), 1.0)])
def test_staged_records_equal_global_loads(cosm, orc, K, make, ratio):
    # binary32 edge lists can stream each colour's records into shared memory
    # ahead of use (COSM_STAGE); the phases and cuts are those of the
    # global-load sweep, bit for bit, also across the segment hand-offs of
    # the wrap-around schedule (records staged again after each hand-off)
    inst = make()
    col, C = orc.color_greedy(inst.n, inst.src, inst.dst)
    out = []
    for env in ({}, {"COSM_STAGE": "1"}, {"COSM_STAGE": "1", "COSM_GRID_CAP": "5"}):
        os.environ["COSM_K"] = str(K)
        os.environ.update(env)
        try:
            s = cosm.Solver(inst.n, inst.src, inst.dst, inst.w, color=col, n_colors=C, dwt_ratio=ratio)
            s.run(301, 6 * K + 1, seed=8)
            out.append((s.get_state(), s.replica_cuts()[0], s.layout()))
        finally:
            for k in ("COSM_K", "COSM_STAGE", "COSM_GRID_CAP"):
                os.environ.pop(k, None)
    assert out[0][2]["K"] == K and out[1][2]["K"] == K
    assert out[1][2]["smem"] > out[0][2]["smem"]  # the staging buffers
    for x, c, _ in out[1:]:
        assert np.array_equal(x, out[0][0]) and np.array_equal(c, out[0][1])


@pytest.mark.parametrize("K", [1, 2, 4])
@pytest.mark.parametrize("threads", [64, 96])
@pytest.mark.parametrize("wmax", [1, 3])
def test_edge_list_tails_and_signed_records(cosm, orc, K, threads, wmax):
    # binary32 edge lists: whole batches of B edges per thread, then one
    # checked batch; a greedy colouring of G(n, m) has colours of every size,
    # so at small thread counts the rem edges left after the whole batches
    # of a colour take every count of valid slots in the checked batch: one
    # sweep against the oracle. With +-1 weights on at most 2^15 slots the
    # sweep reads records carrying the weight's sign (the default); they
    # equal split records and weights bit for bit over whole trials.
    inst = instances.sparse_gnm(700, 2100, 5, wmax=wmax)
    col, C = orc.color_greedy(inst.n, inst.src, inst.dst)
    sizes = np.bincount(col, minlength=C)
    B = {1: 4, 2: 3, 4: 2}[K]
    rems = sizes % (B * threads)
    assert (rems > 0).any() and (rems <= threads).any() and (rems > (B - 1) * threads).any()
    env = {"COSM_K": str(K), "COSM_THREADS": str(threads)}
    out = []
    for split in (False, True):
        os.environ.update(env)
        if split:
            os.environ["COSM_SPLIT_W"] = "1"
        try:
            s, g = _solver(cosm, orc, inst, use_dims=False, color=col, C=C, dwt_ratio=1.0)
            R = 2 * K + 1
            x0 = np.stack([orc.init_phases(inst.n, 6, r) for r in range(R)])
            s.set_state(x0, seed=6)
            alpha = float(np.float32(orc.alpha(3, 1000, A14)))
            s.step(3, alpha)
            x1 = s.get_state()
            assert s.layout()["K"] == K and s.layout()["threads"] == threads
            for r in range(R):
                err, _ = one_sweep_error(orc, g, x0[r], x1[r], alpha, 3, seed=6, replica=r, **_params_kw(s))
                assert err <= TOL_F32, (r, err)
            s.run(201, R, seed=9)
            out.append((x1, s.get_state(), s.replica_cuts()[0]))
        finally:
            for k in list(env) + ["COSM_SPLIT_W"]:
                os.environ.pop(k, None)
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("storage", [1, 2, 3])
@pytest.mark.parametrize("K", [2, 4, 8])
def test_signed_records_equal_split_16bit(cosm, orc, storage, K):
    # binary16, fixed point and bfloat16 edge lists read the records carrying
    # a +-1 weight's sign too: whole trials equal those with split records
    # and weights bit for bit, at every tile width and with checked batches
    # of every fill (96 threads against colours of every size)
    inst = instances.sparse_gnm(700, 2100, 5, wmax=1)
    col, C = orc.color_greedy(inst.n, inst.src, inst.dst)
    env = {"COSM_K": str(K), "COSM_THREADS": "96"}
    out = []
    for split in (False, True):
        os.environ.update(env)
        if split:
            os.environ["COSM_SPLIT_W"] = "1"
        try:
            s, _ = _solver(cosm, orc, inst, storage=storage, use_dims=False, color=col, C=C, dwt_ratio=1.0)
            s.run(201, 2 * K + 1, seed=9)
            assert s.layout()["K"] == K and s.layout()["threads"] == 96
            out.append((s.get_state(), s.replica_cuts()[0]))
        finally:
            for k in list(env) + ["COSM_SPLIT_W"]:
                os.environ.pop(k, None)
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_edge_cases(cosm, orc):
    # single edge, odd n, one replica, one bisector, weights up to 127
    s = cosm.Solver(3, [0], [2], [127], n_bisectors=1)
    s.run(5, 1, seed=0)
    cut, en, rep, spins = s.best()
    assert cut in (0, 127) and rep == 0
    # two-vertex FM, no DWT
    s = cosm.Solver(2, [0], [1], [-1], flags=cosm.NO_DWT)
    s.set_state(np.array([[0.30, 0.20]]))
    s.step(1, 0.01)
    np.testing.assert_allclose(s.get_state()[0], [0.29, 0.21], atol=1e-7)
    # invalid inputs are rejected before any device work
    with pytest.raises(cosm.CosmError):
        cosm.Solver(3, [0, 0], [1, 1], [1, 1])          # duplicate edge
    with pytest.raises(cosm.CosmError):
        cosm.Solver(3, [1], [0], [1])                   # not canonical
    with pytest.raises(cosm.CosmError):
        cosm.Solver(3, [0, 1], [1, 2], [1, 1], color=[0, 0], n_colors=1)  # not a matching
    with pytest.raises(cosm.CosmError):
        cosm.Solver(3, [0], [1], [0])                   # zero weight
    with pytest.raises(cosm.CosmError):
        cosm.Solver(100000, [0], [1], [1])              # too many vertices
    inst = instances.torus2d(16, 16, 0)
    with pytest.raises(cosm.CosmError):
        cosm.Solver(inst.n, inst.src, inst.dst, inst.w, dims=(16, 15))


def test_full_size_workload_sampled(cosm, orc):
    # the 20k-spin torus at the bench's launch configuration (1024 replicas),
    # short trial; sampled replicas checked against the oracle
    inst = instances.torus2d(100, 200, 0)
    s, g = _solver(cosm, orc, inst)
    s.run(60, 1024, seed=21)
    cuts, bps = s.replica_cuts()
    x = s.get_state()
    for r in (0, 1, 511, 1000, 1023):
        best, bp, _, _ = orc.binarize(g, x[r])
        assert cuts[r] == best and bps[r] == bp
    # one more sweep from the exported state, sampled replicas
    alpha = float(np.float32(0.013))
    s.step(61, alpha)
    x1 = s.get_state()
    kw = _params_kw(s)
    for r in (3, 700):
        err, _ = one_sweep_error(orc, g, x[r], x1[r], alpha, 61, seed=21, replica=r, **kw)
        assert err <= TOL_F32


@pytest.mark.parametrize("storage", [1, 3])
def test_full_size_workload_sampled_16bit(cosm, orc, storage):
    # the 20k-spin torus with binary16 / bfloat16 phases at the forms' launch
    # configuration (four replicas per CTA, 1024 replicas): sampled replicas'
    # cuts bit-exact on the final phases, and one more sweep against the
    # oracle's store-per-pass rounding
    inst = instances.torus2d(100, 200, 0)
    s, g = _solver(cosm, orc, inst, storage=storage)
    assert s.layout()["lattice"] == 2
    s.run(60, 1024, seed=22)
    assert s.layout()["K"] == 4
    cuts, bps = s.replica_cuts()
    x = s.get_state()
    for r in (0, 2, 513, 1022, 1023):
        best, bp, _, _ = orc.binarize(g, x[r])
        assert cuts[r] == best and bps[r] == bp
    alpha = float(np.float32(0.013))
    s.step(63, alpha)  # a twist sweep
    x1 = s.get_state()
    kw = _params_kw(s)
    mode, tol = (orc.STORE_F16_PASS, TOL_F16) if storage == 1 else (orc.STORE_BF16_PASS, TOL_BF16)
    for r in (5, 701):
        err, _ = one_sweep_error(orc, g, x[r], x1[r], alpha, 63, seed=22, replica=r, storage=mode, **kw)
        assert err <= tol


@pytest.mark.parametrize("K,flags", [(2, 0), (4, 0), (2, 4)])
def test_paired_f32_lattice_equals_scalar(cosm, orc, K, flags):
    # the f32x2 passes round every lane as the scalar binary32 passes do
    inst = instances.torus2d(24, 32, 5)
    os.environ["COSM_K"] = str(K)
    try:
        s = cosm.Solver.from_instance(inst, flags=flags, dwt_ratio=1.0)
        assert s.layout()["lattice"] == 2
        s.run(400, 3 * K, 21)
        x_pair, c_pair = s.get_state(), s.replica_cuts()[0]
        os.environ["COSM_SCALAR_F32"] = "1"
        s.run(400, 3 * K, 21)
        assert np.array_equal(s.get_state(), x_pair)
        assert np.array_equal(s.replica_cuts()[0], c_pair)
    finally:
        os.environ.pop("COSM_K", None)
        os.environ.pop("COSM_SCALAR_F32", None)


@pytest.mark.parametrize("storage", [1, 3])
@pytest.mark.parametrize("K,flags", [(2, 0), (4, 0), (8, 0), (4, 4)])
def test_paired_16bit_lattice_equals_scalar(cosm, orc, storage, K, flags):
    # binary16 / bfloat16 tiles in f32x2 lanes: every update is wrapped and
    # rounded through the storage type as in the scalar passes
    inst = instances.torus2d(24, 32, 5)
    os.environ["COSM_K"] = str(K)
    try:
        s = cosm.Solver.from_instance(inst, flags=flags, dwt_ratio=1.0, storage=storage)
        assert s.layout()["lattice"] == 2
        s.run(400, 3 * K, 21)
        assert s.layout()["K"] == K
        x_pair, c_pair = s.get_state(), s.replica_cuts()[0]
        os.environ["COSM_SCALAR_F32"] = "1"
        s.run(400, 3 * K, 21)
        assert np.array_equal(s.get_state(), x_pair)
        assert np.array_equal(s.replica_cuts()[0], c_pair)
    finally:
        os.environ.pop("COSM_K", None)
        os.environ.pop("COSM_SCALAR_F32", None)


@pytest.mark.parametrize("L1,L2,threads", [(24, 32, 64), (20, 36, 64), (16, 16, 32), (24, 32, 0), (6, 4, 0),
                                           (10, 28, 96), (8, 30, 0)])
def test_block_pairs_equal_single_blocks(cosm, orc, L1, L2, threads):
    # two-replica binary32 tiles take two 2x2 blocks per thread in the even
    # pass where the block rows have an even width; the phases and cuts equal
    # those of the one-block passes bit for bit, with the twist, wraps of
    # rows and columns, fixed and moving columns (forced thread counts), and
    # an odd width (one-block passes)
    inst = instances.torus2d(L1, L2, 9)
    os.environ["COSM_K"] = "2"
    if threads:
        os.environ["COSM_THREADS"] = str(threads)
    try:
        s = cosm.Solver.from_instance(inst, dwt_ratio=1.0)
        assert s.layout()["lattice"] == 2
        s.run(300, 6, 17)
        x_pair, c_pair = s.get_state(), s.replica_cuts()[0]
        os.environ["COSM_SINGLE_BLOCKS"] = "1"
        s.run(300, 6, 17)
        assert np.array_equal(s.get_state(), x_pair)
        assert np.array_equal(s.replica_cuts()[0], c_pair)
    finally:
        for k in ("COSM_K", "COSM_THREADS", "COSM_SINGLE_BLOCKS"):
            os.environ.pop(k, None)


@pytest.mark.parametrize("storage,dims,scalar", [(0, True, False), (0, True, True), (0, False, False),
                                                 (1, True, False), (1, False, False), (0, True, "K2")])
def test_exact_ties_follow_the_biased_sign(cosm, orc, storage, dims, scalar):
    # phases on a 1/16-turn grid make many pairs coincide (d = 0) or sit
    # exactly opposite (d = 1/2); with a step of 1/256 every operation is
    # exact in binary32, binary16 and FP64, so the sweep must match the
    # oracle bit for bit, ties included (both orientations of wrap edges)
    inst = instances.torus2d(16, 16, 3)
    s, g = _solver(cosm, orc, inst, storage=storage, use_dims=dims)
    R = 4
    rng = np.random.default_rng(5)
    x0 = rng.integers(0, 16, (R, inst.n)) / 16.0
    if scalar == "K2":
        # two-replica tiles: the block-pair passes
        os.environ["COSM_K"] = "2"
    elif scalar:
        os.environ["COSM_SCALAR_F32"] = "1"
    try:
        s.set_state(x0, seed=3)
        s.step(1, 1.0 / 256)
        x1 = s.get_state()
    finally:
        os.environ.pop("COSM_SCALAR_F32", None)
        os.environ.pop("COSM_K", None)
    for r in range(R):
        xo, ties = orc.sweep(g, x0[r], 1.0 / 256, 1, seed=3, replica=r, storage=storage,
                             tie_eps=1e-12, **_params_kw(s))
        assert len(ties) > 0
        assert np.array_equal(x1[r], xo), r


@pytest.mark.parametrize("storage", [0, 1, 2])
def test_edge_order_within_colours_changes_nothing(cosm, orc, storage):
    # the bank-spreading order of each colour class against the plain
    # source-slot order: a colour is a matching, so trials are identical
    inst = instances.sparse_gnm(3000, 9000, 4)
    col, C = orc.color_greedy(inst.n, inst.src, inst.dst)
    kw = dict(color=col, n_colors=C, storage=storage, dwt_ratio=1.0)
    a = cosm.Solver(inst.n, inst.src, inst.dst, inst.w, **kw)
    a.run(200, 6, 9)
    os.environ["COSM_SRC_ORDER"] = "1"
    try:
        b = cosm.Solver(inst.n, inst.src, inst.dst, inst.w, **kw)
    finally:
        os.environ.pop("COSM_SRC_ORDER", None)
    b.run(200, 6, 9)
    assert np.array_equal(a.get_state(), b.get_state())
    assert np.array_equal(a.replica_cuts()[0], b.replica_cuts()[0])


def test_quality_at_ten_thousand_spins(cosm, orc):
    # the unfrustrated gauge-planted 100 x 100 torus reaches its known
    # optimum; the +-J 100 x 100 glass reaches a ground-energy density near
    # the paper's -1.40 for its toroidal glasses (Section III-A)
    inst = instances.gauge_planted(instances.torus2d(100, 100, 5), 6)
    s = cosm.Solver.from_instance(inst, alpha0_deg=25.0, dwt_ratio=1.0)
    s.run(10000, 256, 3)
    cut, energy, rep, spins = s.best()
    assert (cut, energy) == (inst.meta["opt_cut"], inst.meta["ground_energy"])
    glass = instances.torus2d(100, 100, 0)
    s = cosm.Solver.from_instance(glass)
    s.run(20000, 1024, 4)
    cut, energy, rep, spins = s.best()
    assert energy / glass.n < -1.395
    assert orc.energy(glass.src, glass.dst, glass.w, spins) == energy
