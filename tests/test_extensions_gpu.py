"""GPU parity of the single-instance extensions: local fields (eq. (1)),
the drawn twist direction, the optimal bisector and mid-anneal tracking.

Bars: readouts (cuts, energies, bisector positions, spins) bit-exact on
replayed states; whole fixed-point trials (phases, trace, kept readout)
bit-exact; one FP32 sweep with fields within 1e-5 rad, near-ties either
branch."""
import numpy as np
import pytest

import instances
from parity_util import TOL_F32, one_sweep_error

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


def _fields(n, seed, lo=-4, hi=5):
    return np.random.default_rng(seed).integers(lo, hi, n).astype(np.int32)


def _coloured(orc, inst, use_dims=True):
    col, C = orc.color_instance(inst) if use_dims else orc.color_greedy(inst.n, inst.src, inst.dst)
    return col, C, orc.ColouredGraph(inst.n, inst.src, inst.dst, inst.w, col, C)


# ------------------------------------------------------------------ local fields

@pytest.mark.parametrize("storage", [0, 2])
def test_field_readout_bit_exact(cosm, orc, storage):
    inst = instances.sparse_gnm(3001, 9000, 4)
    h = _fields(inst.n, 1)
    col, C, g = _coloured(orc, inst)
    s = cosm.Solver(inst.n, inst.src, inst.dst, inst.w, color=col, n_colors=C, h=h, storage=storage)
    R = 7
    x0 = np.stack([orc.init_phases(inst.n, 3, r) for r in range(R)])
    if storage == 2:
        x0 = orc.q16_grid(x0)
    s.set_state(x0)
    s.readout()
    x = s.get_state()
    cuts, bps = s.replica_cuts()
    en = s.replica_energies()
    B = s.replica_bisectors()
    for r in range(R):
        H, c, sp = orc.readout_fields(g, h, x[r])
        assert (cuts[r], en[r], bps[r], B[r]) == (c, H, -1, 0xC0000000), r
    cut, energy, rep, spins = s.best()
    assert energy == en.min() and rep == int(np.argmin(en))
    assert orc.energy_h(inst.n, inst.src, inst.dst, inst.w, h, spins) == energy


@pytest.mark.parametrize("flags", [0, 2])
def test_field_one_sweep_f32(cosm, orc, flags):
    inst = instances.random_regular(1200, 3, 5)
    h = _fields(inst.n, 2)
    col, C, g = _coloured(orc, inst)
    s = cosm.Solver(inst.n, inst.src, inst.dst, inst.w, color=col, n_colors=C, h=h, flags=flags,
                    dwt_ratio=1.0)
    assert s.layout()["lattice"] == 0
    R = 4
    x0 = np.stack([orc.init_phases(inst.n, 9, r) for r in range(R)])
    for sweep in (1, 3):
        s.set_state(x0, seed=9)
        alpha = float(np.float32(0.0123))
        s.step(sweep, alpha)
        x1 = s.get_state()
        for r in range(R):
            err, ties = one_sweep_error(orc, g, x0[r], x1[r], alpha, sweep, seed=9, replica=r,
                                        dwt_ratio=1.0, flags=flags, h=h)
            assert err < TOL_F32, (sweep, r, err, ties)


CASES_Q = [
    ("torus_fields", lambda: instances.torus2d(16, 16, 0), True, 1),
    ("gnm_fields", lambda: instances.sparse_gnm(500, 1500, 2), False, 2),
    ("reg3_fields_noscs", lambda: instances.random_regular(400, 3, 3), False, 3),
]


@pytest.mark.parametrize("name,make,dims,fseed", CASES_Q, ids=[c[0] for c in CASES_Q])
def test_fixed_point_trials_with_fields_bit_exact(cosm, orc, name, make, dims, fseed):
    inst = make()
    h = _fields(inst.n, fseed)
    col, C, g = _coloured(orc, inst, dims)
    flags = cosm.NO_SCS if "noscs" in name else 0
    s = cosm.Solver(inst.n, inst.src, inst.dst, inst.w, color=col, n_colors=C, h=h, storage=cosm.Q16,
                    dwt_ratio=1.0, flags=flags)
    S, R, seed = 140, 6, 17
    s.run(S, R, seed)
    x = s.get_state()
    en = s.replica_energies()
    cuts, _ = s.replica_cuts()
    out, _, xo, _ = orc.trials_ex(g, S, R, dwt_ratio=1.0, seed=seed, storage=orc.STORE_Q16, h=h,
                                  flags=flags, keep_x=True)
    assert np.array_equal(x, xo), name
    assert np.array_equal(en, out[:, 1]) and np.array_equal(cuts, out[:, 0])
    cut, energy, rep, spins = s.best()
    assert energy == out[:, 1].min()
    assert orc.energy_h(inst.n, inst.src, inst.dst, inst.w, h, spins) == energy


# ------------------------------------------------------------------ twist direction

@pytest.mark.parametrize("dims", [True, False])
def test_random_twist_direction_bit_exact(cosm, orc, dims):
    inst = instances.torus2d(16, 20, 6)
    col, C, g = _coloured(orc, inst, dims)
    s = cosm.Solver.from_instance(inst, color=col, n_colors=C, use_dims=dims, storage=cosm.Q16,
                                  dwt_ratio=1.5, flags=cosm.DWT_RANDOM_DIR)
    assert s.layout()["lattice"] == (2 if dims else 0)
    S, R, seed = 120, 6, 8
    s.run(S, R, seed)
    out, _, xo, _ = orc.trials_ex(g, S, R, dwt_ratio=1.5, seed=seed, storage=orc.STORE_Q16,
                                  flags=orc.DWT_RANDDIR, keep_x=True)
    assert np.array_equal(s.get_state(), xo)
    # the drawn direction changes the trajectory
    plain, _, xp, _ = orc.trials_ex(g, S, R, dwt_ratio=1.5, seed=seed, storage=orc.STORE_Q16, keep_x=True)
    assert not np.array_equal(xo, xp)


# ------------------------------------------------------------------ optimal bisector

@pytest.mark.parametrize("storage", [0, 1, 2])
def test_optimal_bisector_readout_bit_exact(cosm, orc, storage):
    inst = instances.sparse_gnm(5003, 15000, 7, wmax=3)
    col, C, g = _coloured(orc, inst)
    s = cosm.Solver(inst.n, inst.src, inst.dst, inst.w, color=col, n_colors=C, storage=storage,
                    flags=cosm.OPT_BISECTOR)
    R = 9
    x0 = np.stack([orc.init_phases(inst.n, 5, r) for r in range(R)])
    x0[3] = np.round(x0[3] * 64) / 64 % 1.0  # repeated positions and exact antipodes
    s.set_state(x0)
    s.readout()
    x = s.get_state()
    cuts, bps = s.replica_cuts()
    B = s.replica_bisectors()
    en = s.replica_energies()
    W = int(np.sum(inst.w))
    for r in range(R):
        c, b, sp = orc.binarize_opt(g, x[r])
        assert (cuts[r], B[r], bps[r], en[r]) == (c, b, -1, W - 2 * c), r
        assert c >= orc.binarize(g, x[r])[0]
    cut, energy, rep, spins = s.best()
    assert cut == cuts.max() and orc.cut(inst.src, inst.dst, inst.w, spins) == cut


def test_optimal_bisector_after_trials(cosm, orc):
    inst = instances.torus2d(40, 50, 3)
    s = cosm.Solver.from_instance(inst, flags=cosm.OPT_BISECTOR)
    S, R = 400, 37
    s.run(S, R, 5)
    assert s.layout()["launches"] == 3
    x = s.get_state()
    cuts, _ = s.replica_cuts()
    B = s.replica_bisectors()
    g = orc.coloured(inst)
    for r in range(R):
        c, b, _ = orc.binarize_opt(g, x[r])
        assert (cuts[r], B[r]) == (c, b)
    plain = cosm.Solver.from_instance(inst)
    plain.run(S, R, 5)
    assert np.array_equal(plain.get_state(), x)
    assert (cuts >= plain.replica_cuts()[0]).all()


# ------------------------------------------------------------------ tracking

@pytest.mark.parametrize("name,make,dims,flags", [
    ("torus_lattice", lambda: instances.torus2d(16, 16, 0), True, 0),
    ("gnm", lambda: instances.sparse_gnm(600, 1800, 2), False, 0),
    ("gnm_opt", lambda: instances.sparse_gnm(600, 1800, 2), False, 8),
    ("reg3_fields", lambda: instances.random_regular(500, 3, 4), False, 0),
])
def test_fixed_point_tracking_bit_exact(cosm, orc, name, make, dims, flags):
    inst = make()
    h = _fields(inst.n, 6) if "fields" in name else None
    col, C, g = _coloured(orc, inst, dims)
    T, S, R, seed = 25, 160, 7, 3
    s = cosm.Solver(inst.n, inst.src, inst.dst, inst.w, color=col, n_colors=C,
                    dims=inst.dims if dims else (), h=h, storage=cosm.Q16, dwt_ratio=1.0,
                    flags=flags, track_period=T)
    s.run(S, R, seed)
    tr = s.trace()
    out, otr, xo, osp = orc.trials_ex(g, S, R, dwt_ratio=1.0, seed=seed, storage=orc.STORE_Q16,
                                      track=T, h=h, flags=flags, keep_x=True, keep_spins=True)
    assert tr.shape == (R, -(-S // T))
    assert np.array_equal(tr, otr), name
    assert np.array_equal(s.get_state(), xo)
    cuts, bps = s.replica_cuts()
    assert np.array_equal(cuts, out[:, 0]) and np.array_equal(s.replica_energies(), out[:, 1])
    assert np.array_equal(s.replica_bisectors(), out[:, 2].astype(np.uint32))
    assert np.array_equal(bps, out[:, 3])
    cut, energy, rep, spins = s.best()
    assert energy == out[:, 1].min() and rep == int(np.argmin(out[:, 1]))
    assert np.array_equal(spins, osp[rep])


def test_tracking_does_not_change_the_trajectory_f32(cosm, orc):
    inst = instances.torus2d(32, 32, 9)
    a = cosm.Solver.from_instance(inst, track_period=50)
    b = cosm.Solver.from_instance(inst)
    S, R = 520, 20
    a.run(S, R, 4)
    b.run(S, R, 4)
    assert np.array_equal(a.get_state(), b.get_state())
    tr = a.trace()
    W = int(np.sum(inst.w))
    cb, _ = b.replica_cuts()
    assert np.array_equal(tr[:, -1], W - 2 * cb)
    assert np.array_equal(a.replica_energies(), tr.min(axis=1))
    cut, energy, rep, spins = a.best()
    assert orc.energy(inst.src, inst.dst, inst.w, spins) == energy == tr.min()


def test_trace_requires_tracking(cosm):
    inst = instances.torus2d(16, 16, 0)
    s = cosm.Solver.from_instance(inst)
    s.run(10, 4, 1)
    with pytest.raises(cosm.CosmError):
        s.trace()
