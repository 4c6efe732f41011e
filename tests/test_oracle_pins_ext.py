"""Pins of the oracle's local fields, twist direction, optimal bisector and
mid-anneal tracking against hand-worked cases, closed forms, invariants and
brute force (not against the oracle itself)."""
import itertools

import numpy as np
import pytest

import instances

A = 0.01


def _graph(orc, n, edges, colors):
    src = [min(a, b) for a, b, _ in edges]
    dst = [max(a, b) for a, b, _ in edges]
    w = [wt for _, _, wt in edges]
    return orc.ColouredGraph(n, src, dst, w, colors, max(colors) + 1 if colors else 0)


def _empty(orc, n):
    return orc.ColouredGraph(n, [], [], [], [], 0)


# ------------------------------------------------------------------ local fields

def test_field_moves_vertex_towards_reference_or_away(orc):
    # eq. (6) with the partner frozen at 0 and J = h: a positive field pulls
    # x towards 0 by alpha h along the shorter way, a negative one pushes it
    # towards 1/2
    g = _empty(orc, 4)
    x0 = [0.1, 0.9, 0.1, 0.5]
    h = [2, 2, -2, 1]
    x, _ = orc.sweep(g, x0, A, 1, flags=orc.NO_DWT, h=h)
    np.testing.assert_allclose(x, [0.08, 0.92, 0.12, 0.51], atol=1e-15)
    # a zero field leaves the vertex alone
    x, _ = orc.sweep(g, x0, A, 1, flags=orc.NO_DWT, h=[0, 0, 0, 0])
    np.testing.assert_array_equal(x, x0)


def test_field_subsweep_follows_the_colours(orc):
    # one ferromagnetic edge (w = -1) and a field on vertex 0, with the field
    # step flipping the sign of the edge difference: colour first gives
    # (0.29, 0.315); field first would give (0.31, 0.295)
    g = _graph(orc, 2, [(0, 1, -1)], [0])
    x, _ = orc.sweep(g, [0.31, 0.305], A, 1, flags=orc.NO_DWT, h=[1, 0])
    np.testing.assert_allclose(x, [0.29, 0.315], atol=1e-15)
    # simultaneous step (NO_SCS): both forces from the old state
    x, _ = orc.sweep(g, [0.31, 0.305], A, 1, flags=orc.NO_DWT | orc.NO_SCS, h=[1, 0])
    np.testing.assert_allclose(x, [0.29, 0.315], atol=1e-15)
    x, _ = orc.sweep(g, [0.30, 0.305], A, 1, flags=orc.NO_DWT | orc.NO_SCS, h=[1, 0])
    np.testing.assert_allclose(x, [0.30, 0.295], atol=1e-15)


def test_field_readout_is_the_half_circle_around_the_reference(orc):
    g = _empty(orc, 6)
    x = [0.2, 0.25, 0.75, 0.7499, 0.0, 0.5]
    H, c, s = orc.readout_fields(g, [1, 1, 1, 1, 1, 1], x)
    assert list(s) == [1, -1, 1, -1, 1, -1]
    assert c == 0 and H == -sum(s)


def test_energy_with_fields_closed_forms_and_flip_identity(orc):
    # ferromagnetic path with a uniform field: all up costs -(n-1) - n h
    n = 9
    src, dst = np.arange(n - 1), np.arange(1, n)
    w = -np.ones(n - 1, dtype=np.int32)
    assert orc.energy_h(n, src, dst, w, [3] * n, np.ones(n, np.int8)) == -(n - 1) - 3 * n
    # H(s) - H(-s) = -2 sum h s and H(s) + H(-s) = 2 sum w s_i s_j
    inst = instances.sparse_gnm(40, 90, 3)
    rng = np.random.default_rng(1)
    h = rng.integers(-5, 6, inst.n)
    for _ in range(5):
        s = rng.choice([-1, 1], inst.n).astype(np.int8)
        Hp = orc.energy_h(inst.n, inst.src, inst.dst, inst.w, h, s)
        Hm = orc.energy_h(inst.n, inst.src, inst.dst, inst.w, h, -s)
        assert Hp - Hm == -2 * int(np.dot(h, s))
        assert Hp + Hm == 2 * orc.energy(inst.src, inst.dst, inst.w, s)


def test_fields_alone_are_solved_exactly(orc):
    # no edges: every vertex settles in the half of its field's sign
    g = _empty(orc, 50)
    h = np.random.default_rng(2).choice([-5, -3, -1, 1, 2, 4], 50)
    r = orc.trial_ex(g, 300, h=h, seed=3)
    assert np.array_equal(r["spins"], np.sign(h).astype(np.int8))
    assert r["energy"] == -int(np.abs(h).sum())


def _bruteforce_ising(n, src, dst, w, h):
    best = None
    for bits in itertools.product([-1, 1], repeat=n):
        s = np.array(bits)
        H = int(np.sum(np.asarray(w) * s[src] * s[dst]) - np.dot(h, s))
        best = H if best is None else min(best, H)
    return best


def test_trials_with_fields_reach_bruteforce_ground_state(orc):
    inst = instances.sparse_gnm(12, 20, 5)
    h = np.random.default_rng(4).integers(-3, 4, inst.n)
    g = orc.coloured(inst)
    out, *_ = orc.trials_ex(g, 500, 16, h=h, seed=7, dwt_ratio=1.0)
    ground = _bruteforce_ising(inst.n, inst.src, inst.dst, inst.w, h)
    assert out[:, 1].min() == ground
    assert (out[:, 1] >= ground).all()


def test_fixed_point_with_fields_equals_fp64_on_grid(orc):
    inst = instances.random_regular(200, 3, 8)
    g = orc.coloured(inst)
    h = np.random.default_rng(5).integers(-4, 5, inst.n)
    x0 = orc.q16_grid(orc.init_phases(inst.n, 4, 1))
    a = 300 / 65536
    for s in (1, 2, 3):
        xq, _ = orc.sweep(g, x0, a, s, seed=4, replica=1, dwt_ratio=1.0, storage=orc.STORE_Q16, h=h)
        xf, _ = orc.sweep(g, x0, a, s, seed=4, replica=1, dwt_ratio=1.0, h=h)
        assert np.array_equal(xq, xf)
        x0 = xq


# ------------------------------------------------------------------ twist direction

def test_twist_direction_is_word1_top_bit(orc):
    for seed, r, s in ((0, 0, 1), (7, 3, 12), (2 ** 40 + 5, 99, 3000)):
        o = orc.philox4x32_10([s, r, 0, 1], [seed & 0xFFFFFFFF, seed >> 32])
        assert orc.twist_dir(seed, r, s) == (1 if int(o[1]) < 2 ** 31 else -1)
    d = [orc.twist_dir(11, r, s) for r in range(10) for s in range(1, 401)]
    assert abs(np.mean(d)) < 0.1


def test_random_twist_moves_the_window_by_the_drawn_direction(orc):
    g = _empty(orc, 1)
    seed, step_ratio = 5, 1.0
    for s in range(3, 60, 3):
        th = orc.theta(seed, 0, s)
        x0 = (th + 0.01) % 1.0  # inside the window around theta
        d = orc.twist_dir(seed, 0, s)
        x, _ = orc.sweep(g, [x0], A, s, dwt_period=3, dwt_ratio=step_ratio, seed=seed,
                         flags=orc.DWT_RANDDIR)
        assert x[0] == pytest.approx((x0 + d * step_ratio * A) % 1.0, abs=1e-15)
        x, _ = orc.sweep(g, [x0], A, s, dwt_period=3, dwt_ratio=step_ratio, seed=seed)
        assert x[0] == pytest.approx((x0 + step_ratio * A) % 1.0, abs=1e-15)


# ------------------------------------------------------------------ optimal bisector

def test_optimal_bisector_hand_cases(orc):
    # two vertices joined by w = 1 at 0.1 and 0.2 turn: cut 1 from the first
    # position past vertex 0
    g = _graph(orc, 2, [(0, 1, 1)], [0])
    c, B, s = orc.binarize_opt(g, [0.1, 0.2])
    assert c == 1 and B == int(np.floor(0.1 * 2 ** 32)) + 1
    assert s[0] != s[1]
    # antiferromagnetic triangle at 0, 1/3, 2/3: every bisector cuts 2
    t = _graph(orc, 3, [(0, 1, 1), (1, 2, 1), (0, 2, 1)], [0, 1, 2])
    c, B, _ = orc.binarize_opt(t, [0.0, 1 / 3, 2 / 3])
    assert c == 2 and B == 0


def test_optimal_bisector_sorted_sweep_equals_brute_force(orc):
    rng = np.random.default_rng(3)
    for k in range(12):
        inst = instances.sparse_gnm(30 + 5 * k, 70 + 7 * k, k, wmax=3)
        g = orc.coloured(inst)
        x = orc.init_phases(inst.n, 100 + k, 0)
        if k % 3 == 0:  # repeated points and exact antipodes
            x = np.round(x * 16) / 16 % 1.0
        c1, B1, s1 = orc.binarize_opt(g, x)
        c2, B2, s2 = orc.binarize_opt(g, x, brute=True)
        assert (c1, B1) == (c2, B2)
        assert np.array_equal(s1, s2)
        assert orc.cut(g.src, g.dst, g.w, s1) == c1
        # no bisector position beats it, and the P-bisector readouts are bounded by it
        for B in rng.integers(0, 2 ** 31, 300):
            s = np.where(((np.floor(x * 2 ** 32).astype(np.uint64) - np.uint64(B)) % 2 ** 32) < 2 ** 31,
                         1, -1).astype(np.int8)
            assert orc.cut(g.src, g.dst, g.w, s) <= c1
        for P in (1, 7, 100, 256):
            assert orc.binarize(g, x, P)[0] <= c1


def test_optimal_bisector_equals_bisectors_on_antipodal_clusters(orc):
    inst = instances.gauge_planted(instances.torus2d(12, 12, 1), 2)
    g = orc.coloured(inst)
    tau = inst.meta["tau"]
    x = np.where(tau > 0, 0.3, 0.8)
    c, _, s = orc.binarize_opt(g, x)
    assert c == inst.meta["opt_cut"] == orc.binarize(g, x)[0]


# ------------------------------------------------------------------ tracking

def test_tracking_trace_is_the_readouts_of_the_sweeps(orc):
    inst = instances.torus2d(10, 10, 3)
    g = orc.coloured(inst)
    S, T, seed = 130, 20, 9
    r = orc.trial_ex(g, S, track=T, seed=seed, replica=2)
    # replay the same trajectory one sweep at a time and read out by hand
    x = orc.init_phases(g.n, seed, 2)
    W = int(np.sum(inst.w))
    trace = []
    for s in range(1, S + 1):
        x, _ = orc.sweep(g, x, orc.alpha(s, S, 14 / 360), s, seed=seed, replica=2)
        if s % T == 0 or s == S:
            trace.append(W - 2 * orc.binarize(g, x)[0])
    assert list(r["trace"]) == trace
    assert len(trace) == -(-S // T)
    k = int(np.argmin(trace))
    assert r["energy"] == trace[k] and r["sweep"] == min((k + 1) * T, S)
    assert r["cut"] == (W - r["energy"]) // 2
    assert orc.cut(g.src, g.dst, g.w, r["spins"]) == r["cut"]
    np.testing.assert_array_equal(r["x"], x)


def test_tracking_off_equals_the_plain_trial(orc):
    inst = instances.sparse_gnm(60, 150, 2)
    g = orc.coloured(inst)
    best, x, spins, bp = orc.trial(g, 200, seed=4, replica=1)
    r = orc.trial_ex(g, 200, seed=4, replica=1)
    assert (r["cut"], r["p"], r["sweep"]) == (best, bp, 200)
    assert r["B"] == (bp << 31) // 100
    np.testing.assert_array_equal(r["spins"], spins)
    # one readout at the end equals no tracking
    r1 = orc.trial_ex(g, 200, seed=4, replica=1, track=200)
    assert (r1["cut"], r1["energy"], r1["B"]) == (r["cut"], r["energy"], r["B"])


def test_optimal_bisector_readout_in_trials(orc):
    inst = instances.sparse_gnm(80, 200, 6)
    g = orc.coloured(inst)
    for track in (0, 50):
        r = orc.trial_ex(g, 200, seed=2, track=track, flags=orc.OPT_BISECTOR)
        plain = orc.trial_ex(g, 200, seed=2, track=track)
        c, B, s = orc.binarize_opt(g, r["x"])
        assert r["cut"] >= plain["cut"]
        if track == 0:
            assert (r["cut"], r["B"], r["p"]) == (c, B, -1)
            np.testing.assert_array_equal(r["spins"], s)
        else:
            assert r["energy"] == min(plain["energy"], int(np.sum(inst.w)) - 2 * c)
