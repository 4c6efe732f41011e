"""Pins of the FP64 oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: published
known-answer values, values printed in the paper, hand-worked cases of the
paper's equations, closed forms, invariants, library routines and brute
force. A dropped term, a wrong sign, a swapped index or a wrong colour order
in the oracle fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

import instances

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
A14 = 14.0 / 360.0  # alpha_0 = 14 degrees (Table IX), in turns


def _graph(orc, n, edges, colors):
    src = [min(a, b) for a, b, _ in edges]
    dst = [max(a, b) for a, b, _ in edges]
    w = [wt for _, _, wt in edges]
    return orc.ColouredGraph(n, src, dst, w, colors, max(colors) + 1 if colors else 0)


def _circ(a, b):
    d = (np.asarray(a) - np.asarray(b)) % 1.0
    return np.minimum(d, 1.0 - d)


# ------------------------------------------------------------------ Philox

def test_philox_known_answers(orc):
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox_kat.txt")) if l[0] != "#"]
    assert len(rows) == 3
    for r in rows:
        vals = [int(t, 16) for t in r]
        out = orc.philox4x32_10(vals[0:4], vals[4:6])
        assert [int(v) for v in out] == vals[6:10]


def test_init_phases_are_24bit_uniform(orc):
    x = orc.init_phases(40000, seed=7, replica=3)
    assert (x >= 0).all() and (x < 1).all()
    q = x * 2 ** 24
    assert np.array_equal(q, np.floor(q))
    # uniform: mean 1/2, variance 1/12 within sampling error
    assert abs(x.mean() - 0.5) < 5 * math.sqrt(1 / 12 / x.size)
    assert abs(x.var() - 1 / 12) < 0.003
    # replicas and seeds give different streams; same inputs give the same state
    assert not np.array_equal(x, orc.init_phases(40000, 7, 4))
    assert not np.array_equal(x, orc.init_phases(40000, 8, 3))
    assert np.array_equal(x, orc.init_phases(40000, 7, 3))


def test_theta_uniform_and_keyed(orc):
    th = np.array([orc.theta(11, r, s) for r in range(20) for s in range(1, 200)])
    assert (th >= 0).all() and (th < 1).all()
    assert abs(th.mean() - 0.5) < 0.03
    assert orc.theta(11, 0, 3) != orc.theta(11, 1, 3) != orc.theta(12, 1, 3)


# ------------------------------------------------------------------ schedule

def test_alpha_linear_ramp_to_zero(orc):
    S = 1000
    a = np.array([orc.alpha(s, S, A14) for s in range(1, S + 1)])
    assert a[0] == A14 and a[-1] == 0.0
    np.testing.assert_allclose(np.diff(a), -A14 / (S - 1), rtol=1e-9)
    assert orc.alpha(1, 1, A14) == A14


# ------------------------------------------------------------------ eq. (4), wrap

def test_wrap_is_mod_one(orc):
    for y in [0.0, 0.25, 0.999, 1.0, 1.25, -0.25, -1e-300, -0.999, 1.9]:
        r = orc.wrap(y)
        assert 0.0 <= r < 1.0
        assert _circ(r, y % 1.0) < 1e-15 or (y % 1.0 == 1.0 and r == 0.0)
    assert orc.wrap(-1e-300) == 0.0  # rounds to 1.0, which is the point 0


def test_biased_sign_on_minimum_difference(orc):
    deg = 1 / 360
    assert orc.sgn_b(10 * deg, 350 * deg) == 1      # min difference +20 degrees
    assert orc.sgn_b(350 * deg, 10 * deg) == -1     # min difference -20 degrees
    assert orc.sgn_b(0.3, 0.3) == 1                 # eq. (4): >= 0 gives +1
    assert orc.sgn_b(0.75, 0.25) == -1              # exactly opposite: d = -1/2
    assert orc.sgn_b(0.25, 0.75) == -1
    assert orc.sgn_b(0.2, 0.1) == 1 and orc.sgn_b(0.1, 0.2) == -1


# ------------------------------------------------------------------ eq. (6), SCS

def test_two_vertex_ferro_closes_anti_opens(orc):
    a = 0.01
    fm = _graph(orc, 2, [(0, 1, -1)], [0])  # w = -1 -> J = +1 (FM)
    x, _ = orc.sweep(fm, [0.30, 0.20], a, 1, flags=orc.NO_DWT)
    np.testing.assert_allclose(x, [0.29, 0.21], atol=1e-15)
    af = _graph(orc, 2, [(0, 1, 1)], [0])   # w = +1 -> J = -1 (AFM)
    x, _ = orc.sweep(af, [0.30, 0.20], a, 1, flags=orc.NO_DWT)
    np.testing.assert_allclose(x, [0.31, 0.19], atol=1e-15)
    # weight magnitude scales the step (J taken literally in eq. (6))
    fm3 = _graph(orc, 2, [(0, 1, -3)], [0])
    x, _ = orc.sweep(fm3, [0.30, 0.20], a, 1, flags=orc.NO_DWT)
    np.testing.assert_allclose(x, [0.27, 0.23], atol=1e-15)


def test_exact_coincidence_uses_biased_branch(orc):
    # d = 0 -> sgn_b = +1 -> x_i moves by -alpha J, x_j by +alpha J
    fm = _graph(orc, 2, [(0, 1, -1)], [0])
    x, _ = orc.sweep(fm, [0.5, 0.5], 0.01, 1, flags=orc.NO_DWT)
    np.testing.assert_allclose(x, [0.49, 0.51], atol=1e-15)


def test_pair_update_uses_minimum_angular_difference(orc):
    # x_a is 0.01 turn behind x_b across the 0/1 seam: FM pulls them across it
    fm = _graph(orc, 2, [(0, 1, -1)], [0])
    x, _ = orc.sweep(fm, [0.995, 0.005], 0.01, 1, flags=orc.NO_DWT)
    assert _circ(x[0], 0.005) < 1e-12 and _circ(x[1], 0.995) < 1e-12


def test_colour_order_is_applied_in_sequence(orc):
    # path a-b-c: (a,b) colour 0 FM, (b,c) colour 1 AFM; hand-worked result of
    # applying colour 0 then colour 1 (eqs. (11)-(12)); the reverse order
    # gives (0.09, 0.105, 0.31), so this fails if the order is wrong.
    g = _graph(orc, 3, [(0, 1, -1), (1, 2, 1)], [0, 1])
    x, _ = orc.sweep(g, [0.1, 0.105, 0.3], 0.01, 1, flags=orc.NO_DWT)
    np.testing.assert_allclose(x, [0.11, 0.085, 0.31], atol=1e-15)
    g2 = _graph(orc, 3, [(0, 1, -1), (1, 2, 1)], [1, 0])
    x2, _ = orc.sweep(g2, [0.1, 0.105, 0.3], 0.01, 1, flags=orc.NO_DWT)
    np.testing.assert_allclose(x2, [0.09, 0.105, 0.31], atol=1e-15)


def test_alpha_zero_is_identity(orc):
    inst = instances.torus2d(8, 8, 1)
    g = orc.coloured(inst)
    x0 = orc.init_phases(inst.n, 3, 0)
    x, _ = orc.sweep(g, x0, 0.0, 3, dwt_period=3, dwt_ratio=1.0, seed=3)
    assert np.array_equal(x, x0)


def test_edge_order_inside_a_colour_is_free(orc):
    inst = instances.random_regular(200, 3, 5)
    col, Cn = orc.color_greedy(inst.n, inst.src, inst.dst)
    g = orc.ColouredGraph(inst.n, inst.src, inst.dst, inst.w, col, Cn)
    rng = np.random.default_rng(0)
    perm = rng.permutation(inst.m)
    gp = orc.ColouredGraph(inst.n, inst.src[perm], inst.dst[perm], inst.w[perm], col[perm], Cn)
    x0 = orc.init_phases(inst.n, 9, 1)
    for s in (1, 2, 3):
        a, _ = orc.sweep(g, x0, 0.03, s, seed=9, replica=1)
        b, _ = orc.sweep(gp, x0, 0.03, s, seed=9, replica=1)
        assert np.array_equal(a, b)
        x0 = a


def test_sweep_is_deterministic(orc):
    inst = instances.torus2d(16, 16, 2)
    g = orc.coloured(inst)
    x0 = orc.init_phases(inst.n, 1, 5)
    a, _ = orc.sweep(g, x0, 0.02, 6, seed=1, replica=5)
    b, _ = orc.sweep(g, x0, 0.02, 6, seed=1, replica=5)
    assert np.array_equal(a, b)


# ------------------------------------------------------------------ DWT

def test_dwt_window_is_half_of_phase_space(orc):
    # 90-degree windows cover exactly half of the circle (Section II-D)
    xs = np.arange(2 ** 14) / 2 ** 14
    for th in (0.0, 0.3, 0.71234, 1 - 2 ** -24):
        inside = sum(orc.in_window(float(x), th, 0.25) for x in xs)
        assert inside == 2 ** 13


def test_dwt_hand_cases(orc):
    seed, r, s = 21, 2, 6
    th = orc.theta(seed, r, s)
    pts = [th + 0.1, th + 0.5 + 0.12, th + 0.13, th - 0.125, th + 0.125, th + 0.5 - 0.126]
    expect = [1, 1, 0, 1, 0, 0]
    x0 = np.array([p % 1.0 for p in pts])
    empty = orc.ColouredGraph(len(pts), [], [], [], np.zeros(0, dtype=np.int64), 0)
    alpha, ratio = 0.02, 1.5
    x, _ = orc.sweep(empty, x0, alpha, s, dwt_period=3, dwt_ratio=ratio, seed=seed, replica=r)
    moved = _circ(x, x0) > 0
    assert list(moved.astype(int)) == expect
    # every twisted phase moves by the same +ratio*alpha, counter-clockwise
    np.testing.assert_allclose(((x - x0) % 1.0)[moved], ratio * alpha, atol=1e-12)
    # no DWT on a sweep that is not a multiple of the period, or with ratio 0
    x2, _ = orc.sweep(empty, x0, alpha, s + 1, dwt_period=3, dwt_ratio=ratio, seed=seed, replica=r)
    assert np.array_equal(x2, x0)
    x3, _ = orc.sweep(empty, x0, alpha, s, dwt_period=3, dwt_ratio=0.0, seed=seed, replica=r)
    assert np.array_equal(x3, x0)


# ------------------------------------------------------------------ colourings

def test_greedy_colouring_hand_cases(orc):
    # star: three edges at one vertex -> colours 0, 1, 2
    col, Cn = orc.color_greedy(4, [0, 0, 0], [1, 2, 3])
    assert list(col) == [0, 1, 2] and Cn == 3
    # path a-b-c-d in order -> 0, 1, 0
    col, Cn = orc.color_greedy(4, [0, 1, 2], [1, 2, 3])
    assert list(col) == [0, 1, 0] and Cn == 2


def test_greedy_colouring_is_a_partition_into_matchings(orc):
    for inst in (instances.random_regular(1000, 4, 1), instances.sparse_gnm(800, 2000, 2)):
        col, Cn = orc.color_greedy(inst.n, inst.src, inst.dst)
        deg = np.bincount(np.concatenate([inst.src, inst.dst]), minlength=inst.n).max()
        assert Cn <= 2 * deg - 1
        assert orc.validate_partition(inst.n, inst.src, inst.dst, Cn, col) == 0


def test_torus_colouring_gives_perfect_matchings(orc):
    inst = instances.torus2d(16, 16, 0)
    col, Cn = orc.color_torus2d(16, 16, inst.src, inst.dst)
    assert Cn == 4
    assert list(np.bincount(col)) == [128] * 4     # every vertex in every sub-sweep
    assert orc.validate_partition(inst.n, inst.src, inst.dst, 4, col) == 0
    inst3 = instances.torus3d(4, 6, 8, 0)
    col3, C3 = orc.color_torus3d(4, 6, 8, inst3.src, inst3.dst)
    assert C3 == 6 and list(np.bincount(col3)) == [inst3.n // 2] * 6
    assert orc.validate_partition(inst3.n, inst3.src, inst3.dst, 6, col3) == 0


def test_partition_validator_rejects_conflicts(orc):
    assert orc.validate_partition(3, [0, 1], [1, 2], 1, [0, 0]) == 2   # share vertex 1
    assert orc.validate_partition(3, [0, 1], [1, 2], 2, [0, 2]) == 1   # colour out of range
    assert orc.validate_partition(3, [0, 1], [1, 2], 2, [0, 1]) == 0


# ------------------------------------------------------------------ cut / energy / readout

def test_cut_energy_identity_and_paper_figures(orc):
    for row in open(os.path.join(GOLDEN, "paper_cut_energy.txt")):
        if row[0] == "#":
            continue
        _, W, H, cut, *_ = row.split()
        assert (int(W) - int(H)) == 2 * int(cut)
    inst = instances.sparse_gnm(60, 150, 3)
    rng = np.random.default_rng(1)
    for _ in range(20):
        s = rng.choice([-1, 1], size=inst.n).astype(np.int8)
        c = orc.cut(inst.src, inst.dst, inst.w, s)
        H = orc.energy(inst.src, inst.dst, inst.w, s)
        assert inst.total_weight() - H == 2 * c
        assert orc.cut(inst.src, inst.dst, inst.w, -s) == c    # global flip


def test_binarize_recovers_planted_clusters(orc):
    inst = instances.gauge_planted(instances.torus2d(8, 8, 4), 5)
    tau = inst.meta["tau"]
    g = orc.coloured(inst)
    rng = np.random.default_rng(2)
    for centre in (0.0, 0.137, 0.5, 0.93):
        x = (centre + np.where(tau > 0, 0.0, 0.5) + rng.uniform(-0.004, 0.004, inst.n)) % 1.0
        best, bp, cuts, spins = orc.binarize(g, x)
        assert best == inst.meta["opt_cut"]
        assert orc.cut(g.src, g.dst, g.w, spins) == best
        assert (spins == tau).all() or (spins == -tau).all()
        assert cuts[bp] == best and (cuts <= best).all() and bp == int(np.argmax(cuts))


def test_bisector_hand_case(orc):
    # two bisectors (P = 2): lines at 0 and 1/4 turn; points at 0.1 and 0.3
    g = orc.ColouredGraph(2, [0], [1], [1], [0], 1)
    best, bp, cuts, spins = orc.binarize(g, [0.1, 0.3], P=2)
    # bisector 0: both in [0, 1/2) -> same side -> cut 0
    # bisector 1: [1/4, 3/4) holds 0.3 but not 0.1 -> cut 1
    assert list(cuts) == [0, 1] and best == 1 and bp == 1
    assert list(spins) == [-1, 1]


def test_bruteforce_on_planted_and_cycles(orc):
    for seed in range(4):
        inst = instances.gauge_planted(instances.sparse_gnm(14, 30, seed), 10 + seed)
        best, s = orc.bruteforce_maxcut(inst.n, inst.src, inst.dst, inst.w)
        assert best == inst.meta["opt_cut"]
        assert orc.cut(inst.src, inst.dst, inst.w, s) == best
    # odd cycle with unit weights: max cut = n - 1; even cycle: n
    for n in (5, 6, 9, 10):
        src = list(range(n - 1)) + [0]
        dst = list(range(1, n)) + [n - 1]
        best, _ = orc.bruteforce_maxcut(n, src, dst, [1] * n)
        assert best == (n if n % 2 == 0 else n - 1)


def test_binary16_rounding_matches_ieee_library(orc):
    rng = np.random.default_rng(3)
    ys = np.concatenate([rng.uniform(-0.5, 0.5, 5000), rng.uniform(-1e-4, 1e-4, 2000),
                         np.array([0.5, -0.5, 2 ** -25, 3 * 2 ** -26, 2 ** -24 * 1.5])])
    for y in ys:
        assert orc.round_binary16(float(y)) == float(np.float16(y))


def test_f16_storage_keeps_phases_representable(orc):
    inst = instances.random_regular(300, 3, 4)
    g = orc.coloured(inst)
    x0 = np.array([float(np.float16(v - 1.0)) + 1.0 if v >= 0.5 else float(np.float16(v))
                   for v in orc.init_phases(inst.n, 2, 0)]) % 1.0
    x, _ = orc.sweep(g, x0, 0.031, 3, seed=2, dwt_ratio=1.0, storage=orc.STORE_F16)
    gcen = np.where(x >= 0.5, x - 1.0, x)
    assert np.array_equal(gcen.astype(np.float16).astype(np.float64), gcen)
    # and it stays within a few binary16 quanta of the FP64 sweep
    xf, _ = orc.sweep(g, x0, 0.031, 3, seed=2, dwt_ratio=1.0)
    assert _circ(x, xf).max() < 8 * 2 ** -12


def _split_passes(orc, inst):
    """The torus's coloured graph, and its two passes as graphs of their own:
    colours (0, 1) and colours (2, 3) renumbered (0, 1)."""
    col, C = orc.color_instance(inst)
    assert C == 4
    g = orc.ColouredGraph(inst.n, inst.src, inst.dst, inst.w, col, C)
    parts = []
    for lo in (0, 2):
        k = (col == lo) | (col == lo + 1)
        parts.append(orc.ColouredGraph(inst.n, inst.src[k], inst.dst[k], inst.w[k], col[k] - lo, 2))
    return g, parts


def _round_turns(x, dtype):
    torch = pytest.importorskip("torch") if dtype == "bf16" else None
    g = np.where(x >= 0.5, x - 1.0, x)
    if dtype == "f16":
        g = g.astype(np.float16).astype(np.float64)
    else:
        g = torch.tensor(g).to(torch.bfloat16).to(torch.float64).numpy()
    return np.mod(np.where(g < 0, g + 1.0, g), 1.0)


@pytest.mark.parametrize("dtype", ["f16", "bf16"])
@pytest.mark.parametrize("sweep", [2, 3])
def test_pass_rounding_is_two_fp64_passes_each_rounded_once(orc, dtype, sweep):
    # modes 4 / 5: a sweep of the 4-colour torus equals an FP64 sweep of
    # colours (0, 1), one rounding of every phase (numpy / torch conversion),
    # an FP64 sweep of colours (2, 3) with the twist when due, one rounding
    inst = instances.torus2d(8, 12, 3)
    g, (g01, g23) = _split_passes(orc, inst)
    mode = orc.STORE_F16_PASS if dtype == "f16" else orc.STORE_BF16_PASS
    x0 = _round_turns(orc.init_phases(inst.n, 4, 1), dtype)
    a = 0.0331
    x, _ = orc.sweep(g, x0, a, sweep, seed=4, replica=1, dwt_ratio=1.0, storage=mode)
    y, _ = orc.sweep(g01, x0, a, sweep, seed=4, replica=1, dwt_ratio=1.0, flags=orc.NO_DWT)
    y = _round_turns(y, dtype)
    y, _ = orc.sweep(g23, y, a, sweep, seed=4, replica=1, dwt_ratio=1.0)
    y = _round_turns(y, dtype)
    assert np.array_equal(x, y)
    # the rounding cadence matters: every-write rounding gives another state
    xw, _ = orc.sweep(g, x0, a, sweep, seed=4, replica=1, dwt_ratio=1.0,
                      storage=orc.STORE_F16 if dtype == "f16" else orc.STORE_BF16)
    assert not np.array_equal(x, xw)
    assert _circ(x, xw).max() < 4 * (2 ** -12 if dtype == "f16" else 2 ** -9)


def test_bfloat16_rounding_matches_library(orc):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    ys = np.concatenate([rng.uniform(-0.5, 0.5, 5000), rng.uniform(-1e-4, 1e-4, 2000),
                         np.array([0.5, -0.5, 2 ** -25, 3 * 2 ** -26, 0.25 + 2 ** -10])])
    ref = torch.tensor(ys, dtype=torch.float64).to(torch.bfloat16).to(torch.float64).numpy()
    for y, r in zip(ys, ref):
        assert orc.round_bfloat16(float(y)) == float(r)


def test_bf16_storage_keeps_phases_representable(orc):
    torch = pytest.importorskip("torch")
    inst = instances.random_regular(300, 3, 4)
    g = orc.coloured(inst)
    x0 = np.array([orc.round_bfloat16(v - 1.0) + 1.0 if v >= 0.5 else orc.round_bfloat16(v)
                   for v in orc.init_phases(inst.n, 2, 0)]) % 1.0
    x, _ = orc.sweep(g, x0, 0.031, 3, seed=2, dwt_ratio=1.0, storage=orc.STORE_BF16)
    gcen = np.where(x >= 0.5, x - 1.0, x)
    back = torch.tensor(gcen).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(back, gcen)
    # most phases stay within a few bfloat16 quanta of the FP64 sweep; a
    # rounding can flip a sign decision near a tie and move a phase by a
    # whole step, so this is a distribution bound
    xf, _ = orc.sweep(g, x0, 0.031, 3, seed=2, dwt_ratio=1.0)
    assert (_circ(x, xf) > 8 * 2 ** -9).mean() < 0.02


# ------------------------------------------------------------------ conflict trap

def test_circular_conflict_trap_gd_freezes_scs_escapes(orc):
    # 3-variable unfrustrated instance of Fig. 2: ground states up-down-down,
    # Ising energy -3. Edges (0,1), (0,2) antiferromagnetic, (1,2) ferro.
    edges = [(0, 1, 1), (0, 2, 1), (1, 2, -1)]
    g = _graph(orc, 3, edges, [0, 1, 2])
    src, dst, w = g.src, g.dst, g.w
    opt, _ = orc.bruteforce_maxcut(3, src, dst, w)
    assert int(w.sum()) - 2 * opt == -3
    # a state where every variable's simultaneous forces cancel (eq. (8)):
    # x = (310, 7, 194) degrees. With unit couplings H takes only the values
    # -3 and +1, so the frozen state binarizes to +1 at every bisector.
    x0 = np.array([310.0, 7.0, 194.0]) / 360.0
    x = x0.copy()
    for s in range(1, 50):
        x, _ = orc.sweep(g, x, A14, s, flags=orc.NO_SCS | orc.NO_DWT)
    assert np.allclose(x, x0)
    best, _, cuts, spins = orc.binarize(g, x)
    assert orc.energy(src, dst, w, spins) == 1
    # sequential conflict-free search from the same state reaches the ground
    # state within one sweep (Fig. 4)
    x, _ = orc.sweep(g, x0, A14, 1, flags=orc.NO_DWT)
    best, _, _, spins = orc.binarize(g, x)
    assert orc.energy(src, dst, w, spins) == -3


# ------------------------------------------------------------------ quality

def test_cosm_reaches_bruteforce_optimum_small(orc):
    for seed in range(3):
        inst = instances.sparse_gnm(16, 36, 30 + seed)
        opt, _ = orc.bruteforce_maxcut(inst.n, inst.src, inst.dst, inst.w)
        g = orc.coloured(inst)
        cuts, *_ = orc.trials(g, 400, 32, seed=seed, dwt_ratio=1.0)
        assert cuts.max() == opt
        assert (cuts <= opt).all()


def test_cosm_solves_gauge_planted_256(orc):
    inst = instances.gauge_planted(instances.torus2d(16, 16, 3), 4)
    g = orc.coloured(inst)
    cuts, *_ = orc.trials(g, 1000, 16, seed=5)
    assert cuts.max() == inst.meta["opt_cut"]


def test_frustrated_loop_planted_energy(orc):
    inst = instances.frustrated_loop_planted((4, 4), 0.5, 3)
    best, s = orc.bruteforce_maxcut(inst.n, inst.src, inst.dst, inst.w)
    assert inst.total_weight() - 2 * best == inst.meta["ground_energy"]
    tau = inst.meta["tau"].astype(np.int8)
    assert orc.energy(inst.src, inst.dst, inst.w, tau) == inst.meta["ground_energy"]
    big = instances.frustrated_loop_planted((12, 12), 0.4, 7)
    g = orc.coloured(big)
    cuts, *_ = orc.trials(g, 2000, 16, seed=1, alpha0=25 / 360, dwt_ratio=1.0)
    assert cuts.max() == big.meta["opt_cut"]


# ------------------------------------------------------------------ metrics

def test_metrics_match_paper_tables(orc):
    for row in open(os.path.join(GOLDEN, "paper_metrics.txt")):
        if row[0] == "#" or not row.strip():
            continue
        t = row.split()
        ps, r, S = float(t[1]), float(t[2]), float(t[3])
        stt_, tt, ttt_, tol = float(t[4]), t[5], float(t[6]), float(t[7])
        assert orc.r99(ps) == pytest.approx(r, rel=tol)
        assert orc.stt(S, ps) == pytest.approx(stt_, rel=tol)
        if tt != "-":
            assert orc.ttt(float(tt), ps) == pytest.approx(ttt_, rel=tol)
    assert orc.r99(1.0) == 1.0


# ------------------------------------------------------------------ fixed point

def test_q16_mode_equals_fp64_on_grid_inputs(orc):
    # with grid phases and a grid step every FP64 operation is exact, so the
    # fixed-point mode must reproduce the FP64 sweep bit for bit
    inst = instances.random_regular(300, 3, 6)
    g = orc.coloured(inst)
    x0 = orc.q16_grid(orc.init_phases(inst.n, 4, 1))
    a = 417 / 65536
    for s in (1, 2, 3):
        xq, _ = orc.sweep(g, x0, a, s, seed=4, replica=1, dwt_ratio=0.5 * 2, storage=orc.STORE_Q16)
        xf, _ = orc.sweep(g, x0, a, s, seed=4, replica=1, dwt_ratio=1.0)
        assert np.array_equal(xq, xf)
        assert np.array_equal(np.floor(xq * 65536), xq * 65536)
        x0 = xq


def test_q16_step_rounds_to_nearest_grid_point(orc):
    fm = _graph(orc, 2, [(0, 1, -1)], [0])
    x0 = [0.5, 0.25]
    for frac, expect in ((0.49, 100), (0.51, 101), (0.0, 100)):
        a = (100 + frac) / 65536
        x, _ = orc.sweep(fm, x0, a, 1, flags=orc.NO_DWT, storage=orc.STORE_Q16)
        np.testing.assert_array_equal(x, [0.5 - expect / 65536, 0.25 + expect / 65536])


def test_q16_trials_reach_planted_optimum(orc):
    inst = instances.gauge_planted(instances.torus2d(16, 16, 3), 4)
    g = orc.coloured(inst)
    cuts, *_ = orc.trials(g, 1000, 16, seed=5, storage=orc.STORE_Q16)
    assert cuts.max() == inst.meta["opt_cut"]
