"""The identities behind the fixed-point sweeps on packed words, checked on
the CPU in numpy (no GPU, no library): two u16 phases per 32-bit word with
per-half adds modulo 2^16 give exactly the updates of the q << 16 form,
ties and exactly-opposite pairs included, and the twist's 15-bit compare per
half equals the 2^-32-turn window test for every phase on the grid."""
import numpy as np

M32 = np.uint64(0xFFFFFFFF)


def add_u16x2(a, b):
    """Per-half sum modulo 2^16 of two packed words."""
    lo = (a + b) & np.uint64(0xFFFF)
    hi = ((a >> np.uint64(16)) + (b >> np.uint64(16))) & np.uint64(0xFFFF)
    return lo | (hi << np.uint64(16))


def half_signs(v):
    """0xFFFF over each half whose sign bit is set."""
    lo = np.where(v & np.uint64(0x8000), np.uint64(0xFFFF), np.uint64(0))
    hi = np.where(v & np.uint64(0x80000000), np.uint64(0xFFFF0000), np.uint64(0))
    return lo | hi


def both_halves(v):
    v = v & np.uint64(0xFFFF)
    return v | (v << np.uint64(16))


def pair_packed(xi, xj, ap):
    pw, nw = both_halves(ap), both_halves((np.uint64(0x10000) - ap) & np.uint64(0xFFFF))
    ge = half_signs(add_u16x2(xj, ~xi & M32))
    st = (pw & ge) | (nw & ~ge & M32)
    nst = (nw & ge) | (pw & ~ge & M32)
    return add_u16x2(xi, st), add_u16x2(xj, nst)


def pair_widened(qi, qj, ap):
    """The q << 16 form: step +ap where (q_i - q_j) << 16 read as int32 is >= 0."""
    xi, xj = qi << np.uint64(16), qj << np.uint64(16)
    d = (xi - xj) & M32
    step = ap << np.uint64(16)
    st = np.where(d < np.uint64(0x80000000), step, (np.uint64(1 << 32) - step) & M32)
    return ((xi + st) & M32) >> np.uint64(16), ((xj - st) & M32) >> np.uint64(16)


def test_pair_update_on_packed_words_equals_widened_form():
    rng = np.random.default_rng(5)
    n = 1 << 18
    lo_i, hi_i = rng.integers(0, 1 << 16, n, dtype=np.uint64), rng.integers(0, 1 << 16, n, dtype=np.uint64)
    # every difference in the low halves, ties and exact opposites in the high
    lo_j = (lo_i - np.arange(n, dtype=np.uint64)) & np.uint64(0xFFFF)
    hi_j = np.where(np.arange(n) % 3 == 0, hi_i, np.where(np.arange(n) % 3 == 1, hi_i ^ np.uint64(0x8000),
                                                          rng.integers(0, 1 << 16, n, dtype=np.uint64)))
    for ap in (1, 173, 0x7FFF, 0x8000, 0xFFFF):
        ap = np.uint64(ap)
        xi, xj = lo_i | (hi_i << np.uint64(16)), lo_j | (hi_j << np.uint64(16))
        pi, pj = pair_packed(xi, xj, ap)
        for half in (0, 16):
            sh = np.uint64(half)
            wi, wj = pair_widened((xi >> sh) & np.uint64(0xFFFF), (xj >> sh) & np.uint64(0xFFFF), ap)
            assert np.array_equal((pi >> sh) & np.uint64(0xFFFF), wi)
            assert np.array_equal((pj >> sh) & np.uint64(0xFFFF), wj)


def test_twist_compare_per_half_equals_window_test():
    rng = np.random.default_rng(7)
    q = np.arange(1 << 16, dtype=np.uint64)
    cases = [(int(rng.integers(0, 1 << 32)), int(rng.integers(0, 1 << 31))) for _ in range(200)]
    cases += [(0, 1 << 31), (0xFFFF, 0x10000), (0x12345678, 0x5678), (0x12345678, 0x5679), (0xABCD0000, 0),
              (0xFFFFFFFF, 1 << 31), (0x00010001, 0x10001)]
    for c, qw in cases:
        c64, qw64 = np.uint64(c), np.uint64(qw)
        inside32 = (((q << np.uint64(16)) + c64) & np.uint64(0x7FFFFFFF)) < qw64
        ch, cl = np.uint64(c >> 16), np.uint64(c & 0xFFFF)
        T = ((qw64 - cl + np.uint64(0xFFFF)) >> np.uint64(16)) if qw64 > cl else np.uint64(0)
        y = (q + ch) & np.uint64(0x7FFF)
        inside16 = (((y + ((np.uint64(0x10000) - T) & np.uint64(0xFFFF))) & np.uint64(0xFFFF)) >> np.uint64(15)) == 1
        assert np.array_equal(inside32, inside16), (hex(c), hex(qw))


def test_sign_carrying_record_step():
    # alpha w for w = +-1 is alpha's bits plus bit 0 of the record times 2^31
    rng = np.random.default_rng(3)
    alpha = rng.random(1000).astype(np.float32) * np.float32(0.05)
    for s in (0, 1):
        bits = (alpha.view(np.uint32).astype(np.uint64) + np.uint64(s) * np.uint64(1 << 31)) & M32
        assert np.array_equal(bits.astype(np.uint32).view(np.float32), alpha * np.float32(1 - 2 * s))
