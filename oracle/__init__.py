"""Plain FP64 CPU oracle of Cosm -- test infrastructure.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. It shares no code with the CUDA path:
the arithmetic lives in ``cosm_oracle.c`` (plain C, FP64), loaded here with
ctypes; this file only marshals numpy arrays.

Pins for every function are in ``tests/test_oracle_pins.py``. One part is
marked "parity unpinned": trajectory-level agreement over many sweeps (the
switched dynamics are discontinuous, so FP32 and FP64 runs separate after a
near-tie); only per-sweep, replayed-state and distributional comparisons are
meaningful there.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cosm_oracle.c")
_LIB = os.path.join(_HERE, "libcosm_oracle.so")
_lock = threading.Lock()
_lib = None

NO_DWT = 1
NO_SCS = 2
DWT_RANDDIR = 4
OPT_BISECTOR = 8
STORE_F64 = 0
STORE_F16 = 1
STORE_Q16 = 2
STORE_BF16 = 3
# 16-bit storage rounded once per pass of two colours (at the end of each
# pass, the last pass taking the twist first) instead of at every write
STORE_F16_PASS = 4
STORE_BF16_PASS = 5


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable flags only: no -march, no
    -ffast-math, so FP64 results are the same on x86-64 and aarch64)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            P = C.c_void_p
            i32, i64, u64, f64 = C.c_int32, C.c_int64, C.c_uint64, C.c_double
            sig = {
                "orc_philox4x32_10": (None, [P, P, P]),
                "orc_init_phases": (None, [i32, u64, i64, P]),
                "orc_theta": (f64, [u64, i64, i64]),
                "orc_alpha": (f64, [i64, i64, f64]),
                "orc_wrap": (f64, [f64]),
                "orc_sgn_b": (C.c_int, [f64, f64]),
                "orc_round_binary16": (f64, [f64]),
                "orc_round_bfloat16": (f64, [f64]),
                "orc_in_window_q": (C.c_int, [f64, f64, f64]),
                "orc_sweep": (i64, [i32, i32, P, P, P, P, P, f64, i64, i32, f64, f64, u64, i64,
                                    i32, i32, P, f64, P, i64]),
                "orc_binarize": (i32, [i32, i64, P, P, P, P, i32, P, P, P]),
                "orc_cut": (i64, [i64, P, P, P, P]),
                "orc_energy": (i64, [i64, P, P, P, P]),
                "orc_trial": (i64, [i32, i32, P, P, P, P, i64, f64, i32, f64, f64, i32, u64, i64,
                                    i32, i32, P, P, P]),
                "orc_trials": (i32, [i32, i32, P, P, P, P, i64, f64, i32, f64, f64, i32, u64, i64,
                                     i32, i32, i32, P, P, P]),
                "orc_color_greedy": (i32, [i32, i64, P, P, P]),
                "orc_color_torus2d": (i32, [i32, i32, i64, P, P, P]),
                "orc_color_torus3d": (i32, [i32, i32, i32, i64, P, P, P]),
                "orc_validate_partition": (i32, [i32, i64, P, P, i32, P]),
                "orc_bruteforce_maxcut": (i64, [i32, i64, P, P, P, P]),
                "orc_twist_dir": (C.c_int, [u64, i64, i64]),
                "orc_sweep_h": (i64, [i32, i32, P, P, P, P, P, P, f64, i64, i32, f64, f64, u64, i64,
                                      i32, i32, P, f64, P, i64]),
                "orc_energy_h": (i64, [i32, i64, P, P, P, P, P]),
                "orc_readout_fields": (i64, [i32, i64, P, P, P, P, P, P, P]),
                "orc_binarize_opt": (i64, [i32, i64, P, P, P, P, P, P]),
                "orc_binarize_opt_brute": (i64, [i32, i64, P, P, P, P, P, P]),
                "orc_trial_ex": (i64, [i32, i32, P, P, P, P, P, i64, f64, i32, f64, f64, i32, u64,
                                       i64, i32, i32, i32, P, P, P, P]),
                "orc_trials_ex": (i32, [i32, i32, P, P, P, P, P, i64, f64, i32, f64, f64, i32, u64,
                                        i64, i32, i32, i32, i32, P, P, P, P]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


# ---------------------------------------------------------------- primitives

def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def init_phases(n: int, seed: int, replica: int) -> np.ndarray:
    x = np.zeros(n, dtype=np.float64)
    lib().orc_init_phases(n, seed, replica, _p(x))
    return x


def q16_grid(x):
    """Phases on the 2^-16-turn grid (the fixed-point initial state: top 16
    bits of the 24-bit draw)."""
    return np.floor(np.asarray(x, dtype=np.float64) * 65536.0) / 65536.0


def theta(seed: int, replica: int, sweep: int) -> float:
    return lib().orc_theta(seed, replica, sweep)


def alpha(s: int, S: int, alpha0: float) -> float:
    return lib().orc_alpha(s, S, alpha0)


def wrap(y: float) -> float:
    return lib().orc_wrap(y)


def sgn_b(xi: float, xj: float) -> int:
    return lib().orc_sgn_b(xi, xj)


def round_binary16(y: float) -> float:
    return lib().orc_round_binary16(y)


def round_bfloat16(y: float) -> float:
    return lib().orc_round_bfloat16(y)


def in_window(x: float, th: float, W: float) -> int:
    return lib().orc_in_window_q(x, th, W)


# ---------------------------------------------------------------- graphs

class ColouredGraph:
    """Edges sorted by colour (stable), with colour offsets."""

    def __init__(self, n, src, dst, w, color, C_):
        color = np.asarray(color, dtype=np.int64)
        order = np.argsort(color, kind="stable")
        self.n = int(n)
        self.C = int(C_)
        self.src = _i32(np.asarray(src)[order])
        self.dst = _i32(np.asarray(dst)[order])
        self.w = _i32(np.asarray(w)[order])
        self.order = order
        counts = np.bincount(color, minlength=self.C)
        self.off = np.zeros(self.C + 1, dtype=np.int64)
        self.off[1:] = np.cumsum(counts)

    @property
    def m(self):
        return int(self.off[-1])


def color_greedy(n, src, dst):
    src, dst = _i32(src), _i32(dst)
    col = np.zeros(src.shape[0], dtype=np.int32)
    Cn = lib().orc_color_greedy(n, src.shape[0], _p(src), _p(dst), _p(col))
    return col, int(Cn)


def color_torus2d(L1, L2, src, dst):
    src, dst = _i32(src), _i32(dst)
    col = np.zeros(src.shape[0], dtype=np.int32)
    Cn = lib().orc_color_torus2d(L1, L2, src.shape[0], _p(src), _p(dst), _p(col))
    if Cn < 0:
        raise ValueError("not an even-sided 2D torus")
    return col, int(Cn)


def color_torus3d(L1, L2, L3, src, dst):
    src, dst = _i32(src), _i32(dst)
    col = np.zeros(src.shape[0], dtype=np.int32)
    Cn = lib().orc_color_torus3d(L1, L2, L3, src.shape[0], _p(src), _p(dst), _p(col))
    if Cn < 0:
        raise ValueError("not an even-sided 3D torus")
    return col, int(Cn)


def color_instance(inst):
    """Regular pattern for even-sided tori, else the greedy heuristic."""
    d = tuple(inst.dims)
    if len(d) == 2 and all(x % 2 == 0 and x >= 4 for x in d):
        return color_torus2d(d[0], d[1], inst.src, inst.dst)
    if len(d) == 3 and all(x % 2 == 0 and x >= 4 for x in d):
        return color_torus3d(d[0], d[1], d[2], inst.src, inst.dst)
    return color_greedy(inst.n, inst.src, inst.dst)


def validate_partition(n, src, dst, C_, color) -> int:
    src, dst, color = _i32(src), _i32(dst), _i32(color)
    return int(lib().orc_validate_partition(n, src.shape[0], _p(src), _p(dst), C_, _p(color)))


def coloured(inst, color=None, C_=None):
    if color is None:
        color, C_ = color_instance(inst)
    return ColouredGraph(inst.n, inst.src, inst.dst, inst.w, color, C_)


# ---------------------------------------------------------------- dynamics

def _h(h):
    return None if h is None else _i32(h)


def sweep(g: ColouredGraph, x, alpha_, sweep_idx, *, dwt_period=3, dwt_ratio=0.5, window=0.25,
          seed=0, replica=0, flags=0, storage=STORE_F64, force=None, tie_eps=0.0, max_ties=4096,
          h=None):
    """One sweep in place on a copy; returns (x_new, near_ties). h: local
    fields per vertex (None = none)."""
    x = np.array(x, dtype=np.float64, copy=True)
    ties = np.zeros(max_ties, dtype=np.int64)
    f = None if force is None else np.ascontiguousarray(force, dtype=np.int8)
    hh = _h(h)
    nt = lib().orc_sweep_h(g.n, g.C, _p(g.off), _p(g.src), _p(g.dst), _p(g.w), _p(hh), _p(x), alpha_,
                           sweep_idx, dwt_period, dwt_ratio, window, seed, replica, flags, storage,
                           _p(f), tie_eps, _p(ties), max_ties)
    if nt < 0:
        raise MemoryError
    return x, ties[:min(nt, max_ties)].copy()


def binarize(g, x, P=100):
    x = np.ascontiguousarray(x, dtype=np.float64)
    cuts = np.zeros(P, dtype=np.int64)
    best = np.zeros(1, dtype=np.int64)
    spins = np.zeros(g.n, dtype=np.int8)
    bp = lib().orc_binarize(g.n, g.m, _p(g.src), _p(g.dst), _p(g.w), _p(x), P, _p(cuts),
                            _p(best), _p(spins))
    return int(best[0]), int(bp), cuts, spins


def cut(src, dst, w, spins) -> int:
    src, dst, w = _i32(src), _i32(dst), _i32(w)
    s = np.ascontiguousarray(spins, dtype=np.int8)
    return int(lib().orc_cut(src.shape[0], _p(src), _p(dst), _p(w), _p(s)))


def energy(src, dst, w, spins) -> int:
    src, dst, w = _i32(src), _i32(dst), _i32(w)
    s = np.ascontiguousarray(spins, dtype=np.int8)
    return int(lib().orc_energy(src.shape[0], _p(src), _p(dst), _p(w), _p(s)))


def trial(g, S, *, alpha0=14 / 360, dwt_period=3, dwt_ratio=0.5, window=0.25, P=100, seed=0,
          replica=0, flags=0, storage=STORE_F64):
    x = np.zeros(g.n, dtype=np.float64)
    spins = np.zeros(g.n, dtype=np.int8)
    bp = np.zeros(1, dtype=np.int32)
    best = lib().orc_trial(g.n, g.C, _p(g.off), _p(g.src), _p(g.dst), _p(g.w), S, alpha0,
                           dwt_period, dwt_ratio, window, P, seed, replica, flags, storage,
                           _p(x), _p(spins), _p(bp))
    return int(best), x, spins, int(bp[0])


def trials(g, S, replicas, *, alpha0=14 / 360, dwt_period=3, dwt_ratio=0.5, window=0.25, P=100,
           seed=0, flags=0, storage=STORE_F64, threads=None, keep_x=False):
    threads = threads or os.cpu_count() or 1
    cuts = np.zeros(replicas, dtype=np.int64)
    bps = np.zeros(replicas, dtype=np.int32)
    xs = np.zeros((replicas, g.n), dtype=np.float64) if keep_x else None
    used = lib().orc_trials(g.n, g.C, _p(g.off), _p(g.src), _p(g.dst), _p(g.w), S, alpha0,
                            dwt_period, dwt_ratio, window, P, seed, replicas, flags, storage,
                            threads, _p(cuts), _p(bps), _p(xs))
    return cuts, bps, xs, int(used)


def twist_dir(seed: int, replica: int, sweep_idx: int) -> int:
    return int(lib().orc_twist_dir(seed, replica, sweep_idx))


def energy_h(n, src, dst, w, h, spins) -> int:
    """Eq. (1) with local fields: sum w s_i s_j - sum h s."""
    src, dst, w = _i32(src), _i32(dst), _i32(w)
    s = np.ascontiguousarray(spins, dtype=np.int8)
    hh = _h(h)
    return int(lib().orc_energy_h(n, src.shape[0], _p(src), _p(dst), _p(w), _p(hh), _p(s)))


def readout_fields(g, h, x):
    """Fixed-semicircle readout: (energy, cut, spins)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    hh = _h(h)
    c = np.zeros(1, dtype=np.int64)
    spins = np.zeros(g.n, dtype=np.int8)
    H = lib().orc_readout_fields(g.n, g.m, _p(g.src), _p(g.dst), _p(g.w), _p(hh), _p(x), _p(c),
                                 _p(spins))
    return int(H), int(c[0]), spins


def binarize_opt(g, x, brute=False):
    """Optimal bisector: (best cut, position B in 2^-32 turns, spins)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    c = np.zeros(1, dtype=np.int64)
    spins = np.zeros(g.n, dtype=np.int8)
    fn = lib().orc_binarize_opt_brute if brute else lib().orc_binarize_opt
    B = fn(g.n, g.m, _p(g.src), _p(g.dst), _p(g.w), _p(x), _p(c), _p(spins))
    if B < 0:
        raise MemoryError
    return int(c[0]), int(B), spins


def n_readouts(S, track):
    return (S + track - 1) // track if track > 0 else 0


def trial_ex(g, S, *, alpha0=14 / 360, dwt_period=3, dwt_ratio=0.5, window=0.25, P=100, seed=0,
             replica=0, flags=0, storage=STORE_F64, track=0, h=None):
    """One trial with fields / tracking / optimal bisector. Returns a dict:
    cut, energy, B, p, sweep (of the kept readout), x (final phases), spins
    (of the kept readout), trace (energies of the readouts)."""
    x = np.zeros(g.n, dtype=np.float64)
    spins = np.zeros(g.n, dtype=np.int8)
    out = np.zeros(5, dtype=np.int64)
    tr = np.zeros(max(1, n_readouts(S, track)), dtype=np.int64)
    hh = _h(h)
    lib().orc_trial_ex(g.n, g.C, _p(g.off), _p(g.src), _p(g.dst), _p(g.w), _p(hh), S, alpha0,
                       dwt_period, dwt_ratio, window, P, seed, replica, flags, storage, track,
                       _p(x), _p(spins), _p(out), _p(tr))
    return {"cut": int(out[0]), "energy": int(out[1]), "B": int(out[2]), "p": int(out[3]),
            "sweep": int(out[4]), "x": x, "spins": spins, "trace": tr[:n_readouts(S, track)]}


def trials_ex(g, S, replicas, *, alpha0=14 / 360, dwt_period=3, dwt_ratio=0.5, window=0.25, P=100,
              seed=0, flags=0, storage=STORE_F64, track=0, h=None, threads=None, keep_x=False,
              keep_spins=False):
    """Many replicas of trial_ex: out [replicas][5] (cut, energy, B, p, sweep),
    trace [replicas][readouts], x, spins (or None)."""
    threads = threads or os.cpu_count() or 1
    out = np.zeros((replicas, 5), dtype=np.int64)
    nr = n_readouts(S, track)
    tr = np.zeros((replicas, max(1, nr)), dtype=np.int64)
    xs = np.zeros((replicas, g.n), dtype=np.float64) if keep_x else None
    sp = np.zeros((replicas, g.n), dtype=np.int8) if keep_spins else None
    hh = _h(h)
    lib().orc_trials_ex(g.n, g.C, _p(g.off), _p(g.src), _p(g.dst), _p(g.w), _p(hh), S, alpha0,
                        dwt_period, dwt_ratio, window, P, seed, replicas, flags, storage, track,
                        threads, _p(out), _p(tr if nr else None), _p(xs), _p(sp))
    return out, tr[:, :nr], xs, sp


def bruteforce_maxcut(n, src, dst, w):
    src, dst, w = _i32(src), _i32(dst), _i32(w)
    spins = np.zeros(n, dtype=np.int8)
    best = lib().orc_bruteforce_maxcut(n, src.shape[0], _p(src), _p(dst), _p(w), _p(spins))
    return int(best), spins


# ---------------------------------------------------------------- metrics

def r99(ps: float) -> float:
    """Repetitions for 99% success (Appendix A): log(0.01)/log(1-P_s); 1 if P_s = 1."""
    import math
    if ps >= 1.0:
        return 1.0
    if ps <= 0.0:
        return math.inf
    return math.log(1.0 - 0.99) / math.log(1.0 - ps)


def stt(sweeps_per_trial: float, ps: float) -> float:
    """Sweeps-to-target STT = S_trial R99 (Appendix A)."""
    return sweeps_per_trial * r99(ps)


def ttt(t_trial: float, ps: float) -> float:
    """Wall-clock time-to-target TTT = t_trial R99 (Appendix A)."""
    return t_trial * r99(ps)
