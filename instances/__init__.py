"""Seeded synthetic problem instances shaped like the paper's workloads.

This module only draws graphs and weights. It holds none of the solver's
arithmetic (no edge colouring, no phase dynamics, no cut evaluation), so both
the oracle and the CUDA path can take their inputs from it without sharing
method code.

Every draw goes through a counter-based splitmix64 stream written here, so the
same seed gives the same instance on every machine and numpy version.

Conventions
-----------
* An instance is ``Instance(n, src, dst, w, dims, meta)``. Edges are canonical
  (``src < dst``), simple (no loops, no duplicates) and carry a non-zero
  integer Max-Cut weight ``w = -J`` (the sign convention of the Gset files,
  Appendix A). ``H = sum w_ij s_i s_j`` and ``cut = (sum w - H) / 2``.
* ``dims`` is ``(L1, L2)`` for a 2D torus with vertex ``v = r*L2 + c``,
  ``(L1, L2, L3)`` for a 3D torus with ``v = (a*L2 + b)*L3 + c``, else ``()``.

Families (the paper's workloads and their stand-ins):
* ``torus2d``: 2D periodic +-J spin glass, the shape of Gset G72/G77/G81
  (Section III-A: degree 4, bimodal couplings, toroidal).
* ``random_regular``: random d-regular graphs from the configuration model
  with rejection, standing in for the bounded-degree Gset graphs G61/G70
  (Section III-B, Table III).
* ``sparse_gnm``: uniform random G(n, m) with integer weights in [-3, 3] \\ {0}.
* ``gauge_planted``: an unfrustrated gauge-transformed instance whose optimum
  is known at any size (all edges satisfiable).
* ``frustrated_loop_planted``: frustrated loops planted on a periodic 2D/3D
  lattice, following the loop construction of Hen et al., PRA 92, 042325
  (2015); the planted state is a ground state with known energy. It stands in
  for the tile-planted Chook instances of Section III-C, which are not
  available here.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

_MASK = (1 << 64) - 1
_GAMMA = 0x9E3779B97F4A7C15


def _mix64(z: np.ndarray) -> np.ndarray:
    """splitmix64 finaliser on a uint64 array (Steele, Lea, Flood 2014)."""
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= np.uint64(0xBF58476D1CE4E5B9)
        z ^= z >> np.uint64(27)
        z *= np.uint64(0x94D049BB133111EB)
        z ^= z >> np.uint64(31)
    return z


class Stream:
    """Counter-based splitmix64 stream: value k = mix(base + (k+1)*gamma)."""

    def __init__(self, seed: int, tag: int = 0):
        base = np.array([(seed * 0xD1B54A32D192ED03 + tag * 0xABC98388FB8FAC03) & _MASK],
                        dtype=np.uint64)
        self.base = int(_mix64(base)[0])
        self.pos = 0

    def u64(self, count: int) -> np.ndarray:
        k = np.arange(self.pos + 1, self.pos + 1 + count, dtype=np.uint64)
        with np.errstate(over="ignore"):
            z = np.uint64(self.base) + k * np.uint64(_GAMMA)
        self.pos += count
        return _mix64(z)

    def below(self, bound: int, count: int) -> np.ndarray:
        """Integers uniform in [0, bound) (bound < 2**32), multiply-shift map."""
        hi = self.u64(count) >> np.uint64(32)
        return ((hi * np.uint64(bound)) >> np.uint64(32)).astype(np.int64)

    def signs(self, count: int) -> np.ndarray:
        return np.where((self.u64(count) >> np.uint64(63)) == 1, 1, -1).astype(np.int32)


@dataclass
class Instance:
    n: int
    src: np.ndarray
    dst: np.ndarray
    w: np.ndarray
    dims: tuple = ()
    meta: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return int(self.src.shape[0])

    def total_weight(self) -> int:
        return int(self.w.astype(np.int64).sum())


def _canonical(n, a, b, w, meta=None, dims=()):
    a = np.asarray(a, dtype=np.int64)
    b = np.asarray(b, dtype=np.int64)
    lo = np.minimum(a, b).astype(np.int32)
    hi = np.maximum(a, b).astype(np.int32)
    inst = Instance(int(n), lo, hi, np.asarray(w, dtype=np.int32), tuple(dims), dict(meta or {}))
    check_simple(inst)
    return inst


def check_simple(inst: Instance) -> None:
    """Raise if the instance has loops, duplicate edges, zero weights or bad ids."""
    if inst.m == 0:
        return
    if (inst.src >= inst.dst).any():
        raise ValueError("edges must be canonical src < dst without loops")
    if inst.src.min() < 0 or inst.dst.max() >= inst.n:
        raise ValueError("vertex id out of range")
    key = inst.src.astype(np.int64) * inst.n + inst.dst.astype(np.int64)
    if np.unique(key).shape[0] != inst.m:
        raise ValueError("duplicate edge")
    if (inst.w == 0).any():
        raise ValueError("zero weight")


# ----------------------------------------------------------------------------
# 2D and 3D periodic lattices
# ----------------------------------------------------------------------------

def torus2d_edges(L1: int, L2: int):
    """Edges of the L1 x L2 torus: horizontal ones first, then vertical ones."""
    if L1 < 3 or L2 < 3:
        raise ValueError("torus sides must be >= 3 for a simple graph")
    r, c = np.divmod(np.arange(L1 * L2, dtype=np.int64), L2)
    v = r * L2 + c
    right = r * L2 + (c + 1) % L2
    down = ((r + 1) % L1) * L2 + c
    return np.concatenate([v, v]), np.concatenate([right, down])


def torus3d_edges(L1: int, L2: int, L3: int):
    if min(L1, L2, L3) < 3:
        raise ValueError("torus sides must be >= 3 for a simple graph")
    idx = np.arange(L1 * L2 * L3, dtype=np.int64)
    a, rest = np.divmod(idx, L2 * L3)
    b, c = np.divmod(rest, L3)

    def vid(a_, b_, c_):
        return (a_ * L2 + b_) * L3 + c_

    n0 = vid((a + 1) % L1, b, c)
    n1 = vid(a, (b + 1) % L2, c)
    n2 = vid(a, b, (c + 1) % L3)
    return np.concatenate([idx, idx, idx]), np.concatenate([n0, n1, n2])


def torus2d(L1: int, L2: int, seed: int) -> Instance:
    """2D periodic +-J glass: J uniform in {-1,+1}, w = -J (Section III-A)."""
    a, b = torus2d_edges(L1, L2)
    J = Stream(seed, tag=1).signs(a.shape[0])
    return _canonical(L1 * L2, a, b, -J, {"family": "torus2d", "seed": seed}, dims=(L1, L2))


def torus3d(L1: int, L2: int, L3: int, seed: int) -> Instance:
    a, b = torus3d_edges(L1, L2, L3)
    J = Stream(seed, tag=2).signs(a.shape[0])
    return _canonical(L1 * L2 * L3, a, b, -J, {"family": "torus3d", "seed": seed},
                      dims=(L1, L2, L3))


# ----------------------------------------------------------------------------
# Bounded-degree non-lattice graphs
# ----------------------------------------------------------------------------

def random_regular(n: int, d: int, seed: int, max_tries: int = 1000) -> Instance:
    """Random d-regular graph: configuration model, whole pairing redrawn until
    it has neither loops nor multi-edges. Weights uniform in {-1,+1}."""
    if (n * d) % 2:
        raise ValueError("n*d must be even")
    st = Stream(seed, tag=3)
    points = np.repeat(np.arange(n, dtype=np.int64), d)
    for _ in range(max_tries):
        perm = np.argsort(st.u64(points.shape[0]), kind="stable")
        p = points[perm]
        a, b = p[0::2], p[1::2]
        if (a == b).any():
            continue
        lo, hi = np.minimum(a, b), np.maximum(a, b)
        if np.unique(lo * n + hi).shape[0] != lo.shape[0]:
            continue
        order = np.lexsort((hi, lo))
        w = st.signs(lo.shape[0])
        return _canonical(n, lo[order], hi[order], w,
                          {"family": f"random_{d}_regular", "seed": seed})
    raise RuntimeError("configuration model did not give a simple graph")


_W3 = np.array([-3, -2, -1, 1, 2, 3], dtype=np.int32)


def sparse_gnm(n: int, m: int, seed: int, wmax: int = 3) -> Instance:
    """Uniform simple G(n, m); weights uniform in [-wmax, wmax] \\ {0}."""
    if m > n * (n - 1) // 2:
        raise ValueError("too many edges")
    st = Stream(seed, tag=4)
    keys = np.empty(0, dtype=np.int64)
    while keys.shape[0] < m:
        need = 2 * (m - keys.shape[0]) + 16
        a = st.below(n, need)
        b = st.below(n, need)
        ok = a != b
        lo, hi = np.minimum(a, b)[ok], np.maximum(a, b)[ok]
        cand = np.concatenate([keys, lo * n + hi])
        _, first = np.unique(cand, return_index=True)
        keys = cand[np.sort(first)][:m]
    lo, hi = np.divmod(keys, n)
    wv = np.array([v for v in range(-wmax, wmax + 1) if v != 0], dtype=np.int32)
    w = wv[st.below(wv.shape[0], m)]
    order = np.lexsort((hi, lo))
    return _canonical(n, lo[order], hi[order], w[order], {"family": "sparse_gnm", "seed": seed})


# ----------------------------------------------------------------------------
# Planted instances (known optimum)
# ----------------------------------------------------------------------------

def gauge_planted(base: Instance, seed: int) -> Instance:
    """Unfrustrated instance on base's edges: w_ij = -tau_i tau_j |w_ij|.

    The state s = tau satisfies every edge, so the optimum cut is the sum of
    the positive weights and the ground energy is -sum |w|."""
    tau = Stream(seed, tag=5).signs(base.n)
    w = -tau[base.src] * tau[base.dst] * np.abs(base.w)
    inst = Instance(base.n, base.src.copy(), base.dst.copy(), w.astype(np.int32), base.dims,
                    dict(base.meta, family=base.meta.get("family", "") + "+gauge", planted_seed=seed))
    inst.meta["tau"] = tau
    inst.meta["opt_cut"] = int(np.clip(w, 0, None).sum())
    inst.meta["ground_energy"] = -int(np.abs(w).sum())
    return inst


def _lattice_neighbours(dims):
    dims = tuple(int(x) for x in dims)
    n = int(np.prod(dims))
    idx = np.arange(n, dtype=np.int64)
    coords = np.array(np.unravel_index(idx, dims)).T
    nbrs = []
    for ax in range(len(dims)):
        for step in (1, -1):
            c2 = coords.copy()
            c2[:, ax] = (c2[:, ax] + step) % dims[ax]
            nbrs.append(np.ravel_multi_index(c2.T, dims))
    return np.stack(nbrs, axis=1)  # (n, 2*D)


def frustrated_loop_planted(dims, rho: float, seed: int, R: int = 0) -> Instance:
    """Frustrated loops planted on a periodic lattice (Hen et al. 2015).

    ``round(rho*N)`` loops are drawn. Each loop is a non-backtracking random
    walk from a random vertex, stopped when it first revisits a vertex; the
    closed part is the loop. Along a loop every coupling is ferromagnetic
    except one edge chosen at random, so the all-up state leaves exactly one
    edge of each loop unsatisfied, which is each loop's minimum. Loop
    couplings add up; with ``R > 0`` a loop is rejected if it would push any
    |J| above R. A random gauge tau hides the planted state. Edges whose
    couplings cancel to zero are dropped. Planted energy (H = sum w s s at
    s = tau) is sum over loops of (2 - length)."""
    dims = tuple(int(x) for x in dims)
    n = int(np.prod(dims))
    nb = _lattice_neighbours(dims)
    deg = nb.shape[1]
    st = Stream(seed, tag=6)
    coup: dict[tuple[int, int], int] = {}
    n_loops = int(round(rho * n))
    energy = 0
    placed = 0
    tries = 0
    while placed < n_loops:
        tries += 1
        if tries > 50 * max(n_loops, 1) + 1000:
            raise RuntimeError("could not place loops under the R cap")
        rnd = st.u64(64)
        k = 0
        start = int(rnd[k] % np.uint64(n)); k += 1
        path = [start]
        pos = {start: 0}
        prev = -1
        cur = start
        while True:
            if k >= rnd.shape[0]:
                rnd = st.u64(64)
                k = 0
            choices = [int(x) for x in nb[cur] if int(x) != prev]
            nxt = choices[int(rnd[k] % np.uint64(len(choices)))]; k += 1
            if nxt in pos:
                loop = path[pos[nxt]:] + [nxt]
                break
            pos[nxt] = len(path)
            path.append(nxt)
            prev, cur = cur, nxt
        L = len(loop) - 1
        if L < 4:
            continue
        edges = [(min(loop[t], loop[t + 1]), max(loop[t], loop[t + 1])) for t in range(L)]
        bad = int(st.below(L, 1)[0])
        # Hen et al. couplings in H = sum J s s: ferromagnetic J = -1, one +1.
        add = {}
        for t, e in enumerate(edges):
            add[e] = add.get(e, 0) + (1 if t == bad else -1)
        if R > 0 and any(abs(coup.get(e, 0) + dj) > R for e, dj in add.items()):
            continue
        for e, dj in add.items():
            coup[e] = coup.get(e, 0) + dj
        energy += 2 - L
        placed += 1
    tau = Stream(seed, tag=7).signs(n)
    items = sorted((e, j) for e, j in coup.items() if j != 0)
    a = np.array([e[0] for e, _ in items], dtype=np.int64)
    b = np.array([e[1] for e, _ in items], dtype=np.int64)
    jh = np.array([j for _, j in items], dtype=np.int64)
    # Max-Cut weight w = -J_paper = J_Hen, then gauge by tau.
    w = (jh * tau[a] * tau[b]).astype(np.int32)
    inst = _canonical(n, a, b, w, {"family": f"planted_loops_{len(dims)}d", "seed": seed,
                                   "rho": rho, "R": R}, dims=dims)
    inst.meta["tau"] = tau
    inst.meta["ground_energy"] = int(energy)
    inst.meta["opt_cut"] = (inst.total_weight() - int(energy)) // 2
    return inst


def aligned_fields(inst: Instance, strength: int, fraction: float = 1.0, seed: int = 0) -> np.ndarray:
    """Local fields h_i = strength * tau_i on a random `fraction` of the
    vertices (all of them by default), pointing along a planted instance's
    hidden state tau; the other fields are 0. Every field term is then
    lowest at s = tau as well, so tau stays a ground state, with energy
    ground_energy - strength * (number of fields) (eq. (1))."""
    tau = np.asarray(inst.meta["tau"], dtype=np.int64)
    h = int(strength) * tau
    if fraction < 1.0:
        u = (Stream(seed, tag=11).u64(inst.n) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
        h = np.where(u < fraction, h, 0)
    return h.astype(np.int32)


def ragged_batch(count: int, seed: int, n_lo: int = 800, n_hi: int = 20000):
    """A ragged batch of instances: N log-uniform in [n_lo, n_hi]; half 2D +-1
    tori with even sides near N, half G(n, m) graphs with m = round(d*N/2),
    d uniform in [4, 6], weights in [-3, 3] \\ {0}; replicas uniform in
    {64..256}. Returns (instances, replicas)."""
    st = Stream(seed, tag=8)
    u = (st.u64(count) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    ns = np.round(np.exp(np.log(n_lo) + u * (np.log(n_hi) - np.log(n_lo)))).astype(np.int64)
    du = (st.u64(count) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    reps = 64 + st.below(193, count)
    out = []
    for k in range(count):
        n = int(ns[k])
        if k % 2 == 0:
            L1 = max(4, 2 * int(round(np.sqrt(n) / 2)))
            L2 = max(4, 2 * int(round(n / L1 / 2)))
            out.append(torus2d(L1, L2, seed * 100003 + k))
        else:
            d = 4.0 + 2.0 * du[k]
            out.append(sparse_gnm(n, int(round(d * n / 2)), seed * 100003 + k))
    return out, [int(r) for r in reps]
