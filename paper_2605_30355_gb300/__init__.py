"""Cosm (Collective Switched Motion) on GB300: thin Python binding.

Every call marshals arguments into the C ABI of ``include/cosm.h`` implemented
by the in-tree CUDA library ``libcosm.so`` (built by ``build.py``); all steps of
the solver run in that library's kernels. There is no CPU fallback: importing
this package raises if the library is missing, and device calls raise if
the CUDA runtime reports an error.

PyTorch is optional plumbing: a ``torch.cuda.Stream`` may be passed wherever a
stream is accepted, and device tensors may be passed as output buffers.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_HERE = os.path.dirname(os.path.abspath(__file__))
# COSM_LIBRARY=checked loads the checked build (device index checks on)
LIB_PATH = os.path.join(_HERE, "libcosm_checked.so" if os.environ.get("COSM_LIBRARY") == "checked"
                        else "libcosm.so")

OK = 0
ERR_INVALID_ARG = -1
ERR_NOT_A_MATCHING = -2
ERR_PARTITION = -3
ERR_TOO_LARGE = -4
ERR_CUDA = -5
ERR_TIMEOUT = -6
ERR_STATE = -7
ERR_NOMEM = -8
ERR_CHECK = -9

F32 = 0
F16 = 1
Q16 = 2
BF16 = 3
NO_DWT = 1
NO_SCS = 2
DWT_RANDOM_DIR = 4
OPT_BISECTOR = 8
FAULT_DROP_SIGNAL = 1
NO_TARGET = -(1 << 63)  # INT64_MIN: every replica counts as a success

#: every symbol include/cosm.h declares
EXPORTS = (
    "cosm_default_params", "cosm_create", "cosm_destroy", "cosm_run", "cosm_sync", "cosm_get_best",
    "cosm_get_replica_cuts", "cosm_get_state", "cosm_set_state", "cosm_step", "cosm_readout",
    "cosm_solve", "cosm_layout", "cosm_color_greedy", "cosm_color_misra_gries",
    "cosm_color_torus2d", "cosm_color_torus3d", "cosm_validate_partition", "cosm_probe_smem",
    "cosm_solve_static", "cosm_batch_create", "cosm_batch_run", "cosm_batch_sync",
    "cosm_batch_get_best", "cosm_batch_get_replica_cuts", "cosm_batch_get_state", "cosm_batch_tune",
    "cosm_batch_info", "cosm_batch_destroy", "cosm_server_default_config", "cosm_server_create",
    "cosm_server_submit", "cosm_server_poll", "cosm_server_wait", "cosm_server_get_spins",
    "cosm_server_stats", "cosm_server_destroy", "cosm_last_error", "cosm_get_replica_energies",
    "cosm_get_replica_bisectors", "cosm_get_trace", "cosm_qubo_to_ising", "cosm_probe_fp32",
    "cosm_run_range", "cosm_get_success", "cosm_export_state", "cosm_import_state",
    "cosm_set_wait_limit", "cosm_inject_fault", "cosm_batch_layout",
)


class CosmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"cosm error {code}: {msg}")
        self.code = code


class GraphDesc(C.Structure):
    _fields_ = [("n", C.c_int32), ("m", C.c_int64), ("src", C.c_void_p), ("dst", C.c_void_p),
                ("w", C.c_void_p), ("n_colors", C.c_int32), ("color", C.c_void_p),
                ("dims", C.c_int32 * 3), ("h", C.c_void_p)]


class ServerConfig(C.Structure):
    _fields_ = [("memory_budget", C.c_int64), ("max_active", C.c_int32), ("chunk_sweeps", C.c_int32),
                ("threads", C.c_int32), ("reserved", C.c_int32)]


class RequestResult(C.Structure):
    _fields_ = [("status", C.c_int32), ("trials", C.c_int32), ("best_cut", C.c_int64),
                ("energy", C.c_int64), ("best_trial", C.c_int32), ("best_replica", C.c_int32),
                ("t_submit", C.c_double), ("t_admit", C.c_double), ("t_done", C.c_double),
                ("ttt", C.c_double), ("updates", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Params(C.Structure):
    _fields_ = [("alpha0_deg", C.c_double), ("dwt_ratio", C.c_double), ("dwt_period", C.c_int32),
                ("window_deg", C.c_double), ("n_bisectors", C.c_int32), ("storage", C.c_int32),
                ("flags", C.c_int32), ("track_period", C.c_int32)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libcosm.so is not built ({LIB_PATH}); run paper_2605_30355_gb300/build.py "
                          "or __graft_entry__.build()")
    L = C.CDLL(LIB_PATH)
    P, i32, i64, u64 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64
    sig = {
        "cosm_default_params": (None, [P]),
        "cosm_create": (C.c_int, [P, P, P]),
        "cosm_destroy": (None, [P]),
        "cosm_run": (C.c_int, [P, i64, i32, u64, i64, P]),
        "cosm_run_range": (C.c_int, [P, i64, i64, i64, i32, u64, i64, P]),
        "cosm_get_success": (C.c_int, [P, P]),
        "cosm_export_state": (C.c_int, [P, P, i32, P]),
        "cosm_import_state": (C.c_int, [P, P, i32, i32, u64, i64]),
        "cosm_set_wait_limit": (C.c_int, [P, C.c_double]),
        "cosm_inject_fault": (C.c_int, [P, i32]),
        "cosm_probe_fp32": (C.c_int, [i32, P, P]),
        "cosm_sync": (C.c_int, [P]),
        "cosm_get_best": (C.c_int, [P, P, P, P, P]),
        "cosm_get_replica_cuts": (C.c_int, [P, P, P]),
        "cosm_get_state": (C.c_int, [P, P]),
        "cosm_set_state": (C.c_int, [P, P, i32, u64]),
        "cosm_step": (C.c_int, [P, i64, C.c_float, P]),
        "cosm_readout": (C.c_int, [P, P]),
        "cosm_solve": (C.c_int, [P, P, i64, i32, u64, P, P, P, P]),
        "cosm_layout": (C.c_int, [P, P]),
        "cosm_color_greedy": (C.c_int, [i32, i64, P, P, P, P]),
        "cosm_color_misra_gries": (C.c_int, [i32, i64, P, P, P, P]),
        "cosm_color_torus2d": (C.c_int, [i32, i32, i64, P, P, P]),
        "cosm_color_torus3d": (C.c_int, [i32, i32, i32, i64, P, P, P]),
        "cosm_validate_partition": (C.c_int, [i32, i64, P, P, i32, P]),
        "cosm_probe_smem": (C.c_int, [i32, P, P]),
        "cosm_solve_static": (C.c_int, [P, P, i64, i32, u64, P, P, P]),
        "cosm_batch_create": (C.c_int, [i32, P, P, i32, P]),
        "cosm_batch_run": (C.c_int, [P, P, P, P, P]),
        "cosm_batch_sync": (C.c_int, [P]),
        "cosm_batch_get_best": (C.c_int, [P, i32, P, P, P, P]),
        "cosm_batch_get_replica_cuts": (C.c_int, [P, i32, P, P]),
        "cosm_batch_get_state": (C.c_int, [P, i32, P]),
        "cosm_batch_tune": (C.c_int, [P, P, i64, P]),
        "cosm_batch_info": (C.c_int, [P, P]),
        "cosm_batch_layout": (C.c_int, [P, i32, P]),
        "cosm_batch_destroy": (None, [P]),
        "cosm_server_default_config": (None, [P]),
        "cosm_server_create": (C.c_int, [P, P]),
        "cosm_server_submit": (C.c_int, [P, P, P, i64, i32, u64, i64, i32, P]),
        "cosm_server_poll": (C.c_int, [P, i64, P]),
        "cosm_server_wait": (C.c_int, [P, i64, C.c_double, P]),
        "cosm_server_get_spins": (C.c_int, [P, i64, P]),
        "cosm_server_stats": (C.c_int, [P, P]),
        "cosm_server_destroy": (None, [P]),
        "cosm_last_error": (C.c_char_p, []),
        "cosm_get_replica_energies": (C.c_int, [P, P]),
        "cosm_get_replica_bisectors": (C.c_int, [P, P]),
        "cosm_get_trace": (C.c_int, [P, P, i64]),
        "cosm_qubo_to_ising": (C.c_int, [i32, i64, P, P, P, P, P, P, P, P, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    return L


class _Lazy:
    """Loads libcosm.so on first use; raises ImportError if it is not built."""

    _handle = None

    def __getattr__(self, name):
        if _Lazy._handle is None:
            _Lazy._handle = _load()
        return getattr(_Lazy._handle, name)


_lib = _Lazy()


def lib():
    _lib.cosm_last_error  # force the load
    return _Lazy._handle


def _check(rc):
    if rc != OK:
        raise CosmError(rc, _lib.cosm_last_error().decode())
    return rc


def _p(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    return a.ctypes.data_as(C.c_void_p)


def _stream(s):
    if s is None:
        return None
    if hasattr(s, "cuda_stream"):
        return C.c_void_p(s.cuda_stream)
    return C.c_void_p(int(s))


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def default_params(**kw) -> Params:
    p = Params()
    _lib.cosm_default_params(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise TypeError(f"unknown parameter {k}")
        setattr(p, k, v)
    return p


def _desc(n, src, dst, w, color=None, n_colors=0, dims=(), h=None):
    keep = [_i32(src), _i32(dst), _i32(w)]
    d = GraphDesc()
    d.n = int(n)
    d.m = int(keep[0].shape[0])
    d.src, d.dst, d.w = (k.ctypes.data for k in keep)
    if color is not None:
        keep.append(_i32(color))
        d.color = keep[-1].ctypes.data
        d.n_colors = int(n_colors)
    if h is not None:
        keep.append(_i32(h))
        d.h = keep[-1].ctypes.data
    dd = list(dims) + [0] * (3 - len(dims))
    d.dims = (C.c_int32 * 3)(*dd[:3])
    return d, keep


class Solver:
    """One instance on the current CUDA device (cosm_create ... cosm_destroy)."""

    def __init__(self, n, src, dst, w, color=None, n_colors=0, dims=(), params=None, h=None, **kw):
        self.params = params if params is not None else default_params(**kw)
        desc, keep = _desc(n, src, dst, w, color, n_colors, dims, h)
        h = C.c_void_p()
        _check(_lib.cosm_create(C.byref(desc), C.byref(self.params), C.byref(h)))
        self._h = h
        self.n = int(n)
        self.replicas = 0

    @classmethod
    def from_instance(cls, inst, color=None, n_colors=0, use_dims=True, **kw):
        return cls(inst.n, inst.src, inst.dst, inst.w, color, n_colors,
                   inst.dims if use_dims else (), **kw)

    def close(self):
        if getattr(self, "_h", None):
            _lib.cosm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, sweeps, replicas, seed, stream=None, target=None):
        """cosm_run: one trial per replica; `target` is the success cut
        (cosm_get_success counts the replicas that reach it)."""
        self.replicas = int(replicas)
        self.sweeps = int(sweeps)
        _check(_lib.cosm_run(self._h, int(sweeps), int(replicas), int(seed),
                             NO_TARGET if target is None else int(target), _stream(stream)))

    def run_range(self, sweeps, s_from, s_to, replicas, seed, stream=None, target=None):
        """cosm_run_range: sweeps s_from..s_to of a `sweeps`-sweep trial."""
        self.replicas = int(replicas)
        self.sweeps = int(sweeps)
        _check(_lib.cosm_run_range(self._h, int(sweeps), int(s_from), int(s_to), int(replicas), int(seed),
                                   NO_TARGET if target is None else int(target), _stream(stream)))

    def success(self):
        """Replicas of the last readout whose cut reached the run's target."""
        c = C.c_int64()
        _check(_lib.cosm_get_success(self._h, C.byref(c)))
        return int(c.value)

    def export_state(self):
        """cosm_export_state: (phases in the storage type [replica][vertex],
        sweep index)."""
        dt = np.float32 if self.params.storage == F32 else np.uint16
        x = np.zeros((self.replicas, self.n), dtype=dt)
        idx = C.c_int64()
        _check(_lib.cosm_export_state(self._h, _p(x), int(self.params.storage), C.byref(idx)))
        return x, int(idx.value)

    def import_state(self, phases, replicas, seed, sweep_idx):
        """cosm_import_state: a checkpoint from export_state."""
        dt = np.float32 if self.params.storage == F32 else np.uint16
        x = np.ascontiguousarray(phases, dtype=dt)
        if x.size != int(replicas) * self.n:
            raise ValueError("checkpoint size does not match replicas x n")
        self.replicas = int(replicas)
        _check(_lib.cosm_import_state(self._h, _p(x), int(self.params.storage), int(replicas), int(seed),
                                      int(sweep_idx)))

    def set_wait_limit(self, seconds):
        _check(_lib.cosm_set_wait_limit(self._h, float(seconds)))

    def inject_fault(self, kind):
        _check(_lib.cosm_inject_fault(self._h, int(kind)))

    def replica_energies(self):
        out = np.zeros(self.replicas, dtype=np.int64)
        _check(_lib.cosm_get_replica_energies(self._h, _p(out)))
        return out

    def replica_bisectors(self):
        out = np.zeros(self.replicas, dtype=np.uint32)
        _check(_lib.cosm_get_replica_bisectors(self._h, _p(out)))
        return out

    def trace(self):
        """[replica][readout] energies of the last tracked run."""
        T = int(self.params.track_period)
        k = -(-self.sweeps // T) if T > 0 else 0
        out = np.zeros((self.replicas, max(k, 1)), dtype=np.int64)
        _check(_lib.cosm_get_trace(self._h, _p(out), self.replicas * k))
        return out[:, :k]

    def sync(self):
        _check(_lib.cosm_sync(self._h))

    def best(self, spins_out=None):
        cut, en, rep = C.c_int64(), C.c_int64(), C.c_int32()
        spins = spins_out if spins_out is not None else np.zeros(self.n, dtype=np.int8)
        _check(_lib.cosm_get_best(self._h, C.byref(cut), C.byref(en), C.byref(rep), _p(spins)))
        return int(cut.value), int(en.value), int(rep.value), spins

    def replica_cuts(self):
        cuts = np.zeros(self.replicas, dtype=np.int64)
        bps = np.zeros(self.replicas, dtype=np.int32)
        _check(_lib.cosm_get_replica_cuts(self._h, _p(cuts), _p(bps)))
        return cuts, bps

    def get_state(self):
        x = np.zeros((self.replicas, self.n), dtype=np.float64)
        _check(_lib.cosm_get_state(self._h, _p(x)))
        return x

    def set_state(self, phases, seed=0):
        x = np.ascontiguousarray(phases, dtype=np.float64)
        self.replicas = int(x.shape[0])
        _check(_lib.cosm_set_state(self._h, _p(x), self.replicas, int(seed)))

    def step(self, sweep, alpha, stream=None):
        _check(_lib.cosm_step(self._h, int(sweep), float(alpha), _stream(stream)))

    def readout(self, stream=None):
        _check(_lib.cosm_readout(self._h, _stream(stream)))

    def layout(self):
        out = (C.c_int32 * 8)()
        _check(_lib.cosm_layout(self._h, out))
        keys = ("K", "threads", "smem", "occupancy", "lattice", "grid", "launches", "colors")
        return dict(zip(keys, list(out)))


class Batch:
    """Many instances in one run (cosm_batch_*). `instances` is a list of
    objects with n, src, dst, w and dims (and optional colour arrays)."""

    def __init__(self, instances, params=None, colors=None, use_dims=True, **kw):
        self.params = params if params is not None else default_params(**kw)
        self.n = [int(i.n) for i in instances]
        self._keep = []
        descs = (GraphDesc * len(instances))()
        for k, inst in enumerate(instances):
            col, C_ = (colors[k] if colors is not None else (None, 0))
            d, keep = _desc(inst.n, inst.src, inst.dst, inst.w, col, C_,
                            inst.dims if use_dims else ())
            descs[k] = d
            self._keep.append(keep)
        h = C.c_void_p()
        _check(_lib.cosm_batch_create(len(instances), descs, C.byref(self.params), 1, C.byref(h)))
        self._h = h
        self.replicas = [0] * len(instances)

    def close(self):
        if getattr(self, "_h", None):
            _lib.cosm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, sweeps, replicas, seeds, stream=None):
        k = len(self.n)
        sw = np.ascontiguousarray(np.broadcast_to(sweeps, (k,)), dtype=np.int64)
        rp = np.ascontiguousarray(np.broadcast_to(replicas, (k,)), dtype=np.int32)
        sd = np.ascontiguousarray(np.broadcast_to(seeds, (k,)), dtype=np.uint64)
        self.replicas = [int(x) for x in rp]
        _check(_lib.cosm_batch_run(self._h, _p(sw), _p(rp), _p(sd), _stream(stream)))

    def sync(self):
        _check(_lib.cosm_batch_sync(self._h))

    def tune(self, replicas, probe_sweeps=20, stream=None):
        rp = np.ascontiguousarray(np.broadcast_to(replicas, (len(self.n),)), dtype=np.int32)
        _check(_lib.cosm_batch_tune(self._h, _p(rp), int(probe_sweeps), _stream(stream)))

    def best(self, i):
        cut, en, rep = C.c_int64(), C.c_int64(), C.c_int32()
        spins = np.zeros(self.n[i], dtype=np.int8)
        _check(_lib.cosm_batch_get_best(self._h, int(i), C.byref(cut), C.byref(en), C.byref(rep), _p(spins)))
        return int(cut.value), int(en.value), int(rep.value), spins

    def replica_cuts(self, i):
        cuts = np.zeros(self.replicas[i], dtype=np.int64)
        bps = np.zeros(self.replicas[i], dtype=np.int32)
        _check(_lib.cosm_batch_get_replica_cuts(self._h, int(i), _p(cuts), _p(bps)))
        return cuts, bps

    def get_state(self, i):
        x = np.zeros((self.replicas[i], self.n[i]), dtype=np.float64)
        _check(_lib.cosm_batch_get_state(self._h, int(i), _p(x)))
        return x

    def layout(self, i):
        """Layout of instance i in the last run (cosm_batch_layout)."""
        out = (C.c_int32 * 8)()
        _check(_lib.cosm_batch_layout(self._h, int(i), out))
        keys = ("K", "threads", "smem", "occupancy", "lattice", "grid", "launches", "colors")
        return dict(zip(keys, list(out)))

    def info(self):
        out = (C.c_int64 * 8)()
        _check(_lib.cosm_batch_info(self._h, out))
        keys = ("instances", "classes", "units", "launches", "graphs_built", "policy", "threads", "ctas")
        return dict(zip(keys, list(out)))


QUEUED, RUNNING, REACHED, EXHAUSTED = 0, 1, 2, 3


class Server:
    """Continuous-batching request server (cosm_server_*)."""

    def __init__(self, memory_budget=None, max_active=None, chunk_sweeps=None, threads=None):
        cfg = ServerConfig()
        _lib.cosm_server_default_config(C.byref(cfg))
        for k, v in (("memory_budget", memory_budget), ("max_active", max_active),
                     ("chunk_sweeps", chunk_sweeps), ("threads", threads)):
            if v is not None:
                setattr(cfg, k, int(v))
        self.cfg = cfg
        h = C.c_void_p()
        _check(_lib.cosm_server_create(C.byref(cfg), C.byref(h)))
        self._h = h
        self._n = {}

    def close(self):
        if getattr(self, "_h", None):
            _lib.cosm_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, inst, sweeps, replicas, seed, target_cut, max_trials=1, params=None, color=None,
               n_colors=0, use_dims=True, **kw):
        prm = params if params is not None else default_params(**kw)
        desc, keep = _desc(inst.n, inst.src, inst.dst, inst.w, color, n_colors,
                           inst.dims if use_dims else ())
        rid = C.c_int64()
        _check(_lib.cosm_server_submit(self._h, C.byref(desc), C.byref(prm), int(sweeps), int(replicas),
                                       int(seed), int(target_cut), int(max_trials), C.byref(rid)))
        self._n[rid.value] = int(inst.n)
        return int(rid.value)

    def poll(self, rid):
        out = RequestResult()
        _check(_lib.cosm_server_poll(self._h, int(rid), C.byref(out)))
        return out.as_dict()

    def wait(self, rid, timeout=60.0):
        out = RequestResult()
        _check(_lib.cosm_server_wait(self._h, int(rid), float(timeout), C.byref(out)))
        return out.as_dict()

    def spins(self, rid):
        sp = np.zeros(self._n[rid], dtype=np.int8)
        _check(_lib.cosm_server_get_spins(self._h, int(rid), _p(sp)))
        return sp

    def stats(self):
        out = (C.c_int64 * 8)()
        _check(_lib.cosm_server_stats(self._h, out))
        keys = ("queued", "active", "retired", "chunks", "launches", "max_concurrent",
                "peak_footprint", "footprint")
        return dict(zip(keys, list(out)))


def qubo_to_ising(n, qi, qj, qv):
    """QUBO triplets -> (src, dst, w, h, offset) with 4 f(x) = H(s) + offset
    (cosm_qubo_to_ising)."""
    qi, qj = _i32(qi), _i32(qj)
    qv = np.ascontiguousarray(qv, dtype=np.int64)
    nnz = int(qi.shape[0])
    src = np.zeros(max(nnz, 1), np.int32)
    dst = np.zeros(max(nnz, 1), np.int32)
    w = np.zeros(max(nnz, 1), np.int32)
    h = np.zeros(int(n), np.int32)
    m, off = C.c_int64(), C.c_int64()
    _check(_lib.cosm_qubo_to_ising(int(n), nnz, _p(qi), _p(qj), _p(qv), _p(src), _p(dst), _p(w),
                                   C.byref(m), _p(h), C.byref(off)))
    k = int(m.value)
    return src[:k].copy(), dst[:k].copy(), w[:k].copy(), h, int(off.value)


def solve(n, src, dst, w, sweeps, replicas, seed, color=None, n_colors=0, dims=(), params=None,
          replica_cuts=False, **kw):
    """One-shot host-buffer call (cosm_solve): returns (cut, energy, spins, cuts|None)."""
    prm = params if params is not None else default_params(**kw)
    desc, keep = _desc(n, src, dst, w, color, n_colors, dims)
    cut, en = C.c_int64(), C.c_int64()
    spins = np.zeros(int(n), dtype=np.int8)
    cuts = np.zeros(int(replicas), dtype=np.int64) if replica_cuts else None
    _check(_lib.cosm_solve(C.byref(desc), C.byref(prm), int(sweeps), int(replicas), int(seed),
                           C.byref(cut), C.byref(en), _p(spins), _p(cuts)))
    return int(cut.value), int(en.value), spins, cuts


def solve_static(n, src, dst, w, sweeps, replicas, seed, cuts_out, best_p_out, color=None,
                 n_colors=0, params=None, stream=None, **kw):
    """cosm_solve_static: no device allocation inside the library. cuts_out
    (int64) and best_p_out (int32) are caller-owned device buffers of
    `replicas` entries, e.g. torch tensors on the current device."""
    import torch
    for name, t in (("cuts_out", cuts_out), ("best_p_out", best_p_out)):
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor on the current device")
    dev = torch.cuda.current_device()
    for name, t, dt in (("cuts_out", cuts_out, torch.int64), ("best_p_out", best_p_out, torch.int32)):
        if t.device.index != dev:
            raise ValueError(f"{name} must be a CUDA tensor on the current device")
        if t.dtype != dt or not t.is_contiguous() or t.numel() < int(replicas):
            raise ValueError(f"{name} must be a contiguous {dt} tensor of at least {int(replicas)} entries")
    if stream is None:
        stream = torch.cuda.current_stream()
    prm = params if params is not None else default_params(**kw)
    desc, keep = _desc(n, src, dst, w, color, n_colors, ())
    _check(_lib.cosm_solve_static(C.byref(desc), C.byref(prm), int(sweeps), int(replicas), int(seed),
                                  _p(cuts_out), _p(best_p_out), _stream(stream)))


def probe_fp32(iters=4096):
    """Measured FP32 issue rate: (scalar, packed f32x2) FP32 operations per
    SM clock per SM (cosm_probe_fp32)."""
    a, b = C.c_double(), C.c_double()
    _check(_lib.cosm_probe_fp32(int(iters), C.byref(a), C.byref(b)))
    return float(a.value), float(b.value)


def probe_smem(iters=4096):
    """Measured shared-memory read bandwidth: (bytes per SM clock, device GB/s)."""
    bpc, gbps = C.c_double(), C.c_double()
    _check(_lib.cosm_probe_smem(int(iters), C.byref(bpc), C.byref(gbps)))
    return float(bpc.value), float(gbps.value)


def color_greedy(n, src, dst):
    src, dst = _i32(src), _i32(dst)
    col = np.zeros(src.shape[0], dtype=np.int32)
    nc = C.c_int32()
    _check(_lib.cosm_color_greedy(int(n), src.shape[0], _p(src), _p(dst), _p(col), C.byref(nc)))
    return col, int(nc.value)


def color_misra_gries(n, src, dst):
    src, dst = _i32(src), _i32(dst)
    col = np.zeros(src.shape[0], dtype=np.int32)
    nc = C.c_int32()
    _check(_lib.cosm_color_misra_gries(int(n), src.shape[0], _p(src), _p(dst), _p(col), C.byref(nc)))
    return col, int(nc.value)


def color_torus2d(L1, L2, src, dst):
    src, dst = _i32(src), _i32(dst)
    col = np.zeros(src.shape[0], dtype=np.int32)
    _check(_lib.cosm_color_torus2d(int(L1), int(L2), src.shape[0], _p(src), _p(dst), _p(col)))
    return col, 4


def color_torus3d(L1, L2, L3, src, dst):
    src, dst = _i32(src), _i32(dst)
    col = np.zeros(src.shape[0], dtype=np.int32)
    _check(_lib.cosm_color_torus3d(int(L1), int(L2), int(L3), src.shape[0], _p(src), _p(dst), _p(col)))
    return col, 6


def validate_partition(n, src, dst, n_colors, color) -> int:
    src, dst, color = _i32(src), _i32(dst), _i32(color)
    return int(_lib.cosm_validate_partition(int(n), src.shape[0], _p(src), _p(dst), int(n_colors),
                                            _p(color)))


__all__ = ["Solver", "Batch", "Server", "solve", "default_params", "color_greedy", "color_misra_gries",
           "color_torus2d", "color_torus3d", "validate_partition", "CosmError", "EXPORTS"]
