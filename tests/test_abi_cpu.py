"""CPU checks of the C ABI library: it loads, exports every symbol that
include/cosm.h declares, and its host-side colourers and partition checks
agree with the oracle's (bit-exact for the deterministic ones)."""
import os
import re
import subprocess

import numpy as np
import pytest

import instances

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="session")
def cosm():
    from paper_2605_30355_gb300 import build
    build.build()
    import paper_2605_30355_gb300 as cosm
    return cosm


def _declared():
    text = open(os.path.join(ROOT, "include", "cosm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cosm_[a-z0-9_]+)\s*\(", text)))


def test_header_declarations_are_exported(cosm):
    names = _declared()
    assert len(names) >= 19
    assert sorted(cosm.EXPORTS) == names
    out = subprocess.run(["nm", "-D", "--defined-only", cosm.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (cosm_[a-z0-9_]+)\b", out))
    for name in names:
        assert name in exported, name
        assert getattr(cosm.lib(), name)


def test_default_params_are_the_paper_settings(cosm):
    p = cosm.default_params()
    assert (p.alpha0_deg, p.dwt_ratio, p.dwt_period, p.window_deg, p.n_bisectors) == (14.0, 0.5, 3, 90.0, 100)


def test_greedy_colouring_matches_oracle(cosm, orc):
    for inst in (instances.random_regular(2000, 3, 1), instances.random_regular(2000, 4, 2),
                 instances.sparse_gnm(3000, 7500, 3), instances.torus2d(10, 12, 4)):
        a, ca = cosm.color_greedy(inst.n, inst.src, inst.dst)
        b, cb = orc.color_greedy(inst.n, inst.src, inst.dst)
        assert ca == cb and np.array_equal(a, b)


def test_misra_gries_uses_at_most_delta_plus_one(cosm, orc):
    for inst in (instances.random_regular(4000, 3, 5), instances.random_regular(4000, 4, 6),
                 instances.sparse_gnm(2000, 6000, 7), instances.torus3d(4, 4, 6, 8)):
        col, C = cosm.color_misra_gries(inst.n, inst.src, inst.dst)
        delta = np.bincount(np.concatenate([inst.src, inst.dst]), minlength=inst.n).max()
        assert C <= delta + 1
        assert orc.validate_partition(inst.n, inst.src, inst.dst, C, col) == 0


def test_lattice_colourings_match_oracle(cosm, orc):
    t2 = instances.torus2d(16, 20, 0)
    a, _ = cosm.color_torus2d(16, 20, t2.src, t2.dst)
    b, _ = orc.color_torus2d(16, 20, t2.src, t2.dst)
    assert np.array_equal(a, b)
    t3 = instances.torus3d(4, 6, 8, 1)
    a, _ = cosm.color_torus3d(4, 6, 8, t3.src, t3.dst)
    b, _ = orc.color_torus3d(4, 6, 8, t3.src, t3.dst)
    assert np.array_equal(a, b)
    with pytest.raises(cosm.CosmError):
        cosm.color_torus2d(15, 20, t2.src, t2.dst)


def test_partition_validator_agrees_with_oracle(cosm, orc):
    inst = instances.sparse_gnm(300, 900, 9)
    col, C = orc.color_greedy(inst.n, inst.src, inst.dst)
    assert cosm.validate_partition(inst.n, inst.src, inst.dst, C, col) == 0
    bad = col.copy()
    # put two edges sharing a vertex into one colour
    e0 = 0
    v = inst.src[e0]
    e1 = int(np.nonzero((inst.src == v) | (inst.dst == v))[0][1])
    bad[e1] = bad[e0]
    assert orc.validate_partition(inst.n, inst.src, inst.dst, C, bad) == 2
    assert cosm.validate_partition(inst.n, inst.src, inst.dst, C, bad) == cosm.ERR_NOT_A_MATCHING
    bad2 = col.copy()
    bad2[3] = C
    assert cosm.validate_partition(inst.n, inst.src, inst.dst, C, bad2) == cosm.ERR_PARTITION


def test_qubo_to_ising_matches_bruteforce(cosm, orc):
    # 4 f(x) = H(s) + offset for every x in {0,1}^n, x = (1 + s) / 2
    import itertools
    rng = np.random.default_rng(7)
    for trial in range(5):
        n = 7
        nnz = 25
        qi = rng.integers(0, n, nnz)
        qj = rng.integers(0, n, nnz)
        qv = rng.integers(-4, 5, nnz)
        src, dst, w, h, off = cosm.qubo_to_ising(n, qi, qj, qv)
        assert (src < dst).all() and (w != 0).all()
        Q = np.zeros((n, n), dtype=np.int64)
        np.add.at(Q, (qi, qj), qv)
        for bits in itertools.product([0, 1], repeat=n):
            x = np.array(bits)
            s = (2 * x - 1).astype(np.int8)
            f = int(x @ Q @ x)
            assert 4 * f == orc.energy_h(n, src, dst, w, h, s) + off


def test_qubo_to_ising_rejects_bad_input(cosm):
    with pytest.raises(cosm.CosmError) as e:
        cosm.qubo_to_ising(3, [0], [3], [1])
    assert e.value.code == cosm.ERR_INVALID_ARG
    with pytest.raises(cosm.CosmError) as e:
        cosm.qubo_to_ising(3, [0, 1], [1, 0], [100, 100])
    assert e.value.code == cosm.ERR_TOO_LARGE


def test_single_instance_features_rejected_by_batch_and_static(cosm):
    # checked on the host before any device work
    inst = instances.torus2d(8, 8, 1)
    h = np.ones(inst.n, dtype=np.int32)
    with pytest.raises(cosm.CosmError) as e:
        cosm.Batch([inst], track_period=10)
    assert e.value.code == cosm.ERR_INVALID_ARG
    with pytest.raises(cosm.CosmError) as e:
        cosm.Batch([inst], flags=cosm.OPT_BISECTOR)
    assert e.value.code == cosm.ERR_INVALID_ARG
    import ctypes as C
    desc, keep = cosm._desc(inst.n, inst.src, inst.dst, inst.w, h=h)
    b = C.c_void_p()
    p = cosm.default_params()
    rc = cosm.lib().cosm_batch_create(1, C.byref(desc), C.byref(p), 1, C.byref(b))
    assert rc == cosm.ERR_INVALID_ARG
    cuts = np.zeros(4, np.int64)
    bps = np.zeros(4, np.int32)
    rc = cosm.lib().cosm_solve_static(C.byref(desc), C.byref(p), 10, 4, 1, cosm._p(cuts), cosm._p(bps), None)
    assert rc == cosm.ERR_INVALID_ARG


def test_field_and_tracking_parameters_validated(cosm):
    inst = instances.torus2d(8, 8, 1)
    with pytest.raises(cosm.CosmError):
        cosm.Solver.from_instance(inst, track_period=-1)
    with pytest.raises(cosm.CosmError):
        cosm.Solver(inst.n, inst.src, inst.dst, inst.w, h=np.full(inst.n, 40000, np.int32))
    with pytest.raises(cosm.CosmError):
        cosm.Solver(inst.n, inst.src, inst.dst, inst.w, h=np.ones(inst.n, np.int32),
                    flags=cosm.OPT_BISECTOR)


def test_run_control_entries_reject_bad_arguments_on_the_host(cosm):
    # the entries added for run control and failure detection check their
    # arguments before any device work (no GPU needed here)
    import ctypes as C
    L = cosm.lib()
    NULL = None
    assert L.cosm_set_wait_limit(NULL, 1.0) == cosm.ERR_INVALID_ARG
    assert L.cosm_inject_fault(NULL, cosm.FAULT_DROP_SIGNAL) == cosm.ERR_INVALID_ARG
    c = C.c_int64()
    assert L.cosm_get_success(NULL, C.byref(c)) == cosm.ERR_INVALID_ARG
    assert L.cosm_run_range(NULL, 100, 1, 10, 4, 1, cosm.NO_TARGET, NULL) == cosm.ERR_INVALID_ARG
    assert L.cosm_run(NULL, 100, 4, 1, cosm.NO_TARGET, NULL) == cosm.ERR_INVALID_ARG
    buf = np.zeros(16, np.float32)
    assert L.cosm_export_state(NULL, cosm._p(buf), cosm.F32, NULL) == cosm.ERR_INVALID_ARG
    assert L.cosm_import_state(NULL, cosm._p(buf), cosm.F32, 1, 1, 0) == cosm.ERR_INVALID_ARG
    out = (C.c_int32 * 8)()
    assert L.cosm_batch_layout(NULL, 0, out) == cosm.ERR_INVALID_ARG
    a, b = C.c_double(), C.c_double()
    assert L.cosm_probe_fp32(0, C.byref(a), C.byref(b)) == cosm.ERR_INVALID_ARG


def test_static_entry_checks_output_buffers_before_device_work(cosm):
    # host arrays are not device memory: refused with INVALID_ARG, never
    # handed to a kernel (on a machine without a GPU the pointer query fails
    # the same way)
    import ctypes as C
    inst = instances.torus2d(8, 8, 1)
    desc, keep = cosm._desc(inst.n, inst.src, inst.dst, inst.w)
    p = cosm.default_params()
    cuts = np.zeros(4, np.int64)
    bps = np.zeros(4, np.int32)
    rc = cosm.lib().cosm_solve_static(C.byref(desc), C.byref(p), 10, 4, 1, cosm._p(cuts), cosm._p(bps), None)
    assert rc in (cosm.ERR_INVALID_ARG, cosm.ERR_CUDA)
    with pytest.raises(ValueError):
        cosm.solve_static(inst.n, inst.src, inst.dst, inst.w, 10, 4, 1, cuts, bps)
