"""The checked build (libcosm_checked.so: the kernels compiled with device
index checks, a stand-in for a memory checker, which is not available on
this GPU pool) runs every kernel family -- lattice passes in four storages,
edge lists at three tile widths (split records and weights, and records
carrying a +-1 weight's sign), the simultaneous-update ablation, local
fields with tracking and the optimal bisector, the ragged batch, the
wrap-around schedule -- with no check failing (cosm_sync would report
COSM_ERR_CHECK), and gives the normal build's results bit for bit."""
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _cases(cosm):
    """(name, thunk) pairs; each thunk returns arrays of the case's results."""
    import instances

    def single(inst, S, R, seed, env=None, h=None, **kw):
        def run():
            old = {k: os.environ.get(k) for k in (env or {})}
            os.environ.update(env or {})
            try:
                s = cosm.Solver.from_instance(inst, h=h, **kw)
                s.run(S, R, seed)
                s.sync()
                cuts, bps = s.replica_cuts()
                out = [cuts, bps, s.get_state()]
                if kw.get("track_period"):
                    out.append(s.trace())
                cut, en, rep, spins = s.best()
                out.append(np.array([cut, en, rep]))
                out.append(spins)
                s.close()
                return out
            finally:
                for k, v in old.items():
                    if v is None:
                        os.environ.pop(k, None)
                    else:
                        os.environ[k] = v
        return run

    def batch():
        insts = [instances.torus2d(16, 16, 3), instances.sparse_gnm(400, 1100, 4),
                 instances.random_regular(300, 3, 5)]
        b = cosm.Batch(insts, dwt_ratio=1.0)
        b.run([150, 120, 90], [6, 5, 9], [7, 8, 9])
        out = []
        for i in range(3):
            cut, en, rep, spins = b.best(i)
            out += [b.replica_cuts(i)[0], b.get_state(i), np.array([cut, en, rep]), spins]
        b.close()
        return out

    torus = instances.torus2d(16, 20, 1)
    gnm = instances.sparse_gnm(700, 2000, 2)
    reg3 = instances.random_regular(600, 3, 3)  # +-1 weights: records carrying the sign
    planted = instances.frustrated_loop_planted((12, 12), 0.6, 4)
    fields = instances.aligned_fields(planted, 1, 0.2)
    return [
        ("lattice_f32", single(torus, 200, 9, 11)),
        ("lattice_f16", single(torus, 200, 12, 12, storage=cosm.F16)),
        ("lattice_bf16", single(torus, 200, 12, 13, storage=cosm.BF16)),
        ("lattice_q16", single(torus, 200, 12, 14, storage=cosm.Q16)),
        ("edges_f32_k1", single(gnm, 150, 7, 15, env={"COSM_K": "1"}, dwt_ratio=1.0)),
        ("edges_f32_k2", single(gnm, 150, 8, 16, env={"COSM_K": "2"}, dwt_ratio=1.0)),
        ("edges_f32_k4", single(gnm, 150, 8, 17, env={"COSM_K": "4"}, dwt_ratio=1.0)),
        ("edges_signed_k2", single(reg3, 150, 8, 25, env={"COSM_K": "2"}, dwt_ratio=1.0)),
        ("edges_signed_k1", single(reg3, 150, 7, 26, env={"COSM_K": "1"}, dwt_ratio=1.0)),
        ("edges_signed_f16", single(reg3, 150, 8, 27, storage=cosm.F16, dwt_ratio=1.0)),
        ("edges_signed_q16", single(reg3, 150, 8, 28, storage=cosm.Q16, dwt_ratio=1.0)),
        ("edges_f16", single(gnm, 150, 8, 18, storage=cosm.F16, dwt_ratio=1.0)),
        ("edges_q16", single(gnm, 150, 8, 19, storage=cosm.Q16, dwt_ratio=1.0)),
        ("no_scs_f32", single(gnm, 100, 6, 20, flags=cosm.NO_SCS, dwt_ratio=1.0)),
        ("no_scs_q16", single(gnm, 100, 6, 21, storage=cosm.Q16, flags=cosm.NO_SCS, dwt_ratio=1.0)),
        ("fields_tracking", single(planted, 200, 6, 22, h=fields, track_period=25, alpha0_deg=25.0,
                                   dwt_ratio=1.0, flags=cosm.DWT_RANDOM_DIR)),
        ("opt_bisector", single(torus, 120, 5, 23, flags=cosm.OPT_BISECTOR, track_period=40)),
        ("wraparound", single(gnm, 301, 37, 24, env={"COSM_GRID_CAP": "5"}, dwt_ratio=1.0)),
        ("batch", batch),
    ]


def _run_all(cosm):
    res = {}
    for name, thunk in _cases(cosm):
        for k, a in enumerate(thunk()):
            res[f"{name}_{k}"] = np.asarray(a)
    return res


@pytest.mark.gpu
def test_checked_build_runs_clean_and_matches(tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2605_30355_gb300 import build
    build.build()
    build.build(checked=True)
    import paper_2605_30355_gb300 as cosm
    out = tmp_path / "checked.npz"
    env = dict(os.environ, COSM_LIBRARY="checked")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), str(out)], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    got = np.load(out)
    want = _run_all(cosm)
    assert sorted(got.files) == sorted(want)
    for k, v in want.items():
        assert np.array_equal(got[k], v), k


if __name__ == "__main__":
    # the checked build's side: every case through libcosm_checked.so; a
    # failed device check surfaces as COSM_ERR_CHECK from a synchronising call
    import paper_2605_30355_gb300 as cosm
    assert cosm.LIB_PATH.endswith("libcosm_checked.so"), cosm.LIB_PATH
    np.savez(sys.argv[1], **_run_all(cosm))
