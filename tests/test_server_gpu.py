"""Serving loop (continuous batching): a request's result is the same alone
and in a mix of concurrent requests, whatever the chunk size; a one-trial
request equals a plain cosm_run; fixed-point requests equal the oracle's
whole trials for every trial seed the server derives; admission respects
the slot count and the device-memory budget. Integer results (cuts, trial
and replica indices, spins) are compared exactly."""
import numpy as np
import pytest

import instances

pytestmark = pytest.mark.gpu

KEYS = ("status", "trials", "best_cut", "energy", "best_trial", "best_replica")


@pytest.fixture(scope="module")
def cosm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2605_30355_gb300 import build
    build.build()
    import paper_2605_30355_gb300 as cosm
    return cosm


def _requests():
    # (instance, sweeps, replicas, seed, target, max_trials, storage)
    p1 = instances.frustrated_loop_planted((16, 16), 0.5, 1)
    p2 = instances.frustrated_loop_planted((6, 6, 6), 0.4, 2)
    g3 = instances.gauge_planted(instances.torus2d(20, 20, 3), 4)
    r4 = instances.random_regular(700, 3, 5)
    return [(p1, 300, 16, 11, p1.meta["opt_cut"], 6, 1),
            (p2, 400, 8, 12, p2.meta["opt_cut"], 5, 1),
            (g3, 500, 12, 13, g3.meta["opt_cut"], 4, 0),
            (r4, 150, 10, 14, 10 ** 9, 3, 0)]


def _submit(srv, req):
    inst, S, R, seed, tgt, mt, storage = req
    return srv.submit(inst, S, R, seed, tgt, max_trials=mt, storage=storage, alpha0_deg=25.0,
                      dwt_ratio=1.0)


def test_one_trial_request_equals_plain_run(cosm):
    inst = instances.random_regular(800, 3, 1)
    srv = cosm.Server(chunk_sweeps=37)
    rid = srv.submit(inst, 200, 16, 5, 10 ** 9, max_trials=1, dwt_ratio=1.0)
    res = srv.wait(rid, 120)
    solo = cosm.Solver.from_instance(inst, dwt_ratio=1.0)
    solo.run(200, 16, 5)
    cut, energy, rep, spins = solo.best()
    assert res["status"] == cosm.EXHAUSTED and res["trials"] == 1
    assert (res["best_cut"], res["energy"], res["best_replica"]) == (cut, energy, rep)
    assert np.array_equal(srv.spins(rid), spins)
    assert res["updates"] == inst.m * 16 * 200
    srv.close()


def test_same_result_alone_and_in_the_mix(cosm):
    reqs = _requests()
    alone = []
    for req in reqs:
        srv = cosm.Server(chunk_sweeps=500)
        rid = _submit(srv, req)
        res = srv.wait(rid, 300)
        alone.append((tuple(res[k] for k in KEYS), srv.spins(rid)))
        srv.close()
    for chunk in (500, 53):
        srv = cosm.Server(chunk_sweeps=chunk)
        ids = [_submit(srv, req) for req in reqs]
        for rid, (want, spins) in zip(ids, alone):
            res = srv.wait(rid, 300)
            assert tuple(res[k] for k in KEYS) == want
            assert np.array_equal(srv.spins(rid), spins)
        st = srv.stats()
        assert st["retired"] == len(reqs) and st["max_concurrent"] >= 2
        srv.close()
    # planted optima are verified by energy where the target was reached
    for req, (want, _) in zip(reqs, alone):
        if want[0] == cosm.REACHED:
            assert want[2] >= req[4]


def test_fixed_point_requests_equal_oracle_trials(cosm, orc):
    # trial t of a request runs with seed + t * 0x9E3779B97F4A7C15 (mod 2^64);
    # in fixed point each is the oracle's trial bit for bit, so the server's
    # result is the oracle's: per trial the best replica (ties: the lowest),
    # a later trial kept only if strictly better, retired at the target
    p1 = instances.frustrated_loop_planted((12, 12), 0.6, 3)
    p2 = instances.frustrated_loop_planted((4, 4, 6), 0.4, 5)
    r3 = instances.random_regular(300, 3, 6)
    reqs = [(p1, 150, 6, 101, p1.meta["opt_cut"], 4), (p2, 120, 5, 102, p2.meta["opt_cut"], 3),
            (r3, 80, 4, 103, 10 ** 9, 3)]
    srv = cosm.Server(chunk_sweeps=47)
    ids = [srv.submit(inst, S, R, seed, tgt, max_trials=mt, storage=cosm.Q16, alpha0_deg=25.0,
                      dwt_ratio=1.0) for inst, S, R, seed, tgt, mt in reqs]
    for rid, (inst, S, R, seed, tgt, mt) in zip(ids, reqs):
        res = srv.wait(rid, 300)
        g = orc.coloured(inst)
        best, bt, br, bsp, status, trials = None, -1, -1, None, cosm.EXHAUSTED, 0
        for t in range(mt):
            st = (seed + t * 0x9E3779B97F4A7C15) % (1 << 64)
            outs = [orc.trial(g, S, alpha0=25.0 / 360.0, dwt_ratio=1.0, seed=st, replica=r,
                              storage=orc.STORE_Q16) for r in range(R)]
            cuts = [o[0] for o in outs]
            r = int(np.argmax(cuts))
            if best is None or cuts[r] > best:
                best, bt, br, bsp = cuts[r], t, r, outs[r][2]
            trials = t + 1
            if best >= tgt:
                status = cosm.REACHED
                break
        assert (res["status"], res["trials"], res["best_cut"], res["best_trial"], res["best_replica"]) == \
            (status, trials, best, bt, br)
        assert np.array_equal(srv.spins(rid), bsp)
    srv.close()


def test_admission_by_slots_and_memory_budget(cosm):
    inst = instances.torus2d(32, 32, 7)
    probe = cosm.Server()
    rid = probe.submit(inst, 100, 64, 1, 10 ** 9, max_trials=1)
    probe.wait(rid, 120)
    fp = probe.stats()["peak_footprint"]
    probe.close()
    assert fp > 0
    # room for one request at a time: they run one after another
    srv = cosm.Server(memory_budget=int(1.5 * fp), chunk_sweeps=40)
    ids = [srv.submit(inst, 100, 64, s, 10 ** 9, max_trials=1) for s in range(4)]
    res = [srv.wait(r, 120) for r in ids]
    st = srv.stats()
    assert st["max_concurrent"] == 1 and st["peak_footprint"] <= int(1.5 * fp)
    assert all(r["status"] == cosm.EXHAUSTED for r in res)
    # a request larger than the whole budget is refused at submission
    with pytest.raises(cosm.CosmError) as err:
        srv.submit(instances.torus2d(100, 100, 1), 100, 256, 1, 10 ** 9)
    assert err.value.code == cosm.ERR_TOO_LARGE
    srv.close()
    # slot limit
    srv = cosm.Server(max_active=2, chunk_sweeps=40)
    ids = [srv.submit(inst, 100, 8, s, 10 ** 9, max_trials=1) for s in range(6)]
    for r in ids:
        srv.wait(r, 120)
    assert srv.stats()["max_concurrent"] <= 2
    srv.close()
