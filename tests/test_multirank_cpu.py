"""The multi-GPU path on CPU: gloo, world size 2. Replicas shard across
ranks by seed with no exchange on the data path; the only collective is the
max over ranks of the timed region, and the whole-job rate is the units of
all ranks over that time. The reference arm runs on rank 0 only."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, times, out):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.max_over_ranks(times[rank])
    rate = bench.whole_job_rate(1000.0, world, t)
    seeds = [bench.rank_seed(1, r) for r in range(world)]
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, t, rate, seeds))


def test_two_ranks_gloo_max_time_and_rate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    times = [1.5, 2.5]
    procs = [ctx.Process(target=_worker, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, t, rate, seeds in got:
        assert t == 2.5                       # the slowest rank's time
        assert rate == pytest.approx(2 * 1000.0 / 2.5)
        assert len(set(seeds)) == 2           # disjoint Philox keys per rank


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    bench.main(["--impl", "reference", "--steps", "1", "--warmup", "0"])
    assert capsys.readouterr().out == ""


def _best_worker(rank, world, port, cuts, out):
    import numpy as np
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    spins = np.full(8, 1 if rank == 0 else -1, dtype=np.int8)
    spins[rank] = 0  # marks the owner
    best, owner, got = bench.global_best(cuts[rank], spins)
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, best, owner, got.tolist()))


@pytest.mark.parametrize("cuts,want_owner", [([10, 12], 1), ([12, 10], 0), ([7, 7], 0)])
def test_two_ranks_gloo_global_best(cuts, want_owner):
    # the end-of-run exchange: max cut over ranks (ties -> lowest rank) and
    # the owner's spins on every rank
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_best_worker, args=(r, 2, port, cuts, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, best, owner, spins in got:
        assert best == max(cuts) and owner == want_owner
        assert spins[want_owner] == 0 and spins[1 - want_owner] == (1 if want_owner == 0 else -1)


def test_spins_cut_helper():
    import numpy as np

    import bench
    import instances
    inst = instances.torus2d(8, 8, 1)
    s = np.ones(inst.n, dtype=np.int8)
    assert bench.spins_cut(inst, s) == 0
    s[0] = -1
    nb = (inst.src == 0) | (inst.dst == 0)
    assert bench.spins_cut(inst, s) == int(inst.w[nb].sum())
