"""The bench's reporting arithmetic on the CPU: the Wilson interval against
its closed form, the success statistics (P_s, R99 and TTT of Appendix A)
against hand counts, and the method's shared-memory byte count per update
on the bench's workloads."""
import math

import numpy as np
import pytest

import bench
import instances


def test_wilson_interval_closed_form():
    z = 1.96
    # no successes: [0, z^2 / (n + z^2)]
    for n in (10, 1000, 10240):
        lo, hi = bench.wilson(0, n)
        assert lo == 0.0 and hi == pytest.approx(z * z / (n + z * z))
    # all successes mirror it
    lo, hi = bench.wilson(50, 50)
    assert hi == 1.0 and lo == pytest.approx(1.0 - z * z / (50 + z * z))
    # a textbook case: 10 of 20 is symmetric about 1/2
    lo, hi = bench.wilson(10, 20)
    assert lo + hi == pytest.approx(1.0)
    assert hi - lo == pytest.approx(2 * z * math.sqrt(0.25 / 20 + z * z / 1600) / (1 + z * z / 20))
    # the interval contains the estimate and shrinks with n
    for k, n in ((3, 100), (30, 1000), (300, 10000)):
        lo, hi = bench.wilson(k, n)
        assert lo < k / n < hi
    assert bench.wilson(30, 1000)[1] - bench.wilson(30, 1000)[0] > \
        bench.wilson(300, 10000)[1] - bench.wilson(300, 10000)[0]


def test_success_statistics_by_hand():
    cuts = [np.array([10, 12, 12, 9]), np.array([12, 8, 11, 12])]
    st = bench.success_stats(cuts, 12, t_step=2.0, R=4)
    assert st["trials"] == 8 and st["best_cut"] == 12 and st["mean_cut"] == pytest.approx(86 / 8)
    top, lower = st["levels"][0], st["levels"][1]
    assert top["cut"] == 12 and top["hits"] == 4 and top["P_s"] == 0.5
    r99 = math.log(0.01) / math.log(0.5)
    assert top["R99"] == pytest.approx(r99) and top["TTT_s"] == pytest.approx(0.5 * r99)
    assert lower["cut"] == 10 and lower["hits"] == 6
    assert st["levels"][2]["hits"] == 8 and st["levels"][2]["R99"] == 1.0
    # never reached: no R99, no TTT
    none = bench.success_stats([np.array([1, 2])], 100, 1.0, 2)["levels"][0]
    assert none["P_s"] == 0.0 and none["R99"] is None and none["TTT_s"] is None


def test_method_byte_count_per_update():
    prm = dict(dwt_period=3)
    torus = instances.torus2d(100, 200, 0)
    # 4b + 2b n / (m P) + e / K with m = 2n on the torus
    assert bench.algorithmic_bytes(torus, prm, 4, 2, 2) == pytest.approx(16 + 4 / 3 + 0.125 / 2)
    assert bench.algorithmic_bytes(torus, prm, 2, 2, 4) == pytest.approx(8 + 2 / 3 + 0.125 / 4)
    reg3 = instances.random_regular(2000, 3, 1)
    assert bench.algorithmic_bytes(reg3, prm, 4, 0, 2) == pytest.approx(16 + 8 / 4.5 + 5 / 2)
    # no twist: no twist bytes
    assert bench.algorithmic_bytes(reg3, dict(dwt_period=0), 4, 0, 1) == pytest.approx(16 + 5)


def test_cut_distribution_summary():
    d = bench.cut_distribution([np.arange(100), np.arange(100, 200)])
    assert d["trials"] == 200 and d["min"] == 0 and d["max"] == 199
    assert d["mean"] == pytest.approx(99.5) and d["sem"] == pytest.approx(np.arange(200).std() / math.sqrt(200))
