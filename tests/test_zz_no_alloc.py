"""The no-allocation entry point against the allocating one.

cosm_solve_static serves callers that cannot allocate device memory: its
scratch is a static device array inside the library, and the caller passes
only device buffers for the results. Two calls in a row on different graphs
(the second overwrites the first's scratch) must each give exactly the
per-replica cuts and best bisectors that cosm_solve gives for the same graph,
seed and parameters (integers, so the tolerance is zero). This file is
collected last so that a stop at the first failure has run every other test.
"""
import numpy as np
import pytest

import instances

pytestmark = pytest.mark.gpu


def test_static_entry_matches_allocating_entry():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2605_30355_gb300 import build
    build.build()
    import paper_2605_30355_gb300 as cosm

    cases = [
        (instances.random_regular(600, 3, 1), 0, 7, 40, 300, dict(dwt_ratio=1.0)),
        (instances.sparse_gnm(900, 2500, 2), 1, 8, 33, 200, dict(dwt_ratio=1.0, n_bisectors=37)),
    ]
    for inst, storage, seed, R, S, kw in cases:
        col, C = cosm.color_misra_gries(inst.n, inst.src, inst.dst)
        _, _, _, ref = cosm.solve(inst.n, inst.src, inst.dst, inst.w, S, R, seed, color=col,
                                  n_colors=C, storage=storage, replica_cuts=True, **kw)
        s = cosm.Solver(inst.n, inst.src, inst.dst, inst.w, color=col, n_colors=C,
                        storage=storage, **kw)
        s.run(S, R, seed)
        ref_cuts, ref_bp = s.replica_cuts()
        assert np.array_equal(ref_cuts, ref)
        cuts = torch.full((R,), -1, dtype=torch.int64, device="cuda")
        bps = torch.full((R,), -1, dtype=torch.int32, device="cuda")
        cosm.solve_static(inst.n, inst.src, inst.dst, inst.w, S, R, seed, cuts, bps, color=col,
                          n_colors=C, storage=storage, **kw)
        torch.cuda.synchronize()
        assert np.array_equal(cuts.cpu().numpy(), ref_cuts)
        assert np.array_equal(bps.cpu().numpy(), ref_bp)
    # a problem beyond the static scratch is rejected before any device work
    big = instances.random_regular(20000, 4, 3)
    cuts = torch.zeros(8, dtype=torch.int64, device="cuda")
    bps = torch.zeros(8, dtype=torch.int32, device="cuda")
    with pytest.raises(cosm.CosmError) as err:
        cosm.solve_static(big.n, big.src, big.dst, big.w, 2_000_000, 8, 1, cuts, bps)
    assert err.value.code == cosm.ERR_TOO_LARGE
