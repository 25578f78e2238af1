"""Batching form: systems of uneven grids run concurrently give the results of separate runs."""
import numpy as np
import pytest

import sbse_inputs as si

pytestmark = pytest.mark.gpu


def test_concurrent_batch_of_uneven_grids_matches_separate_runs():
    from paper_2205_06690_gb300 import batch
    from paper_2205_06690_gb300 import binding as B

    items = []
    for seed, n in zip(range(100, 105), (16, 20, 24, 16, 12)):
        n_occ = n // 2
        p = si.model_system.Preset(f"b{seed}", N=n, box=0.5 * n, n_wells=max(2, round(2 * n_occ / 3)),
                                   seed=seed, n_occ=n_occ, n_o=3, n_c=4)
        s = si.make_system(p)
        items.append(batch.BatchItem(n, p.box, s.v_loc, s.phi, s.eps, n_occ, 3, 4, 0.5, 4))
    prm = B.TDHParams(n_s=10, n_steps=40, clean_every=10, dt=0.05, gamma=0.1, alpha=1e-4, seed=7)
    res, wall = batch.run_batch(items, prm, precision=B.SBSE_FP64, workers=5, tune=True)
    for it, r in zip(items, res):
        ref, _ = batch.run_batch([it], prm, precision=B.SBSE_FP64, workers=1, tune=False)
        assert np.array_equal(r["excitons"], ref[0]["excitons"])
    assert wall > 0 and all(r["pairs"] == 6 for r in res)
