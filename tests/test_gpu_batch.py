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
    with batch.Batch(items, B.SBSE_FP64) as bt:
        bt.run(prm, workers=5, tune=True)  # the first run goes one system at a time
        res, wall = bt.run(prm, workers=5, tune=True)  # concurrent graph replays
    for it, r in zip(items, res):
        ref, _ = batch.run_batch([it], prm, precision=B.SBSE_FP64, workers=1, tune=False)
        assert np.array_equal(r["excitons"], ref[0]["excitons"])
    assert wall > 0 and all(r["pairs"] == 6 for r in res)


def test_batch_systems_match_oracle_excitons():
    """Three systems of the 64-system batching workload (32^3, seeds 107, 108, 112; 10 pairs, L = 10,
    500 steps) run concurrently through the batching form against the FP64 oracle's excitons stored
    by tests/golden/make_batch_excitons.py (oracle only): FP64 within 1e-6 Ha (the orbitals are
    rebuilt here by the seeded iterative solver and agree with the stored ones only to its
    tolerance; their energies are checked to 1e-8 first), mixed within 5 meV."""
    import json
    import os

    from paper_2205_06690_gb300 import batch
    from paper_2205_06690_gb300 import binding as B

    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "batch_excitons.json")) as f:
        gold = json.load(f)["systems"]
    items = []
    for p in si.batch_presets():
        if str(p.seed) in gold:
            s = si.make_system(p)
            assert np.max(np.abs(s.eps[:p.n_occ + p.n_c] - np.array(gold[str(p.seed)]["eps"]))) < 1e-8
            items.append(batch.BatchItem(p.N, p.box, s.v_loc, s.phi, s.eps, p.n_occ, p.n_o, p.n_c, p.scissor,
                                         p.n_exc, seed=p.seed))
    assert len(items) == 3
    prm = B.TDHParams(n_s=10, n_steps=500, clean_every=10, dt=0.05, gamma=0.1, alpha=1e-4)
    for prec, tol in ((B.SBSE_FP64, 1e-6), (B.SBSE_MIXED, 5.0 / 27211.386245988)):
        with batch.Batch(items, prec) as bt:
            res, _ = bt.run(prm, workers=3, tune=True)
        for it, r in zip(items, res):
            assert np.max(np.abs(r["excitons"] - np.array(gold[str(it.seed)]["excitons_ha"]))) < tol
