"""Writes tests/golden/batch_excitons.json: the FP64 oracle's whole hot path for three systems of
the 64-system batching workload (sbse_inputs.batch_presets: the first three with a 32^3 grid,
seeds 107, 108 and 112; box 8 bohr, 11 wells, N_occ = 16, n_o = 4, n_c = 8, 10 pairs, L = 10
Gaussian stochastic orbitals with the system's seed, 500 steps of dt = 0.05, gamma = 0.1, M = 10,
alpha = 1e-4, scissor 0.5 Ha): the lowest 4 excitons and the orbital energies that identify the
inputs. Only oracle/ computes here (sbse_inputs builds the orbitals); one process per system.

    python tests/golden/make_batch_excitons.py
"""
import json
import multiprocessing as mp
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

SEEDS = (107, 108, 112)


def _system(seed):
    import sbse_inputs as si
    from oracle import tdh
    p = [q for q in si.batch_presets() if q.seed == seed][0]
    s = si.make_system(p)
    g = tdh.Grid(s.N, s.box)
    coeff = tdh.stochastic_coefficients(seed, p.n_s, p.n_occ, "gaussian")
    op = tdh.TDHParams(n_steps=p.n_steps, dt=p.dt, gamma=p.gamma, alpha=p.alpha, clean_every=p.clean_every)
    r = tdh.run(g, s.v_loc, s.phi, s.eps, p.n_occ, p.n_o, p.n_c, p.scissor, coeff, op, p.n_exc)
    return seed, {"excitons_ha": [float(x) for x in r["excitons"]],
                  "eps": [float(x) for x in s.eps[:p.n_occ + p.n_c]], "N": p.N, "n_steps": p.n_steps}


def main():
    t0 = time.time()
    with mp.get_context("spawn").Pool(len(SEEDS)) as pool:
        out = dict(pool.map(_system, SEEDS))
    res = {"systems": {str(k): v for k, v in out.items()}, "coeff_seed": "the system's seed",
           "oracle_seconds": time.time() - t0}
    with open(os.path.join(ROOT, "tests", "golden", "batch_excitons.json"), "w") as f:
        json.dump(res, f, indent=1)
    print(json.dumps({k: v["excitons_ha"] for k, v in res["systems"].items()}))


if __name__ == "__main__":
    main()
