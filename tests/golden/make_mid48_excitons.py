"""Writes tests/golden/mid48_excitons.json: the FP64 oracle's whole hot path on the 48^3 workload
(40 Gaussian wells, seed 1; N_occ = 60, n_o = 8, n_c = 16; all 36 pairs, L = 10 Gaussian
stochastic orbitals with seed 1, 1000 steps of dt = 0.05, gamma = 0.1, M = 10, alpha = 1e-4,
scissor 0.5 Ha): the lowest 10 excitons of A (Eq. 1), the orbital energies that identify the
inputs, and max |W_ij| with sum W_ij dV of a few pairs. Only oracle/ computes here (sbse_inputs
builds the orbitals); the pairs run in parallel processes, one pair each.

    python tests/golden/make_mid48_excitons.py [processes]
"""
import json
import multiprocessing as mp
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

SEED = 1
N_STEPS = 1000


def _pair(args):
    i, j = args
    import numpy as np

    import sbse_inputs as si
    from oracle import tdh
    p = si.preset("mid48")
    z = np.load(os.path.join(ROOT, "_golden_tmp", "sys.npz"))
    g = tdh.Grid(p.N, p.box)
    coeff = tdh.stochastic_coefficients(SEED, p.n_s, p.n_occ, "gaussian")
    op = tdh.TDHParams(n_steps=N_STEPS, dt=p.dt, gamma=p.gamma, alpha=p.alpha, clean_every=p.clean_every)
    w = tdh.screened_potentials(g, z["v_loc"], z["phi"], p.n_occ, p.n_o, coeff, op, pairs=[(i, j)])[(i, j)]
    np.save(os.path.join(ROOT, "_golden_tmp", f"w_{i}_{j}.npy"), w)
    return i, j


def main():
    import numpy as np

    import sbse_inputs as si
    from oracle import tdh
    procs = int(sys.argv[1]) if len(sys.argv) > 1 else (os.cpu_count() or 1)
    os.makedirs(os.path.join(ROOT, "_golden_tmp"), exist_ok=True)
    s = si.make_system(si.preset("mid48"))
    p = s.preset
    pairs = tdh.pair_list(p.n_o)
    np.savez(os.path.join(ROOT, "_golden_tmp", "sys.npz"), phi=s.phi[:p.n_occ], v_loc=s.v_loc)
    t0 = time.time()
    with mp.get_context("spawn").Pool(procs) as pool:
        for i, j in pool.imap_unordered(_pair, pairs):
            print(f"pair ({i},{j}) done at {time.time() - t0:.0f} s", flush=True)
    w = {pr: np.load(os.path.join(ROOT, "_golden_tmp", f"w_{pr[0]}_{pr[1]}.npy")) for pr in pairs}
    g = tdh.Grid(s.N, s.box)
    phi_o, eps_o, phi_c, eps_c = tdh.windows(s.phi, s.eps, p.n_occ, p.n_o, p.n_c)
    K = tdh.exchange_K(g, phi_o, phi_c)
    D = tdh.direct_D(g, phi_o, phi_c, w)
    A = tdh.assemble_A(eps_o, eps_c, p.scissor, K, D)
    ev = tdh.lowest_excitons(A, p.n_exc)
    sample = [(0, 0), (2, 5), (5, 7), (7, 7)]
    out = {
        "workload": "mid48", "seed": SEED, "n_steps": N_STEPS, "coeff": "gaussian",
        "excitons_ha": [float(x) for x in ev],
        "eps": [float(x) for x in s.eps[:p.n_occ + p.n_c]],
        "w_max_abs": {f"{i},{j}": float(np.max(np.abs(w[(i, j)]))) for i, j in sample},
        "w_integral": {f"{i},{j}": float(np.sum(w[(i, j)]) * g.dV) for i, j in sample},
        "oracle_seconds": time.time() - t0, "processes": procs,
    }
    with open(os.path.join(ROOT, "tests", "golden", "mid48_excitons.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out["excitons_ha"]))


if __name__ == "__main__":
    main()
