"""Finite-box correction W(k -> 0) of Sec. III (the paragraph before the algorithm summary): run the
method for one molecule in boxes of several sizes, take each run's average Kohn-Sham potential on
the box boundary (sbse_boundary_potential), fit eps_eff^-1 so that the spectra overlap
(sbse_fit_inverse_dielectric), and lower the scissor of the production run by
W(k -> 0) = eps_eff^-1 v_bndry (sbse_set_scissor). Orchestration only: every number is computed by
the library."""
from __future__ import annotations

import numpy as np

from . import binding as B


def run_box(system, params, pairs, k: int, precision=B.SBSE_MIXED, coeff=None, device: int = 0):
    """Lowest k excitons and v_bndry of one run (all pairs of the system's window)."""
    p = system.preset
    ns = p.n_occ + p.n_c
    with B.Context(device, precision) as c:
        c.set_grid(system.N, system.box, system.v_loc)
        c.set_orbitals(p.n_occ, p.n_o, p.n_c, system.phi[:ns], system.eps[:ns], p.scissor)
        c.apply_W(params, pairs, coeff=coeff)
        c.build_A()
        ev = c.spectrum(k)
        vb = B.sbse_boundary_potential(c.h)
    return ev, vb


def box_sweep(systems, params, k: int, precision=B.SBSE_MIXED, coeff=None, device: int = 0):
    """Excitons E (n_box x k), boundary potentials v (n_box) and the fitted eps_eff^-1."""
    E, v = [], []
    for s in systems:
        pairs = [(i, j) for i in range(s.preset.n_o) for j in range(i, s.preset.n_o)]
        ev, vb = run_box(s, params, pairs, k, precision, coeff, device)
        E.append(ev)
        v.append(vb)
    E = np.array(E)
    v = np.array(v)
    return E, v, B.sbse_fit_inverse_dielectric(E, v)


def w_k0(eps_inv: float, v_bndry: float) -> float:
    """W(k -> 0) = eps_eff^-1 v_bndry; the production scissor is Delta - W(k -> 0)."""
    return eps_inv * v_bndry
