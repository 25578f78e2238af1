"""Finite-box correction W(k -> 0) (Sec. III) through the C ABI against the oracle (GPU only): the
box-size sweep of one molecule (3 wells drawn for an 8 bohr box, centred in boxes of 8, 10, 12 and
15 bohr at h = 0.5), deterministic TDH (L = N_occ with the coefficients passed in), FP64: each
run's excitons and boundary potential against oracle/finite_box.py at 1e-10, the fitted eps_eff^-1
against the oracle's fit, and the corrected spectra overlapping three times better than the raw
ones; the corrected scissor (sbse_set_scissor) lowers a run's excitons by exactly W(k -> 0)."""
import numpy as np
import pytest

import sbse_inputs as si
from oracle import finite_box as fb
from oracle import tdh

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2205_06690_gb300 import binding
    binding.load()
    return binding


def test_box_sweep_matches_oracle_and_overlaps(B):
    from paper_2205_06690_gb300 import finite_box as gfb
    base = si.model_system.Preset("fb", N=16, box=8.0, n_wells=3, seed=7, n_occ=2, n_o=2, n_c=3,
                                  n_steps=150, gamma=0.2)
    systems = [si.make_system(p) for p in si.box_sweep_presets(base, [8.0, 10.0, 12.0, 15.0])]
    coeff = np.sqrt(2.0) * np.eye(2)
    prm = B.TDHParams(n_s=2, n_steps=150, clean_every=10, dt=0.05, gamma=0.2, alpha=1e-4)
    E, v, s_fit = gfb.box_sweep(systems, prm, 4, precision=B.SBSE_FP64, coeff=coeff)
    E_ref, v_ref = [], []
    for s in systems:
        p = s.preset
        g = tdh.Grid(p.N, p.box)
        op = tdh.TDHParams(n_steps=150, dt=0.05, gamma=0.2, alpha=1e-4, clean_every=10)
        E_ref.append(tdh.run(g, s.v_loc, s.phi, s.eps, 2, 2, 3, 0.5, coeff, op, 4)["excitons"])
        v_ref.append(fb.boundary_potential(g, s.v_loc, s.phi[:2]))
    E_ref, v_ref = np.array(E_ref), np.array(v_ref)
    assert np.max(np.abs(E - E_ref)) < 1e-10 * np.max(np.abs(E_ref))
    assert np.max(np.abs(v - v_ref)) < 1e-10 * np.max(np.abs(v_ref))
    assert abs(s_fit - fb.fit_inverse_dielectric(E_ref, v_ref)) < 1e-9
    assert np.max(np.ptp(E - s_fit * v[:, None], axis=0)) < np.max(np.ptp(E, axis=0)) / 3
    # the production run with its scissor lowered by W(k -> 0)
    s = systems[-1]
    p = s.preset
    with B.Context(0, B.SBSE_FP64) as c:
        c.set_grid(s.N, s.box, s.v_loc)
        c.set_orbitals(2, 2, 3, s.phi[:5], s.eps[:5], p.scissor)
        c.apply_W(prm, tdh.pair_list(2), coeff=coeff)
        c.build_A()
        ev0 = c.spectrum(4)
        B.sbse_set_scissor(c.h, p.scissor - gfb.w_k0(s_fit, v[-1]))
        c.build_A()
        ev1 = c.spectrum(4)
    assert np.max(np.abs(ev1 - (ev0 - s_fit * v[-1]))) < 1e-12
    with pytest.raises(B.SbseError):
        B.sbse_fit_inverse_dielectric(E[:1], v[:1])
