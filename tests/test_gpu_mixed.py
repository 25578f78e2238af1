"""Mixed hole-grid representation of the BSE operator (Sec. II.C) through the C ABI against
oracle/mixed.py (GPU only). 8^3 grid with every eigenpair of the dense H0 (so that the occupied
projector and the conduction states are exact), N_occ = n_o = 2, n_c = 3, W from the library's FP64
propagation with the oracle's coefficients (matching the oracle's W to 1e-10):
* one application of A = Q A-bar (both projectors) on a random vector: 1e-9 relative;
* the Chebyshev residues and sigma for the same interval: 1e-8 relative; the Lanczos interval
  encloses the oracle's and agrees with it to 1e-6;
* with the conduction projector the residues equal those of the electron-hole matrix (sbse_absorption
  route) for the same interval."""
import numpy as np
import pytest

from oracle import mixed, spectrum, tdh

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2205_06690_gb300 import binding
    binding.load()
    return binding


def test_mixed_representation_matches_oracle(B, tiny8):
    p, v, e, phi = tiny8
    g = tdh.Grid(p.N, p.box)
    n_occ, n_o, n_c = 2, 2, 3
    coeff = tdh.stochastic_coefficients(3, 6, n_occ, "gaussian")
    op = tdh.TDHParams(n_steps=40, dt=0.05, gamma=0.2, alpha=1e-4, clean_every=10)
    W = tdh.screened_potentials(g, v, phi, n_occ, n_o, coeff, op)
    prm = B.TDHParams(n_s=6, n_steps=40, clean_every=10, dt=0.05, gamma=0.2, alpha=1e-4, seed=3)
    rng = np.random.default_rng(4)
    f = rng.standard_normal((n_o, p.N, p.N, p.N))
    with B.Context(0, B.SBSE_FP64) as c:
        c.set_grid(p.N, p.box, v)
        c.set_orbitals(n_occ, n_o, n_c, phi[:n_occ + n_c], e[:n_occ + n_c], 0.5)
        c.apply_W(prm, tdh.pair_list(n_o))
        for proj, cond in ((B.SBSE_Q_OCCUPIED, False), (B.SBSE_Q_CONDUCTION, True)):
            ref_op = mixed.MixedA(g, v, phi, e, n_occ, n_o, n_c, W, 0.5, conduction_only=cond)
            fq = ref_op.Q(f)
            got = B.sbse_apply_A_mixed(c.h, proj, fq.reshape(n_o, -1)).reshape(fq.shape)
            want = ref_op(fq)
            assert np.max(np.abs(got - want)) < 1e-9 * np.max(np.abs(want))
            f0 = ref_op.start(0)
            lo_r, hi_r = mixed.lanczos_bounds(ref_op, f0, 30)
            lo, hi = B.sbse_mixed_bounds(c.h, proj, 0, 30)
            assert abs(lo - lo_r) < 1e-6 * (hi_r - lo_r) and abs(hi - hi_r) < 1e-6 * (hi_r - lo_r)
            omega = np.linspace(0.0, 4.0, 64)
            sig, R = B.sbse_absorption_mixed(c.h, proj, 0, 96, lo_r, hi_r, 0.05, omega)
            s_ref, R_ref, _ = mixed.absorption(ref_op, 0, 96, lo_r, hi_r, 0.05, omega)
            assert np.max(np.abs(R - R_ref)) < 1e-8 * R_ref[0]
            assert np.max(np.abs(sig - s_ref)) < 1e-8 * np.max(np.abs(s_ref))
            if cond:
                A = c.build_A()
                f0e = spectrum.dipoles(g, phi[n_occ - n_o:n_occ], phi[n_occ:n_occ + n_c], 0)
                cc, w = 0.5 * (lo_r + hi_r), 0.5 * (hi_r - lo_r)
                At = (A - cc * np.eye(len(f0e))) / w
                Re, vp, vv = np.empty(96), None, f0e.copy()
                for n in range(96):
                    Re[n] = f0e @ vv
                    nxt = At @ vv if n == 0 else 2 * At @ vv - vp
                    vp, vv = vv, nxt
                assert np.max(np.abs(R - Re)) < 1e-8 * Re[0]
