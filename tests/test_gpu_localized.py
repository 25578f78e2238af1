"""Localized occupied window (Forward perspective: fewer (i, j) pairs through localized occupied
orbitals) through the C ABI against oracle/localized.py (GPU only). A double well (two equal wells
4 bohr apart, 12^3 grid, every eigenpair of the dense H0), N_occ = n_o = 3, n_c = 3, deterministic
TDH (L = N_occ, coefficients passed in), FP64:
* sbse_localize_occupied's rotation and sbse_pair_weights equal the oracle's (1e-10);
* with every pair kept and no cleaning, the excitons in the localized window equal the canonical
  ones (the rotation is exact; the kick's O(alpha) nonlinearity is below 1e-9 at alpha = 1e-8);
* with the pairs below a pair-density norm threshold screened out (no sbse_apply_W for them,
  SBSE_DIRECT_PARTIAL), the excitons equal the oracle's screened result (1e-10)."""
import numpy as np
import pytest

from oracle import localized as lo
from oracle import tdh
from sbse_inputs import model_system as ms

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2205_06690_gb300 import binding
    binding.load()
    return binding


def _double_well(N=12, box=10.0):
    wells = np.array([[3.0, 0.9, 3.0, 5.0, 5.0], [3.0, 0.9, 7.0, 5.0, 5.0]])
    v = ms.local_potential(N, box, wells)
    e, U = np.linalg.eigh(ms._dense_h0(N, box, v))
    dV = (box / N) ** 3
    return tdh.Grid(N, box), v, e[:6], (U[:, :6].T / np.sqrt(dV)).reshape(6, N, N, N)


def test_localized_window_matches_oracle(B):
    g, v, e, phi = _double_well()
    n_occ = n_o = n_c = 3
    coeff = np.sqrt(3.0) * np.eye(3)
    prm = B.TDHParams(n_s=3, n_steps=80, clean_every=10, dt=0.05, gamma=0.2, alpha=1e-8)
    op = tdh.TDHParams(n_steps=80, dt=0.05, gamma=0.2, alpha=1e-8, clean_every=10)
    pairs = tdh.pair_list(n_o)

    def ctx():
        c = B.Context(0, B.SBSE_FP64)
        c.set_grid(g.N, g.box, v)
        c.set_orbitals(n_occ, n_o, n_c, phi, e, 0.5)
        return c

    prm0 = B.TDHParams(n_s=3, n_steps=80, clean_every=0, dt=0.05, gamma=0.2, alpha=1e-8)
    with ctx() as c:
        c.apply_W(prm0, pairs, coeff=coeff)
        c.build_A()
        ev_canon = c.spectrum(6)
    U_ref, _ = lo.localize(lo.spread_matrices(g, phi[:n_occ]))
    phi_l = phi.copy()
    phi_l[:n_occ] = lo.rotate(phi[:n_occ], U_ref)
    w_ref = lo.pair_weights(g, phi_l[:n_occ])
    with ctx() as c:
        U = B.sbse_localize_occupied(c.h, n_o)
        assert np.max(np.abs(U - U_ref)) < 1e-10
        w = B.sbse_pair_weights(c.h, n_o)
        assert np.max(np.abs(w - np.array([w_ref[i, j] for i, j in pairs]))) < 1e-10
        c.apply_W(prm0, pairs, coeff=coeff)
        c.build_A()
        ev_loc = c.spectrum(6)
        assert np.max(np.abs(ev_loc - ev_canon)) < 1e-9
        # screening: drop the pairs whose pair density is below the median norm
        tau = float(np.median(w))
        kept = [pr for pr, wi in zip(pairs, w) if wi >= tau]
        assert 0 < len(kept) < len(pairs)
    with ctx() as c:
        B.sbse_localize_occupied(c.h, n_o)
        c.apply_W(prm, kept, coeff=coeff)
        with pytest.raises(B.SbseError):
            c.build_A()  # the full direct term needs every pair
        c.build_A(B.SBSE_EXCHANGE | B.SBSE_DIRECT_PARTIAL)
        ev_scr = c.spectrum(6)
    wfull = tdh.screened_potentials(g, v, phi_l, n_occ, n_o, coeff, op)
    wk = {pr: (wfull[pr] if pr in kept else np.zeros_like(wfull[pr])) for pr in pairs}
    phi_o, _, phi_c, eps_c = tdh.windows(phi_l, e, n_occ, n_o, n_c)
    A = lo.assemble_A_block(lo.occupied_block(e[:n_occ], U_ref), eps_c, 0.5, tdh.exchange_K(g, phi_o, phi_c),
                            tdh.direct_D(g, phi_o, phi_c, wk))
    assert np.max(np.abs(ev_scr - tdh.lowest_excitons(A, 6))) < 1e-10 * np.max(np.abs(ev_scr))
