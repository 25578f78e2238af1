"""Pins of the localized-occupied-basis oracle (oracle/localized.py; Forward perspective: localized
occupied orbitals cut the number of (i, j) pairs needing W_ij). CPU only."""
import numpy as np

from oracle import localized as lo
from oracle import tdh
from sbse_inputs import model_system as ms
from conftest import rel_err


def _double_well(N=12, box=10.0):
    """Two equal wells 4 bohr apart along x: the two lowest states are the bonding and antibonding
    combinations of the two single-well ground states."""
    wells = np.array([[3.0, 0.9, 3.0, 5.0, 5.0], [3.0, 0.9, 7.0, 5.0, 5.0]])
    v = ms.local_potential(N, box, wells)
    e, U = np.linalg.eigh(ms._dense_h0(N, box, v))
    dV = (box / N) ** 3
    phi = (U[:, :6].T / np.sqrt(dV)).reshape(6, N, N, N)
    return tdh.Grid(N, box), v, e[:6], phi


def test_localization_splits_bonding_pair_into_left_and_right_states():
    g, v, e, phi = _double_well()
    Z = lo.spread_matrices(g, phi[:2])
    U, hist = lo.localize(Z)
    assert np.max(np.abs(U.T @ U - np.eye(2))) < 1e-13
    assert all(b >= a - 1e-14 for a, b in zip(hist, hist[1:]))
    loc = lo.rotate(phi[:2], U)
    # each localized state sits on one well (wells at x = 3 and x = 7, box 10)
    x = np.arange(g.N) * g.h
    centres = sorted(float(np.sum((loc[k] ** 2).sum(axis=(0, 1)) * x) * g.dV) for k in range(2))
    assert abs(centres[0] - 3.0) < 0.1 and abs(centres[1] - 7.0) < 0.1
    for k in range(2):
        side = x < 5.0 if np.sum((loc[k] ** 2)[:, :, x < 5.0]) > np.sum((loc[k] ** 2)[:, :, x >= 5.0]) else x >= 5.0
        assert np.sum((loc[k] ** 2)[:, :, side]) * g.dV > 0.95
    w0 = lo.pair_weights(g, phi[:2])[0, 1]
    w1 = lo.pair_weights(g, loc)[0, 1]
    assert w1 < 0.2 * w0
    # H0 in the rotated window: equal diagonal (symmetric wells), off-diagonal = half the splitting
    F = lo.occupied_block(e[:2], U)
    assert abs(F[0, 0] - F[1, 1]) < 1e-10 and abs(abs(F[0, 1]) - 0.5 * (e[1] - e[0])) < 1e-12


def test_rotated_window_gives_the_same_excitons_with_all_pairs():
    """Deterministic TDH (L = N_occ: the occupied density and its response do not depend on the
    basis of the occupied span), all pairs kept, no cleaning: A in the localized window (F instead
    of eps_o, K and D of the rotated pairs) has the canonical excitons, up to the O(alpha)
    nonlinearity of the finite kick (alpha = 1e-7 here). (With cleaning, the renormalization of each
    stochastic orbital to its own norm, Eq. 15 reading, depends on the basis at O(dt^2), because the
    propagated reference orbitals leave the occupied span at that order.)"""
    g, v, e, phi = _double_well()
    n_occ, n_o, n_c = 3, 3, 3
    coeff = np.sqrt(n_occ) * np.eye(n_occ)
    op = tdh.TDHParams(n_steps=80, dt=0.05, gamma=0.2, alpha=1e-7, clean_every=0)
    ref = tdh.run(g, v, phi, e, n_occ, n_o, n_c, 0.5, coeff, op, 6)
    U, _ = lo.localize(lo.spread_matrices(g, phi[:n_occ]))
    phi_l = phi.copy()
    phi_l[:n_occ] = lo.rotate(phi[:n_occ], U)
    w = tdh.screened_potentials(g, v, phi_l, n_occ, n_o, coeff, op)
    phi_o, _, phi_c, eps_c = tdh.windows(phi_l, e, n_occ, n_o, n_c)
    K = tdh.exchange_K(g, phi_o, phi_c)
    D = tdh.direct_D(g, phi_o, phi_c, w)
    A = lo.assemble_A_block(lo.occupied_block(e[:n_occ], U), eps_c, 0.5, K, D)
    assert np.max(np.abs(A - A.T)) < 1e-12
    assert np.max(np.abs(tdh.lowest_excitons(A, 6) - ref["excitons"])) < 2e-9


def test_screened_pairs_converge_to_the_full_result():
    """Dropping the pairs whose localized pair density is below tau (their D blocks zero) moves the
    excitons by an amount that shrinks with tau and vanishes at tau = 0."""
    g, v, e, phi = _double_well()
    n_occ, n_o, n_c = 3, 3, 3
    coeff = np.sqrt(n_occ) * np.eye(n_occ)
    op = tdh.TDHParams(n_steps=80, dt=0.05, gamma=0.2, alpha=1e-6, clean_every=10)
    U, _ = lo.localize(lo.spread_matrices(g, phi[:n_occ]))
    phi_l = phi.copy()
    phi_l[:n_occ] = lo.rotate(phi[:n_occ], U)
    wts = lo.pair_weights(g, phi_l[:n_occ])
    w = tdh.screened_potentials(g, v, phi_l, n_occ, n_o, coeff, op)
    phi_o, _, phi_c, eps_c = tdh.windows(phi_l, e, n_occ, n_o, n_c)
    K = tdh.exchange_K(g, phi_o, phi_c)
    F = lo.occupied_block(e[:n_occ], U)

    def excitons(tau):
        kept = {pr: (w[pr] if wts[pr] >= tau else np.zeros_like(w[pr])) for pr in w}
        return tdh.lowest_excitons(lo.assemble_A_block(F, eps_c, 0.5, K, tdh.direct_D(g, phi_o, phi_c, kept)), 6)

    full = excitons(0.0)
    taus = sorted({float(wts[pr]) for pr in w})
    errs = [np.max(np.abs(excitons(t * 1.0000001) - full)) for t in taus[:-1]]
    assert np.max(np.abs(excitons(0.0) - full)) == 0.0
    assert errs[0] <= errs[-1] + 1e-15
