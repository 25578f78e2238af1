"""Pins of the finite-box correction oracle (oracle/finite_box.py; Sec. III, W(k -> 0) =
eps_eff^-1 v_bndry) against closed forms and the behaviour the correction relies on (CPU only)."""
import numpy as np

import sbse_inputs as si
from oracle import finite_box as fb
from oracle import tdh


def test_boundary_set_and_average_closed_form():
    """The boundary of the periodic box has 3N^2 - 3N + 1 points; for f = cos(2 pi ix / N) its mean
    is (N - 1)^2 / (3N^2 - 3N + 1) (the plane ix = 0 contributes N^2 ones, every other ix the 2N - 1
    points with iy = 0 or iz = 0, and sum_{ix != 0} cos(2 pi ix / N) = -1)."""
    for N in (5, 8, 12):
        m = fb.boundary_mask(N)
        assert m.sum() == 3 * N * N - 3 * N + 1
        f = np.broadcast_to(np.cos(2 * np.pi * np.arange(N) / N)[None, None, :], (N, N, N))
        assert abs(fb.boundary_average(f) - (N - 1) ** 2 / (3 * N * N - 3 * N + 1)) < 1e-14


def test_boundary_potential_of_a_point_like_charge_falls_as_inverse_box_edge():
    """For a unit point charge the periodic (G = 0 dropped) potential on the boundary is a
    Madelung-type term, exactly proportional to 1/L; a Gaussian charge of width sigma adds
    2 pi sigma^2 / L^3 (its G != 0 components differ from the point charge's by -2 pi sigma^2 / Omega
    at small G). So L v_bndry - 2 pi sigma^2 / L^2 is the same for three box sizes (0.5 %). The local
    potential's part vanishes for a zero potential."""
    vals = []
    for L in (16.0, 20.0, 24.0):
        N = int(L / 0.5)
        g = tdh.Grid(N, L)
        x = np.arange(N) * g.h - L / 2
        r2 = x[:, None, None] ** 2 + x[None, :, None] ** 2 + x[None, None, :] ** 2
        rho = np.exp(-r2 / 2.0) / (2 * np.pi) ** 1.5  # unit charge, sigma = 1, at the box centre
        phi = np.sqrt(rho / 2.0)[None]  # n0 = 2 phi^2 = rho
        vals.append(L * fb.boundary_potential(g, np.zeros((N, N, N)), phi) - 2 * np.pi / L ** 2)
    assert max(vals) - min(vals) < 0.005 * abs(np.mean(vals))


def test_fit_recovers_a_known_inverse_dielectric_constant():
    rng = np.random.default_rng(0)
    e = rng.uniform(0.3, 0.6, 5)
    v = np.array([0.05, -0.02, -0.06, -0.08])
    E = e[None, :] + 0.3 * v[:, None]
    assert abs(fb.fit_inverse_dielectric(E, v) - 0.3) < 1e-14
    assert abs(fb.fit_inverse_dielectric(E, v + 1.0) - 0.3) < 1e-12  # a common offset of v is irrelevant
    assert np.max(np.ptp(fb.corrected(E, v, 0.3), axis=0)) < 1e-14


def test_correction_makes_the_box_sweep_spectra_overlap():
    """The method on one molecule (3 wells, drawn for an 8 bohr box) in boxes of 8, 10, 12 and 15
    bohr at h = 0.5, deterministic TDH (L = N_occ, no stochastic noise), 150 steps: the lowest
    excitons drift with the box size; lowering them by eps_eff^-1 v_bndry with the fitted
    eps_eff^-1 shrinks the spread across boxes at least threefold, with 0 < eps_eff^-1 < 1."""
    base = si.model_system.Preset("fb", N=16, box=8.0, n_wells=3, seed=7, n_occ=2, n_o=2, n_c=3,
                                  n_steps=150, gamma=0.2)
    E, v = [], []
    for p in si.box_sweep_presets(base, [8.0, 10.0, 12.0, 15.0]):
        s = si.make_system(p)
        g = tdh.Grid(p.N, p.box)
        coeff = np.sqrt(p.n_occ) * np.eye(p.n_occ)
        op = tdh.TDHParams(n_steps=p.n_steps, dt=0.05, gamma=p.gamma, alpha=1e-4, clean_every=10)
        E.append(tdh.run(g, s.v_loc, s.phi, s.eps, p.n_occ, p.n_o, p.n_c, 0.5, coeff, op, 4)["excitons"])
        v.append(fb.boundary_potential(g, s.v_loc, s.phi[:p.n_occ]))
    E, v = np.array(E), np.array(v)
    s_fit = fb.fit_inverse_dielectric(E, v)
    assert 0.0 < s_fit < 1.0
    assert np.max(np.ptp(fb.corrected(E, v, s_fit), axis=0)) < np.max(np.ptp(E, axis=0)) / 3
