"""Pins of the mixed-representation oracle (oracle/mixed.py; Sec. II.C, the operator A = Q A-bar on
hole-grid vectors f_j(r) and its Chebyshev absorption spectrum). CPU only, 8^3 grid with every
eigenpair of the dense H0 (fixture tiny8)."""
import numpy as np
import pytest

from oracle import mixed, spectrum, tdh


@pytest.fixture(scope="module")
def setup(tiny8):
    p, v, e, phi = tiny8
    g = tdh.Grid(p.N, p.box)
    n_occ, n_o, n_c = 2, 2, 3
    coeff = tdh.stochastic_coefficients(3, 6, n_occ, "gaussian")
    op = tdh.TDHParams(n_steps=40, dt=0.05, gamma=0.2, alpha=1e-4, clean_every=10)
    W = tdh.screened_potentials(g, v, phi, n_occ, n_o, coeff, op)
    return g, v, e, phi, n_occ, n_o, n_c, W


def test_conduction_restriction_is_the_matrix_of_eq1(setup):
    """With Q the projector onto the n_c conduction states and f_j = sum_b f_jb phi_b, the
    coefficients <phi_a|(A f)_j> equal sum_{ib} A(ja, ib) f_ib with A assembled from the exchange
    and direct contractions (Eq. 1): the mixed representation reproduces the electron-hole matrix."""
    g, v, e, phi, n_occ, n_o, n_c, W = setup
    op = mixed.MixedA(g, v, phi, e, n_occ, n_o, n_c, W, 0.5, conduction_only=True)
    phi_o, eps_o, phi_c, eps_c = tdh.windows(phi, e, n_occ, n_o, n_c)
    A = tdh.assemble_A(eps_o, eps_c, 0.5, tdh.exchange_K(g, phi_o, phi_c), tdh.direct_D(g, phi_o, phi_c, W))
    coef = np.random.default_rng(1).standard_normal(n_o * n_c)
    f = np.einsum("jb,bxyz->jxyz", coef.reshape(n_o, n_c), phi_c)
    Af = op(f)
    got = np.einsum("jxyz,axyz->ja", Af, phi_c).reshape(-1) * g.dV
    assert np.max(np.abs(got - A @ coef)) < 1e-11 * np.max(np.abs(A @ coef))


def test_operator_is_symmetric_on_the_virtual_space(setup):
    g, v, e, phi, n_occ, n_o, n_c, W = setup
    op = mixed.MixedA(g, v, phi, e, n_occ, n_o, n_c, W, 0.5)
    rng = np.random.default_rng(2)
    f = op.Q(rng.standard_normal((n_o,) + phi.shape[1:]))
    h = op.Q(rng.standard_normal((n_o,) + phi.shape[1:]))
    a, b = op.dot(h, op(f)), op.dot(op(h), f)
    assert abs(a - b) < 1e-12 * max(abs(a), 1.0)


def test_residues_equal_the_spectral_sum_and_bounds_enclose_the_spectrum(setup):
    """The Chebyshev recursion against R_n = sum_k |<v_k|f0>|^2 T_n((E_k - c)/w) from the dense
    matrix of A in the basis phi_c e_j of the whole virtual space (all 510 virtual eigenstates of
    the 8^3 grid), and the Lanczos interval against that matrix's spectrum."""
    g, v, e_all, phi_all, n_occ, n_o, n_c, W = setup
    op = mixed.MixedA(g, v, phi_all, e_all, n_occ, n_o, n_c, W, 0.5)
    vir = phi_all[n_occ:]
    nv = vir.shape[0]
    basis = np.zeros((n_o * nv, n_o) + phi_all.shape[1:])
    for j in range(n_o):
        basis[j * nv:(j + 1) * nv, j] = vir
    M = np.empty((n_o * nv, n_o * nv))
    for col in range(n_o * nv):
        Af = op(basis[col])
        M[:, col] = np.einsum("kjxyz,jxyz->k", basis, Af) * g.dV
    assert np.max(np.abs(M - M.T)) < 1e-10 * np.max(np.abs(M))
    E, V = np.linalg.eigh(0.5 * (M + M.T))
    f0 = op.start(0)
    c0 = np.einsum("kjxyz,jxyz->k", basis, f0) * g.dV
    lo, hi = mixed.lanczos_bounds(op, f0, 40)
    assert lo < E[0] and E[-1] < hi
    c, w = 0.5 * (lo + hi), 0.5 * (hi - lo)
    R = mixed.residues(op, f0, 64, lo, hi)
    wts = (V.T @ c0) ** 2
    R_ref = np.array([np.sum(wts * np.cos(n * np.arccos((E - c) / w))) for n in range(64)])
    assert np.max(np.abs(R - R_ref)) < 1e-9 * R_ref[0]


def test_conduction_restricted_spectrum_equals_the_electron_hole_spectrum(setup):
    """The mixed route with the conduction projector and the electron-hole route of oracle/spectrum.py
    give the same residues and sigma for the same scaling interval."""
    g, v, e, phi, n_occ, n_o, n_c, W = setup
    op = mixed.MixedA(g, v, phi, e, n_occ, n_o, n_c, W, 0.5, conduction_only=True)
    phi_o, eps_o, phi_c, eps_c = tdh.windows(phi, e, n_occ, n_o, n_c)
    A = tdh.assemble_A(eps_o, eps_c, 0.5, tdh.exchange_K(g, phi_o, phi_c), tdh.direct_D(g, phi_o, phi_c, W))
    lo, hi = spectrum.gershgorin(A)
    omega = np.linspace(0.0, 3.0, 50)
    s_m, R_m, _ = mixed.absorption(op, 0, 128, lo, hi, 0.05, omega)
    f0 = spectrum.dipoles(g, phi_o, phi_c, 0)
    R_e = np.empty(128)
    c, w = 0.5 * (lo + hi), 0.5 * (hi - lo)
    At = (A - c * np.eye(len(f0))) / w
    v_prev, vv = None, f0.copy()
    for n in range(128):
        R_e[n] = f0 @ vv
        nxt = At @ vv if n == 0 else 2 * At @ vv - v_prev
        v_prev, vv = vv, nxt
    assert np.max(np.abs(R_m - R_e)) < 1e-11 * R_e[0]
    s_e = spectrum.sigma_chebyshev(R_e, c, w, omega, 0.05)
    assert np.max(np.abs(s_m - s_e)) < 1e-10 * np.max(np.abs(s_e))
