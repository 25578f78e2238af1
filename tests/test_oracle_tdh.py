"""Pins of the oracle's stochastic-TDH engine (Sec. II.B, Eqs. 10-15) on tiny grids (CPU only)."""
import numpy as np
import pytest

from oracle import rpa, tdh
from conftest import rel_err


def _det_coeff(n_occ):
    # deterministic TDH: L = N_occ stochastic orbitals with c = sqrt(N_occ) I gives eta_s = phi_s
    return np.sqrt(n_occ) * np.eye(n_occ)


@pytest.mark.parametrize("feedback", [False, True])
def test_deterministic_tdh_converges_to_casida_at_second_order(tiny8, feedback):
    """TDH of the full occupied set == the linear-response (Casida) damped W^pol up to O(dt^2)."""
    p, v, e, phi = tiny8
    g = tdh.Grid(p.N, p.box)
    n_occ = 2
    rho = phi[0] * phi[1]
    errs = []
    for dt in (0.04, 0.02):
        pr = tdh.TDHParams(n_steps=int(round(4.0 / dt)), dt=dt, gamma=0.5, alpha=1e-6,
                           clean_every=0, feedback=feedback)
        w = tdh.tdh_w_pol(g, v, phi[:n_occ], rho, _det_coeff(n_occ), pr)
        t = np.arange(pr.n_steps + 1) * dt
        wc = rpa.casida_w_pol(g, e, phi, n_occ, rho, t, tdh.time_weights(pr), feedback=feedback)
        errs.append(rel_err(w, wc))
    assert errs[1] < 2e-4
    assert 3.5 < errs[0] / errs[1] < 4.5  # second order in dt


def test_cleaning_is_second_order_for_the_full_set(tiny8):
    """For the full occupied set the occupied-occupied components cancel in the density (Sec. II.B),
    so Eq. (15) changes the deterministic W^pol only at O(alpha)."""
    p, v, e, phi = tiny8
    g = tdh.Grid(p.N, p.box)
    rho = phi[0] * phi[1]
    base = dict(n_steps=100, dt=0.04, gamma=0.5, alpha=1e-5)
    w0 = tdh.tdh_w_pol(g, v, phi[:2], rho, _det_coeff(2), tdh.TDHParams(clean_every=0, **base))
    w1 = tdh.tdh_w_pol(g, v, phi[:2], rho, _det_coeff(2), tdh.TDHParams(clean_every=10, **base))
    assert rel_err(w1, w0) < 1e-4


def test_single_occupied_state_stochastic_equals_deterministic(tiny8):
    """With N_occ = 1 and random signs, n = 2 sum_l |eta_l|^2 = 2 |phi_1|^2 for any L (Eq. 14):
    the stochastic W^pol equals the deterministic one to rounding."""
    p, v, e, phi = tiny8
    g = tdh.Grid(p.N, p.box)
    rho = phi[0] * phi[0]
    pr = tdh.TDHParams(n_steps=60, dt=0.05, gamma=0.3, alpha=1e-4, clean_every=10)
    c = tdh.stochastic_coefficients(11, 10, 1, "sign")
    w_st = tdh.tdh_w_pol(g, v, phi[:1], rho, c, pr)
    w_det = tdh.tdh_w_pol(g, v, phi[:1], rho, np.ones((1, 1)), pr)
    assert rel_err(w_st, w_det) < 1e-11


def test_difference_form_equals_two_set_form(tiny16):
    """The difference-form engine equals the paper's literal propagation of eta^alpha and eta^0."""
    s = tiny16
    g = tdh.Grid(s.N, s.box)
    rho = s.phi[2] * s.phi[3]
    c = tdh.stochastic_coefficients(5, 4, 4, "gaussian")
    pr = tdh.TDHParams(n_steps=40, dt=0.05, gamma=0.1, alpha=1e-4, clean_every=10)
    w1 = tdh.tdh_w_pol(g, s.v_loc, s.phi[:4], rho, c, pr)
    w2 = tdh.tdh_w_pol_two_set(g, s.v_loc, s.phi[:4], rho, c, pr)
    assert rel_err(w1, w2) < 1e-8


def test_norm_conservation_and_renormalisation(tiny16):
    s = tiny16
    g = tdh.Grid(s.N, s.box)
    prop = tdh._Propagator(g, s.v_loc, 0.05)
    c = tdh.stochastic_coefficients(3, 4, 4, "gaussian")
    a = tdh.stochastic_orbitals(c, s.phi[:4]).astype(complex)
    q = tdh.coulomb_periodic(s.phi[2] * s.phi[3], g)
    d = (np.exp(-1e-2j * q) - 1.0)[None] * a
    n0 = np.real(g.inner(a, a))
    u = 0.01 * q
    for _ in range(20):  # unitary split-operator steps: |eta^alpha| conserved
        a, d = prop.half_phase_pair(a, d, u)
        a, d = prop.kinetic(a), prop.kinetic(d)
        a, d = prop.half_phase_pair(a, d, u)
    assert rel_err(np.real(g.inner(a + d, a + d)), n0) < 1e-13
    d2 = tdh.clean(a, d, s.phi[:4], n0, g)
    assert rel_err(np.real(g.inner(a + d2, a + d2)), n0) < 1e-13
    # direct definition of Eq. (15) + renormalisation: eta^alpha <- c (eta0 + Q d) with
    # c = sqrt(N0 / |eta0 + Q d|^2), i.e. d <- c Q d + (c - 1) eta0
    ov = np.einsum("lzyx,szyx->ls", d, s.phi[:4]) * g.dV
    assert np.max(np.abs(ov)) > 1e-6  # the propagated difference is contaminated
    qd = d - np.einsum("ls,szyx->lzyx", ov, s.phi[:4])
    cc = np.sqrt(n0 / np.real(g.inner(a + qd, a + qd)))[:, None, None, None]
    assert rel_err(d2, cc * qd + (cc - 1.0) * a) < 1e-10


def test_kick_leaves_density_unchanged_and_response_is_linear(tiny16):
    s = tiny16
    g = tdh.Grid(s.N, s.box)
    rho = s.phi[2] * s.phi[3]
    c = tdh.stochastic_coefficients(9, 6, 4, "gaussian")
    rec = []
    pr = tdh.TDHParams(n_steps=30, dt=0.05, gamma=0.1, alpha=1e-4, clean_every=10)
    w1 = tdh.tdh_w_pol(g, s.v_loc, s.phi[:4], rho, c, pr, record=rec)
    u0 = rec[0][1]
    u_mid = np.max(np.abs(rec[15][1]))
    assert np.max(np.abs(u0)) < 1e-3 * u_mid  # u(0) = O(alpha^2), u(t > 0) = O(alpha)
    pr2 = tdh.TDHParams(n_steps=30, dt=0.05, gamma=0.1, alpha=0.5e-4, clean_every=10)
    w2 = tdh.tdh_w_pol(g, s.v_loc, s.phi[:4], rho, c, pr2)
    d12 = rel_err(w2, w1)
    pr4 = tdh.TDHParams(n_steps=30, dt=0.05, gamma=0.1, alpha=0.25e-4, clean_every=10)
    w4 = tdh.tdh_w_pol(g, s.v_loc, s.phi[:4], rho, c, pr4)
    assert d12 < 1e-3
    assert 1.6 < d12 / rel_err(w4, w2) < 2.4  # W^pol(alpha) - W^pol(alpha/2) = O(alpha)


def test_stochastic_estimate_unbiased_and_converges_as_inverse_sqrt(tiny8):
    """Without Hartree feedback the stochastic density response is bilinear in eta_l, so
    E[W^pol] = deterministic W^pol (E[c c'] = delta) and the RMS error falls as N_s^-1/2."""
    import sbse_inputs as si
    p = si.model_system.Preset("t8b", N=8, box=8.0, n_wells=6, seed=4, n_occ=6, n_o=2, n_c=2)
    v, e, phi = si.dense_eigensystem(p)
    g = tdh.Grid(8, 8.0)
    n_occ = 6
    rho = phi[4] * phi[5]
    pr = tdh.TDHParams(n_steps=40, dt=0.05, gamma=0.3, alpha=1e-5, clean_every=0,
                       feedback=False)
    w_det = tdh.tdh_w_pol(g, v, phi[:n_occ], rho, _det_coeff(n_occ), pr)
    rms = {}
    for n_s in (2, 8, 32):
        errs = []
        mean = np.zeros_like(w_det)
        for seed in range(24):
            c = tdh.stochastic_coefficients(1000 + seed, n_s, n_occ, "gaussian")
            w = tdh.tdh_w_pol(g, v, phi[:n_occ], rho, c, pr)
            mean += w / 24
            errs.append(np.sum((w - w_det) ** 2))
        rms[n_s] = np.sqrt(np.mean(errs))
        # the seed mean is closer to the deterministic value than a single estimate by ~sqrt(24)
        assert np.sqrt(np.sum((mean - w_det) ** 2)) < 0.45 * rms[n_s]
    slope = np.polyfit(np.log([2, 8, 32]), np.log([rms[2], rms[8], rms[32]]), 1)[0]
    assert -0.65 < slope < -0.35


def test_eigenstate_under_the_split_operator_propagator(tiny8):
    """With u = 0 an eigenstate of H0 = -1/2 Laplacian + V_loc stays itself up to a phase: after
    t = 2, |<phi|psi>| = 1 - O(dt^4) and the phase error of exp(-i eps t) is O(dt^2) (Strang
    splitting), i.e. it drops 4x when dt is halved."""
    p, v, e, phi = tiny8
    g = tdh.Grid(p.N, p.box)
    s = 1
    phase_err = []
    for dt in (0.02, 0.01):
        prop = tdh._Propagator(g, v, dt)
        psi = phi[s].astype(np.complex128)
        n = int(round(2.0 / dt))
        for _ in range(n):
            psi = prop.pv * prop.kinetic(prop.pv * psi)
        ov = g.inner(phi[s], psi)
        assert abs(abs(ov) - 1.0) < 1e-6
        phase_err.append(abs(np.angle(ov * np.exp(1j * e[s] * n * dt))))
    assert phase_err[1] < 1e-4 and 3.5 < phase_err[0] / phase_err[1] < 4.5


def test_deterministic_w_pol_is_symmetric_and_screens(tiny8):
    """Linear response of the full occupied set: <rho2|W^pol rho1> = <rho1|W^pol rho2> in the limit
    dt -> 0 (the discrete time grid breaks the symmetry at O(dt^2): 4x less per halving), with and
    without feedback; <rho|W^pol rho> < 0 and the screened <rho|v + W^pol|rho> is in (0, <rho|v rho>)."""
    p, v, e, phi = tiny8
    g = tdh.Grid(p.N, p.box)
    r1, r2 = phi[0] * phi[1], phi[0] * phi[0] - phi[1] * phi[1]
    for fb in (False, True):
        asym = []
        for dt in (0.04, 0.02):
            pr = tdh.TDHParams(n_steps=int(round(4.0 / dt)), dt=dt, gamma=0.5, alpha=1e-6, clean_every=0,
                               feedback=fb)
            w1 = tdh.tdh_w_pol(g, v, phi[:2], r1, _det_coeff(2), pr)
            w2 = tdh.tdh_w_pol(g, v, phi[:2], r2, _det_coeff(2), pr)
            a, b = np.sum(r2 * w1) * g.dV, np.sum(r1 * w2) * g.dV
            asym.append(abs(a - b) / max(abs(a), abs(b)))
            for r, w in ((r1, w1), (r2, w2)):
                pol = np.sum(r * w) * g.dV
                bare = np.sum(r * tdh.coulomb_periodic(r, g)) * g.dV
                assert pol < 0.0 and 0.0 < bare + pol < bare
        assert asym[1] < 1e-4 and 3.5 < asym[0] / asym[1] < 4.5


def test_tdh_energy_is_conserved_to_second_order_in_dt(tiny8):
    """Time-dependent Hartree conserves E = 2 sum_s <psi_s|H0|psi_s> + 1/2 <dn|v|dn> (spin factor 2
    of Eq. 11, dn = n^alpha - n^0) when the reference density is stationary, i.e. for the full
    occupied set of eigenstates without cleaning: dE/dt = 0 follows from i psi' = (H0 + v dn) psi.
    The split-operator steps of Eq. (10) keep it up to O(dt^2): over the same time span the largest
    excursion |E(t) - E(0)| falls about four times per halving of dt (dt = 0.02 .. 0.005 over 3 au,
    the asymptotic range on this grid). A strong kick (alpha = 0.2) makes the Hartree term visible;
    a wrong sign, factor or time level of u breaks the scaling."""
    p, v, e, phi = tiny8
    g = tdh.Grid(p.N, p.box)
    n_occ = 2
    rho = phi[0] * phi[1]
    k = 2.0 * np.pi / p.box * (np.fft.fftfreq(p.N) * p.N)
    g2 = k[:, None, None] ** 2 + k[None, :, None] ** 2 + k[None, None, :] ** 2

    def energy(a, d):
        psi = a + d
        hpsi = np.fft.ifftn(0.5 * g2 * np.fft.fftn(psi, axes=(1, 2, 3)), axes=(1, 2, 3)) + v * psi
        e_h0 = 2.0 * np.sum((psi.conj() * hpsi).real) * g.dV
        dn = 2.0 * np.sum(np.abs(psi) ** 2 - np.abs(a) ** 2, axis=0)
        return e_h0 + 0.5 * np.sum(dn * tdh.coulomb_periodic(dn, g)) * g.dV

    drift = []
    for dt in (0.02, 0.01, 0.005):
        pr = tdh.TDHParams(n_steps=int(round(3.0 / dt)), dt=dt, gamma=0.0, alpha=0.2, clean_every=0)
        es = []
        tdh.tdh_w_pol(g, v, phi[:n_occ], rho, _det_coeff(n_occ), pr,
                      observe=lambda n, a, d: es.append(energy(a, d)))
        a0 = tdh.stochastic_orbitals(_det_coeff(n_occ), phi[:n_occ]).astype(complex)
        q = tdh.coulomb_periodic(rho, g)
        d0 = (np.exp(-1j * pr.alpha * q) - 1.0)[None] * a0
        drift.append(np.max(np.abs(np.array(es) - energy(a0, d0))))
    assert drift[2] < 1e-7 * abs(energy(a0, d0))
    assert 3.6 < drift[0] / drift[1] < 4.6 and 3.6 < drift[1] / drift[2] < 4.6
    # the H0 part alone is not conserved (the Hartree term exchanges energy with it)
    es_h0 = []
    tdh.tdh_w_pol(g, v, phi[:n_occ], rho, _det_coeff(n_occ), pr,
                  observe=lambda n, a, d: es_h0.append(2.0 * np.sum((np.conj(a + d) * (np.fft.ifftn(
                      0.5 * g2 * np.fft.fftn(a + d, axes=(1, 2, 3)), axes=(1, 2, 3)) + v * (a + d))).real) * g.dV))
    assert np.max(np.abs(np.array(es_h0) - energy(a0, d0))) > 100 * drift[2]


@pytest.mark.parametrize("feedback", [False, True])
def test_static_casida_limit_equals_dense_rpa_solve(tiny8, feedback):
    """The static branch of the linear-response route (weights=None, S = 1/Omega) against the
    paper's W = v + v chi v written out directly on the 8^3 grid: chi0(r, r') =
    -4 sum_{s,c} phi_s phi_c(r) phi_s phi_c(r') / (eps_c - eps_s) over every occupied x virtual pair
    of the dense H0, v the Coulomb operator applied to unit vectors, chi = (1 - chi0 v)^-1 chi0
    (chi = chi0 without Hartree feedback), W^pol rho = v chi v rho."""
    p, v, e, phi = tiny8
    g = tdh.Grid(p.N, p.box)
    n_occ = 2
    ng = p.N ** 3
    rho = phi[0] * phi[1]
    occ = phi[:n_occ].reshape(n_occ, ng)
    vir = phi[n_occ:].reshape(-1, ng)
    chi0 = np.zeros((ng, ng))
    for s_ in range(n_occ):
        prod = occ[s_][None, :] * vir
        chi0 -= 4.0 * (prod.T / (e[n_occ:] - e[s_])) @ prod
    V = np.stack([tdh.coulomb_periodic(np.eye(ng)[r].reshape(rho.shape), g).reshape(-1) for r in range(ng)], axis=1)
    X0 = chi0 * g.dV
    q = V @ rho.reshape(-1)
    dn = np.linalg.solve(np.eye(ng) - X0 @ V, X0 @ q) if feedback else X0 @ q
    w_ref = (V @ dn).reshape(rho.shape)
    w = rpa.casida_w_pol(g, e, phi, n_occ, rho, None, None, feedback=feedback)
    assert rel_err(w, w_ref) < 1e-9
