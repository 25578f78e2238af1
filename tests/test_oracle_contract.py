"""Pins of the oracle's K and D contractions, of A (Eq. 1) and of its spectrum (CPU only)."""
import numpy as np

from oracle import tdh
from conftest import rel_err


def _direct_coulomb_matrix(N, box):
    """v(r, r') of the periodic box on the grid, summed directly over G != 0 (no FFT):
    sum_r' v(r, r') n(r') must equal the FFT Poisson solve, so v = (1/N^3) sum_G 4pi/G^2 e^{iG(r-r')}
    as a matrix acting on grid values (the dV of the integral and 1/Omega combine to 1/N^3)."""
    m = np.fft.fftfreq(N) * N
    G = 2 * np.pi / box * np.array(np.meshgrid(m, m, m, indexing="ij")).reshape(3, -1).T
    G2 = np.sum(G * G, axis=1)
    x = np.arange(N) * box / N
    R = np.array(np.meshgrid(x, x, x, indexing="ij")).reshape(3, -1).T  # (z, y, x) order
    Gk, G2k = G[G2 > 0], G2[G2 > 0]
    ph = np.exp(1j * R @ Gk.T)  # (n_g, nG)
    return np.real((ph * (4 * np.pi / G2k)) @ ph.conj().T) / N ** 3


def test_coulomb_matrix_brute_force_agrees_with_fft_solver():
    N, box = 4, 5.0
    V = _direct_coulomb_matrix(N, box)
    g = tdh.Grid(N, box)
    f = np.random.default_rng(1).standard_normal((N, N, N))
    assert rel_err(tdh.coulomb_periodic(f, g).reshape(-1), V @ f.reshape(-1)) < 1e-12


def test_exchange_and_direct_elements_by_double_sum():
    """(ia|jb) and (phi_a phi_b|W|phi_i phi_j) as explicit double sums over grid points, with
    distinct windows so that a swapped index or a transposed operand changes the result."""
    N, box = 4, 5.0
    g = tdh.Grid(N, box)
    rng = np.random.default_rng(2)
    n_o, n_c = 2, 3
    phi_o = rng.standard_normal((n_o, N, N, N))
    phi_c = rng.standard_normal((n_c, N, N, N))
    V = _direct_coulomb_matrix(N, box)
    dV = g.dV
    K = tdh.exchange_K(g, phi_o, phi_c)
    # a non-local, non-symmetric-looking W(r, r') acting on pair densities
    Wm = V + 0.3 * np.exp(-np.add.outer(np.arange(N ** 3), np.arange(N ** 3)) / 40.0)
    Wm = 0.5 * (Wm + Wm.T)
    w_pairs = {}
    for i in range(n_o):
        for j in range(i, n_o):
            w_pairs[(i, j)] = (Wm @ (phi_o[i] * phi_o[j]).reshape(-1)).reshape(N, N, N)
    D = tdh.direct_D(g, phi_o, phi_c, w_pairs)
    for i in range(n_o):
        for a in range(n_c):
            for j in range(n_o):
                for b in range(n_c):
                    ria = (phi_o[i] * phi_c[a]).reshape(-1)
                    rjb = (phi_o[j] * phi_c[b]).reshape(-1)
                    kref = ria @ V @ rjb * dV
                    assert abs(K[i * n_c + a, j * n_c + b] - kref) < 1e-10 * (1 + abs(kref))
                    rab = (phi_c[a] * phi_c[b]).reshape(-1)
                    rij = (phi_o[i] * phi_o[j]).reshape(-1)
                    dref = rab @ Wm @ rij * dV
                    assert abs(D[i * n_c + a, j * n_c + b] - dref) < 1e-10 * (1 + abs(dref))


def test_A_structure_and_exact_special_cases(tiny16):
    s = tiny16
    n_occ, n_o, n_c = 4, 2, 4
    g = tdh.Grid(s.N, s.box)
    phi_o, eps_o, phi_c, eps_c = tdh.windows(s.phi, s.eps, n_occ, n_o, n_c)
    # couplings switched off: A = diag(eps_a - eps_i + Delta) exactly, eigenvalues = differences
    A0 = tdh.assemble_A(eps_o, eps_c, 0.5)
    expect = np.array([eps_c[a] - eps_o[i] + 0.5 for i in range(n_o) for a in range(n_c)])
    assert np.array_equal(np.diag(A0), expect) and np.count_nonzero(A0 - np.diag(expect)) == 0
    assert np.allclose(tdh.lowest_excitons(A0, 4), np.sort(expect)[:4], rtol=0, atol=1e-15)
    # full A with a stochastic W is symmetric to rounding ((ia|jb) = (jb|ia), W_ji = W_ij)
    pr = tdh.TDHParams(n_steps=20, dt=0.05, gamma=0.01, alpha=1e-4, clean_every=10)
    c = tdh.stochastic_coefficients(0, 10, n_occ, "gaussian")
    out = tdh.run(g, s.v_loc, s.phi, s.eps, n_occ, n_o, n_c, 0.5, c, pr, 4)
    assert np.max(np.abs(out["A"] - out["A"].T)) < 1e-14 * np.max(np.abs(out["A"]))
    assert out["excitons"].shape == (4,) and np.all(np.diff(out["excitons"]) >= 0)


def test_one_by_one_A_by_hand(tiny16):
    """n_o = n_c = 1: A = eps_L - eps_H + Delta + 2 (HL|HL) - (LL|W|HH), each term by hand."""
    s = tiny16
    g = tdh.Grid(s.N, s.box)
    H, Lu = s.phi[3], s.phi[4]
    pr = tdh.TDHParams(n_steps=20, dt=0.05, gamma=0.01, alpha=1e-4, clean_every=10)
    c = tdh.stochastic_coefficients(0, 10, 4, "gaussian")
    out = tdh.run(g, s.v_loc, s.phi, s.eps, 4, 1, 1, 0.5, c, pr, 1)
    ex = np.sum(H * Lu * tdh.coulomb_periodic(H * Lu, g)) * g.dV
    w_hh = tdh.coulomb_periodic(H * H, g) + tdh.tdh_w_pol(g, s.v_loc, s.phi[:4], H * H, c, pr)
    di = np.sum(Lu * Lu * w_hh) * g.dV
    a11 = s.eps[4] - s.eps[3] + 0.5 + 2 * ex - di
    assert abs(out["A"][0, 0] - a11) < 1e-12 and abs(out["excitons"][0] - a11) < 1e-12
