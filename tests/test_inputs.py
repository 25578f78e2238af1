"""The seeded synthetic inputs shared by the oracle and the CUDA path (sbse_inputs): well draws,
the periodic local potential, and the two eigensolvers that produce the orbitals (CPU only)."""
import numpy as np

import sbse_inputs as si
from sbse_inputs import model_system as ms


def test_wells_follow_the_stated_distributions():
    w = ms.gaussian_wells(200, 16.0, 3)
    assert w.shape == (200, 5)
    assert np.all((2.0 <= w[:, 0]) & (w[:, 0] <= 4.0)) and np.all((0.8 <= w[:, 1]) & (w[:, 1] <= 1.2))
    assert np.all((4.0 <= w[:, 2:]) & (w[:, 2:] <= 12.0))
    assert np.array_equal(w, ms.gaussian_wells(200, 16.0, 3))
    assert not np.array_equal(w, ms.gaussian_wells(200, 16.0, 4))


def test_local_potential_of_one_well_is_a_periodic_gaussian():
    N, box = 16, 8.0
    well = np.array([[3.0, 1.0, 4.0, 4.0, 4.0]])
    v = ms.local_potential(N, box, well)
    h = box / N
    x = np.arange(N) * h - 4.0
    r2 = x[:, None, None] ** 2 + x[None, :, None] ** 2 + x[None, None, :] ** 2
    assert np.max(np.abs(v + 3.0 * np.exp(-r2 / 2.0))) < 1e-14
    # a well at the box edge wraps around (minimum image)
    v_edge = ms.local_potential(N, box, np.array([[3.0, 1.0, 0.0, 4.0, 4.0]]))
    assert abs(v_edge[8, 8, 1] - v_edge[8, 8, N - 1]) < 1e-14


def test_lobpcg_orbitals_equal_dense_diagonalisation():
    """On a 12^3 grid the iterative solver (used above 16^3) reproduces the lowest eigenpairs of the
    dense spectral Hamiltonian: eigenvalues to 1e-8, the spanned subspace to 1e-6."""
    N, box = 12, 7.0
    v = ms.local_potential(N, box, ms.gaussian_wells(5, box, 2))
    E, U = np.linalg.eigh(ms._dense_h0(N, box, v))
    e, vec = ms._lobpcg_h0(N, box, v, 6, 2, 1e-8)
    assert np.max(np.abs(e - E[:6])) < 1e-8
    P = U[:, :6] @ U[:, :6].T
    assert np.max(np.abs(P @ vec - vec)) < 1e-6


def test_system_orbitals_are_orthonormal_eigenstates():
    """make_system above 16^3 (iterative path): sum phi_s phi_t dV = delta_st and H0 phi = eps phi
    up to the solver tolerance, eigenvalues ascending."""
    p = ms.Preset("t18", N=18, box=9.0, n_wells=6, seed=5, n_occ=6, n_o=2, n_c=4)
    s = si.make_system(p)
    dV = s.dV
    G = np.einsum("sxyz,txyz->st", s.phi, s.phi) * dV
    assert np.max(np.abs(G - np.eye(10))) < 1e-10
    assert np.all(np.diff(s.eps) >= 0)
    k = ms._kvec(s.N, s.box)
    g2 = k[:, None, None] ** 2 + k[None, :, None] ** 2 + k[None, None, :] ** 2
    for t in range(10):
        hphi = np.real(np.fft.ifftn(0.5 * g2 * np.fft.fftn(s.phi[t]))) + s.v_loc * s.phi[t]
        assert np.sqrt(np.sum((hphi - s.eps[t] * s.phi[t]) ** 2) * dV) < 1e-4


def test_chebyshev_filtered_subspace_equals_dense_diagonalisation():
    """The filtered subspace iteration used on large grids (run here on the CPU): lowest eigenpairs
    of the dense spectral Hamiltonian of a 12^3 grid, eigenvalues to 1e-10, subspace to 1e-8."""
    from sbse_inputs import chfsi
    N, box = 12, 7.0
    v = ms.local_potential(N, box, ms.gaussian_wells(5, box, 2))
    E, U = np.linalg.eigh(ms._dense_h0(N, box, v))
    e, vec = chfsi.lowest_states(N, box, v, 6, 2, tol=1e-10, device="cpu")
    assert np.max(np.abs(e - E[:6])) < 1e-10
    P = U[:, :6] @ U[:, :6].T
    assert np.max(np.abs(P @ vec - vec)) < 1e-8


def test_chebyshev_coarse_grid_start_matches_lobpcg():
    """From 32^3 up the iteration starts from the half-edge problem, Fourier-interpolated: on a
    32^3 grid (seeded from 16^3) it reaches LOBPCG's eigenvalues to 1e-9."""
    from sbse_inputs import chfsi
    N, box = 32, 9.0
    v = ms.local_potential(N, box, ms.gaussian_wells(6, box, 4))
    e1, _ = ms._lobpcg_h0(N, box, v, 5, 4, 1e-9)
    e2, vec = chfsi.lowest_states(N, box, v, 5, 4, tol=1e-8, device="cpu")
    assert np.max(np.abs(e1 - e2)) < 1e-9
    assert np.max(np.abs(vec.T @ vec - np.eye(5))) < 1e-12


def test_learned_form_and_profiling_presets():
    """The learned form's systems: 20-80 wells drawn per seed, N_occ = round(1.5 wells), the 96^3
    system's box on a 64^3 grid; the profiling preset is the 96^3 grid and box with fewer states."""
    import sbse_inputs as si
    ps = si.fno_presets(40, first_seed=1000)
    assert [p.seed for p in ps] == list(range(1000, 1040))
    assert all(20 <= p.n_wells <= 80 and p.n_occ == round(1.5 * p.n_wells) for p in ps)
    assert all(p.N == 64 and p.box == 24.0 and p.n_o == 8 and p.n_c == 8 for p in ps)
    assert len({p.n_wells for p in ps}) > 10  # drawn, not fixed
    assert si.fno_presets(3, first_seed=1000)[0] == ps[0]  # reproducible
    big, prof = si.preset("large96"), si.preset("prof96")
    assert (prof.N, prof.box) == (big.N, big.box) and prof.n_occ < big.n_occ
