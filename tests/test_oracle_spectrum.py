"""Pins of the FP64 oracle of the Chebyshev absorption spectrum (CPU only)."""
import numpy as np

from oracle import spectrum
from oracle.tdh import Grid


def _sym(n, seed):
    rng = np.random.default_rng(seed)
    M = rng.standard_normal((n, n))
    return 0.5 * (M + M.T) + np.diag(np.linspace(0.3, 1.2, n))


def test_residues_of_a_diagonal_matrix_are_chebyshev_polynomials_of_its_entries():
    """A = diag(d), f0 = e_k: R_n = T_n(d~_k) = cos(n arccos d~_k)."""
    d = np.array([0.2, 0.5, 0.9, 1.4])
    A = np.diag(d)
    c, w = spectrum.scaling(A)
    for k in range(len(d)):
        f0 = np.zeros(len(d))
        f0[k] = 1.0
        R = spectrum.residues(A, f0, 40)
        x = (d[k] - c) / w
        assert np.max(np.abs(R - np.cos(np.arange(40) * np.arccos(x)))) < 1e-12


def test_gershgorin_bounds_enclose_the_spectrum_and_scaling_maps_it_inside():
    A = _sym(30, 1)
    lo, hi = spectrum.gershgorin(A)
    E = np.linalg.eigvalsh(A)
    assert lo <= E.min() and E.max() <= hi
    c, w = spectrum.scaling(A)
    assert np.max(np.abs((E - c) / w)) < 1.0
    assert spectrum.gershgorin(np.diag([1.0, -2.0, 3.0])) == (-2.0, 3.0)


def test_chebyshev_spectrum_converges_to_the_eigenpair_sum():
    """Enough terms for the broadening: the expansion equals the exact smoothed spectrum."""
    A = _sym(24, 2)
    f0 = np.random.default_rng(3).standard_normal(24)
    c, w = spectrum.scaling(A)
    s = 0.08 * w / 10.0
    omega = np.linspace(c - w, c + w, 301)
    exact = spectrum.sigma_exact(A, f0, omega, s)
    errs = []
    for n in (100, 400, 1600):
        R = spectrum.residues(A, f0, n)
        errs.append(np.max(np.abs(spectrum.sigma_chebyshev(R, c, w, omega, s) - exact)) / np.max(np.abs(exact)))
    assert errs[2] < 1e-9 and errs[0] > errs[1] > errs[2]


def test_spectral_weight_sum_rule():
    """integral of sigma(omega) / omega d omega = |f0|^2 (the Gaussian is normalised)."""
    A = _sym(16, 4)
    f0 = np.random.default_rng(5).standard_normal(16)
    c, w = spectrum.scaling(A)
    s = 0.02 * w
    omega = np.linspace(c - 1.3 * w, c + 1.3 * w, 20001)
    R = spectrum.residues(A, f0, 1200)
    sig = spectrum.sigma_chebyshev(R, c, w, omega, s)
    integral = np.sum(sig / omega) * (omega[1] - omega[0])
    assert abs(integral - f0 @ f0) < 1e-6 * (f0 @ f0)


def test_dipole_of_a_gaussian_and_its_first_excitation():
    """phi0 = (pi g^2)^(-3/4) exp(-r^2 / 2 g^2), phi1 = sqrt(2) x / g phi0 (both normalised, centred
    in the box): <phi1| x |phi0> = g / sqrt(2); the y and z dipoles vanish by symmetry."""
    N, box, g = 32, 16.0, 1.3
    grid = Grid(N, box)
    x = spectrum.coordinate(grid, 0)
    y = spectrum.coordinate(grid, 1)
    z = spectrum.coordinate(grid, 2)
    phi0 = (np.pi * g * g) ** -0.75 * np.exp(-(x * x + y * y + z * z) / (2 * g * g))
    phi1 = np.sqrt(2.0) * x / g * phi0
    assert abs(grid.inner(phi0, phi0) - 1.0) < 1e-10 and abs(grid.inner(phi1, phi1) - 1.0) < 1e-10
    f = spectrum.dipoles(grid, phi0[None], phi1[None], 0)
    assert abs(f[0] - g / np.sqrt(2.0)) < 1e-10
    assert abs(spectrum.dipoles(grid, phi0[None], phi1[None], 1)[0]) < 1e-12
    assert abs(spectrum.dipoles(grid, phi0[None], phi1[None], 2)[0]) < 1e-12
    # the coordinate axes follow the [z, y, x] array layout
    assert np.all(np.diff(x[0, 0, :]) > 0) and np.all(x[:, :, 3] == x[0, 0, 3])
