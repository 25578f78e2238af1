"""FP64 oracle of the absorption spectrum of the exciton matrix A by a Chebyshev expansion.

TEST INFRASTRUCTURE: imported only by the tests. Not part of the library's compute path.

The spectrum is the dipole-dipole correlation of Sec. II.C, evaluated in the electron-hole basis
(the paragraph after Eq. 18): sigma(omega) = omega <f0| delta(A - omega) |f0>, with the start vector
of dipole elements f0_ia = <phi_a| x |phi_i> and the delta function smoothed (here by a normalised
Gaussian of standard deviation s) and expanded in Chebyshev polynomials of the scaled matrix, so
that only the residues R_n = <f0|T_n(A~)|f0> of repeated applications of A are needed.

Readings of points the paper leaves open (shared with the CUDA path):
  * x is the coordinate along the chosen axis measured from the box centre, x = h i - box / 2
    (i the grid index along that axis); the systems are finite clusters in the middle of the box.
  * A~ = (A - c) / w with c, w from the Gershgorin bounds [lo, hi] of A: c = (lo + hi) / 2,
    w = 1.01 (hi - lo) / 2, so the spectrum of A~ lies strictly inside (-1, 1).
  * The smoothed delta is the Gaussian G_s(e) = exp(-e^2 / 2 s^2) / (s sqrt(2 pi)); its Chebyshev
    coefficients are taken by Chebyshev-Gauss quadrature on K = n_terms nodes
    x_k = cos(pi (k + 1/2) / K), i.e. c_n(omega) = (2 - delta_n0) / K sum_k G_s(E_k - omega) T_n(x_k)
    with E_k = c + w x_k, so sigma(omega) = omega / K sum_k G_s(E_k - omega) D_k,
    D_k = sum_{n < K} (2 - delta_n0) R_n T_n(x_k).

Arrays: orbitals (count, N, N, N) indexed [z, y, x]; electron-hole index ia = i * n_c + a.
"""
from __future__ import annotations

import numpy as np

from .tdh import Grid


def coordinate(grid: Grid, axis: int) -> np.ndarray:
    """x (axis 0), y (1) or z (2) from the box centre, as an (N, N, N) field."""
    c = grid.h * np.arange(grid.N) - 0.5 * grid.box
    shape = [1, 1, 1]
    shape[2 - axis] = grid.N  # arrays are [z, y, x]
    return np.broadcast_to(c.reshape(shape), (grid.N,) * 3)


def dipoles(grid: Grid, phi_o, phi_c, axis: int) -> np.ndarray:
    """f0_ia = <phi_a| x |phi_i> = sum_r phi_a(r) x(r) phi_i(r) dV, index ia = i * n_c + a."""
    x = coordinate(grid, axis)
    n_o, n_c = phi_o.shape[0], phi_c.shape[0]
    f0 = np.empty(n_o * n_c)
    for i in range(n_o):
        for a in range(n_c):
            f0[i * n_c + a] = np.sum(phi_c[a] * x * phi_o[i]) * grid.dV
    return f0


def gershgorin(A) -> tuple[float, float]:
    """Bounds lo <= every eigenvalue <= hi from the Gershgorin discs of the rows of A."""
    d = np.diag(A)
    r = np.sum(np.abs(A), axis=1) - np.abs(d)
    return float(np.min(d - r)), float(np.max(d + r))


def scaling(A) -> tuple[float, float]:
    """Centre c and half-width w of the map A~ = (A - c) / w (see the module reading)."""
    lo, hi = gershgorin(A)
    return 0.5 * (lo + hi), 1.01 * 0.5 * (hi - lo)


def residues(A, f0, n_terms: int) -> np.ndarray:
    """R_n = <f0| T_n(A~) |f0>, n < n_terms, by the three-term recursion of the Chebyshev
    polynomials applied to vectors: v_0 = f0, v_1 = A~ f0, v_{n+1} = 2 A~ v_n - v_{n-1}."""
    c, w = scaling(A)
    At = (A - c * np.eye(A.shape[0])) / w
    R = np.empty(n_terms)
    v_prev, v = None, f0.copy()
    for n in range(n_terms):
        R[n] = f0 @ v
        v_next = At @ v if n == 0 else 2.0 * (At @ v) - v_prev
        v_prev, v = v, v_next
    return R


def gaussian(e, s: float):
    return np.exp(-0.5 * (e / s) ** 2) / (s * np.sqrt(2.0 * np.pi))


def sigma_chebyshev(R, c: float, w: float, omega, s: float) -> np.ndarray:
    """sigma(omega) from the residues (module reading: K = len(R) quadrature nodes)."""
    K = len(R)
    theta = np.pi * (np.arange(K) + 0.5) / K
    n = np.arange(K)
    weights = np.where(n == 0, 1.0, 2.0)
    D = np.cos(np.outer(theta, n)) @ (weights * R)  # D_k
    E = c + w * np.cos(theta)
    omega = np.asarray(omega, dtype=float)
    return omega * (gaussian(E[None, :] - omega[:, None], s) @ D) / K


def sigma_exact(A, f0, omega, s: float) -> np.ndarray:
    """The same smoothed spectrum from the eigenpairs of A: omega sum_k |<v_k|f0>|^2 G_s(E_k - omega)."""
    E, V = np.linalg.eigh(0.5 * (A + A.T))
    wgt = (V.T @ f0) ** 2
    omega = np.asarray(omega, dtype=float)
    return omega * (gaussian(E[None, :] - omega[:, None], s) @ wgt)


def absorption(grid: Grid, phi_o, phi_c, A, axis: int, n_terms: int, s: float, omega):
    """Whole pipeline: dipoles, residues, smoothed spectrum. Returns (sigma, R, f0)."""
    f0 = dipoles(grid, phi_o, phi_c, axis)
    R = residues(A, f0, n_terms)
    c, w = scaling(A)
    return sigma_chebyshev(R, c, w, omega, s), R, f0
