"""FP64 oracle of the finite-box correction W(k -> 0) (Sec. III, the paragraph before the algorithm
summary): the scissor shift is lowered by W(k -> 0) = eps_eff^-1 v_bndry, where v_bndry is the
average Kohn-Sham potential on the box boundary of a run and eps_eff^-1 is the one parameter that
makes the spectra of runs in boxes of several sizes overlap.

TEST INFRASTRUCTURE: imported only by the tests. Never part of the library's compute path.

Readings (the paper prints no formula beyond W(k -> 0) = eps_eff^-1 v_bndry):
  * The model's Kohn-Sham potential is V_loc plus the Hartree potential of the ground-state density
    n0 = 2 sum_{s <= N_occ} |phi_s|^2 (spin factor of Eq. 11), both in the zero-average convention of
    a periodic calculation: V_loc minus its mean, and v n0 with G = 0 dropped (the Coulomb operator
    of the library).
  * The boundary of the periodic box [0, L)^3 is the set of grid points with ix = 0, iy = 0 or iz = 0
    (x = L is x = 0); v_bndry is the plain mean over those 3 N^2 - 3 N + 1 points.
  * "The spectra overlap" is taken in the least-squares sense: with E[b, k] the k-th exciton of the
    run in box b, eps_eff^-1 minimises sum_{b,k} (E[b,k] - s v[b] - mean_b'(E[b',k] - s v[b']))^2,
    i.e. s = sum_{b,k} (E[b,k] - Ebar_k)(v[b] - vbar) / (K sum_b (v[b] - vbar)^2).
  * The corrected excitons of a run are E - s v_bndry (the scissor lowered by W(k -> 0)).
"""
from __future__ import annotations

import numpy as np

from .tdh import Grid, coulomb_periodic


def boundary_mask(N: int) -> np.ndarray:
    """Grid points on the boundary planes of the periodic box, as an (N, N, N) boolean array."""
    m = np.zeros((N, N, N), dtype=bool)
    m[0, :, :] = True
    m[:, 0, :] = True
    m[:, :, 0] = True
    return m


def boundary_average(f: np.ndarray) -> float:
    """Mean of a field over the boundary planes (reading above)."""
    return float(np.mean(f[boundary_mask(f.shape[-1])]))


def ks_potential(grid: Grid, v_loc: np.ndarray, phi_occ: np.ndarray) -> np.ndarray:
    """V_loc - mean(V_loc) + v n0, n0 = 2 sum_s |phi_s|^2 (reading above)."""
    n0 = 2.0 * np.sum(phi_occ ** 2, axis=0)
    return v_loc - np.mean(v_loc) + coulomb_periodic(n0, grid)


def boundary_potential(grid: Grid, v_loc: np.ndarray, phi_occ: np.ndarray) -> float:
    """v_bndry of one run: the boundary average of its Kohn-Sham potential."""
    return boundary_average(ks_potential(grid, v_loc, phi_occ))


def fit_inverse_dielectric(E: np.ndarray, v: np.ndarray) -> float:
    """Least-squares eps_eff^-1 that makes the exciton lists E[b, :] of the boxes b overlap."""
    E = np.asarray(E, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    dv = v - v.mean()
    dE = E - E.mean(axis=0, keepdims=True)
    return float(np.sum(dE * dv[:, None]) / (E.shape[1] * np.sum(dv ** 2)))


def corrected(E: np.ndarray, v: np.ndarray, s: float) -> np.ndarray:
    """Excitons with the scissor lowered by W(k -> 0) = s v_bndry of each run."""
    return np.asarray(E) - s * np.asarray(v)[:, None]
