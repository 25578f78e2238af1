"""FP64 oracle of the localized-occupied-basis route to fewer W_ij (Forward perspective: localized
occupied orbitals reduce the number of (i, j) pairs whose W_ij(r) is needed).

TEST INFRASTRUCTURE: imported only by the tests. Never part of the library's compute path.

Steps (readings of a direction the paper states without formulas):
  * Localize the n_o window of occupied orbitals by an orthogonal rotation phi'_k = sum_i U_ik phi_i
    that maximises the periodic (Gamma-point) localization functional
    Omega(U) = sum_{alpha=x,y,z} sum_k |Z'_alpha,kk|^2,  Z_alpha,ij = sum_r phi_i phi_j e^{i 2 pi x_alpha / L} dV,
    by Jacobi sweeps over pairs (i, j): the rotation angle theta = atan2(R, (P - Q) / 2) / 4 with
    P = sum_alpha |(Z_ii - Z_jj) / 2|^2, Q = sum_alpha |Z_ij|^2, R = sum_alpha Re((Z_ii - Z_jj) / 2 conj(Z_ij))
    maximises the pair's share of Omega exactly.
  * The occupied block of H0 in the rotated window is F = U^T diag(eps_o) U, and A of Eq. (1) in that
    basis reads A_{ia,jb} = delta_ab (eps_a delta_ij - F_ij) + Delta delta_ij delta_ab + 2 K - D (the
    same matrix as in the canonical basis up to the rotation U x 1, hence the same excitons).
  * Pairs are screened by the norm of their pair density, w_ij = (sum_r (phi'_i phi'_j)^2 dV)^1/2;
    pairs below a threshold get no W_ij (their direct elements are taken as zero).
"""
from __future__ import annotations

import numpy as np

from .tdh import Grid


def spread_matrices(grid: Grid, phi_o: np.ndarray) -> np.ndarray:
    """Z[alpha, i, j] = sum_r phi_i phi_j exp(i 2 pi x_alpha / L) dV, alpha = x, y, z (complex)."""
    N = grid.N
    n = phi_o.shape[0]
    ph = np.exp(2j * np.pi * np.arange(N) / N)
    fields = [ph[None, None, :], ph[None, :, None], ph[:, None, None]]  # x, y, z (arrays are [z, y, x])
    P = phi_o.reshape(n, -1)
    Z = np.empty((3, n, n), dtype=np.complex128)
    for a, f in enumerate(fields):
        w = np.broadcast_to(f, (N, N, N)).reshape(-1)
        Z[a] = (P * w[None, :]) @ P.T * grid.dV
    return Z


def localization_functional(Z: np.ndarray) -> float:
    return float(np.sum(np.abs(np.diagonal(Z, axis1=1, axis2=2)) ** 2))


def localize(Z: np.ndarray, max_sweeps: int = 100, tol: float = 1e-12):
    """Jacobi maximisation of Omega. Returns (U, functional values after each sweep)."""
    Z = Z.copy()
    n = Z.shape[1]
    U = np.eye(n)
    hist = [localization_functional(Z)]
    for _ in range(max_sweeps):
        for i in range(n - 1):
            for j in range(i + 1, n):
                u = 0.5 * (Z[:, i, i] - Z[:, j, j])
                z = Z[:, i, j]
                Pv = np.sum(np.abs(u) ** 2)
                Qv = np.sum(np.abs(z) ** 2)
                Rv = np.sum((u * np.conj(z)).real)
                theta = 0.25 * np.arctan2(Rv, 0.5 * (Pv - Qv))
                if abs(theta) < 1e-15:
                    continue
                c, s = np.cos(theta), np.sin(theta)
                G = np.eye(n)
                G[i, i], G[i, j], G[j, i], G[j, j] = c, -s, s, c  # new i = c i + s j, new j = -s i + c j
                Z = np.einsum("ki,akl,lj->aij", G, Z, G)
                U = U @ G
        hist.append(localization_functional(Z))
        if hist[-1] - hist[-2] <= tol * max(1.0, abs(hist[-1])):
            break
    return U, hist


def rotate(phi_o: np.ndarray, U: np.ndarray) -> np.ndarray:
    """phi'_k = sum_i U_ik phi_i."""
    n = phi_o.shape[0]
    return (U.T @ phi_o.reshape(n, -1)).reshape(phi_o.shape)


def occupied_block(eps_o: np.ndarray, U: np.ndarray) -> np.ndarray:
    """F = U^T diag(eps_o) U, the matrix of H0 in the rotated window."""
    return U.T @ np.diag(eps_o) @ U


def pair_weights(grid: Grid, phi_o: np.ndarray) -> np.ndarray:
    """w[i, j] = ||phi_i phi_j||_2 (sum over the grid with dV)."""
    n = phi_o.shape[0]
    P = phi_o.reshape(n, -1)
    return np.sqrt(((P ** 2) @ (P ** 2).T) * grid.dV)


def assemble_A_block(F: np.ndarray, eps_c: np.ndarray, scissor: float, K=None, D=None) -> np.ndarray:
    """A_{ia,jb} = delta_ab (eps_a delta_ij - F_ij) + Delta delta_ij delta_ab + 2 K - D."""
    n_o, n_c = F.shape[0], len(eps_c)
    A = (np.kron(np.eye(n_o), np.diag(eps_c)) - np.kron(F, np.eye(n_c))
         + scissor * np.eye(n_o * n_c))
    if K is not None:
        A = A + 2.0 * K
    if D is not None:
        A = A - D
    return A
