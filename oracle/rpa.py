"""Deterministic linear-response (RPA / Casida) evaluation of the damped W^pol of Eq. (13).

TEST INFRASTRUCTURE: imported only by the tests. Used to pin the TDH engine in `oracle.tdh` on
tiny grids by an independent route (dense linear algebra instead of time stepping).

Derivation (W = v + v chi v, Sec. II.B first paragraph; the TDH response to the kick
psi_s(0) = e^{-i alpha q} phi_s for the full set of occupied states). Write
psi_s(t) = e^{-i eps_s t} (phi_s + sum_c z_sc(t) phi_c) over occupied s and virtual c. To first order
in alpha, Eq. (10) gives i dz_sc/dt = (eps_c - eps_s) z_sc + <phi_c|u|phi_s> with
u = v delta n, delta n = 4 sum_sc Re(z_sc) phi_s phi_c (the spin factor 2 of n = 2 sum|psi|^2), so
with z = x + i y:  x'' = -D (D + 4V) x, x(0) = 0, x'(0) = -alpha D Q, where D = diag(eps_c - eps_s),
V[sc, s'c'] = (phi_s phi_c | v | phi_s' phi_c'), Q[sc] = <phi_s phi_c|q>. In the symmetric variable
x = D^{1/2} y: y'' = -Omega^2 y with Omega^2 = D^{1/2} (D + 4V) D^{1/2}. Hence
u(r, t) = -4 alpha sum_sc w_sc(r) [D^{1/2} E diag(sin(Omega t)/Omega) E^T D^{1/2} Q]_sc with
w_sc = v(phi_s phi_c) and E the eigenvectors of Omega^2, and Eq. (13) becomes
W^pol = -4 sum_sc w_sc [D^{1/2} E diag(S(Omega)/Omega) E^T D^{1/2} Q]_sc, S(Omega) = the same
quadrature of exp(-gamma^2 t^2/2) sin(Omega t) that the TDH engine applies to u. Without Hartree
feedback (V = 0) the modes are the bare transitions, Omega = D. With S -> 1/Omega this is the
static W^pol = v chi v of the paper's W = v + v chi v.
"""
from __future__ import annotations

import numpy as np

from .tdh import Grid, coulomb_periodic


def casida_w_pol(grid: Grid, eps_all, phi_all, n_occ: int, rho, times, weights,
                 feedback: bool = True, coulomb=coulomb_periodic):
    """Damped W^pol for the source rho from all occupied x virtual transitions of a dense H0.

    times, weights: the sample times t_n and the quadrature weights w_n exp(-gamma^2 t_n^2/2) dt
    (as applied by the TDH engine). Pass weights=None for the static limit (S = 1/Omega).
    """
    n_all = phi_all.shape[0]
    occ = phi_all[:n_occ].reshape(n_occ, -1)
    vir = phi_all[n_occ:].reshape(n_all - n_occ, -1)
    n_v = vir.shape[0]
    rho_sc = (occ[:, None, :] * vir[None, :, :]).reshape(n_occ * n_v, -1)
    dE = (eps_all[None, n_occ:] - eps_all[:n_occ, None]).reshape(-1)
    q = coulomb(rho, grid).reshape(-1)
    Q = rho_sc @ q * grid.dV
    w_sc = coulomb(rho_sc.reshape((-1,) + rho.shape), grid).reshape(n_occ * n_v, -1)
    if feedback:
        V = rho_sc @ w_sc.T * grid.dV
        V = 0.5 * (V + V.T)
    else:
        V = np.zeros((len(dE), len(dE)))
    sd = np.sqrt(dE)
    om2 = sd[:, None] * (np.diag(dE) + 4.0 * V) * sd[None, :]
    lam, E = np.linalg.eigh(om2)
    om = np.sqrt(lam)
    if weights is None:
        s_over = 1.0 / om ** 2
    else:
        S = np.sin(np.outer(om, times)) @ weights
        s_over = S / om
    coef = sd * (E @ (s_over * (E.T @ (sd * Q))))
    return (-4.0 * (coef @ w_sc)).reshape(rho.shape)
