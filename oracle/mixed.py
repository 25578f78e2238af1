"""FP64 oracle of the mixed hole-grid representation of the BSE operator (Sec. II.C, "Mixed
Representation Iterative Solution"): A = Q A-bar acting on the vectors f_j(r), one grid function per
occupied window state j,

    (A-bar f)_j = (H0 + Delta - eps_j) f_j + dv phi_j - sum_i f_i W_ij,
    dv = v dn,  dn = 2 sum_i phi_i f_i  (exciton density and its Coulomb potential),

with Q = 1 - sum_{s <= N_occ} |phi_s><phi_s| (the full virtual space), and the absorption spectrum
sigma(omega) = omega <f0| delta(A - omega) |f0> from the residues R_n = <f0| T_n(A~) |f0> of the
Chebyshev recursion, f0_j = Q x phi_j (Eq. for sigma and the expansion of delta(A - omega) that
follows it).

TEST INFRASTRUCTURE: imported only by the tests. Never part of the library's compute path.

Readings:
  * i and j run over the n_o window of occupied states (the pairs (i, j) whose W_ij is prepared);
    W_ji = W_ij. The sum in dn runs over the same window.
  * "Q" may also be the projector onto the n_c conduction states (the electron-hole-basis variant
    the paper describes after Eq. 18); with it A restricted to span{phi_a} is the matrix of Eq. (1).
  * x is the coordinate from the box centre (as in oracle/spectrum.py).
  * The iterated vectors live in the range of Q; A maps the rest to 0, outside any interval that
    encloses the excitons, so the scaled operator is taken on that range: A~ f = Q(A-bar f - c f) / w
    (the shift projected too, which keeps rounding outside the range from being amplified by the
    recursion), with c, w from an interval [lo, hi] enclosing the spectrum (c = (lo + hi) / 2,
    w = (hi - lo) / 2); `lanczos_bounds` provides one: the extreme Ritz values of m Lanczos steps
    from f0 (each vector projected by Q), widened by 5 % of their spread on each side.
  * The smoothed delta and its Chebyshev coefficients are those of oracle/spectrum.py.
"""
from __future__ import annotations

import numpy as np

from .spectrum import coordinate, sigma_chebyshev
from .tdh import Grid, coulomb_periodic


def kinetic(grid: Grid, f: np.ndarray) -> np.ndarray:
    """-1/2 Laplacian (spectral) on real fields, acting on the last three axes."""
    return np.fft.ifftn(0.5 * grid.G2 * np.fft.fftn(f, axes=(-3, -2, -1)), axes=(-3, -2, -1)).real


def project(grid: Grid, basis: np.ndarray, f: np.ndarray, keep: bool) -> np.ndarray:
    """keep=False: f - sum_s phi_s <phi_s|f> (Q = 1 - P); keep=True: sum_s phi_s <phi_s|f>."""
    B = basis.reshape(basis.shape[0], -1)
    F = f.reshape(f.shape[0], -1)
    ov = F @ B.T * grid.dV
    Pf = (ov @ B).reshape(f.shape)
    return Pf if keep else f - Pf


class MixedA:
    """The operator A = Q A-bar on (n_o, N, N, N) arrays f."""

    def __init__(self, grid: Grid, v_loc, phi, eps, n_occ: int, n_o: int, n_c: int, w_pairs: dict,
                 scissor: float, conduction_only: bool = False):
        self.g = grid
        self.v = v_loc
        self.phi_occ = phi[:n_occ]
        self.phi_o = phi[n_occ - n_o:n_occ]
        self.eps_o = eps[n_occ - n_o:n_occ]
        self.phi_c = phi[n_occ:n_occ + n_c]
        self.n_o = n_o
        self.W = w_pairs
        self.scissor = scissor
        self.cond = conduction_only

    def Q(self, f):
        return project(self.g, self.phi_c, f, keep=True) if self.cond else project(self.g, self.phi_occ, f, keep=False)

    def bar(self, f):
        dn = 2.0 * np.sum(self.phi_o * f, axis=0)
        dv = coulomb_periodic(dn, self.g)
        out = kinetic(self.g, f) + self.v[None] * f
        out += (self.scissor - self.eps_o)[:, None, None, None] * f
        out += dv[None] * self.phi_o
        for j in range(self.n_o):
            for i in range(self.n_o):
                out[j] -= f[i] * self.W[(min(i, j), max(i, j))]
        return out

    def __call__(self, f):
        return self.Q(self.bar(f))

    def start(self, axis: int):
        """f0_j = Q x phi_j."""
        return self.Q(coordinate(self.g, axis)[None] * self.phi_o)

    def dot(self, f, g) -> float:
        return float(np.sum(f * g) * self.g.dV)


def lanczos_bounds(op: MixedA, f0, m: int):
    """[lo, hi] from m Lanczos steps started at f0 (module reading)."""
    q_prev = np.zeros_like(f0)
    q = f0 / np.sqrt(op.dot(f0, f0))
    al, be = [], []
    b = 0.0
    for k in range(m):
        z = op(q) - b * q_prev
        a = op.dot(q, z)
        z = op.Q(z - a * q)
        al.append(a)
        b = np.sqrt(op.dot(z, z))
        if k == m - 1 or b == 0.0:
            break
        be.append(b)
        q_prev, q = q, z / b
    T = np.diag(al) + np.diag(be[:len(al) - 1], 1) + np.diag(be[:len(al) - 1], -1)
    th = np.linalg.eigvalsh(T)
    spread = th[-1] - th[0]
    return float(th[0] - 0.05 * spread), float(th[-1] + 0.05 * spread)


def residues(op: MixedA, f0, n_terms: int, lo: float, hi: float) -> np.ndarray:
    """R_n = <f0| T_n(A~) |f0>, A~ = (A - c) / w, by v_{n+1} = 2 A~ v_n - v_{n-1}."""
    c, w = 0.5 * (lo + hi), 0.5 * (hi - lo)
    R = np.empty(n_terms)
    v_prev, v = None, f0.copy()
    for n in range(n_terms):
        R[n] = op.dot(f0, v)
        Av = op.Q(op.bar(v) - c * v) / w
        v_next = Av if n == 0 else 2.0 * Av - v_prev
        v_prev, v = v, v_next
    return R


def absorption(op: MixedA, axis: int, n_terms: int, lo: float, hi: float, s: float, omega):
    """sigma(omega) of the mixed representation. Returns (sigma, R, f0)."""
    f0 = op.start(axis)
    R = residues(op, f0, n_terms, lo, hi)
    return sigma_chebyshev(R, 0.5 * (lo + hi), 0.5 * (hi - lo), omega, s), R, f0
