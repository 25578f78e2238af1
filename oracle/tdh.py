"""FP64 oracle of the stochastic time-dependent-Hartree (TDH) action of W and of A (Eq. 1).

TEST INFRASTRUCTURE: imported only by the tests, the package smoke check and the benchmark's CPU
baseline. Never part of the library's compute path.

Everything follows "Stochastic evaluation of the action of W" (Sec. II.B, Eqs. 10-15) and the
Tamm-Dancoff matrix of Eq. (1) with its exchange and direct elements. Readings of points the paper
leaves open are marked "reading:" below and are the same in the CUDA path.

Array conventions: a field on the N^3 grid is an (N, N, N) array indexed [z, y, x]; a set of fields
is (count, N, N, N). Integrals are sums times dV = h^3.

Parity status: every function here is pinned by a test against something other than itself
(closed forms, brute force, invariants, or the independent linear-response evaluation in
`oracle.rpa`); see tests/test_oracle_*.py.
"""
from __future__ import annotations

import dataclasses

import numpy as np

# ----------------------------------------------------------------------------------------------
# grid and Coulomb operator


class Grid:
    """Periodic cubic grid of N points per axis over a box of edge `box` (bohr)."""

    def __init__(self, N: int, box: float):
        self.N = int(N)
        self.box = float(box)
        self.h = self.box / self.N
        self.dV = self.h ** 3
        m = np.fft.fftfreq(self.N) * self.N  # integer mode numbers; |k| is symmetric at Nyquist
        k = 2.0 * np.pi / self.box * m
        self.G2 = k[:, None, None] ** 2 + k[None, :, None] ** 2 + k[None, None, :] ** 2

    def inner(self, f, g):
        """<f|g> = sum_r conj(f) g dV over the last three axes."""
        return np.sum(np.conj(f) * g, axis=(-3, -2, -1)) * self.dV


def coulomb_periodic(n: np.ndarray, grid: Grid) -> np.ndarray:
    """u = v n with v = 1/|r - r'| on the periodic box: u(G) = 4 pi n(G) / |G|^2, G = 0 dropped.

    The Coulomb operator is the one in the exchange element after Eq. (1) and in Eq. (11); the
    periodic form with the G = 0 term removed is the reading of the paper's finite-box treatment
    (Sec. II.B, last paragraph before the algorithm summary). Acts on the last three axes.
    """
    nh = np.fft.fftn(n, axes=(-3, -2, -1))
    with np.errstate(divide="ignore"):
        kern = np.where(grid.G2 > 0.0, 4.0 * np.pi / np.where(grid.G2 > 0, grid.G2, 1.0), 0.0)
    out = np.fft.ifftn(nh * kern, axes=(-3, -2, -1))
    return out.real if np.isrealobj(n) else out


def coulomb_truncated(n: np.ndarray, grid: Grid) -> np.ndarray:
    """Free-space u = v n for a density n of extent < box/2 about the box centre.

    The box is zero-padded to 2N per axis and the spherically truncated kernel
    4 pi (1 - cos(|G| R_c)) / |G|^2 (value 2 pi R_c^2 at G = 0) with R_c = box is used. This is
    exact (up to sampling) for every pair of charge and evaluation points closer than R_c, and no
    periodic image comes closer than R_c. Used only to pin the grid/G-table conventions against
    the closed-form potential of a Gaussian charge.
    """
    N = grid.N
    M = 2 * N
    big = np.zeros((M, M, M))
    big[:N, :N, :N] = n
    k = 2.0 * np.pi / (2.0 * grid.box) * (np.fft.fftfreq(M) * M)
    G2 = k[:, None, None] ** 2 + k[None, :, None] ** 2 + k[None, None, :] ** 2
    G = np.sqrt(G2)
    rc = grid.box
    with np.errstate(divide="ignore", invalid="ignore"):
        kern = np.where(G2 > 0, 4.0 * np.pi * (1.0 - np.cos(G * rc)) / np.where(G2 > 0, G2, 1.0),
                        2.0 * np.pi * rc * rc)
    u = np.fft.ifftn(np.fft.fftn(big) * kern).real
    return u[:N, :N, :N]


# ----------------------------------------------------------------------------------------------
# stochastic coefficients (Eq. 14): a counter-based splitmix64 stream


_MASK = (1 << 64) - 1
_GOLDEN = 0x9E3779B97F4A7C15


def splitmix64(seed: int, k: int) -> int:
    """Output number k (k = 0, 1, ...) of Vigna's splitmix64 generator started from state `seed`.

    The state advances by the golden-ratio increment before each output, then passes through the
    two xor-shift-multiply rounds and a final xor-shift of the published generator.
    """
    z = (seed + (k + 1) * _GOLDEN) & _MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
    return z ^ (z >> 31)


def stochastic_coefficients(seed: int, n_s: int, n_occ: int, dist: str = "gaussian") -> np.ndarray:
    """Coefficient matrix c[l, s] of the stochastic orbitals eta_l = L^-1/2 sum_s c[l, s] phi_s.

    Eq. (14) uses random signs; the workloads ask for Gaussian-random combinations (reading: both
    are offered, both have E[c c'] = delta). Sign: top bit of output l*n_occ + s (0 -> +1).
    Gaussian: Box-Muller from the 53-bit uniforms u1, u2 of outputs 2(l*n_occ + s) and +1,
    g = sqrt(-2 ln(1 - u1)) cos(2 pi u2).
    """
    c = np.empty((n_s, n_occ))
    for ell in range(n_s):
        for s in range(n_occ):
            idx = ell * n_occ + s
            if dist == "sign":
                c[ell, s] = -1.0 if (splitmix64(seed, idx) >> 63) else 1.0
            elif dist == "gaussian":
                u1 = (splitmix64(seed, 2 * idx) >> 11) * (1.0 / 9007199254740992.0)
                u2 = (splitmix64(seed, 2 * idx + 1) >> 11) * (1.0 / 9007199254740992.0)
                c[ell, s] = np.sqrt(-2.0 * np.log(1.0 - u1)) * np.cos(2.0 * np.pi * u2)
            else:
                raise ValueError(dist)
    return c


# ----------------------------------------------------------------------------------------------
# TDH propagation


@dataclasses.dataclass
class TDHParams:
    n_steps: int = 200
    dt: float = 0.05
    gamma: float = 0.1
    alpha: float = 1e-4
    clean_every: int = 10  # M of Eq. (15); 0 disables cleaning
    feedback: bool = True  # False: propagate with H0 only (u still recorded): W^pol -> v chi0 v


def time_weights(p: TDHParams) -> np.ndarray:
    """Quadrature of Eq. (13) on t_n = n dt, n = 0..N_t (reading: trapezoid, the upper limit of
    the integral truncated at N_t dt): w_n exp(-gamma^2 t_n^2 / 2) dt with w_0 = w_Nt = 1/2."""
    t = np.arange(p.n_steps + 1) * p.dt
    w = np.ones(p.n_steps + 1)
    w[0] = w[-1] = 0.5
    return w * np.exp(-0.5 * p.gamma ** 2 * t * t) * p.dt


def stochastic_orbitals(coeff: np.ndarray, phi_occ: np.ndarray) -> np.ndarray:
    """eta_l = L^-1/2 sum_s c[l, s] phi_s over all N_occ occupied states (Eq. 14)."""
    L = coeff.shape[0]
    n_occ = phi_occ.shape[0]
    return (coeff @ phi_occ.reshape(n_occ, -1)).reshape((L,) + phi_occ.shape[1:]) / np.sqrt(L)


class _Propagator:
    """Split-operator pieces: e^{-i V dt/2} in real space and e^{-i |G|^2 dt / 2} in G space."""

    def __init__(self, grid: Grid, v_loc: np.ndarray, dt: float):
        self.grid = grid
        self.dt = dt
        self.pv = np.exp(-0.5j * dt * v_loc)
        self.kin = np.exp(-0.5j * dt * grid.G2)

    def kinetic(self, x):
        return np.fft.ifftn(self.kin * np.fft.fftn(x, axes=(-3, -2, -1)), axes=(-3, -2, -1))

    def half_phase_pair(self, a, d, u):
        """One half-step potential factor on the pair (eta0, delta eta).

        eta0 feels V only; eta^alpha = eta0 + delta eta feels V + u. With P = e^{-i V dt/2} and
        E = e^{-i u dt/2}: (a, d) -> (P a, P[(E - 1) a + E d]), where
        E - 1 = -2i sin(u dt/4) e^{-i u dt/4} avoids the cancellation of 1 - cos.
        """
        ph = 0.25 * self.dt * u
        em1 = -2j * np.sin(ph) * np.exp(-1j * ph)
        e = np.exp(-2j * ph)
        return self.pv * a, self.pv * (em1 * a + e * d)


def induced_density(a, d):
    """delta n = n^alpha - n^0 = 2 sum_l (2 Re(conj(eta0) d) + |d|^2)  (density of Eq. 11 with
    n = 2 sum_l |eta_l|^2, spin factor 2)."""
    return 2.0 * np.sum(2.0 * (a.conj() * d).real + (d.conj() * d).real, axis=0)


def clean(a, d, phi_occ, n0, grid: Grid):
    """Eq. (15) followed by the renormalisation of each eta^alpha to its initial norm.

    eta^alpha <- eta^0 + Q(eta^alpha - eta^0), Q = 1 - sum_{s<=N_occ} |phi_s><phi_s|, i.e.
    d <- d - sum_s phi_s <phi_s|d>. Then eta^alpha is rescaled by c = sqrt(N0 / |eta^alpha|^2)
    with |eta^alpha|^2 = N0 (1 + x), x = (2 Re<eta0|d> + |d|^2) / N0 (reading: |eta0|^2 = N0 by
    unitarity), so d <- c d + (c - 1) eta0 with c - 1 = -x / (sqrt(1+x) (1 + sqrt(1+x))).
    """
    L = d.shape[0]
    n_occ = phi_occ.shape[0]
    D = d.reshape(L, -1)
    P = phi_occ.reshape(n_occ, -1)
    ov = (D @ P.T) * grid.dV  # <phi_s|d>, phi real
    D = D - ov @ P
    A = a.reshape(L, -1)
    x = (2.0 * np.sum(np.conj(A) * D, axis=1).real + np.sum(np.abs(D) ** 2, axis=1)) * grid.dV
    x = x / n0
    sq = np.sqrt(1.0 + x)
    cm1 = -x / (sq * (1.0 + sq))
    D = (1.0 + cm1)[:, None] * D + cm1[:, None] * A
    return D.reshape(d.shape)


def tdh_w_pol(grid: Grid, v_loc, phi_occ, rho, coeff, p: TDHParams, coulomb=coulomb_periodic,
              record=None, observe=None):
    """Stochastic-TDH W^pol_ij(r) of Eq. (13) for the source density rho = phi_i phi_j.

    Steps (difference form; algebraically the same as propagating eta^alpha and eta^0, Sec. II.B):
      q = v rho; eta0_l from Eq. (14); kick (Sec. II.B, psi_s(0) = e^{-i alpha q} phi_s):
      d_l = (e^{-i alpha q} - 1) eta0_l = -2i sin(alpha q/2) e^{-i alpha q/2} eta0_l.
      For n = 0..N_t-1: if n mod M == 0, clean (Eq. 15, reading: before step n, including n = 0)
      and recompute u_n; accumulate u_n into Eq. (13); split-operator step of Eq. (10):
      half potential step with u_n, kinetic step, u_{n+1} = v delta n from the post-kinetic
      state (reading: the time at which u enters a step), half potential step with u_{n+1}.
      Finally accumulate u_{N_t}. u subtracts the density of the unperturbed set propagated with
      the same H0 (reading of Eq. 11 for stochastic orbitals, which are not stationary).
    Returns W^pol (N, N, N). `record`, if a list, receives (n, u_n) for every accumulated sample;
    `observe`, if given, is called as observe(n + 1, a, d) with the state after each completed step
    (read-only views; nothing it returns is used).
    """
    wts = time_weights(p)
    prop = _Propagator(grid, v_loc, p.dt)
    q = coulomb(rho, grid)
    a = stochastic_orbitals(coeff, phi_occ).astype(np.complex128)
    d = (-2j * np.sin(0.5 * p.alpha * q) * np.exp(-0.5j * p.alpha * q))[None] * a
    n0 = np.real(grid.inner(a, a))
    u = np.zeros_like(rho)
    w = np.zeros_like(rho)

    def potential(a_, d_):
        return coulomb(induced_density(a_, d_), grid)

    for n in range(p.n_steps):
        if p.clean_every and n % p.clean_every == 0:
            d = clean(a, d, phi_occ, n0, grid)
            u = potential(a, d)
        w += (wts[n] / p.alpha) * u
        if record is not None:
            record.append((n, u.copy()))
        up = u if p.feedback else 0.0 * u
        a, d = prop.half_phase_pair(a, d, up)
        a, d = prop.kinetic(a), prop.kinetic(d)
        u = potential(a, d)
        up = u if p.feedback else 0.0 * u
        a, d = prop.half_phase_pair(a, d, up)
        if observe is not None:
            observe(n + 1, a, d)
    w += (wts[p.n_steps] / p.alpha) * u
    if record is not None:
        record.append((p.n_steps, u.copy()))
    return w


def tdh_w_pol_two_set(grid: Grid, v_loc, phi_occ, rho, coeff, p: TDHParams,
                      coulomb=coulomb_periodic):
    """The same W^pol by the paper's literal procedure: propagate the perturbed set eta^alpha and
    the unperturbed set eta^0 separately (Sec. II.B) and take u = v(n^alpha - n^0). Loses
    ~|log10 alpha| digits to cancellation; used only to cross-check `tdh_w_pol`."""
    wts = time_weights(p)
    prop = _Propagator(grid, v_loc, p.dt)
    q = coulomb(rho, grid)
    e0 = stochastic_orbitals(coeff, phi_occ).astype(np.complex128)
    ea = np.exp(-1j * p.alpha * q)[None] * e0
    n0 = np.real(grid.inner(e0, e0))
    L = e0.shape[0]
    n_occ = phi_occ.shape[0]
    P = phi_occ.reshape(n_occ, -1)

    def potential():
        return coulomb(2.0 * np.sum(np.abs(ea) ** 2 - np.abs(e0) ** 2, axis=0), grid)

    u = potential()
    w = np.zeros_like(rho)
    for n in range(p.n_steps):
        if p.clean_every and n % p.clean_every == 0:
            diff = (ea - e0).reshape(L, -1)
            diff = diff - ((diff @ P.T) * grid.dV) @ P
            ea = e0 + diff.reshape(ea.shape)
            norm = np.real(grid.inner(ea, ea))
            ea = ea * np.sqrt(n0 / norm)[:, None, None, None]
            u = potential()
        w += (wts[n] / p.alpha) * u
        up = u if p.feedback else 0.0 * u
        ea = prop.pv * np.exp(-0.5j * p.dt * up) * ea
        e0 = prop.pv * e0
        ea, e0 = prop.kinetic(ea), prop.kinetic(e0)
        u = potential()
        up = u if p.feedback else 0.0 * u
        ea = prop.pv * np.exp(-0.5j * p.dt * up) * ea
        e0 = prop.pv * e0
    w += (wts[p.n_steps] / p.alpha) * u
    return w


# ----------------------------------------------------------------------------------------------
# pairs, contractions, A and its spectrum


def pair_list(n_o: int):
    """Occupied pairs (i, j), i <= j, in the n_o window; n_o (n_o + 1) / 2 of them (Sec. II.B)."""
    return [(i, j) for i in range(n_o) for j in range(i, n_o)]


def windows(phi, eps, n_occ: int, n_o: int, n_c: int):
    """Reading: i runs over the top n_o occupied states (HOMO - n_o + 1 .. HOMO) and a over the
    bottom n_c virtuals (LUMO .. LUMO + n_c - 1), both in ascending energy."""
    return (phi[n_occ - n_o:n_occ], eps[n_occ - n_o:n_occ], phi[n_occ:n_occ + n_c],
            eps[n_occ:n_occ + n_c])


def screened_potentials(grid: Grid, v_loc, phi, n_occ, n_o, coeff, p: TDHParams, pairs=None,
                        coulomb=coulomb_periodic):
    """W_ij(r) = q_ij + W^pol_ij (Sec. II.B, first paragraph) for the requested pairs."""
    phi_occ = phi[:n_occ]
    phi_o = phi[n_occ - n_o:n_occ]
    pairs = pair_list(n_o) if pairs is None else pairs
    out = {}
    for (i, j) in pairs:
        rho = phi_o[i] * phi_o[j]
        out[(i, j)] = coulomb(rho, grid) + tdh_w_pol(grid, v_loc, phi_occ, rho, coeff, p,
                                                     coulomb=coulomb)
    return out


def exchange_K(grid: Grid, phi_o, phi_c, coulomb=coulomb_periodic):
    """K[ia, jb] = (ia|jb) = sum_r phi_i phi_a (r) [v (phi_j phi_b)](r) dV (exchange element after
    Eq. 1). Index ia = i * n_c + a."""
    n_o, n_c = phi_o.shape[0], phi_c.shape[0]
    rho = (phi_o[:, None] * phi_c[None, :]).reshape(n_o * n_c, -1)
    pot = coulomb(rho.reshape((n_o * n_c,) + phi_o.shape[1:]), grid).reshape(n_o * n_c, -1)
    return (rho @ pot.T) * grid.dV


def direct_D(grid: Grid, phi_o, phi_c, w_pairs):
    """D[ia, jb] = (phi_a phi_b | W | phi_i phi_j) = sum_r phi_a phi_b (r) W_ij(r) dV (direct
    element after Eq. 1), with W_ji = W_ij (only i <= j is computed)."""
    n_o, n_c = phi_o.shape[0], phi_c.shape[0]
    D = np.zeros((n_o * n_c, n_o * n_c))
    C = phi_c.reshape(n_c, -1)
    for (i, j), w in w_pairs.items():
        blk = (C * w.reshape(1, -1)) @ C.T * grid.dV  # [a, b]
        D[i * n_c:(i + 1) * n_c, j * n_c:(j + 1) * n_c] = blk
        D[j * n_c:(j + 1) * n_c, i * n_c:(i + 1) * n_c] = blk.T
    return D


def assemble_A(eps_o, eps_c, scissor, K=None, D=None):
    """Eq. (1) with the scissor: A = diag(eps_a - eps_i + Delta) + 2K - D (reading: Delta enters
    only the diagonal, as in Eq. 9; P's eps_a - eps_j times delta_ij equals eps_a - eps_i)."""
    n_o, n_c = len(eps_o), len(eps_c)
    A = np.diag((eps_c[None, :] - eps_o[:, None] + scissor).reshape(-1))
    if K is not None:
        A = A + 2.0 * K
    if D is not None:
        A = A - D
    return A


def lowest_excitons(A, k):
    """Lowest k eigenvalues (ascending) of the symmetric A."""
    return np.linalg.eigvalsh(0.5 * (A + A.T))[:k]


def run(grid: Grid, v_loc, phi, eps, n_occ, n_o, n_c, scissor, coeff, p: TDHParams, k: int,
        pairs=None):
    """The whole hot path: all W_ij, K, D, A and the lowest k excitons."""
    phi_o, eps_o, phi_c, eps_c = windows(phi, eps, n_occ, n_o, n_c)
    w = screened_potentials(grid, v_loc, phi, n_occ, n_o, coeff, p, pairs=pairs)
    K = exchange_K(grid, phi_o, phi_c)
    D = direct_D(grid, phi_o, phi_c, w)
    A = assemble_A(eps_o, eps_c, scissor, K, D)
    return {"W": w, "K": K, "D": D, "A": A, "excitons": lowest_excitons(A, k)}
