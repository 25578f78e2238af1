"""Gaussian-well model systems on a periodic cubic grid.

Grid convention (shared by every consumer): box [0, L)^3 with N points per axis at
r = h*(ix, iy, iz), h = L/N, dV = h^3. A field is stored as a C-ordered array of shape (N, N, N)
indexed [iz, iy, ix], i.e. x is the fastest-varying index of the flattened n_g = N^3 vector.

H0 = -1/2 Laplacian + V_loc, with the spectral (plane-wave) Laplacian on this grid, and
V_loc(r) = -sum_k D_k exp(-|r - R_k|^2_mic / (2 w_k^2)) (minimum-image distance). Each well draws
D ~ U[2, 4] Ha, w ~ U[0.8, 1.2] bohr and R uniform in the inner half [L/4, 3L/4)^3 of the box, in
that order, from numpy.random.default_rng(seed).

The lowest N_occ + n_c eigenpairs of H0 are the orbitals phi_s (real, normalised so that
sum_r phi_s(r)^2 dV = 1, sign fixed so the largest-magnitude entry is positive) and eigenvalues
eps_s: by dense diagonalisation when n_g <= 4096; on grids of edge 64 and more, when a CUDA device
is present, by Chebyshev-filtered subspace iteration on that device (chfsi.py); otherwise by
preconditioned LOBPCG started from seeded random vectors, followed by a Rayleigh-Ritz rotation.
SBSE_EIGENSOLVER=lobpcg|chfsi forces the iterative solver.
"""
from __future__ import annotations

import dataclasses
import hashlib
import os

import numpy as np
import scipy.fft as sfft
from scipy.sparse.linalg import LinearOperator, lobpcg

_WORKERS = max(1, os.cpu_count() or 1)


@dataclasses.dataclass(frozen=True)
class Preset:
    """One synthetic workload: grid, wells, orbital windows and TDH run parameters."""

    name: str
    N: int
    box: float
    n_wells: int
    seed: int
    n_occ: int
    n_o: int
    n_c: int
    n_s: int = 10
    n_steps: int = 200
    dt: float = 0.05
    gamma: float = 0.1
    alpha: float = 1e-4
    clean_every: int = 10
    scissor: float = 0.5
    n_exc: int = 4
    # box edge the wells are drawn for (None: this box); the wells are then centred in this box, so
    # that one molecule can be placed in boxes of several sizes (the box-size sweep of Sec. III)
    well_box: float | None = None

    @property
    def n_pairs(self) -> int:
        return self.n_o * (self.n_o + 1) // 2


# Workloads shaped like the paper's (Sec. III: a 520-electron system on a ~0.85M-point grid,
# L = 10 stochastic orbitals, cleaning every M = 10 steps, gamma = 0.1 Ha) but built from
# Gaussian wells because the molecule, pseudopotentials and DFT orbitals are not available.
PRESETS = {
    "tiny16": Preset("tiny16", N=16, box=8.0, n_wells=4, seed=0, n_occ=4, n_o=2, n_c=4,
                     n_steps=200, gamma=0.01, n_exc=4),
    "mid48": Preset("mid48", N=48, box=16.0, n_wells=40, seed=1, n_occ=60, n_o=8, n_c=16,
                    n_steps=1000, gamma=0.1, n_exc=10),
    "large96": Preset("large96", N=96, box=24.0, n_wells=170, seed=2, n_occ=260, n_o=16,
                      n_c=32, n_steps=2000, gamma=0.1, n_exc=10),
    # the 96^3 grid with fewer states (about 2 GB on the device): kernel-profiler captures of the
    # 96^3 pass kernels, whose work per orbital is that of large96
    "prof96": Preset("prof96", N=96, box=24.0, n_wells=40, seed=3, n_occ=60, n_o=4, n_c=8,
                     n_steps=2000, gamma=0.1, n_exc=4),
}


def preset(name: str) -> Preset:
    return PRESETS[name]


def batch_presets(first_seed: int = 100, count: int = 64):
    """Many small independent systems of uneven grid sizes: grid drawn from {32,40,48,64,80}^3,
    h = 0.25 bohr, N_occ = N/2, n_o = 4, n_c = 8, 500 steps, round(2 N_occ / 3) wells."""
    out = []
    for s in range(first_seed, first_seed + count):
        N = int(np.random.default_rng(s).choice([32, 40, 48, 64, 80]))
        n_occ = N // 2
        out.append(Preset(f"batch{s}", N=N, box=0.25 * N, n_wells=int(round(2 * n_occ / 3)),
                          seed=s, n_occ=n_occ, n_o=4, n_c=8, n_steps=500, gamma=0.1, n_exc=4))
    return out


def fno_presets(count: int, first_seed: int = 1000, N: int = 64, box: float = 24.0, n_steps: int = 2000):
    """Training / evaluation systems of the learned form: 20 to 80 wells (drawn per seed), grid N^3
    over a box of the paper-scale system's edge (so its fields resample onto this grid),
    N_occ = round(1.5 n_wells), n_o = 8, n_c = 8, the paper-scale TDH parameters."""
    out = []
    for s in range(first_seed, first_seed + count):
        n_wells = int(np.random.default_rng(s).integers(20, 81))
        out.append(Preset(f"fno{s}", N=N, box=box, n_wells=n_wells, seed=s, n_occ=int(round(1.5 * n_wells)),
                          n_o=8, n_c=8, n_steps=n_steps, gamma=0.1, n_exc=10))
    return out


def box_sweep_presets(base: Preset, boxes, n_steps: int | None = None):
    """The molecule of `base` (its wells, drawn for base.box) centred in boxes of the given edges at
    the same grid spacing (N = box / h): the runs of the finite-box correction of Sec. III."""
    h = base.box / base.N
    out = []
    for b in boxes:
        N = int(round(b / h))
        out.append(dataclasses.replace(base, name=f"{base.name}_L{b:g}", N=N, box=float(b),
                                       well_box=base.box,
                                       n_steps=base.n_steps if n_steps is None else n_steps))
    return out


def preset_wells(p: Preset) -> np.ndarray:
    """The wells of a preset: drawn for p.well_box (default p.box) and centred in p.box."""
    wb = p.box if p.well_box is None else p.well_box
    w = gaussian_wells(p.n_wells, wb, p.seed)
    w[:, 2:] += 0.5 * (p.box - wb)
    return w


def gaussian_wells(n_wells: int, box: float, seed: int) -> np.ndarray:
    """Rows (D, w, Rx, Ry, Rz) drawn in the order D, w, R per well."""
    rng = np.random.default_rng(seed)
    rows = []
    for _ in range(n_wells):
        depth = rng.uniform(2.0, 4.0)
        width = rng.uniform(0.8, 1.2)
        centre = rng.uniform(box / 4, 3 * box / 4, size=3)
        rows.append((depth, width, centre[0], centre[1], centre[2]))
    return np.array(rows, dtype=np.float64).reshape(n_wells, 5)


def local_potential(N: int, box: float, wells: np.ndarray) -> np.ndarray:
    h = box / N
    x = np.arange(N) * h
    out = np.zeros((N, N, N))
    for depth, width, rx, ry, rz in wells:
        dx = x - rx
        dx -= box * np.round(dx / box)
        dy = x - ry
        dy -= box * np.round(dy / box)
        dz = x - rz
        dz -= box * np.round(dz / box)
        r2 = dz[:, None, None] ** 2 + dy[None, :, None] ** 2 + dx[None, None, :] ** 2
        out -= depth * np.exp(-r2 / (2.0 * width * width))
    return out


def _kvec(N: int, box: float) -> np.ndarray:
    return 2.0 * np.pi / box * (np.fft.fftfreq(N) * N)


def _dense_h0(N: int, box: float, v: np.ndarray) -> np.ndarray:
    k = _kvec(N, box)
    F = np.fft.fft(np.eye(N), axis=0)
    t1 = np.real(np.fft.ifft((0.5 * k * k)[:, None] * F, axis=0))
    eye = np.eye(N)
    # flattened index = ix + N*(iy + N*iz): the x factor is the last Kronecker factor
    T = (np.kron(np.kron(t1, eye), eye) + np.kron(np.kron(eye, t1), eye)
         + np.kron(np.kron(eye, eye), t1))
    return T + np.diag(v.ravel())


def _lobpcg_h0(N: int, box: float, v: np.ndarray, n_states: int, seed: int, tol: float):
    n_g = N ** 3
    k = 2.0 * np.pi / box * (np.fft.fftfreq(N) * N)
    kr = 2.0 * np.pi / box * np.arange(N // 2 + 1)
    g2 = k[:, None, None] ** 2 + k[None, :, None] ** 2 + kr[None, None, :] ** 2
    vcol = v.reshape(N, N, N, 1)

    def apply_h(xm):
        xm = xm.reshape(N, N, N, -1)
        t = sfft.irfftn(sfft.rfftn(xm, axes=(0, 1, 2), workers=_WORKERS) * (0.5 * g2)[..., None],
                        s=(N, N, N), axes=(0, 1, 2), workers=_WORKERS)
        return (t + vcol * xm).reshape(n_g, -1)

    def precond(xm):
        xm = xm.reshape(N, N, N, -1)
        return sfft.irfftn(sfft.rfftn(xm, axes=(0, 1, 2), workers=_WORKERS)
                           / (0.5 * g2 + 1.0)[..., None],
                           s=(N, N, N), axes=(0, 1, 2), workers=_WORKERS).reshape(n_g, -1)

    block = n_states + max(8, n_states // 8)
    x0 = np.random.default_rng(10_000 + seed).standard_normal((n_g, block))
    a_op = LinearOperator((n_g, n_g), matvec=apply_h, matmat=apply_h, dtype=np.float64)
    m_op = LinearOperator((n_g, n_g), matvec=precond, matmat=precond, dtype=np.float64)
    _, vec = lobpcg(a_op, x0, M=m_op, tol=tol, maxiter=500, largest=False)
    q, _ = np.linalg.qr(vec)
    hs = q.T @ apply_h(q)
    e, u = np.linalg.eigh(0.5 * (hs + hs.T))
    vec = q @ u[:, :n_states]
    return e[:n_states], vec


@dataclasses.dataclass
class ModelSystem:
    """Orbitals and grid of one synthetic system (all arrays FP64, C-ordered, x fastest)."""

    preset: Preset
    N: int
    box: float
    v_loc: np.ndarray  # (N, N, N)
    phi: np.ndarray  # (n_occ + n_c, N, N, N), sum phi^2 dV = 1
    eps: np.ndarray  # (n_occ + n_c,)

    @property
    def h(self) -> float:
        return self.box / self.N

    @property
    def dV(self) -> float:
        return self.h ** 3

    @property
    def n_g(self) -> int:
        return self.N ** 3


def _use_chfsi(N: int) -> bool:
    forced = os.environ.get("SBSE_EIGENSOLVER", "")
    if forced:
        return forced == "chfsi"
    if N < 64:
        return False
    try:
        import torch
        return bool(torch.cuda.is_available())
    except ImportError:
        return False


def _cache_path(p: Preset, n_states: int, tol: float):
    root = os.environ.get("SBSE_INPUT_CACHE")
    if not root:
        return None
    key = (f"{p.N}-{p.box}-{p.n_wells}-{p.seed}-{n_states}-{tol}-{'chfsi' if _use_chfsi(p.N) else 'lobpcg'}"
           f"-{p.well_box}")
    return os.path.join(root, "sys_" + hashlib.sha1(key.encode()).hexdigest()[:16] + ".npz")


def make_system(p: Preset, n_states: int | None = None, tol: float = 1e-6) -> ModelSystem:
    """Build V_loc and the lowest n_states (default N_occ + n_c) orbitals of H0."""
    n_states = p.n_occ + p.n_c if n_states is None else n_states
    wells = preset_wells(p)
    v = local_potential(p.N, p.box, wells)
    dV = (p.box / p.N) ** 3
    cache = _cache_path(p, n_states, tol)
    if cache and os.path.exists(cache):
        z = np.load(cache)
        return ModelSystem(p, p.N, p.box, v, z["phi"], z["eps"])
    if p.N ** 3 <= 4096:
        e, vec = np.linalg.eigh(_dense_h0(p.N, p.box, v))
        e, vec = e[:n_states], vec[:, :n_states]
    elif _use_chfsi(p.N):
        from . import chfsi
        e, vec = chfsi.lowest_states(p.N, p.box, v, n_states, p.seed, tol)
    else:
        e, vec = _lobpcg_h0(p.N, p.box, v, n_states, p.seed, tol)
    idx = np.argmax(np.abs(vec), axis=0)
    sign = np.sign(vec[idx, np.arange(vec.shape[1])])
    vec = vec * sign[None, :]
    phi = (vec.T / np.sqrt(dV)).reshape(n_states, p.N, p.N, p.N).copy()
    eps = np.asarray(e, dtype=np.float64).copy()
    if cache:
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        np.savez(cache, phi=phi, eps=eps)
    return ModelSystem(p, p.N, p.box, v, phi, eps)


def dense_eigensystem(p: Preset):
    """All eigenpairs of the dense H0 (small grids only); orbitals normalised with dV."""
    wells = preset_wells(p)
    v = local_potential(p.N, p.box, wells)
    e, vec = np.linalg.eigh(_dense_h0(p.N, p.box, v))
    dV = (p.box / p.N) ** 3
    idx = np.argmax(np.abs(vec), axis=0)
    vec = vec * np.sign(vec[idx, np.arange(vec.shape[1])])[None, :]
    return v, e, (vec.T / np.sqrt(dV)).reshape(-1, p.N, p.N, p.N)


__all__ = ["Preset", "PRESETS", "ModelSystem", "preset", "batch_presets", "box_sweep_presets", "fno_presets",
           "preset_wells", "gaussian_wells",
           "local_potential", "make_system", "dense_eigensystem"]
