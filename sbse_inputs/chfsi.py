"""Lowest eigenpairs of the grid Hamiltonian H0 = -1/2 Laplacian + V_loc by Chebyshev-filtered
subspace iteration (Zhou, Saad, Tiago, Chelikowsky, J. Comput. Phys. 219 (2006) 172), in FP64
with PyTorch tensors on any device.

This is input preparation, not the method: the paper takes its orbitals from a DFT code, here they
are the eigenstates of a Gaussian-well Hamiltonian. On the large grids (96^3 with ~300 states) a
preconditioned LOBPCG on the host takes tens of minutes; the filtered iteration below runs its
batched FFTs and Rayleigh-Ritz products wherever the tensors live (a GPU when one is present) and
starts from the same problem solved on a grid of half the edge, Fourier-interpolated.

Each outer iteration: Y = p_m(H) X with p_m the degree-m Chebyshev polynomial that is bounded on
the unwanted interval [a, b] (a = largest Ritz value of the block, b = an upper bound of the
spectrum) and grows below a; orthonormalise Y (Householder QR); Rayleigh-Ritz (eigh of Y^T H Y);
stop once every wanted Ritz pair has a residual norm below `tol` (Ha, 2-norm of unit vectors).
"""
from __future__ import annotations

import math

import numpy as np


def _torch():
    import torch
    return torch


def _g2_half(N: int, box: float, device):
    """|G|^2 on the half spectrum of a real N^3 field (last axis halved), symmetric Nyquist."""
    torch = _torch()
    k = 2.0 * math.pi / box * torch.fft.fftfreq(N, d=1.0 / N, dtype=torch.float64, device=device)
    kr = 2.0 * math.pi / box * torch.arange(N // 2 + 1, dtype=torch.float64, device=device)
    return k[:, None, None] ** 2 + k[None, :, None] ** 2 + kr[None, None, :] ** 2


class _H:
    """Action of H0 on a block of real vectors (n_g x k, columns C-ordered N^3 fields)."""

    def __init__(self, N: int, box: float, v, chunk: int):
        torch = _torch()
        self.N = N
        self.v = v.reshape(-1)
        self.half_g2 = 0.5 * _g2_half(N, box, v.device)
        self.chunk = chunk
        self.t_max = float(self.half_g2.max())
        self.torch = torch

    def __call__(self, X):
        torch = self.torch
        N = self.N
        out = torch.empty_like(X)
        for c0 in range(0, X.shape[1], self.chunk):
            xs = X[:, c0:c0 + self.chunk].T.reshape(-1, N, N, N)
            t = torch.fft.irfftn(torch.fft.rfftn(xs, dim=(1, 2, 3)) * self.half_g2, s=(N, N, N),
                                 dim=(1, 2, 3))
            out[:, c0:c0 + self.chunk] = t.reshape(xs.shape[0], -1).T
        out += self.v[:, None] * X
        return out


def _rayleigh_ritz(H, Y):
    torch = _torch()
    Q, _ = torch.linalg.qr(Y)
    HQ = H(Q)
    hs = Q.T @ HQ
    e, U = torch.linalg.eigh(0.5 * (hs + hs.T))
    return e, Q @ U, HQ @ U


def _filter(H, X, m: int, a: float, b: float, a0: float):
    """Scaled Chebyshev filter of degree m damping [a, b], normalised at a0 (< a)."""
    e = 0.5 * (b - a)
    c = 0.5 * (b + a)
    sigma = e / (a0 - c)
    tau = 2.0 / sigma
    Y = (H(X) - c * X) * (sigma / e)
    for _ in range(2, m + 1):
        sigma_new = 1.0 / (tau - sigma)
        Yn = (H(Y) - c * Y) * (2.0 * sigma_new / e) - (sigma * sigma_new) * X
        X, Y, sigma = Y, Yn, sigma_new
    return Y


def _interpolate(Xc, Nc: int, N: int):
    """Fourier interpolation of real fields from Nc^3 to N^3 (N > Nc, both even): the coarse
    spectrum (Nyquist plane split evenly) embedded in the fine one; norms scale by (N/Nc)^3."""
    torch = _torch()
    k = Xc.shape[1]
    out = torch.empty((N ** 3, k), dtype=Xc.dtype, device=Xc.device)
    h = Nc // 2
    for c0 in range(0, k, 32):
        xs = Xc[:, c0:c0 + 32].T.reshape(-1, Nc, Nc, Nc)
        F = torch.fft.fftn(xs, dim=(1, 2, 3))
        # split the Nyquist planes between +Nc/2 and -Nc/2 so the interpolant stays real
        idx = torch.cat([torch.arange(0, h), torch.tensor([h]), torch.arange(h, Nc)]).to(Xc.device)
        wts = torch.ones(Nc + 1, dtype=torch.float64, device=Xc.device)
        wts[h] = 0.5
        wts[h + 1] = 0.5
        for ax in (1, 2, 3):
            F = torch.index_select(F, ax, idx)
            shape = [1, 1, 1, 1]
            shape[ax] = Nc + 1
            F = F * wts.reshape(shape)
        Fi = torch.zeros((F.shape[0], N, N, N), dtype=F.dtype, device=F.device)
        pos = torch.cat([torch.arange(0, h + 1), torch.arange(N - h, N)]).to(Xc.device)
        Fi[:, pos[:, None, None], pos[None, :, None], pos[None, None, :]] = F
        xf = torch.fft.ifftn(Fi, dim=(1, 2, 3)).real * (N / Nc) ** 3
        out[:, c0:c0 + 32] = xf.reshape(xf.shape[0], -1).T
    return out


def lowest_states(N: int, box: float, v_loc: np.ndarray, n_states: int, seed: int, tol: float = 1e-6,
                  device=None, degree: int = 24, max_iter: int = 200, coarse: bool = True):
    """The n_states lowest eigenpairs of H0 on the N^3 grid: (eps ascending, vectors n_g x n_states
    with unit 2-norm), as NumPy arrays. `v_loc` is the potential on this grid; with `coarse`, the
    problem on the N/2 grid (potential sampled at the even points) seeds the iteration from N = 32 up."""
    torch = _torch()
    device = torch.device(device or ("cuda" if torch.cuda.is_available() else "cpu"))
    n_g = N ** 3
    k = n_states + max(16, n_states // 10)
    v = torch.as_tensor(np.ascontiguousarray(v_loc), dtype=torch.float64, device=device)
    H = _H(N, box, v, chunk=64)
    if coarse and N >= 32 and N % 4 == 0 and (N // 2) ** 3 > 4 * k:
        Nc = N // 2
        _, Xc = lowest_states(Nc, box, v_loc[::2, ::2, ::2], n_states, seed, tol=max(tol, 1e-4),
                              device=device, degree=degree, max_iter=max_iter, coarse=coarse)
        Xc = torch.as_tensor(Xc, device=device)
        extra = k - Xc.shape[1]
        gen = torch.Generator(device="cpu").manual_seed(20_000 + seed)
        X = torch.cat([_interpolate(Xc, Nc, N),
                       torch.randn((n_g, extra), generator=gen, dtype=torch.float64).to(device)], dim=1)
    else:
        gen = torch.Generator(device="cpu").manual_seed(20_000 + seed)
        X = torch.randn((n_g, k), generator=gen, dtype=torch.float64).to(device)
    b = H.t_max + float(v.max()) + 1e-3 * H.t_max
    e, X, HX = _rayleigh_ritz(H, X)
    for _ in range(max_iter + 1):
        res = float(torch.linalg.vector_norm(HX[:, :n_states] - X[:, :n_states] * e[:n_states], dim=0).max())
        if res < tol:
            break
        a = float(e[-1])
        X = _filter(H, X, degree, a, b, float(e[0]))
        e, X, HX = _rayleigh_ritz(H, X)
    else:
        raise RuntimeError(f"Chebyshev-filtered subspace iteration did not converge: residual {res:.2e}")
    return e[:n_states].cpu().numpy(), X[:, :n_states].cpu().numpy()
