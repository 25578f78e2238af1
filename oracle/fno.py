"""FP64 oracle of the Fourier-neural-operator surrogate for the screened potential W^pol_ij.

TEST INFRASTRUCTURE: imported only by the tests. Not part of the library's compute path.

The paper has no learned component; the surrogate is defined by the workload description: inputs
(rho_ij, V_loc) on the N^3 grid, a lifting to C channels, Fourier layers
    U_l = K_l(V_l) + W_l V_l + b_l,   V_{l+1} = GELU(U_l) (no activation after the last layer),
with the spectral convolution K_l(V) = irfftn( R_l . rfftn(V) restricted to the kept modes ), and
a linear projection to one output channel. Kept modes (m per axis): kx in [0, m) along the
half-spectrum axis x and ky, kz in [0, m) U [N - m, N): 4 m^3 complex modes, each with a C x C
complex weight matrix R_l[mode][c_in][c_out]. GELU(x) = x (1 + erf(x / sqrt 2)) / 2.

Arrays: activations (B, C, N, N, N) indexed [b, c, z, y, x]; spectra (B, C, 2m, 2m, m) indexed
[b, c, kz, ky, kx] with the kz / ky index running over 0..m-1, N-m..N-1.

Gradients are written out from the chain rule (see `backward`) and pinned by finite differences.
"""
from __future__ import annotations

import dataclasses

import numpy as np
from scipy.special import erf


@dataclasses.dataclass
class FNOParams:
    lift_w: np.ndarray  # (C, 2)
    lift_b: np.ndarray  # (C,)
    spec: list          # n_layers x complex (2m, 2m, m, C, C): R[kz, ky, kx, ci, co]
    pw_w: list          # n_layers x (C, C): W[co, ci]
    pw_b: list          # n_layers x (C,)
    proj_w: np.ndarray  # (C,)
    proj_b: float


def kept_index(N: int, m: int) -> np.ndarray:
    """FFT indices kept along the full axes: 0..m-1, N-m..N-1."""
    return np.concatenate([np.arange(m), np.arange(N - m, N)])


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / np.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + erf(x / np.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / np.sqrt(2.0 * np.pi)


def spectral_forward(v, R, m):
    """Truncated rfftn -> per-mode channel mixing -> irfftn with the other modes zero."""
    B, C, N = v.shape[0], v.shape[1], v.shape[2]
    k = kept_index(N, m)
    F = np.fft.rfftn(v, axes=(2, 3, 4))[:, :, k][:, :, :, k][:, :, :, :, :m]  # (B,C,2m,2m,m)
    G = np.einsum("bizyx,zyxio->bozyx", F, R)
    full = np.zeros((B, R.shape[-1], N, N, N // 2 + 1), dtype=complex)
    full[np.ix_(np.arange(B), np.arange(R.shape[-1]), k, k, np.arange(m))] = G
    return np.fft.irfftn(full, s=(N, N, N), axes=(2, 3, 4)), F


def forward(p: FNOParams, x, m: int, keep=False):
    """x: (B, 2, N, N, N) -> (B, N, N, N). keep=True also returns the intermediates."""
    cache = {"x": x, "V": [], "U": [], "F": []}
    v = np.einsum("ci,bizyx->bczyx", p.lift_w, x) + p.lift_b[None, :, None, None, None]
    L = len(p.spec)
    for l in range(L):
        cache["V"].append(v)
        s, F = spectral_forward(v, p.spec[l], m)
        u = s + np.einsum("oi,bizyx->bozyx", p.pw_w[l], v) + p.pw_b[l][None, :, None, None, None]
        cache["U"].append(u)
        cache["F"].append(F)
        v = gelu(u) if l < L - 1 else u
    cache["V"].append(v)
    y = np.einsum("c,bczyx->bzyx", p.proj_w, v) + p.proj_b
    return (y, cache) if keep else y


def backward(p: FNOParams, cache, dy, m: int):
    """Gradients of L with dL/dy = dy, by the chain rule through each layer:
      projection: dW_proj[c] = sum dy V_L[c], dV_L[c] = W_proj[c] dy;
      activation: dU = dV GELU'(U) (identity after the last layer);
      pointwise : dW[co,ci] = sum dU[co] V[ci], db = sum dU, dV += W^T dU;
      spectral  : with S = irfftn(G), the complex gradient dG = dL/dRe G + i dL/dIm G equals
                  c_kx / N^3 * rfftn(dS) on the kept modes (c_0 = 1, c_kx = 2 for kx > 0: the
                  Hermitian completion), dR[ci,co] = sum_b conj(F[ci]) dG[co],
                  dF[ci] = sum_co conj(R[ci,co]) dG[co], and dV(r) = Re sum_k dF_k e^{+i k.r};
      lifting   : dW_lift[c,i] = sum dV_0[c] x[i], db_lift = sum dV_0, dx[i] = sum_c W_lift[c,i] dV_0[c].
    Returns a dict of gradients with the parameter shapes."""
    x = cache["x"]
    N = x.shape[2]
    L = len(p.spec)
    k = kept_index(N, m)
    ckx = np.where(np.arange(m) == 0, 1.0, 2.0)
    g = {"spec": [None] * L, "pw_w": [None] * L, "pw_b": [None] * L}
    vL = cache["V"][L]
    g["proj_w"] = np.einsum("bzyx,bczyx->c", dy, vL)
    g["proj_b"] = float(np.sum(dy))
    dv = p.proj_w[None, :, None, None, None] * dy[:, None]
    for l in range(L - 1, -1, -1):
        u, v, F = cache["U"][l], cache["V"][l], cache["F"][l]
        du = dv * gelu_grad(u) if l < L - 1 else dv
        g["pw_w"][l] = np.einsum("bozyx,bizyx->oi", du, v)
        g["pw_b"][l] = np.sum(du, axis=(0, 2, 3, 4))
        dv_new = np.einsum("oi,bozyx->bizyx", p.pw_w[l], du)
        dS = np.fft.rfftn(du, axes=(2, 3, 4))[:, :, k][:, :, :, k][:, :, :, :, :m]
        dG = dS * (ckx / N ** 3)[None, None, None, None, :]
        g["spec"][l] = np.einsum("bizyx,bozyx->zyxio", np.conj(F), dG)
        dF = np.einsum("zyxio,bozyx->bizyx", np.conj(p.spec[l]), dG)
        B, C = dF.shape[0], dF.shape[1]
        full = np.zeros((B, C, N, N, N), dtype=complex)
        full[np.ix_(np.arange(B), np.arange(C), k, k, np.arange(m))] = dF
        # Re sum_k dF_k e^{+i k.r} = N^3 Re(ifftn(full)) over the kept (half-axis) modes only
        dv_new += np.real(np.fft.ifftn(full, axes=(2, 3, 4))) * N ** 3
        dv = dv_new
    g["lift_w"] = np.einsum("bczyx,bizyx->ci", dv, x)
    g["lift_b"] = np.sum(dv, axis=(0, 2, 3, 4))
    g["x"] = np.einsum("ci,bczyx->bizyx", p.lift_w, dv)
    return g


def init_params(C: int, m: int, n_layers: int, seed: int) -> FNOParams:
    """Seeded initialisation (scaled so activations stay O(1))."""
    rng = np.random.default_rng(seed)
    scale = 1.0 / (C * C)
    spec = [scale * (rng.standard_normal((2 * m, 2 * m, m, C, C))
                     + 1j * rng.standard_normal((2 * m, 2 * m, m, C, C))) for _ in range(n_layers)]
    return FNOParams(
        lift_w=rng.standard_normal((C, 2)) / np.sqrt(2.0),
        lift_b=0.1 * rng.standard_normal(C),
        spec=spec,
        pw_w=[rng.standard_normal((C, C)) / np.sqrt(C) for _ in range(n_layers)],
        pw_b=[0.1 * rng.standard_normal(C) for _ in range(n_layers)],
        proj_w=rng.standard_normal(C) / np.sqrt(C),
        proj_b=0.05,
    )
