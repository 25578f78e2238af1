"""Learned surrogate of the screened potentials W_ij = W (phi_i phi_j) (the workload's learned form;
the paper has none): training pairs from the stochastic TDH of `sbse_apply_W`, training with the
FNO kernels (`sbse_fno_*`), and surrogate-assisted W for all pairs with a random spot check
against fresh propagation; a spot-checked pair whose surrogate W misses the propagated one by more
than `tol` keeps the propagated W, and if most spot checks fail every pair is propagated.

Only argument marshalling happens here: inputs are formed by `sbse_fno_pair_inputs`, the network
runs in the FNO kernels, W is stored by `sbse_surrogate_W`. Device buffers are torch tensors.

Polarisation form (the configured scale): the network predicts only the polarisation part
W^pol_ij = W_ij - q_ij; the bare part q_ij = v(phi_i phi_j) is computed exactly (`sbse_bare_W`) and
the prediction is added to it (`sbse_add_W`). The network's grid may differ from the system's: the
inputs and the prediction are resampled between the two grids of the same box (`sbse_resample`).
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np

from . import binding as B


@dataclasses.dataclass
class Scales:
    """Fixed input / output scales: x = (rho / s_rho, V / s_v), W = s_w y."""
    s_rho: float
    s_v: float
    s_w: float


def _torch():
    import torch
    return torch


def training_pairs(ctx, params: B.TDHParams, pairs, n_g: int, scales: Scales):
    """Propagate `pairs` with the stochastic TDH and return device tensors (x, t) of inputs and
    normalised targets W_ij / s_w."""
    torch = _torch()
    W = ctx.apply_W(params, pairs, copy_out=True)
    n = len(pairs)
    x = torch.empty((n, 2, n_g), dtype=torch.float32, device="cuda")
    B.sbse_fno_pair_inputs(ctx.h, pairs, scales.s_rho, scales.s_v, x.data_ptr())
    t = torch.from_numpy((W / scales.s_w).astype(np.float32)).cuda()
    return x, t


def train(net: B.FNO, x, t, steps: int, batch: int, lr: float, seed: int = 0):
    """Adam on random mini-batches of the pairs; returns the loss history."""
    torch = _torch()
    g = torch.Generator(device="cpu").manual_seed(seed)
    n = x.shape[0]
    losses = []
    xb = torch.empty((batch,) + tuple(x.shape[1:]), dtype=torch.float32, device="cuda")
    tb = torch.empty((batch,) + tuple(t.shape[1:]), dtype=torch.float32, device="cuda")
    for _ in range(steps):
        idx = torch.randperm(n, generator=g)[:batch].cuda()
        xb.copy_(x.index_select(0, idx))
        tb.copy_(t.index_select(0, idx))
        losses.append(net.train_step(batch, xb.data_ptr(), tb.data_ptr(), lr))
    return losses


def surrogate_apply_W(ctx, net: B.FNO, scales: Scales, params: B.TDHParams, pairs, n_g: int,
                      spot_frac: float = 0.05, tol: float = 0.1, seed: int = 0,
                      max_fail_frac: float = 0.5):
    """W_ij for all pairs from the surrogate, then a spot check of a random `spot_frac` of them
    against fresh propagation (at least one pair). Returns a report dict."""
    t0 = time.perf_counter()
    B.sbse_surrogate_W(ctx.h, net.h, pairs, scales.s_rho, scales.s_v, scales.s_w)
    t_sur = time.perf_counter() - t0
    rng = np.random.default_rng(seed)
    n_spot = max(1, int(round(spot_frac * len(pairs))))
    spot = [pairs[k] for k in sorted(rng.choice(len(pairs), size=n_spot, replace=False))]
    w_sur = B.sbse_get_W(ctx.h, spot, n_g)
    t1 = time.perf_counter()
    w_tdh = ctx.apply_W(params, spot, copy_out=True)  # propagated W replaces the spot pairs
    t_tdh = time.perf_counter() - t1
    err = np.linalg.norm(w_sur - w_tdh, axis=1) / np.linalg.norm(w_tdh, axis=1)
    failed = [p for p, e in zip(spot, err) if e > tol]
    fallback = len(failed) > max_fail_frac * n_spot
    if fallback:
        rest = [p for p in pairs if p not in spot]
        if rest:
            ctx.apply_W(params, rest)
    return {"spot_pairs": spot, "spot_rel_err": err.tolist(), "failed": failed, "fallback": fallback,
            "surrogate_s_per_pair": t_sur / len(pairs), "tdh_s_per_pair": t_tdh / len(spot)}


# ---- polarisation form ----------------------------------------------------------------------------

def init_params(net: B.FNO, seed: int = 0) -> np.ndarray:
    """Random initial parameters in the layout of `sbse_fno_set_params`: lift and projection
    weights with variance 1 / fan-in, spectral weights uniform in [0, 1 / width^2) (real and
    imaginary parts), pointwise weights with variance 1 / width, zero biases. Sets and returns them."""
    rng = np.random.default_rng(seed)
    C, m = net.width, net.modes
    parts = [rng.standard_normal(2 * C) / np.sqrt(2.0), np.zeros(C)]
    for _ in range(net.layers):
        parts.append(rng.random(2 * (2 * m) * (2 * m) * m * C * C) / (C * C))
        parts.append(rng.standard_normal(C * C) / np.sqrt(C))
        parts.append(np.zeros(C))
    parts += [rng.standard_normal(C) / np.sqrt(C), np.zeros(1)]
    p = np.concatenate(parts).astype(np.float32)
    assert p.size == net.n_params
    net.set_params(p)
    return p


def net_inputs(ctx, pairs, n_sys: int, n_net: int, scales: Scales):
    """Inputs (rho_ij / s_rho, V_loc / s_v) of the pairs on the network's grid: [n][2][n_net^3]."""
    torch = _torch()
    n = len(pairs)
    x = torch.empty((n, 2, n_sys ** 3), dtype=torch.float32, device="cuda")
    B.sbse_fno_pair_inputs(ctx.h, pairs, scales.s_rho, scales.s_v, x.data_ptr())
    if n_sys == n_net:
        return x
    xr = torch.empty((n, 2, n_net ** 3), dtype=torch.float32, device="cuda")
    B.sbse_resample(ctx.h, 2 * n, n_sys, x.data_ptr(), n_net, xr.data_ptr())
    return xr


def polarisation_targets(ctx, params: B.TDHParams, pairs, n_sys: int, n_net: int):
    """Propagate the pairs and return W^pol = W - q on the network's grid ([n][n_net^3], FP32,
    device, unscaled). The pairs' W in ctx holds q afterwards."""
    torch = _torch()
    W = ctx.apply_W(params, pairs, copy_out=True)
    B.sbse_bare_W(ctx.h, pairs)
    q = B.sbse_get_W(ctx.h, pairs, n_sys ** 3)
    pol = torch.from_numpy((W - q).astype(np.float32)).cuda()
    if n_sys == n_net:
        return pol
    out = torch.empty((len(pairs), n_net ** 3), dtype=torch.float32, device="cuda")
    B.sbse_resample(ctx.h, len(pairs), n_sys, pol.data_ptr(), n_net, out.data_ptr())
    return out


def train_schedule(net: B.FNO, x, t, epochs: int, batch: int, lr0: float, lr1: float, seed: int = 0):
    """Adam over shuffled epochs with a cosine learning-rate decay from lr0 to lr1; returns the mean
    loss of every epoch."""
    torch = _torch()
    g = torch.Generator(device="cpu").manual_seed(seed)
    n = x.shape[0]
    steps = epochs * (n // batch)
    xb = torch.empty((batch,) + tuple(x.shape[1:]), dtype=torch.float32, device="cuda")
    tb = torch.empty((batch,) + tuple(t.shape[1:]), dtype=torch.float32, device="cuda")
    hist, k = [], 0
    for _ in range(epochs):
        perm = torch.randperm(n, generator=g).cuda()
        tot = 0.0
        for b0 in range(0, n - batch + 1, batch):
            idx = perm[b0:b0 + batch]
            xb.copy_(x.index_select(0, idx))
            tb.copy_(t.index_select(0, idx))
            lr = lr1 + 0.5 * (lr0 - lr1) * (1.0 + np.cos(np.pi * k / max(1, steps)))
            tot += net.train_step(batch, xb.data_ptr(), tb.data_ptr(), float(lr))
            k += 1
        hist.append(tot / max(1, n // batch))
    return hist


def surrogate_pol_apply_W(ctx, net: B.FNO, scales: Scales, params: B.TDHParams, pairs, n_sys: int,
                          spot_frac: float = 0.05, tol: float = 1.0, seed: int = 0,
                          max_fail_frac: float = 0.5, seed_step: int = 7919):
    """W_ij = q_ij + surrogate W^pol_ij for all pairs, then a spot check of a random `spot_frac` of
    them (at least one) against fresh propagation. The stochastic W^pol of one propagation carries
    sampling noise, so a spot pair is propagated with two stochastic seeds (params.seed and
    params.seed + seed_step) and the surrogate passes when it is no farther from the first sample
    than the second sample is: ||sur - t1|| <= tol ||t2 - t1||. The spot pairs keep the mean of the
    two samples; if more than `max_fail_frac` of the spot checks fail, every other pair is
    propagated as well (the method-level fallback). Returns a report dict."""
    torch = _torch()
    n_net = net.n
    t0 = time.perf_counter()
    B.sbse_bare_W(ctx.h, pairs)
    rng = np.random.default_rng(seed)
    n_spot = 0 if spot_frac <= 0 else max(1, int(round(spot_frac * len(pairs))))  # 0: no spot check
    spot = [pairs[k] for k in sorted(rng.choice(len(pairs), size=n_spot, replace=False))]
    bmax = net.max_batch
    y = torch.empty((bmax, n_net ** 3), dtype=torch.float32, device="cuda")
    ys = y if n_sys == n_net else torch.empty((bmax, n_sys ** 3), dtype=torch.float32, device="cuda")
    for k0 in range(0, len(pairs), bmax):
        chunk = pairs[k0:k0 + bmax]
        x = net_inputs(ctx, chunk, n_sys, n_net, scales)
        net.forward(len(chunk), x.data_ptr(), y.data_ptr())
        if ys is not y:
            B.sbse_resample(ctx.h, len(chunk), n_net, y.data_ptr(), n_sys, ys.data_ptr())
        B.sbse_add_W(ctx.h, chunk, ys.data_ptr(), scales.s_w)
    torch.cuda.synchronize()
    t_sur = time.perf_counter() - t0
    t1 = time.perf_counter()
    ratio = np.zeros(0)
    if spot:
        w_sur = B.sbse_get_W(ctx.h, spot, n_sys ** 3)
        w1 = ctx.apply_W(params, spot, copy_out=True)
        w2 = ctx.apply_W(dataclasses.replace(params, seed=params.seed + seed_step), spot, copy_out=True)
        B.sbse_set_W(ctx.h, spot, 0.5 * (w1 + w2))
        ratio = np.linalg.norm(w_sur - w1, axis=1) / np.linalg.norm(w2 - w1, axis=1)
    t_tdh = time.perf_counter() - t1
    failed = [p for p, e in zip(spot, ratio) if e > tol]
    fallback = len(failed) > max_fail_frac * n_spot
    t_fb = 0.0
    if fallback:
        rest = [p for p in pairs if p not in spot]
        if rest:
            t2 = time.perf_counter()
            ctx.apply_W(params, rest)
            t_fb = time.perf_counter() - t2
    return {"spot_pairs": spot, "spot_ratio": ratio.tolist(), "failed": failed, "fallback": fallback,
            "surrogate_s": t_sur, "spot_tdh_s": t_tdh, "fallback_s": t_fb,
            "surrogate_s_per_pair": t_sur / len(pairs), "tdh_s_per_pair": t_tdh / max(1, 2 * len(spot))}
