"""Learned surrogate of the screened potentials W_ij = W (phi_i phi_j) (the workload's learned form;
the paper has none): training pairs from the stochastic TDH of `sbse_apply_W`, training with the
FNO kernels (`sbse_fno_*`), and surrogate-assisted W for all pairs with a random spot check
against fresh propagation; a spot-checked pair whose surrogate W misses the propagated one by more
than `tol` keeps the propagated W, and if most spot checks fail every pair is propagated.

Only argument marshalling happens here: inputs are formed by `sbse_fno_pair_inputs`, the network
runs in the FNO kernels, W is stored by `sbse_surrogate_W`. Device buffers are torch tensors.
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
