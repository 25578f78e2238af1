"""One system on several GPUs: the occupied pairs (i, j) are independent W applications (Sec. II.B:
each pair density is propagated on its own, coupled only to the shared stochastic set), so a
system's pairs are split into contiguous blocks, one per rank. Every rank propagates its block
with the same stochastic coefficients (same seed) and contracts its pairs' direct-element columns
locally (sbse_get_direct: n_c^2 numbers per pair); those columns are gathered, which is the one
exchange of the method (n_c^2 x n_o(n_o+1)/2 doubles, about 1.1 MB for the 520-electron system
against 0.96 GB for the W fields themselves), and every rank assembles A from them
(sbse_set_direct, sbse_build_A) and takes its excitons.

Only marshalling happens here: W and D come from the library; the exchange is a
`torch.distributed` all-gather (NCCL with device buffers, gloo with host buffers). `gather_W`
(the W fields themselves) remains for callers that need W on every rank.
"""
from __future__ import annotations

import numpy as np

from . import binding as B


def pair_list(n_o: int):
    """Canonical pair order (0,0), (0,1), ..., (n_o-1, n_o-1), as in the C interface."""
    return [(i, j) for i in range(n_o) for j in range(i, n_o)]


def pair_block(n_pairs: int, rank: int, world: int) -> range:
    """Indices of the contiguous block of pairs owned by `rank` (sizes differ by at most one)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    return range((n_pairs * rank) // world, (n_pairs * (rank + 1)) // world)


def gather_W(w_local: np.ndarray, n_pairs: int, rank: int, world: int, group=None) -> np.ndarray:
    """All-gather the blocks of W (each rank's rows in pair order) into the full n_pairs x n_g array."""
    import torch
    import torch.distributed as dist

    sizes = [len(pair_block(n_pairs, r, world)) for r in range(world)]
    if w_local.shape[0] != sizes[rank]:
        raise ValueError("w_local must hold this rank's block of pairs")
    n_g = w_local.shape[1]
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" \
        else torch.device("cpu")
    buf = torch.zeros((max(sizes), n_g), dtype=torch.float64, device=dev)
    if sizes[rank]:
        buf[:sizes[rank]] = torch.from_numpy(np.ascontiguousarray(w_local)).to(dev)
    outs = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(outs, buf, group=group)
    return np.concatenate([outs[r][:sizes[r]].cpu().numpy() for r in range(world)], axis=0)


def gather_columns(d_local: np.ndarray, n_pairs: int, rank: int, world: int, group=None) -> np.ndarray:
    """All-gather the ranks' direct-element columns (rows ab, one column per pair of the rank's
    block) into the n_c^2 x n_pairs array in canonical pair order."""
    import torch
    import torch.distributed as dist

    sizes = [len(pair_block(n_pairs, r, world)) for r in range(world)]
    if d_local.shape[1] != sizes[rank]:
        raise ValueError("d_local must hold this rank's block of pairs")
    rows = d_local.shape[0]
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" \
        else torch.device("cpu")
    buf = torch.zeros((max(sizes), rows), dtype=torch.float64, device=dev)
    if sizes[rank]:
        buf[:sizes[rank]] = torch.from_numpy(np.ascontiguousarray(d_local.T)).to(dev)
    outs = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(outs, buf, group=group)
    return np.concatenate([outs[r][:sizes[r]].cpu().numpy() for r in range(world)], axis=0).T.copy()


def sharded_excitons(ctx: B.Context, params: B.TDHParams, n_o: int, n_c: int, k: int, rank: int,
                     world: int, group=None):
    """This rank's block of W by propagation and its direct-element columns, the all-gather of
    the columns, then A and its k lowest excitons (on every rank). Returns (A, excitons)."""
    pairs = pair_list(n_o)
    mine = [pairs[i] for i in pair_block(len(pairs), rank, world)]
    if mine:
        ctx.apply_W(params, mine)
        d_local = B.sbse_get_direct(ctx.h, mine, n_c)
    else:
        d_local = np.empty((n_c * n_c, 0))
    B.sbse_set_direct(ctx.h, gather_columns(d_local, len(pairs), rank, world, group))
    A = ctx.build_A()
    return A, ctx.spectrum(k)
