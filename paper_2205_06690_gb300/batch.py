"""Batching form: many independent systems of uneven grid sizes advanced together on one GPU.

A `Batch` keeps one context (device memory, CUDA stream, captured graph of the time loop) per
system; `Batch.run` issues the systems' calls from a pool of host threads (the C calls release the
interpreter lock), so their kernels run concurrently on the GPU and fill it even when one system
alone would not, and from the second run on every system's time loop is a graph replay. The first
run of a batch goes one system at a time: under CUDA's lazy module loading the first launch of a
kernel loads its module, which would invalidate another thread's graph capture in progress; after
one run every kernel is loaded and every graph captured.
`autotune` picks, per grid size, the fastest split-operator variant that the grid supports (three
pass kernels or the persistent step kernel; plain or bulk-copy streamed passes) from a short timed
trial, and caches the choice.
"""
from __future__ import annotations

import concurrent.futures as cf
import dataclasses
import time

import numpy as np

from . import binding as B

_TUNED: dict = {}


@dataclasses.dataclass
class BatchItem:
    n: int
    box: float
    v_loc: np.ndarray
    phi: np.ndarray
    eps: np.ndarray
    n_occ: int
    n_o: int
    n_c: int
    scissor: float
    k: int
    seed: int = 0  # stochastic coefficient seed of the system


def _variants(n: int, precision: int):
    """(persistent, tma_planes) pairs that change the kernels on this grid."""
    if n in (80, 96) and precision == B.SBSE_MIXED:
        return [(0, 1)]  # the two-sweep passes: one variant
    tma = [0, 1] if (precision == B.SBSE_MIXED and n in (32, 40, 48, 64)) else [1]
    return [(p, t) for p in (0, 1) for t in tma]


def autotune(ctx: B.Context, item: BatchItem, params: B.TDHParams, trial_steps: int = 6) -> dict:
    """Time a short propagation with each step variant and keep the fastest (cached per grid)."""
    key = (item.n, item.n_o, params.n_s, ctx.precision)
    if key not in _TUNED:
        trial = dataclasses.replace(params, n_steps=trial_steps, clean_every=0)
        pairs = [(i, j) for i in range(item.n_o) for j in range(i, item.n_o)]
        best = None
        for persistent, tma in _variants(item.n, ctx.precision):
            B.sbse_set_option(ctx.h, B.SBSE_OPT_PERSISTENT, persistent)
            B.sbse_set_option(ctx.h, B.SBSE_OPT_TMA_PLANES, tma)
            ctx.apply_W(trial, pairs)  # warm-up of this variant
            t0 = time.perf_counter()
            ctx.apply_W(trial, pairs)
            dt = time.perf_counter() - t0
            if best is None or dt < best[2]:
                best = (persistent, tma, dt)
        _TUNED[key] = {"persistent": best[0], "tma_planes": best[1], "trial_s": best[2]}
    B.sbse_set_option(ctx.h, B.SBSE_OPT_PERSISTENT, _TUNED[key]["persistent"])
    B.sbse_set_option(ctx.h, B.SBSE_OPT_TMA_PLANES, _TUNED[key]["tma_planes"])
    return _TUNED[key]


class Batch:
    """Contexts of several systems, kept between runs."""

    def __init__(self, items, precision: int = B.SBSE_MIXED, device: int = 0):
        self.items = list(items)
        self.precision = precision
        self.warm = False
        self.ctx = []
        for it in self.items:
            c = B.Context(device, precision)
            c.precision = precision
            c.set_grid(it.n, it.box, it.v_loc)
            c.set_orbitals(it.n_occ, it.n_o, it.n_c, it.phi, it.eps, it.scissor)
            self.ctx.append(c)

    def _one(self, idx: int, params: B.TDHParams, tune: bool):
        it, c = self.items[idx], self.ctx[idx]
        if tune:
            autotune(c, it, params)
        pairs = [(i, j) for i in range(it.n_o) for j in range(i, it.n_o)]
        t0 = time.perf_counter()
        c.apply_W(dataclasses.replace(params, seed=it.seed), pairs)
        c.build_A(copy_out=False)
        ev = c.spectrum(it.k)
        return {"excitons": ev, "seconds": time.perf_counter() - t0, "pairs": len(pairs)}

    def run(self, params: B.TDHParams, workers: int = 8, tune: bool = True):
        """Whole hot path (all pairs, A, excitons) of every system; per-system results and the
        wall time of the batch."""
        t0 = time.perf_counter()
        with cf.ThreadPoolExecutor(max_workers=workers if self.warm else 1) as ex:
            res = list(ex.map(lambda i: self._one(i, params, tune), range(len(self.items))))
        self.warm = True
        return res, time.perf_counter() - t0

    def close(self):
        for c in self.ctx:
            c.close()
        self.ctx = []

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def run_batch(items, params: B.TDHParams, precision: int = B.SBSE_MIXED, workers: int = 8,
              tune: bool = True, device: int = 0):
    """One run of a fresh batch (contexts created and destroyed here)."""
    with Batch(items, precision, device) as b:
        return b.run(params, workers, tune)
