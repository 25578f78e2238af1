"""Batching form: many independent systems of uneven grid sizes advanced together on one GPU.

A `Batch` keeps one context (device memory, CUDA stream, captured graph of the time loop) per
system; `Batch.run` issues the systems' calls from a pool of host threads (the C calls release the
interpreter lock), so their kernels run concurrently on the GPU and fill it even when one system
alone would not, and from the second run on every system's time loop is a graph replay. The first
run of a batch goes one system at a time: under CUDA's lazy module loading the first launch of a
kernel loads its module, which would invalidate another thread's graph capture in progress; after
one run every kernel is loaded and every graph captured.
`autotune` picks, per grid size and pair count, the fastest split-operator variant that the grid
supports (three pass kernels or the persistent step kernel; plain or bulk-copy streamed passes;
all pairs per pass or L2-sized chunks of pairs) from a short timed trial, and caches the choice.
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


# pair-chunk sizes tried (SBSE_OPT_CHUNK_MB; 0 = every pair in one pass): one chunk near half of L2
_CHUNKS_MB = (0, 64)


def _variants(n: int, precision: int, pair_bytes: float):
    """(persistent, tma_planes, chunk_mb) triples that change the kernels or their launches on this
    grid; chunking is tried only where the pair batch does not fit in one chunk."""
    chunks = [c for c in _CHUNKS_MB if c == 0 or pair_bytes > c * 2 ** 20]
    if n in (80, 96) and precision == B.SBSE_MIXED:
        return [(0, 1, c) for c in chunks]  # the two-sweep passes
    tma = [0, 1] if (precision == B.SBSE_MIXED and n in (32, 40, 48, 64)) else [1]
    out = []
    for p in (0, 1):
        for t in tma:
            for c in chunks:
                if p == 0 or c == 0:  # the persistent kernel takes every pair at once
                    out.append((p, t, c))
    return out


def autotune(ctx: B.Context, item: BatchItem, params: B.TDHParams, trial_steps: int = 6) -> dict:
    """Time a short propagation with each step variant and keep the fastest (cached per grid)."""
    key = (item.n, item.n_o, params.n_s, ctx.precision)
    if key not in _TUNED:
        trial = dataclasses.replace(params, n_steps=trial_steps, clean_every=0)
        pairs = [(i, j) for i in range(item.n_o) for j in range(i, item.n_o)]
        pair_bytes = len(pairs) * params.n_s * item.n ** 3 * (8 if ctx.precision == B.SBSE_MIXED else 16)
        best = None
        for persistent, tma, chunk in _variants(item.n, ctx.precision, pair_bytes):
            _set(ctx, persistent, tma, chunk)
            ctx.apply_W(trial, pairs)  # warm-up of this variant
            t0 = time.perf_counter()
            ctx.apply_W(trial, pairs)
            dt = time.perf_counter() - t0
            if best is None or dt < best[3]:
                best = (persistent, tma, chunk, dt)
        _TUNED[key] = {"persistent": best[0], "tma_planes": best[1], "chunk_mb": best[2], "trial_s": best[3]}
    t = _TUNED[key]
    _set(ctx, t["persistent"], t["tma_planes"], t["chunk_mb"])
    return t


def _set(ctx, persistent: int, tma: int, chunk_mb: int):
    B.sbse_set_option(ctx.h, B.SBSE_OPT_PERSISTENT, persistent)
    B.sbse_set_option(ctx.h, B.SBSE_OPT_TMA_PLANES, tma)
    B.sbse_set_option(ctx.h, B.SBSE_OPT_CHUNK_MB, chunk_mb)


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
