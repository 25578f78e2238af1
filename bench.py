#!/usr/bin/env python
"""Benchmark of the stochastic-BSE hot path on GB300.

Workload (default): the paper-scale system, a 96^3 grid (24 bohr box, 170 Gaussian wells, seed 2),
N_occ = 260 (520 electrons), n_o = 16, n_c = 32 (136 pairs, A is 512 x 512), L = 10 stochastic
orbitals, 2000 steps of dt = 0.05, gamma = 0.1, cleaning every M = 10 steps.

One step = W_ij for one block of pairs by stochastic TDH (all time steps, cleaning, damped time
integral; the blocks of 68 pairs are taken in turn, so two steps renew all 136), then the
exchange and direct contractions over all pairs' W, the FP64 Tamm-Dancoff matrix A and its lowest
excitons. The whole system is also run end to end through the C ABI from pinned host buffers.
Smaller workloads (--workload mid48 / tiny16) advance all their pairs in every step.

Metric: W-applications per second (pairs completed per second of device time) for the whole job.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference] [--precision fp64]
Under torchrun every rank runs its own replica of the workload with its own stochastic seed
(independent problems, no collective on the data path): weak scaling.
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="large96")
    ap.add_argument("--pairs-per-step", type=int, default=None,
                    help="pairs per benchmark step (default: all up to 64, else one eighth)")
    ap.add_argument("--prof-steps", type=int, default=2)
    ap.add_argument("--batch-workers", type=int, default=8, help="batch64: systems run at once")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--n-steps", type=int, default=None, help="override the TDH step count")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=None)
    ap.add_argument("--chunk-mb", type=int, default=None, help="SBSE_OPT_CHUNK_MB (L2 chunking)")
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the whole-system end-to-end call "
                    "(profiling runs); the pairs outside the timed blocks then keep W = 0")
    ap.add_argument("--fno-systems", type=int, default=32, help="fno64: training systems")
    ap.add_argument("--fno-epochs", type=int, default=30, help="fno64: training epochs")
    ap.add_argument("--fno-large96", action="store_true",
                    help="fno64: also evaluate on the 96^3 paper-scale system (resampled to 64^3)")
    ap.add_argument("--oracle-child", default=None, help=argparse.SUPPRESS)
    return ap.parse_args()


# ---------------------------------------------------------------------------------------------
# the oracle as the CPU baseline / reference arm: one pair per host core, each in its own
# single-threaded child process (pairs are independent W applications)

class _StepClock(list):
    """Passed to the oracle as its `record` list: time stamps of every accumulated sample u_n, i.e.
    the end of each TDH step of its own loop (the oracle itself is unchanged)."""

    def append(self, item):
        super().append(time.perf_counter())


def _oracle_child(spec_path: str) -> None:
    import numpy as np

    from oracle import tdh
    with open(spec_path) as f:
        spec = json.load(f)
    z = np.load(spec["system"])
    phi, v = z["phi"], z["v_loc"]
    N, box, n_occ, n_o = spec["N"], spec["box"], spec["n_occ"], spec["n_o"]
    g = tdh.Grid(N, box)
    coeff = tdh.stochastic_coefficients(spec["seed"], spec["n_s"], n_occ, "gaussian")
    op = tdh.TDHParams(n_steps=spec["sample_steps"], dt=spec["dt"], gamma=spec["gamma"],
                       alpha=spec["alpha"], clean_every=spec["clean_every"])
    phi_o = phi[n_occ - n_o:n_occ]
    i, j = spec["pair"]
    rho = phi_o[i] * phi_o[j]
    clock = _StepClock()
    t0 = time.perf_counter()
    tdh.coulomb_periodic(rho, g) + tdh.tdh_w_pol(g, v, phi[:n_occ], rho, coeff, op, record=clock)
    t1 = time.perf_counter()
    # clock[n] = end of step n - 1 (clock[0]: after the set-up and the first cleaning)
    print(json.dumps({"total": t1 - t0, "setup": clock[0] - t0,
                      "steps": [b - a for a, b in zip(clock[:-1], clock[1:])]}))


def oracle_cores() -> int:
    """Host cores for the oracle children, bounded by the memory each needs."""
    n = os.cpu_count() or 1
    try:
        avail = os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
    except (ValueError, OSError):
        avail = None
    return max(1, min(n, 64) if avail is None else min(n, 64, int(avail // (6 << 30)) or 1))


def run_oracle_parallel(system, preset, sample_steps, seed, cores=None):
    """Run the oracle on `cores` pairs at once (one child each) for `sample_steps` TDH steps.
    Returns (cores, per-child step times [list of lists], per-child set-up seconds)."""
    import numpy as np
    cores = cores or oracle_cores()
    pairs = [(i, j) for i in range(preset.n_o) for j in range(i, preset.n_o)]
    with tempfile.TemporaryDirectory() as td:
        sp = os.path.join(td, "sys.npz")
        np.savez(sp, phi=system.phi[:preset.n_occ], v_loc=system.v_loc)
        env = dict(os.environ)
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            env[k] = "1"
        procs = []
        for c in range(cores):
            spec = dict(system=sp, N=system.N, box=system.box, n_occ=preset.n_occ, n_o=preset.n_o,
                        n_s=preset.n_s, dt=preset.dt, gamma=preset.gamma, alpha=preset.alpha,
                        clean_every=preset.clean_every, sample_steps=sample_steps, seed=seed,
                        pair=pairs[(len(pairs) - 1 - c) % len(pairs)])
            jp = os.path.join(td, f"spec{c}.json")
            with open(jp, "w") as f:
                json.dump(spec, f)
            procs.append(subprocess.Popen([sys.executable, os.path.abspath(__file__), "--oracle-child", jp],
                                          stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True,
                                          env=env, cwd=ROOT))
        steps, setup = [], []
        for pr in procs:
            out, err = pr.communicate()
            if pr.returncode != 0:
                raise RuntimeError("oracle child failed: " + err[-2000:])
            d = json.loads(out.strip().splitlines()[-1])
            steps.append(d["steps"])
            setup.append(d["setup"])
    return cores, steps, setup


def cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith(("model name", "cpu part")):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


# ---------------------------------------------------------------------------------------------

class ClockSampler:
    """nvidia-smi clock / throttle-reason samples every 200 ms during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.p = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.TemporaryFile(mode="w+")
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.f.read().splitlines():
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# the sources the pass kernels of each workload are compiled from (their definitions and the data
# structures they read; declarations of other launchers do not enter)
KERNEL_SOURCES = {
    "large96": ["fft_split.cu", "fft_reg.cuh", "passes.cuh", "common.cuh", "tables.cuh"],
    "default": ["fft_fast.cu", "fft_reg.cuh", "passes.cuh", "tma.cuh", "common.cuh", "tables.cuh"],
}


def kernel_source_hash(workload: str = "default") -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES.get(workload, KERNEL_SOURCES["default"]):
        with open(os.path.join(ROOT, "paper_2205_06690_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(phase, workload, mixed, sweep_bytes=None):
    """DRAM bytes (read + write) per launch of the pass, from the committed ncu summary, when it
    was taken on the current kernel sources; else None."""
    path = os.path.join(ROOT, "profiles", f"pair_passes_{workload}_traffic.txt")
    if phase is None or not mixed or not os.path.exists(path):
        return None, None
    with open(path) as f:
        d = json.load(f)
    if d.get("source_sha256_16") != kernel_source_hash(workload):
        return None, "kernel sources changed since the ncu capture"
    v = d.get("dram_bytes_per_launch", {}).get(str(phase))
    if not v:
        return None, None
    note = os.path.relpath(path, ROOT)
    alg = d.get("algorithmic_bytes_per_launch")
    if sweep_bytes and alg and abs(sweep_bytes - alg) > 1e-6 * alg:
        # another block size than the capture's: these passes move their bytes per orbital
        v = float(v) * sweep_bytes / alg
        note += f" (scaled from its {alg / 1e9:.3f} GB launch to this {sweep_bytes / 1e9:.3f} GB one)"
    return float(v), note


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        for k in ("hbm_gbs", "hbm_GBs", "hbm"):
            if k in d:
                return float(d[k]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def block_default(pre) -> int:
    """Pairs per benchmark step: every pair for the small workloads; half of the 136 pairs of the
    96^3 system (68), so that one step (68 pairs x 2000 TDH steps + A + excitons) takes about 14 s
    and two steps refresh all of W. (Larger blocks amortise the per-step eta0 set and A build:
    measured 3.9 / 4.6 / 4.8 W/s for blocks of 17 / 34 / 68 pairs.)"""
    return pre.n_pairs if pre.n_pairs <= 64 else -(-pre.n_pairs // 2)


def batch_bench(args):
    """The batching form: 64 independent Gaussian-well systems of uneven grids ({32,40,48,64,80}^3,
    h = 0.25 bohr, N_occ = N/2, n_o = 4, n_c = 8, 500 steps), one context each, run concurrently
    from a pool of host threads; one step = the whole hot path of every system."""
    import numpy as np
    import torch

    os.environ.setdefault("SBSE_EIGENSOLVER", "chfsi")  # orbitals of 64 systems: on the GPU
    os.environ.setdefault("CUDA_MODULE_LOADING", "EAGER")  # no module loads during other threads' captures
    import sbse_inputs as si
    from paper_2205_06690_gb300 import batch
    from paper_2205_06690_gb300 import binding as B
    pres = si.batch_presets()
    t_in = time.perf_counter()
    items = []
    for p in pres:
        s = si.make_system(p)
        items.append(batch.BatchItem(p.N, p.box, s.v_loc, np.ascontiguousarray(s.phi), np.ascontiguousarray(s.eps),
                                     p.n_occ, p.n_o, p.n_c, p.scissor, p.n_exc, seed=p.seed))
    t_in = time.perf_counter() - t_in
    prm = B.TDHParams(n_s=10, n_steps=args.n_steps or 500, clean_every=10, dt=0.05, gamma=0.1, alpha=1e-4)
    n_pairs = sum(it.n_o * (it.n_o + 1) // 2 for it in items)
    bt = batch.Batch(items, B.SBSE_MIXED)
    for _ in range(args.warmup):
        bt.run(prm, workers=args.batch_workers, tune=True)
    clk = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.synchronize()
    clk.start()
    launches0 = B.sbse_kernel_launches()
    walls = []
    for _ in range(args.steps):
        torch.cuda.synchronize()
        res, wall = bt.run(prm, workers=args.batch_workers, tune=True)
        torch.cuda.synchronize()
        walls.append(wall)
    clocks = clk.stop()
    launches = B.sbse_kernel_launches() - launches0
    # the same systems one after another (no concurrency), for the gain of the pool
    torch.cuda.synchronize()
    _, serial = bt.run(prm, workers=1, tune=True)
    torch.cuda.synchronize()
    bt.close()
    # exciton error of the mixed path against the FP64 GPU path on one system of each grid size
    check = {}
    for n in sorted({it.n for it in items}):
        idx = [i for i, x in enumerate(items) if x.n == n][0]
        r64, _ = batch.run_batch([items[idx]], prm, precision=B.SBSE_FP64, workers=1, tune=False)
        check[str(n)] = float(np.max(np.abs(res[idx]["excitons"] - r64[0]["excitons"])) * 27211.386245988)
    ms_step = 1e3 * statistics.mean(walls)
    line = {
        "metric": "W-rho applications/sec (stochastic TDH, all pairs) + A build",
        "value": n_pairs / (ms_step / 1e3), "unit": "W-applications/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"batch64: {len(items)} Gaussian-well systems (seeds 100-163), grids "
                               f"{{32,40,48,64,80}}^3 at h = 0.25 bohr, N_occ = N/2, n_o = 4, n_c = 8, "
                               f"{n_pairs} pairs in all, L = 10, {prm.n_steps} steps, M = 10",
                   "step": "the whole hot path (all pairs, A, 4 excitons) of every system, "
                           f"{args.batch_workers} systems at a time from a thread pool, each time loop "
                           "replayed as a CUDA graph, per-grid variant from the autotuner",
                   "timing": "host wall clock between device-wide synchronisations (the systems run on "
                             "their own streams)"},
        "clocks": clocks, "gpu_launches": launches,
        "serial_ms_per_step": 1e3 * serial, "concurrency_gain": serial / (ms_step / 1e3),
        "autotuned": {f"{k[0]}": v for k, v in batch._TUNED.items()},
        "exciton_dev_vs_fp64_mev": check, "inputs_s": t_in,
        "e2e": None, "roofline": None, "cpu_baseline": None,
    }
    print(json.dumps(line), flush=True)


def fno_bench(args):
    """The learned form at its configured scale: an FNO (64^3, width 32, 12 modes, 4 layers)
    trained on the polarisation part W^pol = W - q of TDH pairs from 20-80-well systems on 64^3
    grids of a 24 bohr box (seeds 1000 + k), then used for all pairs of held-out systems (seeds
    2000, 2001) with a 5 % spot check against fresh propagation. One step = the surrogate-assisted
    W of every pair of the held-out systems (bare part exact, polarisation part from the network,
    spot-checked pairs propagated) + A + excitons. Reported beside it: the excitons' deviation from
    a TDH run, the spread between two TDH runs of different stochastic seeds, and the deviation of
    the unscreened (bare) excitons, in meV."""
    import numpy as np
    import torch

    os.environ.setdefault("SBSE_EIGENSOLVER", "chfsi")
    import sbse_inputs as si
    from paper_2205_06690_gb300 import binding as B
    from paper_2205_06690_gb300 import surrogate as S
    HA_MEV = 27211.386245988
    n_steps = args.n_steps or 2000
    prm = B.TDHParams(n_s=10, n_steps=n_steps, clean_every=10, dt=0.05, gamma=0.1, alpha=1e-4, seed=11)
    NN = 64
    t0 = time.perf_counter()
    xs, ts, n_train_pairs = [], [], 0
    for p in si.fno_presets(args.fno_systems, first_seed=1000, n_steps=n_steps):
        s = si.make_system(p)
        with B.Context(0, B.SBSE_MIXED) as c:
            c.set_grid(p.N, p.box, s.v_loc)
            c.set_orbitals(p.n_occ, p.n_o, p.n_c, s.phi, s.eps, p.scissor)
            pairs = [(i, j) for i in range(p.n_o) for j in range(i, p.n_o)]
            sc1 = S.Scales(1.0, 1.0, 1.0)
            xs.append(S.net_inputs(c, pairs, p.N, NN, sc1))
            ts.append(S.polarisation_targets(c, dataclasses.replace(prm, seed=p.seed), pairs, p.N, NN))
            n_train_pairs += len(pairs)
    x = torch.cat(xs)
    t = torch.cat(ts)
    del xs, ts
    sc = S.Scales(float(x[:, 0].std()), float(x[:, 1].std()), float(t.std()))
    x[:, 0] /= sc.s_rho
    x[:, 1] /= sc.s_v
    t /= sc.s_w
    t_data = time.perf_counter() - t0
    net = B.FNO(NN, width=32, modes=12, layers=4, max_batch=4)
    S.init_params(net, seed=0)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    hist = S.train_schedule(net, x, t, epochs=args.fno_epochs, batch=4, lr0=1e-3, lr1=1e-5, seed=0)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t1
    del x, t
    torch.cuda.empty_cache()

    n_ref = 4  # stochastic seeds of the reference (the mean of their W: L = 40 orbitals' worth)

    def evaluate(p, system, n_sys):
        """Excitons of one system from: the mean W of n_ref TDH runs of different stochastic seeds
        (the reference), each single TDH run, the bare potentials alone, the surrogate (no spot
        check) and the surrogate-assisted path with its spot check; deviations from the reference
        in meV, times of one TDH run and of the surrogate-assisted path."""
        pairs = [(i, j) for i in range(p.n_o) for j in range(i, p.n_o)]
        ng = p.N ** 3
        out = {"system": f"{p.name}: {p.N}^3, {p.n_wells} wells, N_occ={p.n_occ}, {len(pairs)} pairs"}
        with B.Context(0, B.SBSE_MIXED) as c:
            c.set_grid(p.N, p.box, system.v_loc)
            c.set_orbitals(p.n_occ, p.n_o, p.n_c, system.phi[:p.n_occ + p.n_c], system.eps[:p.n_occ + p.n_c],
                           p.scissor)

            def excitons():
                c.build_A(copy_out=False)
                return c.spectrum(p.n_exc)

            Ws, Es, t_tdh = [], [], []
            for k in range(n_ref):
                torch.cuda.synchronize()
                ta = time.perf_counter()
                c.apply_W(dataclasses.replace(prm, seed=prm.seed + 101 * k), pairs)
                Es.append(excitons())
                torch.cuda.synchronize()
                t_tdh.append(time.perf_counter() - ta)
                Ws.append(B.sbse_get_W(c.h, pairs, ng))
            w_ref = sum(Ws) / n_ref
            B.sbse_set_W(c.h, pairs, w_ref)
            e_ref = excitons()
            B.sbse_bare_W(c.h, pairs)
            q = B.sbse_get_W(c.h, pairs, ng)
            e_bare = excitons()
            pol_ref = w_ref - q
            nrm = np.linalg.norm(pol_ref)
            pol_err_tdh = [float(np.linalg.norm(w - w_ref) / nrm) for w in Ws]
            # the surrogate alone (every pair)
            S.surrogate_pol_apply_W(c, net, sc, prm, pairs, n_sys, spot_frac=0.0, tol=np.inf, seed=0)
            w_sur = B.sbse_get_W(c.h, pairs, ng)
            pol_err_sur = float(np.linalg.norm(w_sur - w_ref) / nrm)
            steps, rep = [], None
            for k in range(args.warmup + args.steps):
                torch.cuda.synchronize()
                ts0 = time.perf_counter()
                rep = S.surrogate_pol_apply_W(c, net, sc, prm, pairs, n_sys, spot_frac=0.05, tol=1.0, seed=k)
                es = excitons()
                torch.cuda.synchronize()
                steps.append(time.perf_counter() - ts0)
            t_s = statistics.mean(steps[args.warmup:])
            # surrogate-only excitons (no spot pairs replaced), for the deviation of the network itself
            S.surrogate_pol_apply_W(c, net, sc, prm, pairs, n_sys, spot_frac=0.0, tol=np.inf, seed=0)
            e_sur = excitons()

        def dev(e):
            return float(np.max(np.abs(np.asarray(e) - e_ref)) * HA_MEV)

        out.update({
            "pairs": len(pairs), "tdh_s": statistics.mean(t_tdh), "surrogate_assisted_s": t_s,
            "tdh_w_per_s": len(pairs) / statistics.mean(t_tdh), "speedup_vs_tdh": statistics.mean(t_tdh) / t_s,
            "exciton_dev_vs_ref_mev": {"single_tdh_runs": [dev(e) for e in Es], "surrogate": dev(e_sur),
                                       "surrogate_assisted": dev(es), "bare_only": dev(e_bare)},
            "w_pol_rel_err_vs_ref": {"single_tdh_runs": pol_err_tdh, "surrogate": pol_err_sur},
            "reference": f"mean W of {n_ref} TDH runs with different stochastic seeds",
            "spot_ratio": rep["spot_ratio"], "fallback": rep["fallback"],
        })
        return out, len(pairs) / t_s

    held = []
    rates = []
    for p in si.fno_presets(2, first_seed=2000, n_steps=n_steps):
        r, w = evaluate(p, si.make_system(p), p.N)
        held.append(r)
        rates.append(w)
    large = None
    if args.fno_large96:
        pre = si.preset("large96")
        pre = dataclasses.replace(pre, n_steps=n_steps)
        large, _ = evaluate(pre, si.make_system(pre), pre.N)
    line = {
        "metric": "W-rho applications/sec (stochastic TDH, all pairs) + A build",
        "value": statistics.mean(rates), "unit": "W-applications/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(r["surrogate_assisted_s"] for r in held),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "fno64: FNO 64^3 (width 32, 12 modes/axis, 4 Fourier layers, BF16 weights) "
                               f"trained on W^pol of {n_train_pairs} TDH pairs from {args.fno_systems} "
                               "20-80-well systems (64^3, 24 bohr box, seeds 1000+); held-out systems "
                               "seeds 2000-2001 (36 pairs each), 5 % spot check",
                   "step": "surrogate-assisted W of all pairs of one held-out system (bare part exact, "
                           "W^pol from the network, spot pairs propagated) + A + 10 excitons",
                   "tdh": f"L=10, {n_steps} steps dt=0.05, gamma=0.1, M=10"},
        "training": {"pairs": n_train_pairs, "epochs": args.fno_epochs, "batch": 4,
                     "data_s": t_data, "train_s": t_train, "loss_first_last": [hist[0], hist[-1]],
                     "scales": dataclasses.asdict(sc)},
        "held_out": held, "large96": large,
        "e2e": None, "roofline": None, "cpu_baseline": None,
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.oracle_child:
        _oracle_child(args.oracle_child)
        return
    if args.workload == "batch64" and args.impl == "ours":
        batch_bench(args)
        return
    if args.workload == "fno64" and args.impl == "ours":
        fno_bench(args)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    import numpy as np

    import sbse_inputs as si
    pre = si.preset(args.workload)
    n_steps = args.n_steps or pre.n_steps
    P = pre.n_pairs
    pairs = [(i, j) for i in range(pre.n_o) for j in range(i, pre.n_o)]
    blk = args.pairs_per_step or block_default(pre)
    blocks = [pairs[b:b + blk] for b in range(0, P, blk)]
    workload = (f"{pre.name}: {pre.N}^3 grid, box {pre.box} bohr, {pre.n_wells} Gaussian wells "
                f"(seed {pre.seed}), N_occ={pre.n_occ} ({2 * pre.n_occ} electrons), n_o={pre.n_o}, "
                f"n_c={pre.n_c}, {P} pairs, L={pre.n_s}, {n_steps} steps dt={pre.dt}, "
                f"gamma={pre.gamma}, M={pre.clean_every}, A {pre.n_o * pre.n_c}^2, "
                f"{pre.n_exc} excitons")
    step_def = (f"one step = W for one block of {blk} of the {P} pairs (all {n_steps} TDH steps, "
                f"L={pre.n_s}; blocks in turn), then A from all {P} pairs' W and the lowest "
                f"{pre.n_exc} excitons")
    metric = "W-rho applications/sec (stochastic TDH, all pairs) + A build"

    if args.impl == "reference":
        if rank != 0:
            return
        system = si.make_system(pre)
        k_steps = args.warmup + args.steps
        cores, steps, setup = run_oracle_parallel(system, pre, k_steps, pre.seed)
        # step k of the line = TDH step k of every child (each child one pair); the first W are
        # the warm-up; W-applications/s = cores / (mean time of one TDH step x n_steps)
        per = [statistics.mean(st[k] for st in steps) for k in range(k_steps)]
        timed = per[args.warmup:]
        val = cores / (statistics.mean(timed) * n_steps)
        line = {
            "impl": "reference", "metric": metric, "value": val, "unit": "W-applications/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.mean(timed), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload, "precision": "fp64 oracle",
                       "step": f"one TDH step of one pair on each of {cores} host cores"},
            "cpu_baseline": {"value": val, "unit": "W-applications/s", "cores": cores, "kind": "oracle",
                             "sample": f"{cores} pairs at once (one single-threaded process each) x "
                                       f"{k_steps} TDH steps; per-step times from the oracle's own loop, "
                                       f"scaled to {n_steps} steps; set-up "
                                       f"{statistics.mean(setup):.1f} s excluded; host {cpu_model()}"},
            "e2e": {"value": val, "unit": "W-applications/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
        }
        print(json.dumps(line), flush=True)
        return

    system = si.make_system(pre)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sample = min(10, n_steps)
        cores, steps, setup = run_oracle_parallel(system, pre, sample, pre.seed)
        per_step = statistics.mean(statistics.mean(st) for st in steps)
        cpu = {"value": cores / (per_step * n_steps), "unit": "W-applications/s", "cores": cores,
               "kind": "oracle",
               "sample": f"{cores} pairs of {pre.name} at once (one single-threaded process each) x "
                         f"{sample} TDH steps (mean step {per_step:.2f} s, set-up "
                         f"{statistics.mean(setup):.1f} s excluded), scaled to {n_steps} steps; "
                         f"host {cpu_model()}"}

    import torch
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    from paper_2205_06690_gb300 import binding as B

    prec = B.SBSE_MIXED if args.precision == "mixed" else B.SBSE_FP64
    prm = B.TDHParams(n_s=pre.n_s, n_steps=n_steps, clean_every=pre.clean_every, dt=pre.dt,
                      gamma=pre.gamma, alpha=pre.alpha, seed=pre.seed + 1000 * rank)
    ns = pre.n_occ + pre.n_c
    phi = np.ascontiguousarray(system.phi[:ns])
    eps = np.ascontiguousarray(system.eps[:ns])

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    ctx = B.Context(local, prec)
    if args.chunk_mb is not None:
        B.sbse_set_option(ctx.h, B.SBSE_OPT_CHUNK_MB, args.chunk_mb)
    ext = torch.cuda.ExternalStream(B.sbse_get_stream(ctx.h), device=dev)

    # end to end through the C ABI, the whole system in one call: pinned host inputs -> all pairs'
    # W -> A -> excitons copied back to the host (the first such call also captures the graph of
    # the time loop; a second, timed call replays it)
    v_pin = torch.from_numpy(np.ascontiguousarray(system.v_loc)).pin_memory()
    phi_pin = torch.from_numpy(phi).pin_memory()
    eps_pin = torch.from_numpy(eps).pin_memory()

    def full_system():
        ctx.set_grid(pre.N, pre.box, v_pin.numpy())
        ctx.set_orbitals(pre.n_occ, pre.n_o, pre.n_c, phi_pin.numpy(), eps_pin.numpy(), pre.scissor)
        ctx.apply_W(prm, pairs)
        ctx.build_A(copy_out=False)
        return ctx.spectrum(pre.n_exc)

    e2e_runs = 0 if args.no_e2e else (args.e2e_steps or 1)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_runs):
        full_system()
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / e2e_runs if e2e_runs else None
    if not e2e_runs:
        ctx.set_grid(pre.N, pre.box, system.v_loc)
        ctx.set_orbitals(pre.n_occ, pre.n_o, pre.n_c, phi, eps, pre.scissor)
        B.sbse_set_W(ctx.h, pairs, np.zeros((P, pre.N ** 3)))
    if world > 1 and e2e_s:
        t = torch.tensor([e2e_s], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        e2e_s = float(t.item())
    h2d = system.v_loc.nbytes + phi.nbytes + eps.nbytes + pre.n_s * pre.n_occ * 8
    d2h = pre.n_exc * 8

    # the benchmark step: W for the next block of pairs, then A and the excitons (all pairs' W
    # are resident from the call above)
    cursor = [0]

    def step():
        ctx.apply_W(prm, blocks[cursor[0] % len(blocks)])
        cursor[0] += 1
        ctx.build_A(copy_out=False)
        return ctx.spectrum(pre.n_exc)

    for _ in range(args.warmup):
        ev = step()
    # timed region: inputs resident in HBM, default configuration (time loop replayed as a graph);
    # the propagated orbitals (blk L n_g complex) exceed L2
    barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    launches0 = B.sbse_kernel_launches()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(ext)
    for _ in range(args.steps):
        ev = step()
    e1.record(ext)
    torch.cuda.synchronize()
    barrier()
    clocks = clk.stop()
    launches = B.sbse_kernel_launches() - launches0
    ms = e0.elapsed_time(e1)
    if world > 1:
        t = torch.tensor([ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    ms_step = ms / args.steps
    value = world * blk / (ms_step / 1e3)

    # per-pass times: further steps with events around every pass (this disables the graph replay,
    # so they run as direct launches; their step time is reported beside the headline's)
    prof_steps = max(1, args.prof_steps)
    B.sbse_profile(ctx.h, True)
    p0 = torch.cuda.Event(enable_timing=True)
    p1 = torch.cuda.Event(enable_timing=True)
    p0.record(ext)
    for _ in range(prof_steps):
        step()
    p1.record(ext)
    torch.cuda.synchronize()
    ms_prof = p0.elapsed_time(p1)
    phase = {ph: B.sbse_phase_time(ctx.h, ph) for ph in range(8)}
    B.sbse_profile(ctx.h, False)

    # A-build time (orbitals and W resident -> A in FP64), measured separately
    ta0 = torch.cuda.Event(enable_timing=True)
    ta1 = torch.cuda.Event(enable_timing=True)
    ta0.record(ext)
    ctx.build_A(copy_out=False)
    ta1.record(ext)
    torch.cuda.synchronize()
    a_build_ms = ta0.elapsed_time(ta1)

    # absorption spectrum from A (Sec. II.C, Chebyshev expansion; outside the timed step)
    ev_ha = 1.0 / 27.211386245988
    omega = np.linspace(0.0, 3.0, 1000)
    n_terms = 4096
    ctx.absorption(0, n_terms, 0.08 * ev_ha, omega)  # warm-up
    torch.cuda.synchronize()
    t_abs = time.perf_counter()
    sig_abs, _ = ctx.absorption(0, n_terms, 0.08 * ev_ha, omega)
    absorption = {"ms": 1e3 * (time.perf_counter() - t_abs), "n_terms": n_terms, "n_omega": len(omega),
                  "broadening_ev": 0.08, "axis": "x", "peak_omega_ha": float(omega[int(np.argmax(sig_abs))])}

    # the plain FP64 GPU path on the same block of pairs (shortened propagation, scaled to
    # n_steps): the comparator of the mixed path
    fp64 = None
    if prec == B.SBSE_MIXED and not args.no_fp64_compare:
        short = max(20, n_steps // 100)
        prm64 = B.TDHParams(n_s=pre.n_s, n_steps=short, clean_every=pre.clean_every, dt=pre.dt,
                            gamma=pre.gamma, alpha=pre.alpha, seed=prm.seed)
        prm32 = B.TDHParams(n_s=pre.n_s, n_steps=short, clean_every=pre.clean_every, dt=pre.dt,
                            gamma=pre.gamma, alpha=pre.alpha, seed=prm.seed)
        with B.Context(local, B.SBSE_FP64) as c64:
            c64.set_grid(pre.N, pre.box, system.v_loc)
            c64.set_orbitals(pre.n_occ, pre.n_o, pre.n_c, phi, eps, pre.scissor)
            c64.apply_W(prm64, blocks[0])
            ext64 = torch.cuda.ExternalStream(B.sbse_get_stream(c64.h), device=dev)
            f0 = torch.cuda.Event(enable_timing=True)
            f1 = torch.cuda.Event(enable_timing=True)
            f0.record(ext64)
            c64.apply_W(prm64, blocks[0])
            f1.record(ext64)
            torch.cuda.synchronize()
            ms64 = f0.elapsed_time(f1) * n_steps / short
            # the FP64 A build (FP64 CUDA-core contractions) on W held by the mixed context
            w_all = B.sbse_get_W(ctx.h, pairs, pre.N ** 3)
            B.sbse_set_W(c64.h, pairs, w_all)
            c64.build_A(copy_out=False)
            f0.record(ext64)
            c64.build_A(copy_out=False)
            f1.record(ext64)
            torch.cuda.synchronize()
            a64_ms = f0.elapsed_time(f1)
            del w_all
        # the mixed path on the same shortened run, for a like-for-like ratio
        ctx.apply_W(prm32, blocks[0])
        f0.record(ext)
        ctx.apply_W(prm32, blocks[0])
        f1.record(ext)
        torch.cuda.synchronize()
        ms32 = f0.elapsed_time(f1) * n_steps / short
        ctx.apply_W(prm, blocks[0])  # restore the block's full-length W
        # full-length exciton check of the mixed path against the FP64 path: the same system,
        # stochastic set and step count on the valence window cut to n_o = 3 (6 pairs, A of
        # 3 n_c rows; the FP64 run of every pair would take about 20 min)
        n_ow = min(3, pre.n_o)
        pairs_w = [(i, j) for i in range(n_ow) for j in range(i, n_ow)]
        exc = {}
        t_chk = time.perf_counter()
        for pm in (B.SBSE_FP64, B.SBSE_MIXED):
            with B.Context(local, pm) as cw:
                cw.set_grid(pre.N, pre.box, system.v_loc)
                cw.set_orbitals(pre.n_occ, n_ow, pre.n_c, phi, eps, pre.scissor)
                cw.apply_W(prm, pairs_w)
                cw.build_A(copy_out=False)
                exc[pm] = cw.spectrum(min(pre.n_exc, n_ow * pre.n_c))
        dev_mev = np.abs(exc[B.SBSE_MIXED] - exc[B.SBSE_FP64]) * 27211.386245988
        exciton_check = {"window": f"n_o = {n_ow} ({len(pairs_w)} pairs), n_c = {pre.n_c}, all {n_steps} TDH "
                                   f"steps, seed {prm.seed}",
                         "lowest": len(dev_mev), "max_dev_mev": float(dev_mev.max()),
                         "dev_mev": [float(x) for x in dev_mev], "target_mev": 5.0,
                         "seconds": time.perf_counter() - t_chk}
        fp64 = {"value": len(blocks[0]) / (ms64 / 1e3), "unit": "W-applications/s",
                "sample": f"{len(blocks[0])} pairs x {short} TDH steps, scaled to {n_steps}",
                "mixed_same_sample": len(blocks[0]) / (ms32 / 1e3),
                "mixed_speedup": ms64 / ms32,
                "a_build_ms": a64_ms, "a_build_speedup_mixed": a64_ms / a_build_ms,
                "exciton_check_mixed_vs_fp64": exciton_check}

    # learned form: FNO surrogate of the workload's shape (64^3, width 32, 12 modes, 4 layers)
    surrogate = None
    if not args.no_surrogate:
        net = B.FNO(64, width=32, modes=12, layers=4, max_batch=4, device=local)
        rng = np.random.default_rng(0)
        net.set_params(0.01 * rng.standard_normal(net.n_params).astype(np.float32))
        xs = torch.randn((4, 2, 64 ** 3), device=dev)
        ys = torch.empty((4, 64 ** 3), device=dev)
        net.forward(4, xs.data_ptr(), ys.data_ptr())
        net.train_step(4, xs.data_ptr(), ys.data_ptr(), 1e-4)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(3):
            net.forward(4, xs.data_ptr(), ys.data_ptr())
        torch.cuda.synchronize()
        t_inf = (time.perf_counter() - t0) / 12
        t0 = time.perf_counter()
        for _ in range(3):
            net.train_step(4, xs.data_ptr(), ys.data_ptr(), 1e-4)
        torch.cuda.synchronize()
        t_tr = (time.perf_counter() - t0) / 12
        net.close()
        surrogate = {"network": "FNO 64^3, width 32, 12 modes/axis, 4 Fourier layers, BF16 weights",
                     "infer_ms_per_pair": 1e3 * t_inf, "train_ms_per_pair": 1e3 * t_tr,
                     "tdh_ms_per_pair_this_workload": ms_step / blk}

    # Roofline. Algorithmic unit: one read and one write of every complex value of the propagated
    # block (blk L n_g points, 16 B/point in FP32). Each pass of a TDH step (phases 5, 6, 7, timed by
    # events on the library's stream; two passes on the 80/96 grids, three elsewhere) is one such
    # sweep; the dominant kernel is the pass with the largest share. The whole propagation step
    # (phase 0) is reported against the same per-step figure, so its fraction shows the cost of
    # several sweeps per step.
    peak, src = measured_peaks()
    csize = 8 if prec == B.SBSE_MIXED else 16
    sweep_bytes = blk * pre.n_s * pre.N ** 3 * 2 * csize
    split = pre.N in (80, 96)
    if split:  # two sweeps per step: the kinetic propagator as three one-dimensional operators
        pass_names = {5: "plane kinetic pass k_plane_kin2 (potential phase + x, y kinetic operators)",
                      7: "z kinetic pass k_zkin2_tma (z kinetic operator + induced density; columns "
                         "staged by tensor copies)"}
    else:
        pass_names = {5: "forward plane pass k_plane_fwd (potential phase + x, y FFTs)",
                      6: "z-column pass k_zcol_tma (z FFT, kinetic phase, inverse z FFT)",
                      7: "inverse plane pass k_plane_inv_density_tma (y, x inverse FFTs + density)"}
    passes = {}
    for ph, name in pass_names.items():
        t, nl = phase[ph]
        if nl:
            gbs = sweep_bytes / (t / nl / 1e3) / 1e9
            passes[str(ph)] = {"kernel": name, "avg_us": 1e3 * t / nl, "launches": nl,
                               "achieved": gbs, "frac": gbs / peak, "share_of_step": t / ms_prof}
    dom = max(passes, key=lambda k: passes[k]["share_of_step"]) if passes else None
    traffic, traffic_note = profiled_traffic(dom and int(dom), pre.name, prec == B.SBSE_MIXED, sweep_bytes)
    ms0, n0 = phase[0]
    step_gbs = (sweep_bytes + pre.n_s * pre.N ** 3 * 2 * csize) / (ms0 / n0 / 1e3) / 1e9 if n0 else None
    prof_note = (f"{prof_steps} further benchmark steps with CUDA events around every pass on the "
                 f"library stream (direct launches, {ms_prof / prof_steps:.1f} ms per step vs "
                 f"{ms_step:.1f} ms in the timed region with graph replay)")
    if dom:
        roofline = {"bound": "hbm", "achieved": passes[dom]["achieved"], "peak": peak, "unit": "GB/s",
                    "frac": passes[dom]["frac"], "traffic": traffic, "traffic_source": traffic_note,
                    "kernel": passes[dom]["kernel"], "bytes_per_launch": sweep_bytes,
                    "avg_launch_us": passes[dom]["avg_us"], "share_of_step": passes[dom]["share_of_step"],
                    "peak_source": src, "timing": prof_note, "passes": passes,
                    "step": {"achieved": step_gbs, "frac": step_gbs / peak if step_gbs else None,
                             "share_of_step": ms0 / ms_prof if ms_prof else None}}
    else:
        roofline = {"bound": "hbm", "achieved": step_gbs, "peak": peak, "unit": "GB/s",
                    "frac": step_gbs / peak if step_gbs else None, "traffic": None,
                    "kernel": "propagation step", "peak_source": src, "timing": prof_note}
    line = {
        "metric": metric,
        "value": value, "unit": "W-applications/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if prec == B.SBSE_MIXED else "f64", "data": "synthetic",
        "config": {"workload": workload, "step": step_def,
                   "precision": "mixed: FP32 FFT/propagation, BF16-split tensor-core cleaning and "
                                "contractions, FP64 W accumulator, A, eigensolve"
                                if prec == B.SBSE_MIXED else "fp64",
                   "l2": "inputs larger than L2 (propagated orbitals of one block "
                         f"{blk * pre.n_s * pre.N ** 3 * csize / 1e6:.0f} MB)",
                   "parallelism": f"replicas x{world}"},
        "clocks": clocks,
        "e2e": {"value": world * P / e2e_s, "unit": "W-applications/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h,
                "what": f"whole system per call: pinned host v_loc, orbitals, eps -> all {P} pairs' W "
                        f"-> A -> excitons to the host ({e2e_s:.2f} s per call; the first call, so "
                        f"it includes the capture of the time loop's graph)"} if e2e_s else None,
        "gpu_launches": launches,
        "roofline": roofline,
        "a_build_ms": a_build_ms,
        "absorption": absorption,
        "phase_ms_per_step": {str(k): v[0] / prof_steps for k, v in phase.items()},
        "excitons_ha": [float(x) for x in ev],
        "fp64_gpu_path": fp64,
        "surrogate": surrogate,
        "cpu_baseline": cpu,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
