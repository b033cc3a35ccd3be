"""Benchmark of the z_re(x) path on GB300: one JSON line on rank 0.

A step is one amber_solve (radiation field -> rank -> abundance matching) of
one seeded synthetic 1024^3 realisation (box 1000 h^-1 Mpc, l_mfp 5,
history z_mid 8, dz 4, Az 3), inputs resident in HBM.  Multi-GPU runs are
independent replicas (one realisation per GPU, no collective on the data
path), so value = all ranks' cells / max-over-ranks time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl amber|reference] [--n 1024]

--impl reference times the FP64 CPU oracle (the only other implementation
of the method) on a bounded sample of the same workload.

At one GPU the line also carries "batched" (48 realisations of 128^3 and
256^3 as a loop of plain solves vs one graph of one launch per stage), "serving"
(p50/p99 latency and cells/s of a Poisson request stream at 200 req/s over
128^3/256^3/512^3 grids with cached rank orders) and "library_context"
(cuFFT and CUB timings at the same size); --no-extras skips them.
"""
from __future__ import annotations

import argparse
import hashlib
import re
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "z_re cells/s at 1024^3 (plain vs batched) at oracle tol; serving p50/p99 ms"
HIST = (8.0, 4.0, 3.0)
L_MFP = 5.0


def _workload(n: int, box: float) -> dict:
    return {"workload": f"single instance {n}^3 z_re solve (radiation field, rank, abundance match)",
            "n": n, "cells": n ** 3, "box_mpc_h": box, "l_mfp": L_MFP,
            "history": {"z_mid": HIST[0], "dz": HIST[1], "Az": HIST[2], "n_table": 2000},
            "inputs": "seeded synthetic Gaussian-recipe source and mass fields (realisation r uses seed 1000+r)",
            "l2": "inputs larger than L2 (each field 4 B/cell; 4.3 GB at 1024^3 vs 129 MB L2)",
            "parallelism": "replicas"}


def reduce_max(x: float, dist, device) -> float:
    """Max of a per-rank scalar over all ranks (the slowest rank sets the time)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(cells_per_rank: int, world_size: int, ms_max: float) -> float:
    """Cells per second of the whole job: every rank's cells over the slowest rank's time."""
    return cells_per_rank * world_size / (ms_max / 1e3)


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ---------------------------------------------------------------------------
# Reference arm: the FP64 CPU oracle on bounded samples
# ---------------------------------------------------------------------------

_ORACLE_ARGS = None


def _oracle_init(S, m, box):
    global _ORACLE_ARGS
    _ORACLE_ARGS = (S, m, box)


def _oracle_solve(_):
    from oracle import amber_oracle as O
    S, m, box = _ORACLE_ARGS
    O.solve(S, m, box, L_MFP, *HIST)
    return 1


class OraclePool:
    """The FP64 oracle, as it stands, one realisation per process on every host core.

    Processes are spawned (never forked after CUDA is initialised) and take the
    sample's fields once; numpy's FFT in the oracle is single-threaded, so each
    process is one core."""

    def __init__(self, n_sample: int, box: float, workers: int | None = None):
        import multiprocessing as mp
        from paper_2109_10375_gb300 import synth
        S, m = synth.realisation(n_sample, box, 0)
        self.S, self.m = S.double().numpy(), m.double().numpy()
        self.box, self.ns = box, n_sample
        self.workers = workers or os.cpu_count() or 1
        for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ.setdefault(v, "1")
        self.pool = mp.get_context("spawn").Pool(self.workers, initializer=_oracle_init,
                                                  initargs=(self.S, self.m, self.box))
        self.pool.map(_oracle_solve, range(self.workers))  # start-up and imports, untimed

    def single(self, min_seconds: float, max_reps: int = 50):
        """Cells/s of one process solving one realisation after another."""
        from oracle import amber_oracle as O
        t0 = time.perf_counter()
        reps = 0
        while True:
            O.solve(self.S, self.m, self.box, L_MFP, *HIST)
            reps += 1
            el = time.perf_counter() - t0
            if el >= min_seconds or reps >= max_reps:
                return reps * self.ns ** 3 / el, reps, el

    def parallel(self, tasks: int):
        """Wall time of `tasks` realisations spread over all processes."""
        t0 = time.perf_counter()
        self.pool.map(_oracle_solve, range(tasks), chunksize=1)
        return time.perf_counter() - t0

    def close(self):
        self.pool.close()
        self.pool.join()


def oracle_baseline(n_sample: int, box: float, seconds: float) -> dict:
    """cpu_baseline: all-core oracle throughput on a bounded sample (single-core alongside)."""
    pool = OraclePool(n_sample, box)
    try:
        one, reps1, el1 = pool.single(min(seconds / 3, 5.0))
        per_task = n_sample ** 3 / one
        rounds = max(1, int(round(seconds / per_task)))
        tasks = rounds * pool.workers
        el = pool.parallel(tasks)
    finally:
        pool.close()
    return {"value": tasks * n_sample ** 3 / el, "unit": "cells/s", "cores": pool.workers, "kind": "oracle",
            "sample": f"{tasks} x {n_sample}^3 realisation(s) of the same recipe and cell size on "
                      f"{pool.workers} processes, {el:.1f} s",
            "single_core_value": one,
            "single_core_sample": f"{reps1} x {n_sample}^3 in one process, {el1:.1f} s"}


def oracle_accuracy(S_h, m_h, J, z, n: int, box: float) -> dict:
    """Error of the workload's GPU results (J and z_re of one solve) against
    the FP64 oracle's whole path on the same input fields, every cell: the
    oracle runs as it stands (oracle.solve_large: the steps of oracle.solve on
    all host cores).  Tolerances: intensity relative L2 <= 1e-5 and max
    relative <= 1e-4 (denominator max(|J|, 5e-2 rms J), the FP32 reading);
    z_re off by more than 1e-3 in at most 1e-4 of the cells."""
    import numpy as np
    from oracle import amber_oracle as O
    t0 = time.perf_counter()
    workers = max(1, min(16, os.cpu_count() or 1))
    S64 = S_h.numpy().astype(np.float64)
    m64 = m_h.numpy().astype(np.float64)
    J_o, order_o, z_o = O.solve_large(S64, m64, box, L_MFP, *HIST, workers=workers)
    del S64, m64, order_o
    J_o = J_o.reshape(-1)
    d = J.reshape(-1).astype(np.float64)
    d -= J_o
    rms = float(np.sqrt(np.mean(J_o * J_o)))
    rel_l2 = float(np.linalg.norm(d) / np.linalg.norm(J_o))
    max_abs = float(np.max(np.abs(d)))
    np.abs(d, out=d)
    d /= np.maximum(np.abs(J_o), 5e-2 * rms)
    max_rel = float(d.max())
    del d, J_o
    dz = np.abs(z.reshape(-1).astype(np.float64) - z_o)
    out = {"against": f"FP64 oracle (oracle.solve_large, {workers} host processes) on the same {n}^3 inputs, "
                      "every cell",
           "J_rel_l2": rel_l2, "J_max_rel": max_rel, "J_max_abs_over_rms": max_abs / rms,
           "J_max_rel_denominator": "max(|J_oracle|, 5e-2 rms(J_oracle))",
           "zre_frac_dz_gt_1e-3": float(np.mean(dz > 1e-3)), "zre_max_abs_dz": float(dz.max()),
           "zre_median_abs_dz": float(np.median(dz)),
           "tolerances": {"J_rel_l2": 1e-5, "J_max_rel": 1e-4, "zre_frac_dz_gt_1e-3": 1e-4},
           "host_seconds": time.perf_counter() - t0}
    out["within_tolerance"] = bool(rel_l2 <= 1e-5 and max_rel <= 1e-4 and out["zre_frac_dz_gt_1e-3"] <= 1e-4)
    return out


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    n = args.n
    box = 1000.0 * n / 1024
    ns = args.cpu_sample_n
    box_s = box * ns / n  # same cell size as the workload
    pool = OraclePool(ns, box_s)
    try:
        # a step: one realisation of the sample per host core, all at once
        for _ in range(args.warmup):
            pool.parallel(pool.workers)
        el = 0.0
        for _ in range(args.steps):
            el += pool.parallel(pool.workers)
    finally:
        pool.close()
    value = args.steps * pool.workers * ns ** 3 / el
    sample = (f"{pool.workers} x {ns}^3 realisations per step (same recipe and cell size), one per process, "
              f"{args.steps} steps")
    line = {"metric": METRIC, "value": value, "unit": "cells/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": _workload(n, box), "impl": "reference",
            "cpu_baseline": {"value": value, "unit": "cells/s", "cores": pool.workers, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "cells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# Clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        # the raw samples go to $AMBER_CLOCKS_DIR (default: the system's
        # temporary directory); their summary is part of the JSON line
        d = os.environ.get("AMBER_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(d, f"clocks_rank{gpu_index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": 0}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# Roofline bookkeeping: algorithmic bytes per launch of each kernel
# ---------------------------------------------------------------------------

def model_bytes(n: int, sort_passes: int) -> dict:
    """Algorithmic HBM bytes per step of each kernel kind, on the scope table's
    byte model ("model A"): every FFT pass reads and writes 4 B/cell (the half
    spectrum counted as 4 B/cell), the histogram reads 4, the digit passes move
    12 (first: key in, key + index out), 16 (middle) and 12 (last: no key out)
    B/cell, and the matching reads the order and the rank-order masses (4 + 4)
    and writes z (4).  112 B/cell for four 8-bit passes, 96 for three."""
    C = n ** 3
    sort = (12 + 16 * (sort_passes - 2) + 12) * C if sort_passes >= 2 else 8 * C
    return {"fft_r2c_x": 8 * C, "fft_y_fwd": 8 * C, "fft_z_conv": 8 * C, "fft_y_inv": 8 * C, "fft_c2r_x": 8 * C,
            "sort_histogram": 4 * C, "sort_pass": sort, "scan_assign": 8 * C, "scatter_back": 4 * C,
            "mass_reduce": 0, "thresholds": 0}


def design_bytes(n: int, sort_passes: int) -> dict:
    """Algorithmic bytes per step of each kernel as this design moves them:
    the half spectrum at its true size, the mass riding through the sort as a
    second payload (+8 B/cell per pass), and the scan's (cell, z) pairs
    written and read back by the scatter to cell order."""
    C = n ** 3
    H = 8 * n * n * (n // 2 + 1)  # half spectrum, complex64
    if sort_passes == 1:
        sort = 16 * C                       # J 4 + mass 4 in, order 4 + mass 4 out
    else:
        sort = (20 + 24 * (sort_passes - 2) + 20) * C  # first / middle / last pass
    return {
        "fft_r2c_x": 4 * C + H, "fft_y_fwd": 2 * H, "fft_z_conv": 2 * H, "fft_y_inv": 2 * H,
        "fft_c2r_x": H + 4 * C,
        "sort_histogram": 4 * C,            # digit histograms (the key range comes with the inverse x pass)
        "sort_pass": sort,
        "mass_reduce": 4 * C, "thresholds": 0, "scan_assign": 16 * C, "scatter_back": 12 * C,
    }


# The translation unit that holds each kernel kind; its hash covers that unit
# and every csrc/ header it includes, directly or not.
_KERNEL_SOURCES = {"fft": "fft_f32.cu", "sort": "sort.cu", "scan_assign": "assign.cu", "scatter_back": "assign.cu",
                   "thresholds": "assign.cu", "mass_reduce": "assign.cu"}


def _src_hash(kernel: str = None, read=None) -> str:
    """Hash of the sources a kernel kind is built from: its translation unit
    and the csrc/ headers it includes (all sources when no kernel is named).
    read(name) returns a file's bytes (default: the working tree)."""
    d = os.path.join(ROOT, "paper_2109_10375_gb300", "csrc")
    read = read or (lambda f: open(os.path.join(d, f), "rb").read())
    names = sorted(os.listdir(d))
    if kernel is not None:
        unit = _KERNEL_SOURCES.get(kernel.split("_")[0], _KERNEL_SOURCES.get(kernel))
        todo, seen = [unit], set()
        while todo:
            f = todo.pop()
            if f in seen or f not in names:
                continue
            seen.add(f)
            todo += re.findall(rb'#include\s+"([^"]+)"', read(f))
            todo = [t.decode() if isinstance(t, bytes) else t for t in todo]
        names = sorted(seen)
    h = hashlib.sha256()
    for f in names:
        h.update(read(f))
    return h.hexdigest()[:16]


def _traffic(kernel: str, n: int):
    """DRAM bytes per launch from the committed ncu summary, if it matches the sources."""
    p = os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        d = json.load(open(p))
    except Exception:
        return None
    k = d.get("kernels", {}).get(kernel)
    if not k or k.get("src_hash") != _src_hash(kernel):
        return None
    return k["bytes_per_launch"] * (n ** 3) / k["cells"]


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0}, "fallback"


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def run_amber(args):
    import torch
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2109_10375_gb300 import binding as B, synth

    n = args.n
    box = 1000.0 * n / 1024
    C = n ** 3
    S, m = synth.realisation(n, box, rank, device="cuda")
    # pinned host buffers of the end-to-end measurement, taken while host
    # memory is fresh (filled from S and m here, read back near the end)
    S_h = torch.empty(S.shape, dtype=torch.float32, pin_memory=True)
    m_h = torch.empty(S.shape, dtype=torch.float32, pin_memory=True)
    z_h = [torch.empty(S.shape, dtype=torch.float32, pin_memory=True) for _ in range(2)]
    S_h.copy_(S)
    m_h.copy_(m)
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    h = B.history(*HIST)
    ctx = B.Context(C, device=local)
    if args.fuse_histogram is not None:
        ctx.set_tuning(n, fuse_histogram=args.fuse_histogram)
    if args.zpass_tma is not None:
        ctx.set_tuning(n, zpass_tma=args.zpass_tma)
    z = torch.empty_like(S)
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        ctx.solve(S, m, box, L_MFP, h, out=z)
    st = ctx.sync_status()
    if st != 0:
        raise RuntimeError(f"device status after warm-up: {B.status_string(st)}")

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # --- device-resident timed region (kernel timing events on the same stream)
    ctx.profile(True)
    ctx.profile_reset()
    clk = ClockSampler(local)
    clk.start()
    time.sleep(0.3)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        ctx.solve(S, m, box, L_MFP, h, out=z)
    e1.record(stream)
    barrier()
    clocks = clk.stop()
    ms = e0.elapsed_time(e1) / args.steps
    prof = ctx.profile_read()
    ctx.profile(False)
    passes = ctx.sort_passes()  # digit passes of the timed solves' ranking
    tuning = ctx.get_tuning(n)  # the choices the timed solves ran with
    st = ctx.sync_status()
    if st != 0:
        raise RuntimeError(f"device status after timed region: {B.status_string(st)}")
    ms_max = reduce_max(ms, dist, "cuda")

    # --- the other weightings of the matched fraction (same step, same inputs)
    weightings = {}
    if rank == 0 and ws == 1 and not args.no_extras:
        for name, wgt in (("mass_growth", B.AMBER_WEIGHT_MASS_GROWTH), ("volume", B.AMBER_WEIGHT_VOLUME)):
            hw = B.history(*HIST, weighting=wgt)
            for _ in range(2):
                ctx.solve(S, m, box, L_MFP, hw, out=z)
            ctx.profile(True)
            ctx.profile_reset()
            reps = 3
            e0.record(stream)
            for _ in range(reps):
                ctx.solve(S, m, box, L_MFP, hw, out=z)
            e1.record(stream)
            torch.cuda.synchronize()
            pw = ctx.profile_read()
            ctx.profile(False)
            st = ctx.sync_status()
            if st != 0:
                raise RuntimeError(f"device status ({name}): {B.status_string(st)}")
            wms = e0.elapsed_time(e1) / reps
            weightings[name] = {"ms_per_step": wms, "cells_per_s": C / (wms / 1e3),
                                "scan_assign_ms": pw["scan_assign"][0] / reps,
                                "thresholds_ms": pw["thresholds"][0] / reps}

    # --- tomographic matching: three redshift intervals, each with its own
    # source field (here the workload's source and two drifted copies)
    tomographic = {}
    if rank == 0 and ws == 1 and not args.no_extras:
        S1 = (0.7 * S + 0.3 * torch.roll(S, 7, dims=0)).contiguous()
        S2 = (0.4 * S + 0.6 * torch.roll(S, 7, dims=0)).contiguous()
        zt = torch.empty_like(S)
        bounds = [20.0, 8.6, 7.2, 5.0]
        ctx.solve_tomographic([S, S1, S2], bounds, m, box, L_MFP, h, out=zt)
        torch.cuda.synchronize()
        e0.record(stream)
        ctx.solve_tomographic([S, S1, S2], bounds, m, box, L_MFP, h, out=zt)
        e1.record(stream)
        torch.cuda.synchronize()
        st = ctx.sync_status()
        if st != 0:
            raise RuntimeError(f"device status (tomographic): {B.status_string(st)}")
        tms = e0.elapsed_time(e1)
        tomographic = {"intervals": len(bounds) - 1, "bounds": bounds, "ms": tms, "cells_per_s": C / (tms / 1e3)}
        del S1, S2, zt
        torch.cuda.empty_cache()

    # --- analysis of the z_re fields (Sec. 2.3) at the workload's size: the
    # plain and growth-rescaled fields' normalised forms, their auto and cross
    # shell spectra, and the PDF of their fractional difference
    analysis = {}
    if rank == 0 and ws == 1 and not args.no_extras:
        za, zb = torch.empty_like(S), torch.empty_like(S)
        ctx.solve(S, m, box, L_MFP, h, out=za)
        ctx.solve(S, m, box, L_MFP, B.history(*HIST, weighting=B.AMBER_WEIGHT_MASS_GROWTH), out=zb)
        da, _ = ctx.delta_z(za)
        db, _ = ctx.delta_z(zb)
        ps = ctx.power_spectrum(da, db, box)
        ctx.epsilon_z_pdf(zb, za, -0.05, 0.05, 200)
        torch.cuda.synchronize()

        def timed(fn, reps=3):
            e0.record(stream)
            for _ in range(reps):
                fn()
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / reps

        analysis = {"what": f"{n}^3 z_re fields, plain and growth-rescaled weighting",
                    "delta_z_ms": timed(lambda: ctx.delta_z(za, out=da)),
                    "power_spectrum_cross_ms": timed(lambda: ctx.power_spectrum(da, db, box)),
                    "power_spectrum_auto_ms": timed(lambda: ctx.power_spectrum(da, None, box)),
                    "epsilon_pdf_ms": timed(lambda: ctx.epsilon_z_pdf(zb, za, -0.05, 0.05, 200)),
                    "shells": int(ps["modes"].numel())}
        st = ctx.sync_status()
        if st != 0:
            raise RuntimeError(f"device status (analysis): {B.status_string(st)}")
        del za, zb, da, db, ps

    # --- the source-field pipeline that makes S and the mass field (Sec. 3.2,
    # 3.3): 2LPT displacements of one particle per cell from a linear field,
    # TSC matter density and ESF-L halo density (CIC), both interlaced
    source_pipeline = {}
    if rank == 0 and ws == 1 and not args.no_extras:
        d_lin = synth.gaussian_density(n, box, 2000, sigma=1.0, device="cuda").float()
        D1 = 0.25  # linear field scaled to sigma 0.25 at the target redshift
        D2 = -3.0 / 7.0 * D1 ** 2
        psi = ctx.lpt_displacement(d_lin, box, D1, D2)
        rho_m = ctx.mesh_density(psi, box, 3, True)
        f = ctx.esf_fcoll(d_lin, box, 2.0 * box / n, 1.686 / D1, 1.0)
        rho_h = ctx.mesh_density(psi, box, 2, True, mass=f)
        torch.cuda.synchronize()

        def once(fn):
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1)

        source_pipeline = {
            "what": f"{n}^3 particles and mesh; linear field sigma 1 scaled by D1 = {D1}",
            "lpt_2nd_order_ms": once(lambda: ctx.lpt_displacement(d_lin, box, D1, D2)),
            "tsc_interlaced_ms": once(lambda: ctx.mesh_density(psi, box, 3, True, out=rho_m)),
            "esf_fcoll_sharpk_ms": once(lambda: ctx.esf_fcoll(d_lin, box, 2.0 * box / n, 1.686 / D1, 1.0, out=f)),
            "cic_interlaced_weighted_ms": once(lambda: ctx.mesh_density(psi, box, 2, True, mass=f, out=rho_h)),
            "rho_m_mean": float(rho_m.double().mean()), "rho_h_mean": float(rho_h.double().mean())}
        st = ctx.sync_status()
        if st != 0:
            raise RuntimeError(f"device status (source pipeline): {B.status_string(st)}")
        del d_lin, psi, rho_m, f, rho_h
        torch.cuda.empty_cache()

    # the workload's intensity and z_re, kept on the host for the comparison
    # with the oracle (the cpu_baseline leg, after every GPU measurement)
    J_keep = z_keep = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline and not args.no_accuracy:
        Jbuf = torch.empty_like(S)
        ctx.solve(S, m, box, L_MFP, h, out=z, J_out=Jbuf)
        st = ctx.sync_status()
        if st != 0:
            raise RuntimeError(f"device status (accuracy solve): {B.status_string(st)}")
        J_keep, z_keep = Jbuf.cpu().numpy(), z.cpu().numpy()
        del Jbuf

    # --- end to end through the C ABI with host buffers: amber_solve_host
    # copies the step's inputs in from pinned host memory, solves and copies
    # z_re out, all on its stream.  Each call runs its copies and its solve in
    # order, so the contexts take turns on their own streams: while one
    # solves, the others copy.
    del S, m
    torch.cuda.empty_cache()
    ctxs2 = [ctx] + [B.Context(C, device=local) for _ in range(args.e2e_contexts - 1)]
    for cx in ctxs2[1:]:
        if args.fuse_histogram is not None:
            cx.set_tuning(n, fuse_histogram=args.fuse_histogram)
        if args.zpass_tma is not None:
            cx.set_tuning(n, zpass_tma=args.zpass_tma)
    streams = [torch.cuda.Stream() for _ in ctxs2]
    z_h = z_h + [torch.empty(z.shape, dtype=torch.float32, pin_memory=True) for _ in range(len(ctxs2) - len(z_h))]
    e_steps = max(2, args.steps)  # the same K as the device-timed steps

    def pipeline(steps):
        """steps host-to-host solves alternating over the two contexts; ms per step"""
        barrier()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for st_ in streams:
            st_.wait_event(f0)
        for i in range(steps):
            b = i % len(ctxs2)
            ctxs2[b].solve_host(S_h, m_h, box, L_MFP, h, z_h[b], stream=streams[b])
        for st_ in streams:
            ev = torch.cuda.Event()
            ev.record(st_)
            stream.wait_event(ev)
        f1.record(stream)
        barrier()
        return f0.elapsed_time(f1) / steps

    pipeline(len(ctxs2))  # warm-up: every context's first use
    # three timed trials; the median one is reported (the host side of the
    # copies is shared with the rest of the machine)
    trials = [pipeline(e_steps) for _ in range(3)]
    e2e_ms = sorted(trials)[1]
    e2e_ms = reduce_max(e2e_ms, dist, "cuda")
    # the copies alone, for context
    S_d, z_d = torch.empty(z.shape, device="cuda"), torch.empty(z.shape, device="cuda")
    c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    c0.record(stream)
    S_d.copy_(S_h, non_blocking=True)
    S_d.copy_(m_h, non_blocking=True)
    c1.record(stream)
    torch.cuda.synchronize()
    h2d_gbps = 8 * C / (c0.elapsed_time(c1) / 1e3) / 1e9
    c0.record(stream)
    z_h[0].copy_(z_d, non_blocking=True)
    c1.record(stream)
    torch.cuda.synchronize()
    d2h_gbps = 4 * C / (c0.elapsed_time(c1) / 1e3) / 1e9
    del S_d, z_d
    for cx in ctxs2:
        st = cx.sync_status()
        if st != 0:
            raise RuntimeError(f"device status after end-to-end steps: {B.status_string(st)}")
    for cx in ctxs2[1:]:
        cx.close()
    # the autotuner needs device copies of the workload's fields
    S_d = [torch.empty(z.shape, device="cuda")]
    m_d = [torch.empty(z.shape, device="cuda")]
    S_d[0].copy_(S_h)
    m_d[0].copy_(m_h)
    # the autotuner's measurement of this workload (after the timed steps,
    # which ran the default choices)
    tune = None
    if rank == 0 and ws == 1 and not args.no_extras:
        tune = ctx.autotune(S_d[0], m_d[0], box, L_MFP)
        st = ctx.sync_status()
        if st != 0:
            raise RuntimeError(f"device status after autotuning: {B.status_string(st)}")
    del S_d, m_d, z_h

    # each timed bracket is one kernel launch, except the histogram's, which
    # also holds the one-CTA digit-offset scan (k_sort_offsets) -- alone when
    # the inverse x pass counted the digits
    fused = bool(tuning.get("fuse_histogram")) and tuning["sort_digit_bits"] == 8
    launches_per_step = (sum(v[1] for v in prof.values()) + (0 if fused else prof["sort_histogram"][1])) / args.steps
    mb, db = model_bytes(n, passes), design_bytes(n, passes)
    kernels = {}
    for k, (ms_k, cnt) in prof.items():
        if cnt == 0:
            continue
        ms_step = ms_k / args.steps
        kernels[k] = {"ms_per_step": ms_step, "launches_per_step": cnt / args.steps,
                      "model_bytes_per_step": mb.get(k, 0), "design_bytes_per_step": db.get(k, 0),
                      "GBps_model": (mb.get(k, 0) / (ms_step / 1e3) / 1e9) if ms_step > 0 else None,
                      "GBps_design": (db.get(k, 0) / (ms_step / 1e3) / 1e9) if ms_step > 0 else None}
    dom = max(kernels, key=lambda k: kernels[k]["ms_per_step"])
    peaks, src = _peaks()
    peak = peaks["hbm_gbs"]
    achieved = kernels[dom]["GBps_model"]
    path_model = sum(mb.get(k, 0) for k in kernels)
    path_design = sum(db.get(k, 0) for k in kernels)
    cpu, accuracy = None, None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        ns = args.cpu_sample_n
        cpu = oracle_baseline(ns, box * ns / n, args.cpu_seconds)
        if not args.no_accuracy:
            accuracy = oracle_accuracy(S_h, m_h, J_keep, z_keep, n, box)
    del J_keep, z_keep, S_h, m_h

    extras = {}
    if tune is not None:
        extras["autotune"] = tune
    if rank == 0 and ws == 1 and not args.no_extras:
        ctx.close()
        torch.cuda.empty_cache()
        extras["batched"] = run_batched(B, synth, torch)
        torch.cuda.empty_cache()
        extras["serving"] = run_serving(torch)
        torch.cuda.empty_cache()
        extras["library_context"] = run_library_context(torch, synth, n, box)

    if rank == 0:
        line = {"metric": METRIC, "value": whole_job_rate(C, ws, ms_max), "unit": "cells/s", "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": _workload(n, box),
                "e2e": {"value": whole_job_rate(C, ws, e2e_ms), "unit": "cells/s", "h2d_bytes_per_step": 8 * C,
                        "d2h_bytes_per_step": 4 * C, "ms_per_step": e2e_ms, "steps": e_steps,
                        "call": "amber_solve_host (pinned host buffers in and out, copies on the call's stream)",
                        "overlap": f"{len(ctxs2)} contexts take turns on their own streams: while one solves, "
                                   "the others copy",
                        "h2d_GBps_alone": h2d_gbps, "d2h_GBps_alone": d2h_gbps,
                        "trials_ms": trials, "reported": "median of 3 timed trials"},
                "gpu_launches": int(round(launches_per_step * args.steps)),
                "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                             "unit": "GB/s", "frac": achieved / peak, "traffic": _traffic(dom, n),
                             "peak_source": src, "peak_kind": "measured copy bandwidth (burst)",
                             "bytes_model": "scope-table model A (sort 12+16+..+12 B/cell per pass set)",
                             "model_bytes_per_launch": mb[dom] / max(1, kernels[dom]["launches_per_step"]),
                             "launch_ms": kernels[dom]["ms_per_step"] / max(1, kernels[dom]["launches_per_step"]),
                             "path_bytes_per_cell": path_model / C,
                             "path_frac": (path_model / (ms_max / 1e3) / 1e9) / peak,
                             "design_bytes_per_cell": {"kernel": db[dom] / C, "path": path_design / C},
                             "design_frac": {"kernel": kernels[dom]["GBps_design"] / peak,
                                             "path": (path_design / (ms_max / 1e3) / 1e9) / peak},
                             "sort_passes": passes},
                "kernels": kernels,
                "tuning": {k: tuning[k] for k in ("fft_variant", "sort_digit_bits", "sort_match", "fuse_histogram",
                                                 "zpass_tma")},
                "clocks": clocks,
                "cpu_baseline": cpu}
        if accuracy is not None:
            line["accuracy"] = accuracy
        if weightings:
            line["weightings"] = weightings
        if tomographic:
            line["tomographic"] = tomographic
        if analysis:
            line["analysis"] = analysis
        if source_pipeline:
            line["source_pipeline"] = source_pipeline
        line.update(extras)
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_batched(B, synth, torch, reps: int = 3):
    """48 realisations (32 x 128^3, 16 x 256^3): a loop of plain solves vs one graph launch."""
    g = __import__("numpy").random.default_rng(2024)
    specs = [(128, 100.0)] * 32 + [(256, 200.0)] * 16
    items = []
    for r, (n, box) in enumerate(specs):
        S, m = synth.realisation(n, box, r, device="cuda")
        hist = (float(g.uniform(6.5, 9.0)), float(g.uniform(2.0, 6.0)), float(g.uniform(1.5, 5.0)))
        items.append((S, m, box, float(g.uniform(1.0, 20.0)), B.history(*hist), torch.empty_like(S)))
    cells = sum(it[0].numel() for it in items)
    ctxs = [B.Context(256 ** 3)]
    stream = torch.cuda.current_stream()
    # the autotuner picks each size's FFT variant, digit width and digit-peer
    # method on that size's first realisation; plain loop and batch then
    # share the choices (the batch finds the sizes tuned)
    tuning = {}
    for n_t in (128, 256):
        it = next(x for x in items if x[0].shape[0] == n_t)
        t = ctxs[0].autotune(it[0], it[1], it[2], it[3])
        for c in ctxs[1:]:
            c.set_tuning(n_t, t["fft_variant"], t["sort_digit_bits"], t["sort_match"])
        tuning[str(n_t)] = t
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # plain: the single-instance path, one call after another
    for it in items:
        ctxs[0].solve(*it[:5], out=it[5])
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        for it in items:
            ctxs[0].solve(*it[:5], out=it[5])
    e1.record(stream)
    torch.cuda.synchronize()
    plain_ms = e0.elapsed_time(e1) / reps
    batch = B.Batch(ctxs, items)
    nodes = batch.kernel_nodes()
    batch.launch()
    torch.cuda.synchronize()
    e0.record(stream)
    # an NVTX range over the timed replays lets a profiler capture just them
    torch.cuda.nvtx.range_push("batch_replay")
    for _ in range(reps):
        batch.launch()
    torch.cuda.nvtx.range_pop()
    e1.record(stream)
    torch.cuda.synchronize()
    graph_ms = e0.elapsed_time(e1) / reps
    st = max(c.sync_status() for c in ctxs)
    batch.close()
    for c in ctxs:
        c.close()
    return {"workload": "48 realisations: 32 x 128^3 (box 100) + 16 x 256^3 (box 200), l_mfp U[1,20], "
                        "z_mid U[6.5,9], dz U[2,6], Az U[1.5,5]",
            "cells": cells, "tuning": tuning, "plain_loop_ms": plain_ms,
            "plain_loop_cells_per_s": cells / (plain_ms / 1e3),
            "graph_ms": graph_ms, "graph_cells_per_s": cells / (graph_ms / 1e3), "speedup": plain_ms / graph_ms,
            "form": "one launch per stage over all 48 items (per grid size for the transforms, per digit width "
                    "for the sort), captured once",
            "graph_kernel_nodes": nodes, "status": st}


def run_serving(torch, n_requests: int = 800, rate: float = 200.0):
    """Poisson request stream over mixed grids with a cache of rank orders."""
    from paper_2109_10375_gb300 import serve
    reqs = serve.poisson_requests(n_requests, rate=rate, seed=7)
    srv = serve.Server(n_slots=6, max_n=512, cache_bytes=40e9)
    srv.prepare(reqs)
    warm = serve.poisson_requests(60, rate=rate, seed=8)  # untimed: first launches, allocator
    srv.run(warm, realtime=True)
    srv.run(reqs, realtime=True)
    out = serve.summarize(reqs)
    out.update({"rate_per_s": rate, "mix": {"128^3": 0.6, "256^3": 0.3, "512^3": 0.1}, "realisations": 20,
                "history_only_fraction": 0.7, "slots": len(srv.slots),
                "cache": "rank order per (realisation, grid, l_mfp, delta_c); transformed source per "
                         "(realisation, grid, delta_c)",
                "waits_for_hbm": srv.waiting_hbm, "evictions": srv.evictions})
    srv.close()
    return out


def run_library_context(torch, synth, n: int, box: float, reps: int = 3):
    """Library routines at the workload's size, for context only (not on the path):
    cuFFT R2C + C2R through torch.fft, and torch.sort (CUB radix sort) of the
    intensity with its int64 permutation."""
    S, _ = synth.realisation(n, box, 0, device="cuda")
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    fft_ms = timed(lambda: torch.fft.irfftn(torch.fft.rfftn(S), s=S.shape))
    torch.cuda.empty_cache()
    sort_ms = timed(lambda: torch.sort(S.view(-1), descending=True, stable=True))
    torch.cuda.empty_cache()
    # the store pattern of the scatter back to cell order: every cell written
    # once, in random order within windows of 2^23 consecutive cells taken one
    # after another (torch's scatter_, one 4-byte store per element)
    C = n ** 3
    W = min(1 << 23, C)
    g = torch.Generator(device="cuda")
    g.manual_seed(11)
    idx = torch.empty(C, dtype=torch.int64, device="cuda")
    for w0 in range(0, C, W):
        idx[w0:w0 + W] = torch.randperm(W, device="cuda", generator=g) + w0
    src = S.view(-1)
    dst = torch.empty_like(src)
    store_ms = timed(lambda: dst.scatter_(0, idx, src))
    del S, idx, src, dst
    torch.cuda.empty_cache()
    return {"what": f"library routines at {n}^3 for context (not on the path)",
            "cufft_rfftn_irfftn_ms": fft_ms, "torch_sort_stable_ms": sort_ms,
            "random_store": {"ms": store_ms, "stores_per_s": C / (store_ms / 1e3),
                             "pattern": "torch scatter_ of every cell once, random within 2^23-cell windows"}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="amber", choices=["amber", "reference"])
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--cpu-sample-n", type=int, default=128)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fuse-histogram", type=int, choices=[0, 1], default=None,
                    help="override the size's choice of digit counts in the inverse x pass (8-bit digits)")
    ap.add_argument("--zpass-tma", type=int, choices=[0, 1], default=None,
                    help="override the size's choice of the TMA-staged z pass")
    ap.add_argument("--e2e-contexts", type=int, default=3,
                    help="contexts (each with its own stream) the end-to-end steps rotate over")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the oracle comparison of the workload's J and z_re (minutes of host time)")
    ap.add_argument("--no-extras", action="store_true", help="skip the batched and serving measurements")
    ap.add_argument("--batched-only", action="store_true",
                    help="run only the batched measurement (48 realisations) and print it as one JSON line")
    args = ap.parse_args()
    if args.batched_only:
        import torch
        from paper_2109_10375_gb300 import binding as B, synth
        print(json.dumps({"batched": run_batched(B, synth, torch)}))
        return 0
    if args.warmup < 3 and args.impl == "amber":
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_amber(args)


if __name__ == "__main__":
    sys.exit(main())
