#!/usr/bin/env python
"""Benchmark of the GB300 PIC step: particle-steps per second, Picard iterations included,
mixed precision against FP64 at the stated energy drift, with the rooflines of the particle
kernels.

Default workload (the large two-stream configuration): the 3D periodic two-stream problem
on a 128^3 mesh with 134,217,728 electrons (32 per beam per cell), beams +-0.2 c, thermal
spread 1e-4, dt = 0.1, Picard tolerance 1e-13, split-orbit closed-form weights.  One step is
one full implicit time step: every Picard iteration of Algorithm 1 plus the final
consistency sweep, with the cell sort, the orbit-current scatters, the continuity +
Crank--Nicolson mesh solves and the orbit pushes.  The headline is the mixed path (FP32
Picard iterations, FP64 refinement to mixed_tol64 and the FP64 final sweep); the FP64 path
runs on the same input beside it.  Synthetic, seeded inputs (pic_inputs).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload NAME] [--precision mixed|fp64] [--probe-peaks]

Multi-GPU runs (torchrun, one rank per GPU) are independent replicas with distinct
seeds: the method is not sharded, so there is no data-path collective; only the timing
barrier and the max-over-ranks reduction touch the process group.
--impl reference times the FP64 CPU oracle (the reference arm of this benchmark) on a
bounded sample of the same workload, on all host cores (one independent sample per core).
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "twostream-128c-134M"
METRIC = "particle-steps/s incl. Picard iters, mixed vs FP64 at stated energy drift; %HBM"
UNIT = "particle-steps/s"
MIXED_TOL64 = 1e-9        # FP64 refinement tolerance of the mixed path (energy error is second order in it)
# FP64 ALU peak of the GB300: 152 SMs x 2 FP64 FMA (4 flop) per clock per SM x 2070 MHz (the
# recipe's SM count and maximum clock; pic_probe_fma_rates measures the per-SM rate live).
FP64_PEAK_TFLOPS = 152 * 4 * 2.070e9 / 1e12
HBM_FALLBACK_GBS = 6800.0
SUB_CELLS = 16            # the CPU oracle's sample: a periodic sub-box of SUB_CELLS^3 cells
CPU_STEPS = 10            # timed oracle steps of the cpu_baseline leg

# Algorithmic FP64 flops (add, mul = 1, FMA = 2; the scatter's atomic adds counted) of the
# fused push + next-orbit scatter kernel, counted from the kernel source per particle and per
# knot-free orbit piece:
FLOPS_PER_PARTICLE = 190
FLOPS_PER_PUSH_PIECE = 409
FLOPS_PER_SCATTER_PIECE = 150
# The survey's lower estimate of the same work (its per-orbit count split into a per-particle part
# and a per-piece part: weights 110, grad phi 24, A^(m) and C 72, contraction 48, transverse 72,
# D sum 48 and scatter 24 per piece; point gather 36, push and orbit 30, next-orbit weights 20 per
# particle), reported beside the source count so that both fractions are visible.
MIN_FLOPS_PER_PARTICLE = 86
MIN_FLOPS_PER_PIECE = 398
# Bytes per particle-iteration of the FP32 push (read cell 4, offset 12, v^n 12, increment 12;
# write the new increment 12).
BYTES32_PER_PARTICLE = 52
# DRAM bytes (read + write) per launch from one ncu capture of the kernel version in the tree,
# keyed by kernel and workload, with how the figure was obtained (absent: not captured for this
# version).  The 128^3 run is too large for a multi-pass capture, so its k_push figure is the
# 32^3 capture (2,097,152 particles, third Picard iteration) scaled by the particle count: the
# kernel's traffic is its particle streams, 141.7 B per particle-iteration there.
NCU_TRAFFIC = {
    ("k_push", "twostream-32c-2M"): (297.07e6, "ncu capture, one launch (dram read 259.32 MB + write 37.75 MB)"),
    ("k_push", "twostream-128c-134M"): (297.07e6 * 64, "the 32^3 capture scaled by particles (x 64)"),
    ("k_push32", "twostream-32c-2M"): (96.43e6, "ncu capture, one launch (dram read 86.57 MB + write 9.86 MB)"),
    ("k_push32", "twostream-128c-134M"): (96.43e6 * 64, "the 32^3 capture scaled by particles (x 64)"),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--mixed-tol64", type=float, default=MIXED_TOL64)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-other", action="store_true", help="skip the other precision's run")
    ap.add_argument("--no-mixed", action="store_true", help="alias of --no-other")
    ap.add_argument("--deterministic", action="store_true", help="bitwise reproducible mode")
    ap.add_argument("--ops", default="central2", choices=["central2", "spectral"],
                    help="spatial operators: central differences or the paper's spectral operators (FFT)")
    ap.add_argument("--shape-order", type=int, default=1, choices=[1, 2, 3],
                    help="B-spline degree r; r > 1 runs the split Gauss rule with 2 nq - 1 >= 3 r (FP64)")
    ap.add_argument("--probe-peaks", action="store_true", help="print the measured FMA rates and exit")
    return ap.parse_args()


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(value, pg, device):
    """The largest of one float over all ranks (the whole job's time is its slowest rank's), or
    the value itself in a single-process run.  ``pg`` is torch.distributed (NCCL on the GPU
    box, gloo in the CPU tests); ``device`` holds the reduction tensor."""
    if pg is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, count, seconds):
    """Whole-job throughput: the units all ranks processed, divided by the slowest rank's time."""
    return units_per_rank * world * count / seconds


def measured_peaks():
    """HBM GB/s from the generated MEASURED_PEAKS.json, else the recipe's fallback."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "of measured (MEASURED_PEAKS.json hbm_gbs)"
    except Exception:
        return HBM_FALLBACK_GBS, "of fallback (6.8 TB/s)"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.path = tempfile.mktemp(suffix=".csv")
        self.dev = device_index
        self.proc = None

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.dev), "-lms", "200"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---- the CPU oracle on a bounded sample (cpu_baseline and the reference arm) ------------------

def oracle_sample(w, run=0):
    """A bounded sample of workload ``w`` for the CPU oracle: a periodic sub-box of SUB_CELLS^3
    cells with the workload's cell size (the whole mesh when it is that small), one particle per
    beam per cell, the workload's beam speed, thermal spread, perturbation amplitude, dt and
    Picard tolerance.  The oracle's cost per particle-step is that of the full workload: it is
    dominated by the particle work (the mesh solve of 16^3 nodes is a few percent of it)."""
    import pic_inputs as pi
    sub = tuple(min(SUB_CELLS, a) for a in w.n)
    Ls = tuple(w.L[a] * sub[a] / w.n[a] for a in range(3))
    x, v, q, m = pi.random_twostream(sub, Ls, 1, w.v0, w.eps, w.vth, w.seed + 50 + run)
    return sub, Ls, x, v, q, m


def sample_text(w):
    sub = tuple(min(SUB_CELLS, a) for a in w.n)
    npart = 2 * sub[0] * sub[1] * sub[2]
    return (f"{npart} particles in a periodic {sub[0]}x{sub[1]}x{sub[2]}-cell sub-box with the {w.name} cell size "
            f"(1 per beam per cell; same beams, spread, dt, tau)")


def time_oracle(name, steps, warmup, run=0):
    """Oracle particle-steps/s over `steps` timed steps (after `warmup`) of one sample, one thread."""
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    import pic_inputs as pi
    from oracle import pic as opic
    w = pi.WORKLOADS[name]
    n, Ls, x, v, q, m = oracle_sample(w, run)
    cfg = opic.Config(n=n, L=Ls, dt=w.dt, picard_tol=w.picard_tol, picard_max=w.picard_max)
    st = opic.init(x, v, q, m, cfg)
    for _ in range(warmup):
        st, info = opic.step(st, cfg)
    t0 = time.perf_counter()
    iters = 0
    for _ in range(steps):
        st, info = opic.step(st, cfg)
        iters += info["iterations"]
    secs = time.perf_counter() - t0
    return {"particles": int(x.shape[0]), "steps": steps, "secs": secs, "iterations": iters}


def _oracle_worker(name, steps, warmup, run, queue):
    queue.put(time_oracle(name, steps, warmup, run))


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def time_oracle_all_cores(name, steps, warmup):
    """One independent oracle sample per host core (spawned processes, one numpy thread each),
    all at once: throughput = all particle-steps over the slowest process's timed region."""
    import multiprocessing as mp
    cores = host_cores()
    os.environ["OMP_NUM_THREADS"] = "1"
    ctx = mp.get_context("spawn")
    queue = ctx.Queue()
    procs = [ctx.Process(target=_oracle_worker, args=(name, steps, warmup, r, queue)) for r in range(cores)]
    for p in procs:
        p.start()
    res = [queue.get() for _ in procs]
    for p in procs:
        p.join()
    secs = max(r["secs"] for r in res)
    units = sum(r["particles"] * r["steps"] for r in res)
    iters = sum(r["iterations"] for r in res) / max(sum(r["steps"] for r in res), 1)
    return units / secs, secs, iters, cores


def run_reference(args, world, rank):
    """The reference arm: the FP64 oracle as it stands on all host cores, K timed steps of one
    bounded sample per core after W warm-up steps (rank 0 only)."""
    import pic_inputs as pi
    if rank != 0:
        return
    w = pi.WORKLOADS[args.workload]
    value, secs, mean_it, cores = time_oracle_all_cores(w.name, args.steps, args.warmup)
    sample = (f"per core: {sample_text(w)}; {cores} independent samples at once (one process per core, numpy "
              f"single thread), {args.steps} timed steps after {args.warmup} warm-up")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / max(args.steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "grid": list(w.n), "dt": w.dt, "picard_tol": w.picard_tol,
                   "mean_picard_iterations": mean_it, "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ---- the GPU arm ------------------------------------------------------------------------------

def run_ensemble(args, world, rank, local):
    """--workload ensemble-<R>: R independent runs (pic_inputs.ensemble_runs: meshes 16^3..48^3,
    8..64 particles per cell, v0 in [0.1, 0.3], eps in [1e-4, 1e-2]) stepped together through
    pic_ensemble_step, against the same runs stepped one after another with pic_step.  The
    runs use their own streams, so the timed region is bracketed by device-wide
    synchronisations and timed on the host clock."""
    import torch
    import __graft_entry__ as ge
    ge.build()
    import pic_inputs as pi
    from paper_2606_15035_gb300 import sim

    torch.cuda.set_device(local)
    nruns = int(args.workload.split("-")[1])
    runs = pi.ensemble_runs(nruns, seed=pi.twostream.ENSEMBLE_SEED + 1000 * rank)
    prec = 1 if args.precision == "mixed" else 0
    items = []
    for r in runs:
        x, v, q, m = pi.ensemble_particles(r)
        items.append((sim.pic_config_default(n=r.n, L=r.L, dt=r.dt, picard_tol=r.picard_tol, picard_max=r.picard_max,
                                             precision=prec, mixed_tol64=args.mixed_tol64 if prec else 0.0),
                      x, v, q, m))
    total = sum(r.n_particles for r in runs)
    ens = sim.PicEnsemble(items, autotune=True)
    e0 = [run.energy().total for run in ens.runs]
    drift = 0.0
    for _ in range(args.warmup):
        ens.step(1)
        drift = max(drift, max(abs(run.energy().total - a) / a for run, a in zip(ens.runs, e0)))
    for run in ens.runs:
        run.profile(True)
    sampler = ClockSampler(local)
    sampler.start()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    infos = []
    for _ in range(args.steps):
        inf, _ = ens.step(1)
        infos.append(inf)
        drift = max(drift, max(abs(run.energy().total - a) / a for run, a in zip(ens.runs, e0)))
    torch.cuda.synchronize()
    t_ens = time.perf_counter() - t0
    clk = sampler.stop()
    profs = [run.profile(False) for run in ens.runs]
    # the same runs one after another (each on its own stream, pic_step)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for run in ens.runs:
        run.step(1)
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t0
    # end to end: every run's state through pinned host memory around each ensemble step
    e2e = None
    if not args.no_e2e:
        from paper_2606_15035_gb300._lib import PicStateView
        views, nbytes = [], 0
        for run in ens.runs:
            N = run.ncell
            host = [torch.empty(3 * run.np, dtype=torch.float64, pin_memory=True) for _ in range(4)]
            host += [torch.empty(N, dtype=torch.float64, pin_memory=True) for _ in range(3)]
            host += [torch.empty(3 * N, dtype=torch.float64, pin_memory=True) for _ in range(2)]
            nbytes += sum(t.numel() * 8 for t in host)
            view = PicStateView(*[t.data_ptr() for t in host], 0)
            sim.pic_get_state(run.ctx, view)
            views.append((view, host))
        k_e2e = max(1, min(args.steps, 3))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(k_e2e):
            for run, (view, _) in zip(ens.runs, views):
                sim.pic_set_state(run.ctx, view)
            ens.step(1)
            for run, (view, _) in zip(ens.runs, views):
                sim.pic_get_state(run.ctx, view)
        torch.cuda.synchronize()
        t_e2e = time.perf_counter() - t0
        e2e = {"value": whole_job_rate(total, world, k_e2e, t_e2e), "unit": UNIT, "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": nbytes, "steps": k_e2e,
               "what": "every run: pic_set_state from pinned host, then pic_ensemble_step(1), then pic_get_state"}
    iters = sum(i.total_iterations for inf in infos for i in inf) / max(sum(i.steps_done for inf in infos for i in inf), 1)
    # pieces of the FP64 push launches only (the profile sums FP64 and FP32-pair iterations)
    fp64_part = [p.push_launches / max(p.push_launches + p.pushpair_launches, 1) for p in profs]
    flops = sum(p.particle_pushes * FLOPS_PER_PARTICLE + f * (p.push_pieces * FLOPS_PER_PUSH_PIECE +
                p.scatter_pieces * FLOPS_PER_SCATTER_PIECE) for p, f in zip(profs, fp64_part))
    push_ms = sum(p.push_ms for p in profs)
    tuning = sorted({tuple(t) for t in ens.tuning})
    ens.close()
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(pi.WORKLOADS["twostream-32c-2M"])
        cpu["sample"] += " (the ensemble's runs have meshes of 16^3 to 48^3 cells at this cell size scale)"
    if rank != 0:
        return
    value = total * args.steps / t_ens
    achieved = flops / (push_ms / 1e3) / 1e12 if push_ms > 0 else None
    line = {
        "metric": METRIC, "value": value * world, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_ens / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == 0 else "f32+f64", "data": "synthetic",
        "config": {"workload": args.workload, "runs": nruns, "particles_per_gpu": total,
                   "meshes": sorted({r.n[0] for r in runs}), "precision": args.precision,
                   "mixed_tol64": args.mixed_tol64 if prec else None,
                   "mean_picard_iterations": iters, "relative_energy_drift": drift,
                   "drift_definition": "max over runs and steps of |E^n - E^0| / E^0",
                   "timing": "host clock between device-wide synchronisations (runs on their own streams)",
                   "autotuned_blocks_per_sm (fp64, fp32)": tuning,
                   "l2": "inputs larger than L2"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / FP64_PEAK_TFLOPS if achieved else None, "traffic": None,
                     "kernel": "k_push (all runs; algorithmic flops over the summed k_push event durations)",
                     "peak_note": "derived: 152 SMs x 4 flop/clk x 2070 MHz"},
        "sequential": {"value": total / t_seq, "unit": UNIT,
                       "what": "the same runs, one pic_step each, one after another"},
        "cpu_baseline": cpu, "e2e": e2e,
        "gpu_launches": int(sum(p.launches for p in profs)), "clocks": clk,
    }
    print(json.dumps(line))


def cpu_baseline(w):
    """The oracle on bounded samples of workload w: CPU_STEPS timed steps on one core, then one
    independent sample per host core at once."""
    one = time_oracle(w.name, CPU_STEPS, 0)
    v1 = one["particles"] * one["steps"] / one["secs"]
    vall, secs, _, cores = time_oracle_all_cores(w.name, CPU_STEPS, 0)
    return {"value": vall, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"per core: {sample_text(w)}, {CPU_STEPS} steps ({secs:.1f} s); {cores} samples at once, "
                      f"one process per core, numpy single thread",
            "single_core": {"value": v1, "unit": UNIT, "cores": 1,
                            "sample": f"{sample_text(w)}, {CPU_STEPS} steps ({one['secs']:.1f} s)"}}


def kernel_shares(prof, ms):
    phases = {"k_push (FP64 iterations)": prof.push_ms, "k_push (FP64 final sweep)": prof.commit_ms,
              "k_local": prof.local_ms, "k_push32": prof.push32_ms, "mesh phases": prof.mesh_ms,
              "first scatters": prof.scatter_ms, "sort": prof.sort_ms,
              "k_push_df (FP32-pair iterations)": prof.pushpair_ms}
    return {k: v / ms for k, v in phases.items()} if ms > 0 else {}


def mean_pieces(prof, npart):
    """Orbit pieces per particle of the iteration pushes (FP64 and FP32-pair; the profile sums
    both) and of their next-orbit scatters."""
    n = (prof.push_launches + prof.pushpair_launches) * npart
    return (prof.push_pieces / n, prof.scatter_pieces / n) if n else (0.0, 0.0)


def fp64_push_roofline(prof, workload):
    """k_push (FP64 push + next-orbit scatter) against the FP64 ALU peak."""
    pushes = prof.particle_pushes
    if not prof.push_launches or prof.push_ms <= 0:
        return None
    npart = pushes // prof.push_launches
    mp, msc = mean_pieces(prof, npart)
    push_pieces, scatter_pieces = mp * pushes, msc * pushes    # the FP64 launches' share of the pieces
    flops = (pushes * FLOPS_PER_PARTICLE + push_pieces * FLOPS_PER_PUSH_PIECE
             + scatter_pieces * FLOPS_PER_SCATTER_PIECE)
    achieved = flops / (prof.push_ms / 1e3) / 1e12
    min_flops = pushes * (MIN_FLOPS_PER_PARTICLE + MIN_FLOPS_PER_PIECE * mp)
    achieved_min = min_flops / (prof.push_ms / 1e3) / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP64_PEAK_TFLOPS,
            "flops_basis": "counted from the kernel source (add, mul = 1, FMA = 2): 190 per particle + 409 per push "
                           "piece + 150 per scatter piece",
            "frac_survey_minimum": achieved_min / FP64_PEAK_TFLOPS,
            "survey_minimum_basis": "86 per particle + 398 per orbit piece (the survey's per-orbit estimate)",
            "traffic": NCU_TRAFFIC.get(("k_push", workload), (None, None))[0],
            "traffic_unit": "DRAM bytes per launch (ncu dram read + write)",
            "traffic_source": NCU_TRAFFIC.get(("k_push", workload), (None, "not captured"))[1],
            "kernel": "k_push (fused FP64 orbit push + next-orbit current scatter, Picard iterations)",
            "peak_note": "FP64 ALU, of derived: 152 SMs x 4 flop/clk x 2070 MHz (the live probe is in fma_probe)",
            "launches": int(prof.push_launches), "ms_per_launch": prof.push_ms / prof.push_launches,
            "flops_per_launch": flops / prof.push_launches,
            "mean_orbit_pieces": mp}


def final_sweep_roofline(prof, workload, npart):
    """The FP64 final sweep (k_push, commit: the push of the accepted orbit, no scatter) against
    the FP64 ALU peak.  Its orbit is the one the last iteration scattered, so its pieces per
    particle are taken as the iterations' scatter pieces per particle."""
    if not prof.commit_launches or prof.commit_ms <= 0:
        return None
    _, msc = mean_pieces(prof, npart)
    flops = prof.commit_launches * npart * (FLOPS_PER_PARTICLE + FLOPS_PER_PUSH_PIECE * msc)
    achieved = flops / (prof.commit_ms / 1e3) / 1e12
    min_flops = prof.commit_launches * npart * (MIN_FLOPS_PER_PARTICLE + MIN_FLOPS_PER_PIECE * msc)
    return {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP64_PEAK_TFLOPS,
            "flops_basis": "counted from the kernel source (add, mul = 1, FMA = 2): 190 per particle + 409 per push "
                           "piece (no scatter in the final sweep)",
            "frac_survey_minimum": min_flops / (prof.commit_ms / 1e3) / 1e12 / FP64_PEAK_TFLOPS,
            "survey_minimum_basis": "86 per particle + 398 per orbit piece (the survey's per-orbit estimate)",
            "traffic": None, "traffic_unit": "DRAM bytes per launch (ncu dram read + write)",
            "traffic_source": "not captured for the commit variant",
            "kernel": "k_push (FP64 final sweep: push of the accepted orbit, commit, residual sums)",
            "peak_note": "FP64 ALU, of derived: 152 SMs x 4 flop/clk x 2070 MHz (the live probe is in fma_probe)",
            "launches": int(prof.commit_launches), "ms_per_launch": prof.commit_ms / prof.commit_launches,
            "flops_per_launch": flops / prof.commit_launches, "mean_orbit_pieces": msc}


def pair_push_summary(prof, npart, step_ms):
    """The FP32-pair iteration push (k_push_df): FP64-class results from FP32-pair arithmetic on
    the FP32 pipes, latency-bound; reported beside the rooflines with its rate in FP64-equivalent
    flops (the FP64 push's count for the same work), which is not a roofline fraction."""
    if not prof.pushpair_launches or prof.pushpair_ms <= 0:
        return None
    mp, msc = mean_pieces(prof, npart)
    flops = npart * (FLOPS_PER_PARTICLE + FLOPS_PER_PUSH_PIECE * mp + FLOPS_PER_SCATTER_PIECE * msc)
    ms_l = prof.pushpair_ms / prof.pushpair_launches
    return {"kernel": "k_push_df (FP32-pair push + next-orbit current scatter)", "launches": int(prof.pushpair_launches),
            "ms_per_launch": ms_l, "share_of_step": prof.pushpair_ms / step_ms if step_ms > 0 else None,
            "fp64_equivalent_tflops": flops / (ms_l / 1e3) / 1e12,
            "note": "FP32 pipes, four blocks per SM; the FP64 push's flop count for the same work, per launch time"}


def fp32_push_roofline(prof, workload, npart, hbm_gbs, hbm_note):
    """k_push32 (FP32 push + next-orbit scatter) against the HBM peak."""
    if not prof.push32_launches or prof.push32_ms <= 0:
        return None
    bytes_per_launch = float(BYTES32_PER_PARTICLE) * npart
    gbs = bytes_per_launch * prof.push32_launches / (prof.push32_ms / 1e3) / 1e9
    return {"bound": "hbm", "achieved": gbs, "peak": hbm_gbs, "unit": "GB/s", "frac": gbs / hbm_gbs,
            "traffic": NCU_TRAFFIC.get(("k_push32", workload), (None, None))[0],
            "traffic_source": NCU_TRAFFIC.get(("k_push32", workload), (None, "not captured"))[1], "peak_note": hbm_note,
            "kernel": "k_push32 (FP32 orbit push + next-orbit current scatter)",
            "bytes_per_particle_iteration": BYTES32_PER_PARTICLE, "launches": int(prof.push32_launches),
            "ms_per_launch": prof.push32_ms / prof.push32_launches,
            "chunks_untiled": (prof.push32_chunks_global / prof.push32_chunks) if prof.push32_chunks else None}


def main():
    args = parse()
    if args.no_mixed:
        args.no_other = True
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    if args.workload.startswith("ensemble-"):
        run_ensemble(args, world, rank, local)
        return
    import torch
    import __graft_entry__ as ge
    ge.build()
    import pic_inputs as pi
    from paper_2606_15035_gb300 import sim
    from paper_2606_15035_gb300._lib import PicStateView

    torch.cuda.set_device(local)
    if args.probe_peaks:
        f64, f32 = sim.pic_probe_fma_rates()
        print(json.dumps({"fp64_fma_tflops": f64 / 1e12, "fp32_fma_tflops": f32 / 1e12,
                          "fp64_derived_tflops": FP64_PEAK_TFLOPS, "device": torch.cuda.get_device_name()}))
        return
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist
    w = pi.WORKLOADS[args.workload]
    x, v, q, m = pi.workload_particles(w, run=rank)
    stream = torch.cuda.current_stream()
    hbm_gbs, hbm_note = measured_peaks()

    def timed(precision, with_clocks):
        """W warm-up steps, then K timed steps between barriers, CUDA events on the library's
        stream; the total energy after every step (inside the timed region) gives the drift
        max_n |E^n - E^0| / E^0 over all W + K steps."""
        extra = {"ops": 1 if args.ops == "spectral" else 0, "deterministic": int(args.deterministic)}
        if args.shape_order > 1:
            extra.update(shape_order=args.shape_order, quadrature=1, nq=(3 * args.shape_order + 2) // 2)
        if precision == "mixed":
            extra.update(precision=1, mixed_tol64=args.mixed_tol64)
        cfg = sim.pic_config_default(n=w.n, L=w.L, dt=w.dt, picard_tol=w.picard_tol, picard_max=w.picard_max,
                                     **extra)
        sm = sim.PicSim(cfg, x, v, q, m)
        e0 = sm.energy().total
        drift = 0.0
        for _ in range(args.warmup):
            sm.step(1)
            drift = max(drift, abs(sm.energy().total - e0) / e0)
        sm.profile(True)                  # reset accumulators, profiling on
        sampler = ClockSampler(local) if with_clocks else None
        if sampler:
            sampler.start()
        if pg:
            pg.barrier()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        it = it32 = done = 0
        ev0.record(stream)
        for _ in range(args.steps):
            inf = sm.step(1)
            it += inf.total_iterations
            it32 += inf.total_iterations_fp32
            done += inf.steps_done
            drift = max(drift, abs(sm.energy().total - e0) / e0)
        ev1.record(stream)
        torch.cuda.synchronize()
        if pg:
            pg.barrier()
        clk = sampler.stop() if sampler else None
        pr = sm.profile(False)
        t_ms = max_over_ranks(ev0.elapsed_time(ev1), pg, "cuda")
        ev_h, ej_h, kind_h = sm.residual_history()
        kinds = {0: "fp64", 1: "fp32", 2: "fp32-pair", 3: "final-sweep residual of v*"}
        fin = lambda z: float(z) if np.isfinite(z) else None   # strict JSON: no Infinity
        history = [[fin(a), fin(b), kinds[int(k)]] for a, b, k in zip(ev_h, ej_h, kind_h)]
        return {"sim": sm, "prof": pr, "ms": t_ms, "drift": drift, "clocks": clk,
                "iters": it / max(done, 1), "iters32": it32 / max(done, 1), "history": history}

    head = timed(args.precision, True)
    s, prof, ms = head["sim"], head["prof"], head["ms"]
    value = whole_job_rate(w.n_particles, world, args.steps, ms / 1e3)
    shares = kernel_shares(prof, ms)
    r64 = fp64_push_roofline(prof, w.name)
    r32 = fp32_push_roofline(prof, w.name, w.n_particles, hbm_gbs, hbm_note)
    rfs = final_sweep_roofline(prof, w.name, w.n_particles)
    pair_push = pair_push_summary(prof, w.n_particles, ms)
    # the dominant kernel of the step with a roofline (FP64 or FP32 pipes, HBM) carries the
    # roofline object; the FP32-pair push, when it runs, is reported beside it (pair_push)
    cands = {"k_push (FP64 iterations)": r64, "k_push (FP64 final sweep)": rfs, "k_push32": r32}
    ranked = sorted((k for k in cands if cands[k] and k in shares), key=lambda k: -shares[k])
    roofline = cands[ranked[0]] if ranked else None
    if args.shape_order > 1 and roofline is r64 and roofline:
        roofline = dict(roofline, achieved=None, frac=None)   # the flop counts are those of the linear closed forms
    local_solves = None
    if prof.local_launches:
        local_solves = {"kernel": "k_local", "share_of_step": prof.local_ms / ms if ms > 0 else None,
                        "ms_per_launch": prof.local_ms / prof.local_launches,
                        "solves_per_launch": prof.local_solves / prof.local_launches,
                        "evals_per_solve": prof.local_evals / prof.local_solves if prof.local_solves else None}

    # end to end through the public API: the full state crosses host <-> device every step
    e2e = None
    if not args.no_e2e:
        N = w.n[0] * w.n[1] * w.n[2]
        npart = w.n_particles
        host = {k: torch.empty(3 * npart, dtype=torch.float64, pin_memory=True) for k in ("x", "v", "P", "vprev")}
        host.update({k: torch.empty(N, dtype=torch.float64, pin_memory=True) for k in ("phi", "psi", "rho")})
        host.update({k: torch.empty(3 * N, dtype=torch.float64, pin_memory=True) for k in ("A", "U")})
        order = ("x", "v", "P", "vprev", "phi", "psi", "rho", "A", "U")
        view = PicStateView(*[host[k].data_ptr() for k in order], 0)
        sim.pic_get_state(s.ctx, view)
        nbytes = sum(t.numel() * 8 for t in host.values())
        k_e2e = max(1, min(args.steps, 3))
        if pg:
            pg.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(k_e2e):
            sim.pic_set_state(s.ctx, view)        # step inputs: host -> device
            sim.pic_step(s.ctx, 1)
            sim.pic_get_state(s.ctx, view)        # step result: device -> host
        torch.cuda.synchronize()
        t_e2e = max_over_ranks(time.perf_counter() - t0, pg, "cuda")
        e2e = {"value": whole_job_rate(w.n_particles, world, k_e2e, t_e2e), "unit": UNIT,
               "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes, "steps": k_e2e,
               "what": "pic_set_state from pinned host + pic_step(1) + pic_get_state to pinned host, per step"}
        del host
    s.close()

    # the other precision on the same workload ("mixed vs FP64 at stated energy drift")
    other = None
    if not args.no_other and args.shape_order == 1:
        oname = "fp64" if args.precision == "mixed" else "mixed"
        o = timed(oname, False)
        o["sim"].close()
        po = o["prof"]
        other = {"precision": oname, "value": whole_job_rate(w.n_particles, world, args.steps, o["ms"] / 1e3),
                 "unit": UNIT, "ms_per_step": o["ms"] / args.steps, "relative_energy_drift": o["drift"],
                 "mean_picard_iterations": o["iters"], "mean_fp32_iterations": o["iters32"],
                 "residual_history_last_step": o["history"],
                 "kernel_shares": kernel_shares(po, o["ms"]),
                 "fp64_push_roofline": fp64_push_roofline(po, w.name),
                 "fp32_push_roofline": fp32_push_roofline(po, w.name, w.n_particles, hbm_gbs, hbm_note)}
    fma = None
    try:
        f64, f32 = sim.pic_probe_fma_rates()
        fma = {"fp64_tflops": f64 / 1e12, "fp32_tflops": f32 / 1e12, "what": "pic_probe_fma_rates, live"}
    except Exception as e:  # the probe is evidence beside the derived peak, never a value
        fma = {"error": str(e)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w)
    if rank == 0:
        mixed_desc = (f"mixed: FP32 Picard iterations (cell index + FP32 offsets), one FP32-pair iteration, "
                      f"then the FP64 final sweep commits that iterate once it measures its residual "
                      f"||G(v*) - v*|| / ||G(v*)|| <= {args.mixed_tol64:g} (else FP64 iterations to e_v, e_J <= "
                      f"{args.mixed_tol64:g} first)")
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32+f64",
            "data": "synthetic",
            "config": {"workload": w.name, "grid": list(w.n), "particles_per_gpu": w.n_particles, "dt": w.dt,
                       "picard_tol": w.picard_tol, "picard_max": w.picard_max,
                       "precision": "fp64" if args.precision == "fp64" else mixed_desc,
                       "orbits": ("split at knots, closed form" if args.shape_order == 1 else
                                  f"split at the knots of the degree-{args.shape_order} B-spline, "
                                  f"{(3 * args.shape_order + 2) // 2}-point Gauss rule per piece"),
                       "shape_order": args.shape_order, "ops": args.ops,
                       "deterministic": bool(args.deterministic),
                       "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
                       "l2": f"inputs larger than L2 (FP64 particle state {w.n_particles * 120 / 1e9:.1f} GB "
                             f"per GPU: x, v, P, v^(n-1), iterate)",
                       "mean_picard_iterations": head["iters"], "mean_fp32_iterations": head["iters32"],
                       "relative_energy_drift": head["drift"],
                       "residual_history_last_step": head["history"],
                       "drift_definition": "max over the W + K steps of |E^n - E^0| / E^0, E^0 at pic_init; "
                                           "the energy is evaluated after every step, inside the timed region"},
            "roofline": roofline,
            "kernel_shares": shares,
            "fp32_push_roofline": r32,
            "final_sweep_roofline": rfs,
            "pair_push": pair_push,
            "local_solves": local_solves,
            "fma_probe": fma,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(prof.launches),
            "clocks": head["clocks"],
            "other_precision": other,
            "speedup_vs_other": (value / other["value"]) if other else None,
        }
        print(json.dumps(line))
    if pg:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
