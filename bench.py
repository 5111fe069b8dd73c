#!/usr/bin/env python
"""Benchmark of the GB300 PIC step: particle-steps per second, Picard iterations included.

Workload (one step = one full implicit time step: every Picard iteration of Algorithm 1
plus the final consistency sweep, with the cell sort, the orbit-current scatters, the
continuity + Crank--Nicolson mesh solves and the orbit pushes): the 3D periodic cold
two-stream problem on a 32^3 mesh with 2,097,152 electrons (32 per beam per cell),
beams +-0.2 c, thermal spread 1e-4, dt = 0.1, Picard tolerance 1e-13, FP64, split-orbit
closed-form weights.  Synthetic, seeded inputs (pic_inputs).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU runs (torchrun, one rank per GPU) are independent replicas with distinct
seeds: the method is not sharded, so there is no data-path collective; only the timing
barrier and the max-over-ranks reduction touch the process group.
--impl reference times the FP64 CPU oracle (the reference arm of this benchmark) on a
bounded sample of the same workload.
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

WORKLOAD = "twostream-32c-2M"
METRIC = "particle-steps/s incl. Picard iters, mixed vs FP64 at stated energy drift; %HBM"
UNIT = "particle-steps/s"
# FP64 ALU peak of the GB300: 152 SMs x 2 FP64 FMA (4 flop) per clock per SM x 2070 MHz.
FP64_PEAK_TFLOPS = 152 * 4 * 2.070e9 / 1e12
SAMPLE_PARTICLES = 65536


# Algorithmic FP64 flops (add, mul = 1, FMA = 2; the scatter's atomic adds counted) of the
# fused push + next-orbit scatter kernel, counted from the kernel source per particle and per
# knot-free orbit piece (see the design notes):
FLOPS_PER_PARTICLE = 190
FLOPS_PER_PUSH_PIECE = 409
FLOPS_PER_SCATTER_PIECE = 150
# DRAM bytes (read + write) of one k_push launch on the 32^3 x 2.1M workload, from an ncu
# capture of this kernel version (dram__bytes_read.sum + dram__bytes_write.sum).
KPUSH_TRAFFIC_BYTES = {"twostream-32c-2M": 297.3e6}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--deterministic", action="store_true", help="bitwise reproducible mode")
    ap.add_argument("--ops", default="central2", choices=["central2", "spectral"],
                    help="spatial operators: central differences or the paper's spectral operators (FFT)")
    ap.add_argument("--shape-order", type=int, default=1, choices=[1, 2, 3],
                    help="B-spline degree r; r > 1 runs the split Gauss rule with 2 nq - 1 >= 3 r (FP64)")
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


def oracle_sample(w, npart):
    """A bounded sample of the workload for the CPU oracle: the same mesh, box and physics
    with a strided subset of the particle pairs (charge rescaled to keep neutrality)."""
    import pic_inputs as pi
    x, v, q, m = pi.workload_particles(w)
    half = x.shape[0] // 2
    stride = max(1, (2 * half) // npart)
    pairs = np.arange(0, half, stride)[: npart // 2]
    idx = np.concatenate([pairs, pairs + half])
    scale = x.shape[0] / idx.size
    return x[idx], v[idx], q * scale, m * scale


def time_oracle(w, npart, steps, warmup):
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    from oracle import pic as opic
    x, v, q, m = oracle_sample(w, npart)
    cfg = opic.Config(n=w.n, L=w.L, dt=w.dt, picard_tol=w.picard_tol, picard_max=w.picard_max)
    st = opic.init(x, v, q, m, cfg)
    for _ in range(warmup):
        st, info = opic.step(st, cfg)
    t0 = time.perf_counter()
    iters = 0
    for _ in range(steps):
        st, info = opic.step(st, cfg)
        iters += info["iterations"]
    dt_s = time.perf_counter() - t0
    return x.shape[0] * steps / dt_s, dt_s, iters / max(steps, 1), x.shape[0]


def run_reference(args, world, rank):
    import pic_inputs as pi
    if rank != 0:
        return
    w = pi.WORKLOADS[args.workload]
    value, secs, mean_it, nsample = time_oracle(w, SAMPLE_PARTICLES, args.steps, args.warmup)
    sample = (f"{nsample} particles (strided pairs of the {w.n_particles}-particle workload, same 32^3 mesh and "
              f"physics), {args.steps} timed steps after {args.warmup} warm-up, numpy single thread")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / max(args.steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "grid": list(w.n), "particles": nsample, "dt": w.dt,
                   "picard_tol": w.picard_tol, "mean_picard_iterations": mean_it},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


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
                                             precision=prec),
                      x, v, q, m))
    total = sum(r.n_particles for r in runs)
    ens = sim.PicEnsemble(items, autotune=True)
    e0 = [run.energy().total for run in ens.runs]
    if args.warmup > 0:
        ens.step(args.warmup)
    for run in ens.runs:
        run.profile(True)
    sampler = ClockSampler(local)
    sampler.start()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    infos, _ = ens.step(args.steps)
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
    drift = max(abs(run.energy().total - a) / a for run, a in zip(ens.runs, e0))
    iters = sum(i.total_iterations for i in infos) / max(sum(i.steps_done for i in infos), 1)
    flops = sum(p.particle_pushes * FLOPS_PER_PARTICLE + p.push_pieces * FLOPS_PER_PUSH_PIECE +
                p.scatter_pieces * FLOPS_PER_SCATTER_PIECE for p in profs)
    tuning = sorted({tuple(t) for t in ens.tuning})
    ens.close()
    if rank != 0:
        return
    value = total * args.steps / t_ens
    line = {
        "metric": METRIC, "value": value * world, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_ens / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == 0 else "f32+f64", "data": "synthetic",
        "config": {"workload": args.workload, "runs": nruns, "particles_per_gpu": total,
                   "meshes": sorted({r.n[0] for r in runs}), "precision": args.precision,
                   "mean_picard_iterations": iters, "relative_energy_drift_max": drift,
                   "timing": "host clock between device-wide synchronisations (runs on their own streams)",
                   "autotuned_blocks_per_sm (fp64, fp32)": tuning,
                   "l2": "inputs larger than L2"},
        "roofline": {"bound": "alu", "achieved": flops / t_ens / 1e12, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": flops / t_ens / 1e12 / FP64_PEAK_TFLOPS, "traffic": None,
                     "kernel": "k_push (all runs, algorithmic flops over the whole timed region)"},
        "sequential": {"value": total / t_seq, "unit": UNIT,
                       "what": "the same runs, one pic_step each, one after another"},
        "cpu_baseline": None, "e2e": None,
        "gpu_launches": int(sum(p.launches for p in profs)), "clocks": clk,
    }
    print(json.dumps(line))


def main():
    args = parse()
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
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist
    w = pi.WORKLOADS[args.workload]
    x, v, q, m = pi.workload_particles(w, run=rank)
    stream = torch.cuda.current_stream()

    def timed(precision, with_clocks):
        """W warm-up steps, then K timed steps between barriers, CUDA events on the library's stream."""
        extra = {"ops": 1 if args.ops == "spectral" else 0, "deterministic": int(args.deterministic)}
        if args.shape_order > 1:
            extra.update(shape_order=args.shape_order, quadrature=1, nq=(3 * args.shape_order + 2) // 2)
        cfg = sim.pic_config_default(n=w.n, L=w.L, dt=w.dt, picard_tol=w.picard_tol, picard_max=w.picard_max,
                                     precision=1 if precision == "mixed" else 0, **extra)
        sm = sim.PicSim(cfg, x, v, q, m)
        e_start = sm.energy().total
        if args.warmup > 0:
            sm.step(args.warmup)
        sm.profile(True)                  # reset accumulators, profiling on
        sampler = ClockSampler(local) if with_clocks else None
        if sampler:
            sampler.start()
        if pg:
            pg.barrier()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        inf = sm.step(args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        if pg:
            pg.barrier()
        clk = sampler.stop() if sampler else None
        pr = sm.profile(False)
        t_ms = max_over_ranks(ev0.elapsed_time(ev1), pg, "cuda")
        drift_ = abs(sm.energy().total - e_start) / e_start
        return sm, inf, pr, t_ms, drift_, clk

    s, info, prof, ms_max, drift, clocks = timed(args.precision, True)
    ms = ms_max
    value = whole_job_rate(w.n_particles, world, args.steps, ms_max / 1e3)

    # roofline of the dominant kernel (the fused push + scatter, FP64 ALU bound)
    pushes = prof.particle_pushes
    flops = (pushes * FLOPS_PER_PARTICLE + prof.push_pieces * FLOPS_PER_PUSH_PIECE
             + prof.scatter_pieces * FLOPS_PER_SCATTER_PIECE)
    mean_pieces = prof.push_pieces / pushes if pushes else None
    push_s = prof.push_ms / 1e3
    achieved = flops / push_s / 1e12 if push_s > 0 else None
    if args.shape_order > 1:
        achieved = None   # the flop counts above are those of the linear closed forms
    roofline = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": (achieved / FP64_PEAK_TFLOPS) if achieved else None,
                "traffic": KPUSH_TRAFFIC_BYTES.get(w.name) if args.precision == "fp64" else None,
                "traffic_unit": "bytes per launch (ncu dram read + write)",
                "kernel": "k_push (fused orbit push + next-orbit current scatter, FP64)",
                "peak_note": "FP64 ALU: 152 SMs x 4 flop/clk x 2070 MHz (derived; probe measured 1.203 TFLOP/s "
                             "at 2010 MHz)",
                "share_of_step": (prof.push_ms / ms) if ms > 0 else None,
                "mean_orbit_pieces": mean_pieces}
    # the particle-local solves of the creeping particles (their own kernel, after each push)
    local = None
    if prof.local_launches:
        local = {"kernel": "k_local", "share_of_step": prof.local_ms / ms if ms > 0 else None,
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
        k_e2e = max(1, min(args.steps, 5))
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

    # the other precision on the same workload ("mixed vs FP64 at stated energy drift")
    other = None
    if args.precision == "fp64" and not args.no_mixed and args.shape_order == 1:
        sm2, inf2, pr2, ms2, drift2, _ = timed("mixed", False)
        sm2.close()
        # per particle-iteration: read cell 4 + offset 12 + v^n 12 + increment 12, write 12
        bytes32 = 52.0 * w.n_particles * pr2.push32_launches
        hbm32 = bytes32 / (pr2.push32_ms / 1e3) / 1e9 if pr2.push32_ms > 0 else None
        other = {
            "precision": "mixed: FP32 iterations (cell index + FP32 offsets), FP64 refinement to the same tau "
                         "and FP64 final sweep",
            "value": whole_job_rate(w.n_particles, world, args.steps, ms2 / 1e3), "unit": UNIT,
            "ms_per_step": ms2 / args.steps,
            "relative_energy_drift": drift2,
            "mean_picard_iterations": inf2.total_iterations / max(inf2.steps_done, 1),
            "mean_fp32_iterations": inf2.total_iterations_fp32 / max(inf2.steps_done, 1),
            "fp32_push_roofline": {"bound": "hbm", "achieved": hbm32, "peak": 6804.8, "unit": "GB/s",
                                   "frac": (hbm32 / 6804.8) if hbm32 else None, "traffic": None,
                                   "kernel": "k_push32 (FP32 orbit push + next-orbit scatter)",
                                   "bytes_per_particle_iteration": 52},
            "share_fp32_push": pr2.push32_ms / ms2 if ms2 > 0 else None,
            "share_fp64_push": pr2.push_ms / ms2 if ms2 > 0 else None,
        }

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cv, secs, mit, nsample = time_oracle(w, SAMPLE_PARTICLES, 1, 0)
        cpu = {"value": cv, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"1 step of {nsample} particles (strided pairs of the workload, same 32^3 mesh and physics), "
                         f"{secs:.1f} s, numpy single thread"}
    s.close()
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32+f64",
            "data": "synthetic",
            "config": {"workload": w.name, "grid": list(w.n), "particles_per_gpu": w.n_particles, "dt": w.dt,
                       "picard_tol": w.picard_tol,
                       "precision": "fp64" if args.precision == "fp64" else
                                    "mixed: FP32 iterations, FP64 refinement and final sweep",
                       "orbits": ("split at knots, closed form" if args.shape_order == 1 else
                                  f"split at the knots of the degree-{args.shape_order} B-spline, "
                                  f"{(3 * args.shape_order + 2) // 2}-point Gauss rule per piece"),
                       "shape_order": args.shape_order,
                       "ops": args.ops,
                       "deterministic": bool(args.deterministic),
                       "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
                       "l2": f"inputs larger than L2 (FP64 particle state {w.n_particles * 120 / 1e9:.1f} GB "
                             f"per GPU: x, v, P, v^(n-1), iterate)",
                       "mean_picard_iterations": info.total_iterations / max(info.steps_done, 1),
                       "mean_fp32_iterations": info.total_iterations_fp32 / max(info.steps_done, 1),
                       "relative_energy_drift": drift},
            "roofline": roofline,
            "local_solves": local,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(prof.launches),
            "clocks": clocks,
            "mixed": other,
        }
        print(json.dumps(line))
    if pg:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
