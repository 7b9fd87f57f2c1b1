#!/usr/bin/env python3
"""Benchmark of the LLG hot path: RK4 steps of a 256x256x16 film, FP32, one B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl b300|reference]

One step = one classical RK4 step: four effective-field evaluations, each two
kernels -- k_yz (y transform, the demag product along z, inverse y transform)
and k_x (inverse x transform fused with exchange, anisotropy, Zeeman, LLG, the
RK4 update, and the x transform of the next stage's state) --
on synthetic inputs (seeded random unit vectors).  The L2 cache is flushed
between timed steps (a 512 MiB write), so every step starts cold.

Prints one JSON line (rank 0).  Multi-GPU runs (torchrun) run one independent
replica per rank: a single film does not shard without a global transpose.
The reference arm (--impl reference) times the FP64 CPU oracle on the host.
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "LLG cell-steps/s at 256×256×16 (FP32 vs split-prec vs batched); adjoint/fwd time"
UNIT = "cell-steps/s"
FLUSH_BYTES = 512 << 20


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="b300", choices=["b300", "reference"])
    ap.add_argument("--workload", default="film_256x256x16")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the batched-sweep and adjoint measurements")
    ap.add_argument("--extras", default="all",
                    help="comma list of the extra measurements to run: batched, adjoint, sp4, sp3, split, cufft, "
                         "noalloc (default all)")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "split_bf16", "split_fp16"],
                    help="the z product of the timed steps: FP32 direct sum or the tensor-core split forms")
    ap.add_argument("--batch-max-steps", type=int, default=20000,
                    help="field sweep run to convergence: step cap per film (the workload's 20,000)")
    ap.add_argument("--ref-max-steps", type=int, default=8,
                    help="reference arm: at most this many oracle RK4 steps are executed and timed")
    return ap.parse_args()


def dist_info():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
CLOCK_QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
REASON_NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]


class ClockSampler:
    def __init__(self, gpu_index):
        self.path = tempfile.mktemp(prefix="clocks_", suffix=".csv")
        self.proc = None
        self.gpu = gpu_index

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={CLOCK_QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.3)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        sm, mx, reasons = [], [], set()
        try:
            for line in open(self.path):
                p = [v.strip() for v in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    sm.append(float(p[1]))
                    mx.append(float(p[2]))
                except ValueError:
                    continue
                for name, v in zip(REASON_NAMES, p[5:9]):
                    if v.lower() == "active":
                        reasons.add(name)
        except OSError:
            pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# roofline bookkeeping
# ---------------------------------------------------------------------------
def _padded(grid):
    nx, ny, nz = grid
    px = 1 if nx == 1 else 1 << (2 * nx - 2).bit_length()
    py = 1 if ny == 1 else 1 << (2 * ny - 2).bit_length()
    hx = 1 if px == 1 else px // 2 + 1
    hy = 1 if py == 1 else py // 2 + 1
    return px, py, hx, hy


def algorithmic_bytes(grid):
    """Compulsory HBM bytes per launch of each kernel class of this implementation
    (FP32 RK4 stage).

    yz: read the x-transformed field S and the transformed tensor Kh, write S
    x:  read S, m_stage, m0; accumulator r/w (averaged over the 4 stages:
        1.5 x 12 B/cell); write the next stage (12 B/cell) and S
    """
    nx, ny, nz = grid
    N = nx * ny * nz
    px, py, hx, hy = _padded(grid)
    S = hx * 3 * nz * ny * 8
    Kh = hx * 6 * nz * hy * 4
    v = 12 * N
    return {"yz": 2 * S + Kh, "x": S + v + v + 1.5 * v + v + S}


def method_bytes(grid):
    """The method's algorithmic bytes per field evaluation (three passes: x forward,
    fused y/z with the spectral product, x inverse with the LLG/RK4 update), per
    pass, in bytes for the whole grid: the fewest a zero-padded FFT convolution
    moves when the spectrum does not fit on chip -- one round trip of the
    half spectrum (3 components x 8 B x hx/nx per cell) per transform direction,
    the transformed tensor's octant (6 components x 4 B x hx hy (pz/2 + 1)) and
    the RK4 state.  At 256 x 256 x 16: 36.1 + 73.9 + 84.1 = 194.1 B per cell and
    evaluation, 776 B per cell and RK4 step."""
    nx, ny, nz = grid
    N = nx * ny * nz
    px, py, hx, hy = _padded(grid)
    pz = 1 if nz == 1 else 1 << (2 * nz - 2).bit_length()
    spec = 3 * 8 * hx * ny * nz            # half spectrum after the x transform
    tens = 6 * 4 * hx * hy * (pz // 2 + 1)  # real octant of the transformed tensor
    a1 = 12 * N + spec                      # read m, write the spectrum
    a2 = spec + tens + spec                 # read spectrum + tensor, write spectrum
    a3 = spec + 12 * N + 12 * N + 24 * N + 12 * N   # spectrum, m_stage, m0, acc r/w, next stage
    return {"a1": a1, "a2": a2, "a3": a3, "eval": a1 + a2 + a3}


def _fft_pruned(L):
    """Flops of a length-L complex FFT whose upper half of inputs is zero (or whose
    upper half of outputs is discarded): one radix-2 split into two half-length
    FFTs (5 (L/2) log2 (L/2) each) after L/2 complex twiddle products (6 flops)."""
    if L <= 1:
        return 0
    return 5 * L * (math.log2(L) - 1) + 3 * L


def algorithmic_flops(grid):
    """FP32 flops per launch of each kernel class (FP32 RK4 stage), counted for
    the method as the paper states it (eq. 12-14: a zero-padded 3-D FFT
    convolution), not for this implementation's direct sum along z:

    yz: per kx column, the forward and inverse y transforms of the 3 nz rows
        (length py, half the inputs zero / half the outputs dropped), and per
        (kx, ky) the z transforms of length PZ = 2^ceil(log2(2 nz - 1)) of the 3
        components both ways plus the 3x3 tensor product per kz (9 complex-by-
        real products and 6 complex adds = 30 flops)
    x:  per (y, z) row, the real inverse and forward x transforms of the 3
        components (a half-length complex FFT, pruned, plus 5 px flops of pre-
        or post-processing each), plus about 100 flops per cell for exchange,
        anisotropy, Zeeman, the LLG right-hand side and the RK4 update
    """
    nx, ny, nz = grid
    px = 1 if nx == 1 else 1 << (2 * nx - 2).bit_length()
    py = 1 if ny == 1 else 1 << (2 * ny - 2).bit_length()
    hx = 1 if px == 1 else px // 2 + 1
    pz = 1 if nz == 1 else 1 << (2 * nz - 2).bit_length()
    col = 6 * nz * _fft_pruned(py) + py * (6 * _fft_pruned(pz) + 30 * pz)
    rfft = (_fft_pruned(px // 2) + 5 * px) if px > 1 else 0
    return {"yz": hx * col, "x": ny * nz * 6 * rfft + 100 * nx * ny * nz}


# FP32 peak derived from the unit counts and the maximum clock, used only when
# the probe cannot run: SMs x 128 FP32 lanes x 2 flops (one FMA) x 2032 MHz
def derived_fp32_tflops(sms):
    return sms * 128 * 2 * 2.032e9 / 1e12


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def stored_traffic(kernel):
    """DRAM bytes per launch from a committed ncu capture, if the kernel source is unchanged since."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        d = json.load(open(p))[kernel]
    except Exception:
        return None
    src = os.path.join(ROOT, "paper_1501_07293_b300", "csrc", d.get("source", "field_kernels.cuh"))
    try:
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
    except OSError:
        return None
    return d["bytes_per_launch"] if sha == d.get("source_sha256") else None


# ---------------------------------------------------------------------------
# oracle timing (CPU baseline / reference arm)
# ---------------------------------------------------------------------------
def time_oracle(w, nsteps, warmup):
    """Oracle RK4 steps on the full film; returns (cell-steps/s, cores given, seconds, steps, utilisation)."""
    from oracle import to_xyz
    from oracle.llg import Film
    from paper_1501_07293_b300 import inputs
    mat = w.mat
    film = Film(w.grid, w.delta, mat.Ms, mat.A, mat.Ku, mat.alpha, mat.gamma, b_ext=w.b_ext)
    m = to_xyz(inputs.workload_state(w))
    for _ in range(warmup):
        m = film.rk4_step(m, w.dt)
    c0, t0 = time.process_time(), time.perf_counter()
    for _ in range(nsteps):
        m = film.rk4_step(m, w.dt)
    wall = time.perf_counter() - t0
    cpu = time.process_time() - c0
    from oracle.demag import WORKERS
    # cores: the host cores the oracle's transforms are given (scipy.fft workers,
    # the process's CPU affinity); utilisation: CPU time over wall time
    return w.ncells * nsteps / wall, WORKERS, wall, nsteps, cpu / wall


def reference_arm(args, w):
    rank, world, _ = dist_info()
    if rank != 0:
        return
    n = max(1, min(args.steps, args.ref_max_steps))
    warm = min(args.warmup, 1)
    val, cores, wall, n, util = time_oracle(w, n, warm)
    sample = (f"{n} RK4 steps of the full {w.grid[0]}x{w.grid[1]}x{w.grid[2]} film (FP64 numpy/scipy oracle, "
              f"{warm} warm-up step), of the {args.steps} requested; FFTs on {cores} cores, "
              f"mean utilisation {util:.1f} cores")
    out = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
           "steps": n, "warmup": warm, "ms_per_step": 1e3 * wall / n, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": w.name, "grid": list(w.grid), "integrator": "rk4", "dt_s": w.dt,
                      "l2": "n/a (CPU)"},
           "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
           "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------
# B300 arm
# ---------------------------------------------------------------------------
def bench_batched(args, steps=40, warmup=5, seq_steps=20):
    """The field-sweep workload: 256 independent films of uneven size, RK4.

    * persistent vs grouped schedule: aggregate cell-steps/s over `steps` steps;
    * the same films one context at a time (seq_steps steps each, CUDA events
      around the steps only): the batching speed-up;
    * the workload as specified: mm_batch_run until each film's max |dm/dt| is
      below 1e3 rad/s (checked every 100 steps) or args.batch_max_steps steps.
    Under torchrun the films are sharded over the ranks by estimated cost (no
    data-path collective); values are all films' cell-steps over the slowest rank."""
    import torch
    from paper_1501_07293_b300 import inputs
    from paper_1501_07293_b300.shard import max_over_ranks, partition
    from paper_1501_07293_b300.solver import Batch, Solver
    rank, world, _ = dist_info()
    films_all = inputs.film_batch()
    mine = partition([f.grid for f in films_all], world)[rank]
    films = [films_all[i] for i in mine]
    mat = inputs.BATCH_MATERIAL
    stream = torch.cuda.current_stream()
    cells = sum(f.grid[0] * f.grid[1] * f.grid[2] for f in films_all)
    peak, _ = measured_peaks()
    step_bytes = sum(4 * method_bytes(f.grid)["eval"] for f in films_all)

    def make_batch():
        b = Batch([f.grid for f in films], inputs.BATCH_DELTA, mat.Ms, mat.A, mat.Ku, mat.alpha, mat.gamma)
        for j, f in enumerate(films):
            b.films[j].set_field(f.b_ext)
            b.films[j].set_m(torch.from_numpy(inputs.initial_state("tilted_x", f.grid, f.seed)).cuda())
        return b

    def timed(fn, n):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        fn(n)
        e1.record(stream)
        torch.cuda.synchronize()
        return max_over_ranks(e0.elapsed_time(e1), device="cuda")

    b = make_batch()
    sched = {}
    for name in ("persistent", "grouped"):
        b.set_schedule(name)
        b.step(warmup, inputs.BATCH_DT)
        l0 = b.launch_count()
        ms = timed(lambda n: b.step(n, inputs.BATCH_DT), steps)
        b.sync()
        sched[name] = {"ms_per_step": ms / steps, "value": cells * steps / (ms * 1e-3), "unit": UNIT,
                       "gpu_launches_per_step": (b.launch_count() - l0) / steps,
                       "hbm_frac": step_bytes / (ms / steps * 1e-3) / 1e9 / peak}
    groups = b.group_count()
    b.close()
    best = "persistent" if sched["persistent"]["ms_per_step"] <= sched["grouped"]["ms_per_step"] else "grouped"

    # one context at a time (the plain single-film path), the same films
    seq_ms = 0.0
    for f in films:
        s = Solver(f.grid, inputs.BATCH_DELTA, mat.Ms, mat.A, mat.Ku, mat.alpha, mat.gamma)
        s.set_field(f.b_ext)
        s.set_m(torch.from_numpy(inputs.initial_state("tilted_x", f.grid, f.seed)).cuda())
        s.step(3, inputs.BATCH_DT)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        s.step(seq_steps, inputs.BATCH_DT)
        e1.record(stream)
        torch.cuda.synchronize()
        seq_ms += e0.elapsed_time(e1)   # local: ranks hold different numbers of films
        s.close()
    seq_ms = max_over_ranks(seq_ms, device="cuda")
    seq_ms_per_step = seq_ms / seq_steps

    # the workload as specified: to |dm/dt| < 1e3 rad/s or the step cap
    b = make_batch()
    b.set_schedule(best)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    nsteps = b.run(args.batch_max_steps, inputs.BATCH_DT, 1e3, check_every=100)
    e1.record(stream)
    torch.cuda.synchronize()
    run_ms = max_over_ranks(e0.elapsed_time(e1), device="cuda")
    wall = time.perf_counter() - t0
    cell_steps = sum(f.grid[0] * f.grid[1] * f.grid[2] * n for f, n in zip(films, nsteps))
    final_dmdt = b.max_dmdt()
    b.close()
    srt = sorted(nsteps)
    out = {"workload": "256 films, nx 32..256, ny 8..128, nz 1..4, fields -50..50 mT, RK4 dt 1e-13 s",
           "cells": cells, "groups": groups, "films_per_rank": len(films),
           "sharding": f"by film over {world} rank(s), cost-balanced",
           "schedules": sched, "schedule_used": best,
           "value": sched[best]["value"], "unit": UNIT, "ms_per_step": sched[best]["ms_per_step"],
           "hbm_frac": sched[best]["hbm_frac"],
           "bytes_model": "sum over films of 4 x the method's bytes per field evaluation (passes a1 + a2 + a3)",
           "one_context_at_a_time": {"ms_per_step": seq_ms_per_step, "value": cells / (seq_ms_per_step * 1e-3),
                                     "steps_timed_per_film": seq_steps},
           "speedup_over_one_context_at_a_time": seq_ms_per_step / sched[best]["ms_per_step"],
           "speedup_persistent_over_grouped": sched["grouped"]["ms_per_step"] / sched["persistent"]["ms_per_step"],
           "run_to_convergence": {"tol_rad_per_s": 1e3, "check_every": 100, "max_steps": args.batch_max_steps,
                                  "device_ms": run_ms, "wall_s": wall,
                                  "value": cell_steps / (run_ms * 1e-3) if world == 1 else None,
                                  "steps_min": srt[0], "steps_median": srt[len(srt) // 2], "steps_max": srt[-1],
                                  "films_stopped_early": int(sum(1 for n in nsteps if n < args.batch_max_steps)),
                                  "max_dmdt_at_stop_median": float(np.median(final_dmdt))},
           "l2": "working set larger than L2 (no flush)"}
    return out

def bench_adjoint(args, reps=3):
    """Differentiation study: 128x128x4 film, 500 RK4 steps, checkpoint every 50; adjoint / forward time."""
    import torch
    from paper_1501_07293_b300 import inputs
    from paper_1501_07293_b300.solver import Solver
    w = inputs.film_128x128x4()
    mat = w.mat
    s = Solver(w.grid, w.delta, mat.Ms, mat.A, 0.0, mat.alpha, mat.gamma)
    h = torch.from_numpy(inputs.zeeman_map(w.grid, 5001)).cuda()
    ku = torch.from_numpy(inputs.ku_map(w.grid, 5002)).cuda()
    s.set_field((0.0, 0.0, 0.0), h, ku)
    m0 = torch.from_numpy(inputs.workload_state(w)).cuda()
    g = torch.full_like(m0, 1e-5)
    stream = torch.cuda.current_stream()
    budget = 2.0 * 2**30   # the second variant: 2 GiB of recorded segments
    fwd, adj, adjb = [], [], []
    for r in range(reps + 1):
        e = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
        s.set_m(m0)
        torch.cuda.synchronize()
        e[0].record(stream)
        s.step(w.steps, w.dt)
        e[1].record(stream)
        s.set_adjoint_memory(0)
        s.set_m(m0)
        e[2].record(stream)
        s.adjoint(w.steps, w.dt, 50, g)
        e[3].record(stream)
        s.set_adjoint_memory(budget)
        s.set_m(m0)
        e[4].record(stream)
        s.adjoint(w.steps, w.dt, 50, g)
        e[5].record(stream)
        torch.cuda.synchronize()
        if r:   # first round warms up (graph capture, workspace allocation)
            fwd.append(e[0].elapsed_time(e[1]))
            adj.append(e[2].elapsed_time(e[3]))
            adjb.append(e[4].elapsed_time(e[5]))
    s.close()
    f, a, ab = statistics.median(fwd), statistics.median(adj), statistics.median(adjb)
    nx, ny, nz = w.grid
    slot = 12 * (8 * 50 + 1) * nx * ny * nz
    nseg = (w.steps + 49) // 50
    rec = max(1, min(8, nseg, int(budget // slot)))
    return {"workload": "film_128x128x4, 500 RK4 steps, checkpoint every 50, gradients w.r.t. m0, h, Ku",
            "forward_ms": f, "adjoint_ms": a, "adjoint_over_forward": a / f,
            "note": "adjoint time includes its own forward pass with checkpoints and the recomputation "
                    "of every segment but the last",
            "with_recording_budget": {"budget_bytes": budget, "segments_recorded": rec, "segments_recomputed": nseg - rec,
                                      "adjoint_ms": ab, "adjoint_over_forward": ab / f,
                                      "note": "mm_set_adjoint_memory: the forward pass keeps the stage data of its "
                                              "last segments; the gradients are bitwise the same"}}


def bench_sp4(args, sample_every=1000):
    """The paper's validation run: standard problem 4 on 166x42x1 cells of 3 nm in
    the paper's mode (explicit Euler at dt = 5 fs, tensor without the self offset),
    the full 150,000-step protocol as a device field program, <m> recorded every
    1000 steps inside the step graph (obs_every), no host round trip in the run."""
    import torch
    from paper_1501_07293_b300 import inputs
    from paper_1501_07293_b300.solver import Solver
    w = inputs.sp4_film()
    mat = w.mat
    s = Solver(w.grid, w.delta, mat.Ms, mat.A, mat.Ku, mat.alpha, mat.gamma, integrator="euler",
               self_term=False, obs_every=sample_every)
    m0 = torch.from_numpy(inputs.workload_state(w)).cuda()
    s.set_m(m0)
    s.set_program(inputs.sp4_schedule(w.dt))
    s.step(1, w.dt)   # graph capture
    s.set_m(m0)
    s.set_time(0.0)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = s.launch_count()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e0.record(stream)
    s.step(w.steps, w.dt)
    e1.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    ms = e0.elapsed_time(e1)
    rec = s.series()
    means = rec[:, 2:5]
    out = {"workload": "muMAG standard problem 4 protocol, 166x42x1 cells of 3 nm, Euler dt 5 fs, "
                       "150,000 steps, self offset skipped (paper mode), <m> every 1000 steps on the device",
           "steps": w.steps, "ms_per_step": ms / w.steps, "wall_s": wall, "records": int(rec.shape[0]),
           "value": w.ncells * w.steps / (ms * 1e-3), "unit": UNIT,
           "gpu_launches": s.launch_count() - l0,
           "mean_m_at_50000_steps": means[50000 // sample_every - 1].tolist(),
           "mean_m_final": means[-1].tolist()}
    s.close()
    return out

def bench_split(args, fp32_ms, steps=30, warmup=3):
    """The split-precision forms (tensor-core z DFT with BF16 / FP16 hi+lo operands):
    RK4 step time at 256x256x16 under the main protocol, the effective field's
    relative L2 distance from the FP32 path, and the precision study (512x512x8
    vortex, RK4): along 20 FP32 steps, the split field's distance from the FP32
    field at every step's state."""
    import torch
    from paper_1501_07293_b300 import inputs
    from paper_1501_07293_b300.solver import Solver
    w = inputs.film_256x256x16()
    mat = w.mat
    m0 = torch.from_numpy(inputs.workload_state(w)).cuda()
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    ref = Solver(w.grid, w.delta, mat.Ms, mat.A, mat.Ku, mat.alpha, mat.gamma)
    ref.set_field(w.b_ext)
    ref.set_m(m0)
    H32 = ref.heff(15).double()
    ref.close()
    out = {"workload": w.name, "fp32_ms_per_step": fp32_ms}
    for prec in ("split_bf16", "split_fp16"):
        s = Solver(w.grid, w.delta, mat.Ms, mat.A, mat.Ku, mat.alpha, mat.gamma, precision=prec)
        s.set_field(w.b_ext)
        s.set_m(m0)
        H = s.heff(15).double()
        err = float(torch.linalg.norm(H - H32) / torch.linalg.norm(H32))
        s.set_m(m0)
        for _ in range(warmup):
            flush.zero_()
            s.step(1, w.dt)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        torch.cuda.synchronize()
        for k in range(steps):
            flush.zero_()
            ev[k][0].record(stream)
            s.step(1, w.dt)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in ev) / steps
        kt = s.step_timed(5, w.dt)
        out[prec] = {"ms_per_step": ms, "value": w.ncells / (ms * 1e-3), "unit": UNIT,
                     "speedup_vs_fp32": fp32_ms / ms, "yz_ms_per_launch": kt[1] / 20,
                     "heff_rel_l2_vs_fp32": err}
        s.close()
    # precision study (512x512x8 vortex): along 20 FP32 RK4 steps, at every step's
    # state, the FP32 and split fields against the FP64 oracle at 42 sampled cells
    # (eq. 13 at each cell plus the eq. 5/7 exchange field; Ku and the applied
    # field are zero), and the split fields against the FP32 field everywhere
    from oracle import to_xyz
    from oracle.demag import demag_at_cells
    from oracle.exchange import exchange_field
    from oracle.tensor import demag_tensor
    w3 = inputs.film_512x512x8()
    nx, ny, nz = w3.grid
    m3 = torch.from_numpy(inputs.workload_state(w3)).cuda()
    f32 = Solver(w3.grid, w3.delta, w3.mat.Ms, w3.mat.A, w3.mat.Ku, w3.mat.alpha, w3.mat.gamma)
    sp = {p: Solver(w3.grid, w3.delta, w3.mat.Ms, w3.mat.A, w3.mat.Ku, w3.mat.alpha, w3.mat.gamma, precision=p)
          for p in ("split_bf16", "split_fp16")}
    K = demag_tensor(*w3.grid, delta=w3.delta)
    rng = np.random.default_rng(3008)
    cells = sorted({(0, 0, 0), (nx - 1, ny - 1, nz - 1), (nx // 2, ny // 2, 0), (nx // 2, ny // 2, nz - 1),
                    (0, ny // 2, nz // 2), (nx - 1, 0, 0)} |
                   {(int(rng.integers(nx)), int(rng.integers(ny)), int(rng.integers(nz))) for _ in range(36)})
    f32.set_m(m3)
    vs_fp32 = {p: [] for p in sp}
    vs_oracle = {p: [] for p in ["fp32"] + list(sp)}
    for step in range(20):
        state = f32.get_m()
        Hr = f32.heff(15).double()
        f32.set_m(state)
        mo = to_xyz(state.cpu().numpy())
        Hex = exchange_field(mo, w3.mat.Ms, w3.mat.A, w3.delta)
        Ho = demag_at_cells(mo, w3.mat.Ms, cells, K=K) + np.array([Hex[:, i, j, k] for (i, j, k) in cells])
        fields = {"fp32": Hr}
        for p, sv in sp.items():
            sv.set_m(state)
            fields[p] = sv.heff(15).double()
            vs_fp32[p].append(float(torch.linalg.norm(fields[p] - Hr) / torch.linalg.norm(Hr)))
        for p, H in fields.items():
            Hc = H.cpu().numpy()
            Hg = np.array([[Hc[a, k, j, i] for a in range(3)] for (i, j, k) in cells])
            vs_oracle[p].append(float(np.linalg.norm(Hg - Ho) / np.linalg.norm(Ho)))
        f32.step(1, w3.dt)
    out["precision_study_512x512x8"] = {
        "steps": 20, "oracle_cells": len(cells),
        "heff_rel_l2_vs_fp64_oracle_sampled": {p: {"per_step": e, "max": max(e)} for p, e in vs_oracle.items()},
        "heff_rel_l2_vs_fp32_path": {p: {"max": max(e), "mean": sum(e) / len(e)} for p, e in vs_fp32.items()}}
    f32.close()
    for sv in sp.values():
        sv.close()
    # trajectory error: 20 RK4 steps of a 128x128x8 copy of the vortex film (same
    # material and recipe), each precision against the FP64 oracle's trajectory
    from oracle.llg import Film
    grid_s = (128, 128, 8)
    ms = inputs.initial_state("vortex", grid_s, 3008)
    film = Film(grid_s, w3.delta, w3.mat.Ms, w3.mat.A, w3.mat.Ku, w3.mat.alpha, w3.mat.gamma)
    mo20 = film.run(to_xyz(ms), w3.dt, 20, "rk4")
    traj = {}
    for p in ("fp32", "split_bf16", "split_fp16"):
        sv = Solver(grid_s, w3.delta, w3.mat.Ms, w3.mat.A, w3.mat.Ku, w3.mat.alpha, w3.mat.gamma, precision=p)
        sv.set_m(torch.from_numpy(ms).cuda())
        sv.step(20, w3.dt)
        mg = to_xyz(sv.get_m().cpu().numpy())
        traj[p] = {"max_abs_state_error_after_20_steps": float(np.abs(mg - mo20).max())}
        sv.close()
    out["trajectory_128x128x8_vs_fp64_oracle"] = traj
    return out


def bench_noalloc(args, reps=20):
    """mm_heff_noalloc (tensor set-up + one field evaluation, no allocation) against
    mm_heff on a context (tensor built once at creation), 128 x 128 x 4, CUDA events."""
    import torch
    from paper_1501_07293_b300 import inputs
    from paper_1501_07293_b300.solver import Solver, TERM_ALL, heff_noalloc, noalloc_status
    w = inputs.film_128x128x4()
    mat = w.mat
    m = torch.from_numpy(inputs.workload_state(w)).cuda()
    s = Solver(w.grid, w.delta, mat.Ms, mat.A, mat.Ku, mat.alpha, mat.gamma)
    s.set_m(m)
    mn = s.get_m().clone()
    H = torch.empty_like(mn)
    stream = torch.cuda.current_stream()

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    ctx_ms = timed(lambda: s.heff(TERM_ALL, out=H))
    na_ms = timed(lambda: heff_noalloc(w.grid, w.delta, mat.Ms, mat.A, mat.Ku, (0, 0, 0), mn, H))
    noalloc_status()
    s.close()
    return {"workload": "128x128x4 effective field", "mm_heff_ms": ctx_ms, "mm_heff_noalloc_ms": na_ms,
            "note": "mm_heff_noalloc rebuilds the FP64 tensor on every call"}


def bench_cufft(args, ours_ms_per_stage, reps=20):
    """Timed comparison only: the demagnetising convolution of one field evaluation as
    a library pipeline -- cuFFT (through torch.fft) R2C of the three zero-padded
    components on the px x py x 2nz grid, the 3x3 symmetric product with six
    spectral tensor components, C2R of the three results -- against one stage of
    our kernels (k_yz + k_x, which also do the exchange/anisotropy/Zeeman/LLG/RK4
    work and the next x transform).  The tensor values do not change the cost,
    so random spectra of the right shape stand in for them."""
    import torch
    from paper_1501_07293_b300 import inputs
    w = inputs.film_256x256x16()
    nx, ny, nz = w.grid
    px, py, pz = 2 * nx, 2 * ny, 2 * nz
    g = torch.Generator(device="cuda").manual_seed(7)
    M = torch.zeros(3, px, py, pz, device="cuda")
    M[:, :nx, :ny, :nz] = torch.randn(3, nx, ny, nz, device="cuda", generator=g)
    K = torch.randn(6, px, py, pz // 2 + 1, device="cuda", generator=g)   # xx yy zz xy xz yz
    pairs = [[0, 3, 4], [3, 1, 5], [4, 5, 2]]
    stream = torch.cuda.current_stream()

    def conv():
        Mh = torch.fft.rfftn(M, dim=(1, 2, 3))
        H = [sum(K[pairs[a][b]] * Mh[b] for b in range(3)) for a in range(3)]
        return torch.fft.irfftn(torch.stack(H), s=(px, py, pz), dim=(1, 2, 3))[:, :nx, :ny, :nz]

    for _ in range(3):
        conv()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        conv()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    return {"workload": f"demag convolution of {w.name}, padded {px}x{py}x{pz}, cuFFT via torch.fft",
            "cufft_pipeline_ms_per_field_eval": ms, "ours_ms_per_stage": ours_ms_per_stage,
            "ours_speedup": ms / ours_ms_per_stage,
            "note": "timed comparison only; not on any product path"}


TABLE1_GPU_SINGLE_MS = {8: 22.58, 16: 23.97, 32: 26.89, 64: 76.24}   # the paper's Table 1 (GTX 650 Ti)


def bench_sp3(args, steps=500, warmup=20):
    """Table 1's shapes: per-step time of explicit Euler on the standard-problem-3
    cube, n = 8 .. 64, graph replays, working set resident in L2 (as in the
    paper's steady-state loop).  The paper's GTX 650 Ti numbers are context."""
    import torch
    from paper_1501_07293_b300 import inputs
    from paper_1501_07293_b300.solver import Solver
    from paper_1501_07293_b300.tune import autotune
    stream = torch.cuda.current_stream()
    rows = []
    for n in (8, 16, 32, 64, 128):
        w = inputs.sp3_cube(n)
        mat = w.mat
        s = Solver(w.grid, w.delta, mat.Ms, mat.A, mat.Ku, mat.alpha, mat.gamma, integrator="euler")
        s.set_m(torch.from_numpy(inputs.workload_state(w)).cuda())
        tuned = autotune(s, w.dt)   # the y/z launch shape for this size (fused or split, ky block)
        s.step(warmup, w.dt)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        s.step(steps, w.dt)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        rows.append({"n": n, "ms_per_step": ms, "cell_steps_per_s": n ** 3 / (ms * 1e-3),
                     "yz_route": "fused" if tuned["yz_route"] == 1 else f"split, ky block {s.tuning()[1]}",
                     "paper_gtx650ti_single_ms": TABLE1_GPU_SINGLE_MS.get(n)})
        s.close()
    return {"workload": "muMAG standard problem 3 cube n^3, Euler, FP32, one field evaluation per step",
            "steps": steps, "rows": rows}


def b300_arm(args, w):
    import torch
    import torch.distributed as dist

    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1501_07293_b300 import inputs
    from paper_1501_07293_b300.solver import Solver

    mat = w.mat
    # set-up: the FP64 tensor (eq. 10/11 near the source, its multipole series
    # beyond 12 cells) and its FP64 transforms; mm_create synchronises
    torch.cuda.synchronize()
    t_setup0 = time.perf_counter()
    s = Solver(w.grid, w.delta, mat.Ms, mat.A, mat.Ku, mat.alpha, mat.gamma, precision=args.precision)
    setup_ms = 1e3 * (time.perf_counter() - t_setup0)
    s.set_field(w.b_ext)
    m0 = inputs.workload_state(w)
    m0_dev = torch.from_numpy(m0).cuda()
    s.set_m(m0_dev)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            dist.barrier()

    def max_over_ranks(v):
        if world == 1:
            return v
        t = torch.tensor([v], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    # warm-up (graph capture happens on the first step)
    for _ in range(max(args.warmup, 0)):
        flush.zero_()
        s.step(1, w.dt)
    torch.cuda.synchronize()

    # ---- timed region: K steps, L2 flushed between steps (outside the events) ----
    K = args.steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    launches0 = s.launch_count()
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t_wall0 = time.perf_counter()
        for k in range(K):
            flush.zero_()
            ev[k][0].record(stream)
            s.step(1, w.dt)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall0
    barrier()
    launches = s.launch_count() - launches0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_dev = sum(step_ms) / 1e3
    t_max = max_over_ranks(t_dev)
    value = world * w.ncells * K / t_max
    s.sync()

    # ---- per-kernel device times (event-bracketed eager replay of the same steps) ----
    kt = np.zeros(3)
    nk = min(K, 10)
    for _ in range(nk):
        flush.zero_()
        torch.cuda.synchronize()
        kt += s.step_timed(1, w.dt)
    per_launch_ms = {"yz": kt[1] / (4 * nk), "x": kt[2] / (4 * nk)}
    names = ["yz", "x"]
    kernels = {"yz": "k_yz", "x": "k_x"}
    alg = algorithmic_bytes(w.grid)
    meth = method_bytes(w.grid)
    ncell = w.ncells
    # the method's bytes per launch of each kernel class: y/z = pass a2; x = pass a3
    # plus the spectrum write of the next stage's x transform (a1 without its read
    # of m, which this implementation takes from registers)
    mb = {"yz": meth["a2"], "x": meth["a3"] + meth["a1"] - 12 * ncell}
    flops = algorithmic_flops(w.grid)
    dom = max(names, key=lambda n: per_launch_ms[n])
    peak, peak_kind = measured_peaks()
    # FP32 ceiling: measured by the library's FMA-chain probe on this device
    from paper_1501_07293_b300.solver import fp32_probe_tflops
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    fp32 = {"scalar_fma_tflops": fp32_probe_tflops(False, 1 << 12),
            "packed_fma2_tflops": fp32_probe_tflops(True, 1 << 12),
            "sms": sms, "derived_tflops": derived_fp32_tflops(sms)}
    fp32_peak = max(fp32["scalar_fma_tflops"], fp32["packed_fma2_tflops"])
    kernel_table = {}
    for n in names:
        t = per_launch_ms[n] * 1e-3
        kernel_table[n] = {"ms_per_launch": float(per_launch_ms[n]),
                           "method_bytes": float(mb[n]), "impl_bytes": float(alg[n]),
                           "alg_flops": float(flops[n]), "GBps": float(mb[n] / t / 1e9),
                           "TFLOPs": float(flops[n] / t / 1e12),
                           "hbm_frac": float(mb[n] / t / 1e9 / peak),
                           "alu_frac": float(flops[n] / t / 1e12 / fp32_peak),
                           "hbm_floor_ms": float(mb[n] / (peak * 1e9) * 1e3),
                           "alu_floor_ms": float(flops[n] / (fp32_peak * 1e12) * 1e3)}
    kd = kernel_table[dom]
    roofline = {"bound": "hbm", "kernel": kernels[dom], "achieved": kd["GBps"], "peak": peak,
                "peak_kind": peak_kind, "unit": "GB/s", "frac": kd["hbm_frac"],
                "traffic": stored_traffic(kernels[dom]),
                "bytes_per_launch": kd["method_bytes"],
                "bytes_model": "the method's pass a2 (y/z + product): read and write the half spectrum, "
                               "read the tensor octant",
                "alu": {"achieved": kd["TFLOPs"], "peak": fp32_peak, "unit": "TFLOP/s", "frac": kd["alu_frac"],
                        "peak_kind": "measured (FMA-chain probe, the faster of scalar and packed)",
                        "flops_per_launch": kd["alg_flops"]}}

    # ---- end to end through the C ABI with host buffers ----
    m_host = torch.from_numpy(m0.copy()).pin_memory()
    out_host = torch.empty_like(m_host).pin_memory()
    Ke = min(K, 20)
    eve = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(Ke)]
    torch.cuda.synchronize()
    for k in range(Ke):
        flush.zero_()
        eve[k][0].record(stream)
        s.set_m(m_host)                # host -> device (pinned), normalise
        s.step(1, w.dt)
        s.get_m(out_host)              # device -> host (pinned)
        eve[k][1].record(stream)
    torch.cuda.synchronize()
    t_e2e = max_over_ranks(sum(a.elapsed_time(b) for a, b in eve) / 1e3)
    e2e = world * w.ncells * Ke / t_e2e
    nbytes = 3 * w.ncells * 4

    extra = {}
    want = set() if args.no_extras else (
        {"batched", "adjoint", "sp4", "sp3", "split", "cufft", "noalloc"} if args.extras == "all"
        else set(args.extras.split(",")))
    if "batched" in want:
        extra["batched"] = bench_batched(args)   # every rank: the films are sharded
    if rank == 0:                                # single-GPU measurements: rank 0 only
        if "adjoint" in want:
            extra["adjoint"] = bench_adjoint(args)
        if "sp4" in want:
            extra["sp4_protocol"] = bench_sp4(args)
        if "sp3" in want:
            extra["sp3_table1"] = bench_sp3(args)
        if "split" in want:
            extra["split_precision"] = bench_split(args, 1e3 * t_max / K)
        if "cufft" in want:
            extra["cufft_comparison"] = bench_cufft(args, float(per_launch_ms["yz"] + per_launch_ms["x"]))
        if "noalloc" in want:
            extra["noalloc"] = bench_noalloc(args)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        val, cores, wall, n, util = time_oracle(w, 2, 0)
        cpu = {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{n} RK4 steps of the full {w.grid[0]}x{w.grid[1]}x{w.grid[2]} film, "
                         f"FP64 numpy/scipy oracle (FFTs on {cores} cores, mean utilisation "
                         f"{util:.1f} cores), {wall:.1f} s"}

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_max / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "grid": list(w.grid), "delta_m": w.delta, "integrator": "rk4",
                       "dt_s": w.dt, "variant": args.precision,
                       "l2": "flushed between timed steps (512 MiB write outside the events)",
                       "parallelism": "replicas" if world > 1 else "single"},
            "roofline": roofline,
            "kernels": kernel_table,
            "step_fraction_of_hbm_roofline": (4 * meth["eval"] * K / t_max / 1e9) / peak,   # per GPU
            "step_bytes_per_cell": 4 * meth["eval"] / ncell,
            "fp32_peak": fp32,
            "setup_ms": setup_ms,
            "wall_s_timed_region": t_wall,
            "clocks": clk.summary(),
            "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
                    "path": "mm_set_m(pinned host) + mm_step(1) + mm_get_m(pinned host)"},
            "gpu_launches": launches,
            "cpu_baseline": cpu,
            **extra,
        }
        print(json.dumps(out), flush=True)
    s.close()
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse_args()
    from paper_1501_07293_b300 import inputs
    w = inputs.WORKLOADS[args.workload]
    if args.impl == "reference":
        reference_arm(args, w)
    else:
        b300_arm(args, w)


if __name__ == "__main__":
    main()
