#!/usr/bin/env python
"""Benchmark of the GB300 J-FFT solver on the 2D 1024 x 1024 workload.

Workload (one "step" = one pass of the whole path over the sweep):
  2D plane-strain periodic cell, 1024 x 1024 bilinear quads with 4 Gauss points, FP64;
  density from 16 random Fourier modes with |k| <= 8 (seed 0), affinely mapped to
  [0, 1]; E = E_min + (1 - E_min) rho^2 with contrast 1/E_min in {1e2, 1e4, 1e6};
  nu = 0.3; C_ref = mean material; the three Mandel unit load cases, solved as one
  batch with per-load convergence; Green-Jacobi and Green; relative residual 1e-8.
  Per contrast: material setup (E, J^1/2, Alg. 1 symbol) + one Green-Jacobi solve
  and one Green solve of the three loads -> 18 PCG solves per step.

value: solves/s with the density field resident in HBM and outputs written to
device buffers; e2e: the same through the C ABI with host buffers (pinned), the
host->device copy of the density and the device->host read of u, C_hom, iteration
counts and residuals inside the timed region.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank runs an independent replica (the path has no
exchange step), rank 0 prints one JSON line with the max-over-ranks time.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

SHAPE = (1024, 1024)
MODES, KMAX, SEED = 16, 8.0, 0
EXPONENT, NU, TOL = 2.0, 0.3, 1e-8
CONTRASTS = (1e2, 1e4, 1e6)
PRECONDS = ("green_jacobi", "green")
N_LOADS = 3
METRIC = "PCG solves/s"
WORKLOAD = ("2D plane-strain periodic cell, 1024x1024 Q1 quads (4 Gauss points), FP64; smooth density "
            "(16 Fourier modes, |k|<=8), E = 1/c + (1-1/c) rho^2, c in {1e2,1e4,1e6}, nu 0.3, C_ref mean; "
            "3 Mandel unit loads; Green-Jacobi and Green PCG to 1e-8 relative residual")
PROFILED_STEPS = 1   # steps of the per-kernel profiling pass after the timed steps
FP64_PEAK_TFLOPS = 152 * 2.070e9 * 4 / 1e12   # SMs x max clock x FP64 flop/clk/SM (2 DFMA)
ITER_COUNTS = os.path.join(ROOT, "oracle", "data", "iters_2d_1024.json")


def hbm_peak_gbs():
    """Measured HBM copy bandwidth of this machine (MEASURED_PEAKS.json), else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# ----------------------------------------------------------------- helpers
def env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, power, reasons = [], [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
                power.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None, "samples": len(sm), "reasons": sorted(reasons)}


def flops_per_unit(kernel, shape, d=2):
    kernel = kernel[:-4] if kernel.endswith("_f32") else kernel
    """Algorithmic FLOPs of one kernel for one load case (one right-hand side).

    FFT passes use the conventional 5 L log2 L per complex transform of length L
    (2.5 n log2 n for a real transform of length n); the symbol block multiply of a
    real symmetric d x d block by a complex vector costs 2 d^2 mults + 2 d (d-1)
    adds per frequency; J^1/2 scalings one multiply per real value. The Q1 operator
    counts the flops of its Walsh-Hadamard mode form (74 per node in 2D, see the
    design notes), FMA = 2 flops."""
    n0, n1 = shape
    N = n0 * n1
    M = n1 // 2
    F = n0 * (M + 1)
    if kernel == "fft_lines":
        return d * (M + 1) * 2 * 5 * n0 * math.log2(n0) + F * (2 * d * d * 2 + 2 * d * (d - 1))
    if kernel == "fft_rows_real_fwd":
        return d * n0 * 2.5 * n1 * math.log2(n1) + d * N          # + J^1/2 scaling
    if kernel == "fft_cols_real_inv":
        return d * n0 * 2.5 * n1 * math.log2(n1) + 3 * d * N      # + J^1/2 scaling and r.z
    if kernel == "apply_K":
        return 74 * N + 2 * d * N                                  # operator + fused p.q
    return None


def traffic_bytes_per_unit(kernel, shape, d=2):
    """Compulsory DRAM bytes of one kernel for one load case; kernels whose name ends in
    _f32 move FP32 data (s = 4 bytes per real), the others FP64 (s = 8)."""
    s = 4 if kernel.endswith("_f32") else 8
    k = kernel[:-4] if kernel.endswith("_f32") else kernel
    n0, n1 = shape
    N = n0 * n1
    F = n0 * (n1 // 2 + 1)
    table = {
        "fft_lines": 2 * d * F * 2 * s + F * 3 * s,              # spectrum in + out, symbol table
        "fft_rows_real_fwd": d * N * s + d * F * 2 * s + N * s,   # r, spectrum, J^1/2 scale
        "fft_cols_real_inv": d * F * 2 * s + 2 * d * N * s + N * s,   # spectrum, z, r (dot), scale
        "apply_K": 2 * d * N * s + N * s,                         # p, q, E
        "cg_xr": 6 * d * N * s,                                   # x, r read+write, p, q
        "cg_p": 3 * d * N * s,                                    # p read+write, z
    }
    return table.get(k)


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch with all three
# loads active, from the ncu capture summarised in profiles/fp64_2d_1024_gj_kernels.md
# (1024 x 1024, Green-Jacobi, contrast 1e4), for kernels unchanged since that capture; the
# FP32 kernels have no capture of all three loads active (their traffic stays null).
NCU_TRAFFIC_PER_LAUNCH = {"fft_lines": 63.11e6 + 0.93e6, "apply_K": 59.86e6 + 11.20e6,
                          "fft_cols_real_inv": 110.95e6 + 25.91e6, "fft_rows_real_fwd": 59.18e6 + 13.78e6}


def aggregate(ms_local, world, solves_per_step, dist=None, device=None):
    """Whole-job throughput of N independent replicas: every rank ran the same
    per-rank workload; the job time is the slowest rank's time (max over ranks, the
    only collective), value = N x solves per step / that time. Returns (ms, value)."""
    ms = float(ms_local)
    if dist is not None and world > 1:
        import torch
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, world * solves_per_step / (ms / 1e3)


# ----------------------------------------------------------------- CPU side
def cpu_sample(seconds_budget=25.0):
    """Time the oracle as it stands on a bounded sample of the workload (single process).

    Sample: oracle setup (assembled sparse K, Alg. 1 symbol, diagonal) at 1024 x 1024
    for contrast 1e4, the right-hand side and post-processing of one load, and a few
    Green-Jacobi and Green PCG iterations on that load."""
    from oracle import assemble, material, pcg, post, solve as osolve
    from synthetic import smooth_density
    rho = smooth_density(SHAPE, MODES, KMAX, SEED)
    E = material.young_from_density(rho, 1e-4, 1.0, EXPONENT)
    t0 = time.perf_counter()
    prob = osolve.setup(SHAPE, E, NU)
    t_setup = time.perf_counter() - t0
    eps = np.eye(3)[0]
    t0 = time.perf_counter()
    f = assemble.assemble_rhs(SHAPE, E, prob.C, eps)
    t_rhs = time.perf_counter() - t0
    per_it = {}
    for pc in PRECONDS:
        k = 3
        t0 = time.perf_counter()
        res = pcg.pcg(prob.apply_K, prob.minv(pc), f, 0.0, k)
        per_it[pc] = (time.perf_counter() - t0) / k
    t0 = time.perf_counter()
    u = post.remove_mean(res.x)
    post.element_stress(SHAPE, E, prob.C, eps, u)
    post.homogenised_stress(SHAPE, E, prob.C, eps, u)
    np.linalg.norm(f - prob.apply_K(u))
    t_post = time.perf_counter() - t0
    return {"t_setup": t_setup, "t_rhs": t_rhs, "t_iter": per_it, "t_post": t_post}


def cpu_extrapolate(sample, iters):
    """Seconds for one step (the 18 solves) from the sampled costs and iteration counts
    iters[(contrast, precond)] = list of per-load counts."""
    total = len(CONTRASTS) * sample["t_setup"]
    for (c, pc), its in iters.items():
        total += sum(sample["t_rhs"] + n * sample["t_iter"][pc] + sample["t_post"] for n in its)
    return total


def oracle_iteration_counts():
    with open(ITER_COUNTS) as fh:
        rows = json.load(fh)["solves"]
    out = {}
    for r in rows:
        if r.get("symbol", "alg1") != "alg1":
            continue
        out.setdefault((r["contrast"], r["precond"]), [0, 0, 0])[r["load"]] = r["iters"]
    return out


def run_cpu_sample_subprocess():
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = "import json, bench; print('CPUSAMPLE ' + json.dumps(bench.cpu_sample()))"
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, stdout=subprocess.PIPE,
                       stderr=subprocess.PIPE, text=True, timeout=900)
    for line in r.stdout.splitlines():
        if line.startswith("CPUSAMPLE "):
            return json.loads(line[len("CPUSAMPLE "):])
    raise RuntimeError("oracle sample failed: " + r.stderr[-2000:])


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], stdout=subprocess.PIPE, text=True).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


# ----------------------------------------------------------------- reference arm
def reference_arm(args):
    rank = env_int("RANK", 0)
    if rank != 0:
        return 0
    iters = oracle_iteration_counts()
    for _ in range(args.warmup):
        pass  # the oracle has no warm-up state; samples below are independent
    secs = []
    samples = []
    for _ in range(args.steps):
        s = run_cpu_sample_subprocess()
        samples.append(s)
        secs.append(cpu_extrapolate(s, iters))
    step_s = statistics.mean(secs)
    value = len(CONTRASTS) * len(PRECONDS) * N_LOADS / step_s
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": list(SHAPE), "contrasts": list(CONTRASTS),
                   "preconditioners": list(PRECONDS), "loads": N_LOADS, "tol": TOL},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": 1, "kind": "oracle",
                         "sample": ("per step: oracle setup at 1024x1024 (contrast 1e4), one load's rhs and "
                                    "post-processing, 3 Green-Jacobi and 3 Green iterations; scaled to the 18 "
                                    "solves with the oracle's own iteration counts (oracle/data/iters_2d_1024.json)"),
                         "cpu": cpu_model()},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------- GPU arm
def main():
    global CONTRASTS, PRECONDS
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--contrasts", default=",".join(f"{c:g}" for c in CONTRASTS),
                    help="subset of the contrast sweep (profiling runs)")
    ap.add_argument("--preconds", default=",".join(PRECONDS), help="subset of the preconditioners (profiling runs)")
    ap.add_argument("--legs", default="fp64,mixed", help="precision legs to run (profiling runs)")
    ap.add_argument("--no-cells", action="store_true", help="skip the small-cell batch leg")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving leg")
    ap.add_argument("--no-bf16", action="store_true", help="skip the BF16-material variant of the mixed leg")
    ap.add_argument("--no-graphs", action="store_true",
                    help="launch every kernel from the host (profilers cannot see kernels inside conditional graphs)")
    ap.add_argument("--serving-requests", type=int, default=40,
                    help="requests of the seeded serving stream to replay (the full stream has 2000)")
    args = ap.parse_args()
    CONTRASTS = tuple(float(c) for c in args.contrasts.split(","))
    PRECONDS = tuple(args.preconds.split(","))
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return reference_arm(args)

    rank, world, local = env_int("RANK", 0), env_int("WORLD_SIZE", 1), env_int("LOCAL_RANK", 0)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = run_cpu_sample_subprocess()   # before any CUDA call in this process

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    import __graft_entry__
    __graft_entry__.build()
    from paper_2508_02613_gb300.jfft import Solver
    from synthetic import smooth_density

    stream = torch.cuda.current_stream()
    rho_h = smooth_density(SHAPE, MODES, KMAX, SEED)
    rho_d = torch.tensor(rho_h, device="cuda")
    eps_h = np.eye(3)
    eps_d = torch.tensor(eps_h, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    uuid = str(getattr(torch.cuda.get_device_properties(local), "uuid", ""))
    smi_id = ("GPU-" + uuid) if uuid and not uuid.startswith("GPU-") else (uuid or local)
    solves_per_step = len(CONTRASTS) * len(PRECONDS) * N_LOADS

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
            torch.cuda.synchronize()

    def run_leg(precision, material_bf16=False, light=False):
        """Warm-up, one recording pass (iterations, time to tolerance per solve call),
        then the timed steps with per-kernel CUDA events and clock sampling (light: one
        warm-up and the timed steps only, no per-kernel events)."""
        s = Solver(SHAPE, rho_h, NU, kind="density", e_min=1.0 / CONTRASTS[0], e_max=1.0, exponent=EXPONENT,
                   stream=stream.cuda_stream, io="device", max_loads=N_LOADS, precision=precision,
                   graphs=not args.no_graphs, autotune=True, material_bf16=material_bf16)

        def step(record=None):
            for c in CONTRASTS:
                s.set_material(rho_d, e_min=1.0 / c)
                for pc in PRECONDS:
                    if record is not None:
                        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                        e0.record(stream)
                    out = s.solve(eps_d, TOL, pc, want_stress=False)
                    if record is not None:
                        e1.record(stream)
                        e1.synchronize()
                        record[(c, pc)] = {"iters": [int(v) for v in out["iters"].cpu().tolist()],
                                           "refine": [int(v) for v in out["refine_steps"].cpu().tolist()],
                                           "rel_res": [float(v) for v in out["rel_res"].cpu().tolist()],
                                           "ms": e0.elapsed_time(e1)}

        for _ in range(1 if light else args.warmup):
            step()
        barrier()
        rec = {}
        step(rec)
        barrier()
        clocks = ClockSampler(smi_id)
        clocks.start()
        n0 = s.launch_count
        r0 = s.graph_replays
        times = []
        for _ in range(args.steps):
            flush.fill_(1.0)   # L2 flush (256 MiB > 129 MB L2), outside the timed interval
            barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            barrier()
            times.append(e0.elapsed_time(e1))
        launches = s.launch_count - n0
        replays = s.graph_replays - r0
        tuning = s.tuning
        clk = clocks.stop()
        if light:
            s.close()
            ms, value = aggregate(statistics.mean(times), world, solves_per_step, dist, "cuda")
            return {"ms": ms, "value": value, "times": times, "rec": rec, "launches": launches, "clocks": clk}
        # Per-kernel durations: one more step with a CUDA event pair around every kernel
        # launch (the PCG chunk then runs as a replayed graph with event nodes instead of
        # the device-side loop, which cannot hold event nodes).
        s.set_profiling(True)
        prof_times = []
        for _ in range(PROFILED_STEPS):
            flush.fill_(1.0)
            barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            barrier()
            prof_times.append(e0.elapsed_time(e1))
        prof = s.profile()
        s.set_profiling(False)
        s.close()
        ms, value = aggregate(statistics.mean(times), world, solves_per_step, dist, "cuda")
        return {"ms": ms, "value": value, "times": times, "rec": rec, "prof": prof, "launches": launches,
                "graph_replays": replays, "profiled_step_ms": prof_times, "tuning": tuning,
                "clocks": clk}

    def roofline(leg, alu):
        """Dominant kernel with its achieved rate, from the per-kernel CUDA events of the
        profiling pass that repeats the timed steps. Units are right-hand-side applications:
        per load, one operator and one preconditioner per PCG iteration."""
        n_units = sum(sum(r["iters"]) for r in leg["rec"].values()) * PROFILED_STEPS
        rows = sorted(((k, v[0], v[1]) for k, v in leg["prof"].items()), key=lambda r: -r[2])
        total_ms = sum(r[2] for r in rows)
        peak_gbs, peak_kind = hbm_peak_gbs()
        for name, nl, tot in rows:
            byt = traffic_bytes_per_unit(name, SHAPE)
            fl = flops_per_unit(name, SHAPE)
            if byt is None or fl is None:
                continue
            out = {"kernel": name, "launches": nl, "avg_launch_ms": tot / nl, "share": tot / total_ms,
                   "traffic": None, "algorithmic_bytes_per_unit": byt, "units": n_units}
            if name in NCU_TRAFFIC_PER_LAUNCH:
                out["traffic"] = NCU_TRAFFIC_PER_LAUNCH[name]
                out["traffic_note"] = ("DRAM bytes of one 3-load launch (ncu); the algorithmic bytes of that "
                                       f"launch are {3 * byt:.4g} (L2 keeps part of the fields)")
            gbs = n_units * byt / (tot / 1e3) / 1e9
            tfl = n_units * fl / (tot / 1e3) / 1e12
            if alu:
                out.update({"bound": "alu", "achieved": tfl, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                            "frac": tfl / FP64_PEAK_TFLOPS, "hbm_GBps_algorithmic": gbs,
                            "peak_note": "FP64 ALU: 152 SMs x 2.07 GHz x 4 flop/clk/SM (probe: 1.197 TFLOP/s DFMA)"})
            else:
                out.update({"bound": "hbm", "achieved": gbs, "peak": peak_gbs, "unit": "GB/s", "frac": gbs / peak_gbs,
                            "peak_note": f"HBM copy bandwidth, {peak_kind} (burst)"})
            return out
        return None

    def cells_leg():
        """The 32 x 32 workload (16 modes |k| <= 4, seeds 0-9, E = 1e-4 + (1 - 1e-4) rho^2,
        nu 0.3, eps_xx, tolerance 1e-6) as a batch of 1520 cells (ten seeds x 152) in one
        launch per preconditioner, beside the same solves through one handle per cell."""
        from paper_2508_02613_gb300.jfft import Cells
        from synthetic import smooth_density
        shape, n_rep = (32, 32), 152
        rho10 = np.stack([smooth_density(shape, 16, 4.0, sd) for sd in range(10)])
        fields = np.concatenate([rho10] * n_rep)
        eps1 = np.array([[1.0, 0.0, 0.0]])
        cb = Cells(shape, max_cells=len(fields), max_loads=1, stream=stream.cuda_stream)
        single = Solver(shape, rho10[0], NU, kind="density", e_min=1e-4, e_max=1.0, exponent=2.0,
                        stream=stream.cuda_stream, max_loads=1)
        out = {"workload": "32x32, 16 modes |k|<=4, seeds 0-9 x 152 copies, contrast 1e4, rho^2, nu 0.3, eps_xx, tol 1e-6",
               "cells": len(fields), "dtype": "f64"}
        # FP64 flops per cell and PCG iteration (model): operator ~120 per element, two
        # packed complex 2D FFTs at 5 log2(N) per node each, symbol block 16, vectors 20
        flops_it = 32 * 32 * (120 + 2 * 5 * 10 + 16 + 20)
        for pc in ("green_jacobi", "green"):
            kw = dict(kind="density", e_min=1e-4, e_max=1.0, exponent=2.0)
            cb.solve(fields, NU, eps1, 1e-6, pc, **kw)
            ts = []
            for _ in range(3):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                res = cb.solve(fields, NU, eps1, 1e-6, pc, **kw)
                e1.record(stream)
                e1.synchronize()
                ts.append(e0.elapsed_time(e1))
            ms = statistics.mean(ts)
            its = res["iters"][:10, 0].tolist()
            t_single = []
            for sd in range(10):
                single.set_material(rho10[sd], e_min=1e-4)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                one = single.solve(eps1, 1e-6, pc, want_stress=False)
                e1.record(stream)
                e1.synchronize()
                t_single.append(e0.elapsed_time(e1))
            n_it = float(res["iters"].sum())
            out[pc] = {"solves_per_s": len(fields) / (ms / 1e3), "batch_ms": ms,
                       "us_per_solve": 1e3 * ms / len(fields), "iters_seeds_0_9": [int(v) for v in its],
                       "single_handle_ms_per_solve": statistics.mean(t_single),
                       "single_handle_iters": int(one["iters"][0]),
                       "batch_speedup": statistics.mean(t_single) / (ms / len(fields)),
                       "rel_res_max": float(res["rel_res"].max()),
                       "fp64_tflops_model": n_it * flops_it / (ms / 1e3) / 1e12,
                       "fp64_peak_tflops": FP64_PEAK_TFLOPS}
        cb.close()
        single.close()
        return out

    def serving_leg():
        """The serving stream: seeded requests with Poisson arrivals at 50/s, grids drawn from
        2D {256^2 .. 2048^2} and 3D {64^3, 128^3, 256^3}, contrast log-uniform in [1e2, 1e6],
        nu uniform in [0.2, 0.4], 1..d(d+1)/2 load cases, Green-Jacobi to 1e-8, mixed precision,
        replayed in real time into the request server (4 workers). One smooth field per grid
        (16 modes in 2D, 32 in 3D, |k| <= 8, seed 0; rho^2 in 2D, rho^3 in 3D) serves every
        request of that grid; contrast and nu vary per request. The first 8 requests are also
        solved one after another in plain FP64 (a new handle each, as a serial service would)."""
        from paper_2508_02613_gb300.jfft import Server
        from synthetic import smooth_density
        rng = np.random.default_rng(0)
        grids = [(256, 256), (512, 512), (1024, 1024), (2048, 2048), (64, 64, 64), (128, 128, 128),
                 (256, 256, 256)]
        n = args.serving_requests
        reqs, t_arr = [], 0.0
        for _ in range(n):
            t_arr += rng.exponential(1.0 / 50.0)
            gsh = grids[int(rng.integers(len(grids)))]
            d = len(gsh)
            ds = d * (d + 1) // 2
            reqs.append((t_arr, gsh, float(10.0 ** rng.uniform(2, 6)), float(rng.uniform(0.2, 0.4)),
                         int(rng.integers(1, ds + 1))))
        fields = {gsh: smooth_density(gsh, 16 if len(gsh) == 2 else 32, 8.0, 0) for gsh in grids}
        srv = Server(max_active=4)
        t0 = time.perf_counter()
        ids = []
        for (ta, gsh, c, nu, nl) in reqs:
            while time.perf_counter() - t0 < ta:
                time.sleep(0.0005)
            d = len(gsh)
            ids.append(srv.submit(gsh, fields[gsh], nu, np.eye(d * (d + 1) // 2)[:nl], TOL, "green_jacobi", "mixed",
                                  kind="density", e_min=1.0 / c, e_max=1.0, exponent=2.0 if d == 2 else 3.0))
        outs = [srv.wait(i) for i in ids]
        wall = time.perf_counter() - t0
        st = srv.stats()
        srv.close()
        lat = sorted(o["latency_s"] for o in outs)
        pct = lambda q: lat[min(len(lat) - 1, int(math.ceil(q * len(lat))) - 1)]
        # serial plain FP64 on the first 8 requests
        t_ser = 0.0
        n_ser = min(8, n)
        for (ta, gsh, c, nu, nl) in reqs[:n_ser]:
            d = len(gsh)
            t1 = time.perf_counter()
            s1 = Solver(gsh, fields[gsh], nu, kind="density", e_min=1.0 / c, e_max=1.0,
                        exponent=2.0 if d == 2 else 3.0, max_loads=d * (d + 1) // 2)
            s1.solve(np.eye(d * (d + 1) // 2)[:nl], TOL, "green_jacobi", want_u=False, want_stress=False)
            s1.close()
            t_ser += time.perf_counter() - t1
        served_first = sum(o["run_s"] for o in outs[:n_ser])
        return {"workload": ("seeded stream, Poisson 50/s, 2D {256^2..2048^2} + 3D {64^3,128^3,256^3}, contrast "
                             "log-U[1e2,1e6], nu U[0.2,0.4], 1..d* loads, Green-Jacobi to 1e-8, mixed precision"),
                "requests": n, "of_stream": 2000, "offered_per_s": 50.0, "max_active": 4,
                "wall_s": wall, "solves_per_s": n / wall,
                "p50_latency_s": pct(0.50), "p99_latency_s": pct(0.99),
                "mean_queue_s": statistics.mean(o["queued_s"] for o in outs),
                "max_rel_res": max(float(o["rel_res"].max()) for o in outs),
                "all_converged": all(o["status"] == 0 for o in outs),
                "solvers": {k: st[k] for k in ("solvers_created", "solvers_reused", "solvers_evicted", "peak_used")},
                "serial_fp64_first8_solves_per_s": n_ser / t_ser,
                "served_mixed_first8_run_s_sum": served_first,
                "note": "offered load exceeds capacity, so latency percentiles are queue-dominated"}

    legs = args.legs.split(",")
    fp64 = run_leg("fp64") if "fp64" in legs else None
    mixed = run_leg("mixed") if "mixed" in legs else None
    bf16 = run_leg("mixed", material_bf16=True, light=True) if ("mixed" in legs and not args.no_bf16) else None
    if fp64 is None:   # profiling run of the mixed leg only: report it in the fp64 slots too
        fp64 = mixed
    ms, value, launches = fp64["ms"], fp64["value"], fp64["launches"]
    iters = {k: v["iters"] for k, v in fp64["rec"].items()}
    prof = fp64["prof"]
    roof = roofline(fp64, alu=True)

    # ---- e2e through the C ABI with host buffers (FP64, the value's configuration)
    e2e = None
    if not args.no_e2e:
        sh = Solver(SHAPE, rho_h, NU, kind="density", e_min=1.0 / CONTRASTS[0], e_max=1.0, exponent=EXPONENT,
                    stream=stream.cuda_stream, io="host", max_loads=N_LOADS, pinned=True)
        rho_pin = torch.empty(SHAPE, dtype=torch.float64, pin_memory=True).numpy()
        rho_pin[...] = rho_h
        h2d = d2h = 0

        def step_host():
            nonlocal h2d, d2h
            for c in CONTRASTS:
                sh.set_material(rho_pin, e_min=1.0 / c)
                h2d += rho_pin.nbytes
                for pc in PRECONDS:
                    out = sh.solve(eps_h, TOL, pc, want_stress=False)
                    h2d += eps_h.nbytes
                    d2h += out["u"].nbytes + out["C_hom"].nbytes + out["iters"].nbytes + out["rel_res"].nbytes

        for _ in range(3):
            step_host()
        barrier()
        h2d = d2h = 0
        t0 = time.perf_counter()
        for _ in range(args.steps):
            step_host()
        barrier()
        t_e2e_ms, e2e_value = aggregate((time.perf_counter() - t0) / args.steps * 1e3, world, solves_per_step,
                                        dist, "cuda")
        e2e = {"value": e2e_value, "unit": "solves/s",
               "h2d_bytes_per_step": h2d // args.steps, "d2h_bytes_per_step": d2h // args.steps}
        sh.close()

    cells_line = cells_leg() if not args.no_cells else None
    serving_line = serving_leg() if not args.no_serving else None

    mixed_line = None if mixed is None else {
        "value": mixed["value"], "unit": "solves/s", "ms_per_step": mixed["ms"], "speedup_vs_fp64": fp64["ms"] / mixed["ms"],
        "dtype": "f32 inner PCG (operator, FFT, preconditioner, vectors) + f64 scalars, residual and solution",
        "roofline": roofline(mixed, alu=False), "clocks": mixed["clocks"], "gpu_launches": mixed["launches"] // args.steps,
        "time_to_tol_ms": {f"{pc}@{c:g}": round(v["ms"], 3) for (c, pc), v in mixed["rec"].items()},
        "iters": {f"{pc}@{c:g}": v["iters"] for (c, pc), v in mixed["rec"].items()},
        "refine_steps": {f"{pc}@{c:g}": v["refine"] for (c, pc), v in mixed["rec"].items()},
        "rel_res_max": max(max(v["rel_res"]) for v in mixed["rec"].values()),
        "kernels_ms_total": {k: round(v[1], 3) for k, v in mixed["prof"].items()},
        "graph_replays": mixed["graph_replays"],
        "tuning": mixed["tuning"],
        "profiled_step_ms": mixed["profiled_step_ms"],
    }
    if mixed_line is not None and bf16 is not None:
        mixed_line["material_bf16"] = {
            "value": bf16["value"], "unit": "solves/s", "ms_per_step": bf16["ms"],
            "speedup_vs_fp32_material": mixed["ms"] / bf16["ms"], "speedup_vs_fp64": fp64["ms"] / bf16["ms"],
            "note": "mixed precision with the FP32 operator reading E from a BF16 copy (options.material_bf16)",
            "time_to_tol_ms": {f"{pc}@{c:g}": round(v["ms"], 3) for (c, pc), v in bf16["rec"].items()},
            "iters": {f"{pc}@{c:g}": v["iters"] for (c, pc), v in bf16["rec"].items()},
            "rel_res_max": max(max(v["rel_res"]) for v in bf16["rec"].values())}
    clk = fp64["clocks"]
    times = fp64["times"]

    cpu_line = None
    if cpu is not None:
        cpu_step = cpu_extrapolate(cpu, {k: v for k, v in iters.items()})
        cpu_line = {"value": solves_per_step / cpu_step, "unit": "solves/s", "cores": 1, "kind": "oracle",
                    "sample": ("oracle setup at 1024x1024 (contrast 1e4), one load's rhs and post-processing, "
                               "3 Green-Jacobi and 3 Green iterations, scaled to this step's 18 solves with the "
                               "GPU run's iteration counts"),
                    "cpu": cpu_model(), "sample_seconds": cpu}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": list(SHAPE), "contrasts": list(CONTRASTS),
                       "preconditioners": list(PRECONDS), "loads": N_LOADS, "tol": TOL,
                       "parallelism": f"replicas x{world}",
                       "l2": "256 MiB buffer written before each timed step (outside the timed interval)",
                       "launch_shapes": "plan-time autotuner (options.autotune)"},
            "roofline": roof, "cpu_baseline": cpu_line, "e2e": e2e, "gpu_launches": launches // args.steps,
            "clocks": clk, "mixed": mixed_line, "small_cells": cells_line, "serving": serving_line,
            "detail": {"iters": {f"{pc}@{c:g}": v for (c, pc), v in iters.items()},
                       "time_to_tol_ms": {f"{pc}@{c:g}": round(v["ms"], 3) for (c, pc), v in fp64["rec"].items()},
                       "rel_res_max": max(max(v["rel_res"]) for v in fp64["rec"].values()),
                       "kernels_ms_total": {k: round(v[1], 3) for k, v in prof.items()},
                       "kernel_launches": {k: v[0] for k, v in prof.items()},
                       "graph_replays": fp64["graph_replays"],
                       "tuning": fp64["tuning"],
                       "profiled_step_ms": fp64["profiled_step_ms"],
                       "step_ms": times},
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
