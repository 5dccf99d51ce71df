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

value: solves/s with the density field resident in HBM and every output of
jfft_solve (u, element stress, C_hom, iteration counts, residuals) written to device
buffers; e2e: the same through the C ABI with host buffers (pinned), the host->device
copy of the density and the device->host read of every output inside the timed region.

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
SQRT2 = math.sqrt(2.0)
# 3D configurations (trilinear hexes, 8 Gauss points, nu 0.3, E = 1/c + (1 - 1/c) rho^3,
# Green-Jacobi PCG to a relative residual of 1e-8): one timed solve per precision.
CONFIGS_3D = {
    "3d_128": {"shape": (128, 128, 128), "modes": 32, "kmax": 6.0, "contrast": 1e5,
               "loads": np.eye(6), "precisions": ("fp64", "mixed"),
               "workload": ("3D periodic cell, 128^3 trilinear hexes (8 Gauss points), smooth density (32 Fourier "
                            "modes, |k|<=6), E = 1/c + (1-1/c) rho^3, c = 1e5, nu 0.3; all 6 Mandel unit loads in "
                            "one batched solve; Green-Jacobi PCG to 1e-8 relative residual")},
    "3d_512": {"shape": (512, 512, 512), "modes": 32, "kmax": 12.0, "contrast": 1e6,
               "loads": np.array([[0.0, 0.0, 0.0, 0.0, 0.0, SQRT2]]), "precisions": ("fp64", "mixed", "mixed_bf16"),
               "workload": ("3D periodic cell, 512^3 trilinear hexes (8 Gauss points, 4.0e8 DOF), smooth density "
                            "(32 Fourier modes, |k|<=12), E = 1/c + (1-1/c) rho^3, c = 1e6, nu 0.3; single load "
                            "eps_xy = 1 (Mandel sqrt(2) e_6); Green-Jacobi PCG to 1e-8 relative residual")},
}
# Profiling-only configurations (selectable with --only-3d, never part of the default run):
# 256^3 with the 512^3 recipe and its single load, for ncu captures whose DRAM bytes scale
# to 512^3 by the node count (x 8); a 512^3 capture would hold tens of GB on the device.
PROFILE_CONFIGS_3D = {
    "3d_256": {"shape": (256, 256, 256), "modes": 32, "kmax": 12.0, "contrast": 1e6,
               "loads": np.array([[0.0, 0.0, 0.0, 0.0, 0.0, SQRT2]]), "precisions": ("fp64", "mixed"),
               "workload": ("3D periodic cell, 256^3 trilinear hexes (8 Gauss points), the 512^3 recipe (smooth "
                            "density, 32 Fourier modes, |k|<=12, E = 1/c + (1-1/c) rho^3, c = 1e6, nu 0.3, single "
                            "load eps_xy = 1); Green-Jacobi PCG to 1e-8 relative residual; profiling stand-in for "
                            "512^3")},
}
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


def operator_flops_per_element(d):
    """FP64/FP32 operations of the Walsh-Hadamard mode-form Q1 element (csrc/element.cuh),
    counted by walking the same loops: the forward butterfly of d components (d stages of
    2^(d-1) add/sub pairs), the mode-force map (one FMA per normal term and per shear
    term, FMA = 2 flops), the E scaling (the force-free zero mode left out), the
    transposed butterfly and the accumulation of the corner forces into the nodes.
    70 in 2D, 309 in 3D."""
    nc = 1 << d
    popc = lambda m: bin(m).count("1")  # noqa: E731
    mbit = lambda a: 1 << (d - 1 - a)  # noqa: E731
    fma = 0
    for mu in range(nc):
        if popc(mu) >= d:
            continue
        for a in range(d):
            if mu & mbit(a):
                continue
            fma += sum(1 for b in range(d) if not mu & mbit(b))
            fma += sum(2 for b in range(d) if not mu & mbit(b) and b != a)
            fma += sum(1 for c in range(d) if mu & mbit(c))
    wht = d * d * (nc // 2) * 2
    return wht + 2 * fma + d * (nc - 1) + wht + d * nc


def _grid_terms(shape):
    d = len(shape)
    N = int(np.prod(shape))
    F = N // shape[-1] * (shape[-1] // 2 + 1)
    return d, N, F


def flops_per_unit(kernel, shape):
    """Algorithmic FLOPs of one kernel for one load case (one right-hand side).

    FFT passes use the conventional 5 L log2 L per complex transform of length L
    (2.5 n log2 n for a real transform of length n); the symbol block multiply of a
    real symmetric d x d block by a complex vector costs 2 d^2 mults + 2 d (d-1)
    adds per frequency; J^1/2 scalings one multiply per real value; the operator the
    mode-form count of operator_flops_per_element per node plus the fused p.q."""
    k = kernel[:-4] if kernel.endswith("_f32") else kernel
    d, N, F = _grid_terms(shape)
    n = shape
    rows = N // n[-1]                            # real lines along the last axis
    real_fft = d * rows * 2.5 * n[-1] * math.log2(n[-1])
    if k == "fft_rows_real_fwd":
        return real_fft + d * N
    if k == "fft_rows_real_fwd_xr":                # + x += alpha p, r -= alpha q, ||r||^2
        return real_fft + d * N + 6 * d * N
    if k == "fft_cols_real_inv":
        return real_fft + 3 * d * N
    if k in ("fft_rows_cplx_fwd", "fft_cols_cplx_inv"):   # 3D middle axis
        return d * (F // n[1]) * 5 * n[1] * math.log2(n[1])
    if k == "fft_lines":
        return d * (F // n[0]) * 2 * 5 * n[0] * math.log2(n[0]) + F * (2 * d * d * 2 + 2 * d * (d - 1))
    if k == "apply_K":
        return operator_flops_per_element(d) * N + 2 * d * N
    return None


def traffic_bytes_per_unit(kernel, shape, material_bytes=None):
    """Compulsory DRAM bytes of one kernel for one load case; kernels whose name ends in
    _f32 move FP32 data (s = 4 bytes per real), the others FP64 (s = 8). The material
    field is read once per launch for all loads; it is charged to each load here at
    ``material_bytes`` per voxel (s by default, 2 for a BF16 copy)."""
    s = 4 if kernel.endswith("_f32") else 8
    se = s if material_bytes is None else material_bytes
    k = kernel[:-4] if kernel.endswith("_f32") else kernel
    d, N, F = _grid_terms(shape)
    ncmp = d * (d + 1) // 2
    table = {
        "fft_lines": 2 * d * F * 2 * s + F * ncmp * s,           # spectrum in + out, symbol table
        "fft_rows_real_fwd": d * N * s + d * F * 2 * s + N * s,   # r, spectrum, J^1/2 scale
        # with the PCG update: x, r read + write, p, q, spectrum, J^1/2 scale
        "fft_rows_real_fwd_xr": 6 * d * N * s + d * F * 2 * s + N * s,
        "fft_rows_cplx_fwd": 2 * d * F * 2 * s,                   # spectrum in + out
        "fft_cols_cplx_inv": 2 * d * F * 2 * s,
        "fft_cols_real_inv": d * F * 2 * s + 2 * d * N * s + N * s,   # spectrum, z, r (dot), scale
        "apply_K": 2 * d * N * s + N * se,                        # p, q, E
        "cg_xr": 6 * d * N * s,                                   # x, r read+write, p, q
        "cg_p": 3 * d * N * s,                                    # p read+write, z
    }
    return table.get(k)


def source_fingerprint():
    """sha256 (16 hex digits) over the CUDA sources, the header and the build flags: an
    ncu capture is only reported next to the kernels it measured."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_2508_02613_gb300", "csrc")
    files = sorted(os.path.join(csrc, f) for f in os.listdir(csrc) if f.endswith((".cu", ".cuh")))
    files += [os.path.join(ROOT, "include", "jfft.h"), os.path.join(ROOT, "paper_2508_02613_gb300", "build.py")]
    h = hashlib.sha256()
    for f in files:
        h.update(os.path.basename(f).encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(workload):
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) recorded in the
    committed ncu summaries under profiles/, as lines
        traffic: workload=<w> kernel=<k> loads=<n> dram_bytes=<b> sources=<fingerprint>
    Only lines whose fingerprint matches the current sources are used: a capture of an
    older kernel reads as no capture. A summary may declare the current sources equivalent
    to captured ones, for changes that leave every kernel's device code and launch shape as
    they were (host-side fixes), with a line
        equivalent: sources=<current fingerprint> captured=<fingerprint> reason=<text>
    Returns {kernel: (bytes per launch, loads, file)}."""
    out = {}
    fp = source_fingerprint()
    pdir = os.path.join(ROOT, "profiles")
    if not os.path.isdir(pdir):
        return out
    lines = []
    for name in sorted(os.listdir(pdir)):
        if not name.endswith((".md", ".txt")):
            continue
        with open(os.path.join(pdir, name)) as fh:
            lines += [(name, line.strip().strip("`")) for line in fh]
    accepted = {fp}
    for _, line in lines:
        if line.startswith("equivalent:"):
            kv = dict(t.split("=", 1) for t in line[len("equivalent:"):].split() if "=" in t)
            if kv.get("sources") == fp and kv.get("captured"):
                accepted.add(kv["captured"])
    for name, line in lines:
        if not line.startswith("traffic:"):
            continue
        kv = dict(t.split("=", 1) for t in line[len("traffic:"):].split() if "=" in t)
        if kv.get("workload") == workload and kv.get("sources") in accepted:
            out[kv["kernel"]] = (float(kv["dram_bytes"]), int(kv.get("loads", 1)), name)
    return out


def roofline(prof, n_units, shape, alu, workload, material_bytes=None, profiled_steps=1, every=False):
    """Dominant kernel with its achieved rate, from the per-kernel CUDA events (summed event
    time per kernel name) of a profiling pass that repeats the timed work. Units are
    right-hand-side applications: per load, one operator and one preconditioner per PCG
    iteration; ``n_units`` of them in the profiled pass. ``alu``: report against the FP64
    ALU peak derived from the unit counts (FP64 kernels), else against measured HBM.
    ``every``: the same object for every kernel with a byte and flop model, largest share
    first (a list), limited to the kernels launched once per PCG iteration (at least half
    as many launches as the dominant kernel): the setup and initial-residual kernels run
    once per solve, so the per-iteration unit count does not apply to them."""
    rows = sorted(((k, v[0], v[1]) for k, v in prof.items()), key=lambda r: -r[2])
    found = []
    total_ms = sum(r[2] for r in rows)
    peak_gbs, peak_kind = hbm_peak_gbs()
    captured = ncu_traffic(workload)
    for name, nl, tot in rows:
        byt = traffic_bytes_per_unit(name, shape, material_bytes)
        fl = flops_per_unit(name, shape)
        # the dominant kernel needs both models; the list also takes byte-only kernels
        # (vectors) on HBM-bound legs
        if byt is None or (fl is None and (alu or not every)):
            continue
        out = {"kernel": name, "launches": nl, "avg_launch_ms": tot / nl, "share": tot / total_ms,
               "units": n_units, "algorithmic_bytes_per_unit": byt, "algorithmic_flops_per_unit": fl,
               "traffic": None}
        if name in captured:
            tb, loads, src = captured[name]
            out["traffic"] = tb
            out["traffic_note"] = (f"ncu DRAM bytes of one launch with {loads} load(s) active ({src}); the "
                                   f"algorithmic bytes of that launch are {loads * byt:.4g}")
        else:
            out["traffic_note"] = "no ncu capture of the current kernel sources for this workload"
        gbs = n_units * byt / (tot / 1e3) / 1e9
        tfl = n_units * fl / (tot / 1e3) / 1e12 if fl is not None else None
        if alu:
            out.update({"bound": "alu", "achieved": tfl, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                        "frac": tfl / FP64_PEAK_TFLOPS, "hbm_GBps_algorithmic": gbs,
                        "peak_note": "FP64 ALU, derived: 152 SMs x 2.07 GHz x 4 flop/clk/SM (2 DFMA)"})
        else:
            out.update({"bound": "hbm", "achieved": gbs, "peak": peak_gbs, "unit": "GB/s", "frac": gbs / peak_gbs,
                        "peak_note": f"HBM copy bandwidth, {peak_kind} (MEASURED_PEAKS.json hbm_gbs)"})
        if not every:
            return out
        if not found or nl >= 0.5 * found[0]["launches"]:
            found.append(out)
    return found if every else None


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


# Small instances of the benchmark recipes on which every mixed-precision result is
# compared with the oracle solved to 1e-13 (the full-size grids are beyond the oracle's
# reach inside a benchmark run): the 2D sweep's recipe at 32^2 and 256^2 (contrast 1e4,
# rho^2, 3 loads) and the 3D recipe at 16^3 (32 modes |k| <= 6, rho^3, contrast 1e5, 6 loads).
ERR_CASES = {
    "2d_32": {"shape": (32, 32), "modes": 16, "kmax": 8.0, "exponent": 2.0, "contrast": 1e4, "nloads": 3},
    "2d_256": {"shape": (256, 256), "modes": 16, "kmax": 8.0, "exponent": 2.0, "contrast": 1e4, "nloads": 3},
    "3d_16": {"shape": (16, 16, 16), "modes": 32, "kmax": 6.0, "exponent": 3.0, "contrast": 1e5, "nloads": 6},
}


def oracle_reference_solutions(path):
    """Oracle solutions (Green-Jacobi PCG to 1e-13, zero-mean u and C_hom) of ERR_CASES,
    written to ``path`` (npz); part of the CPU-side leg, run before any CUDA call."""
    from oracle import material, solve as osolve
    from synthetic import smooth_density
    arrays = {}
    for key, c in ERR_CASES.items():
        rho = smooth_density(c["shape"], c["modes"], c["kmax"], SEED)
        E = material.young_from_density(rho, 1.0 / c["contrast"], 1.0, c["exponent"])
        prob = osolve.setup(c["shape"], E, NU)
        ref = osolve.solve(prob, np.eye(c["nloads"]), 1e-13, "green_jacobi")
        arrays[key + "_u"] = ref.u
        arrays[key + "_C_hom"] = ref.C_hom
    np.savez(path, **arrays)


def run_oracle_reference_subprocess(path):
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = f"import bench; bench.oracle_reference_solutions({path!r})"
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, stdout=subprocess.PIPE,
                       stderr=subprocess.PIPE, text=True, timeout=900)
    if r.returncode != 0:
        raise RuntimeError("oracle reference solutions failed: " + r.stderr[-2000:])
    return dict(np.load(path))


def cpu_openmp_sample():
    """The C PCG baseline (oracle/cbase: matrix-free operator, textbook radix-2 FFT, OpenMP
    on every host core) on a bounded sample: at 1024 x 1024 (contrast 1e4) the oracle's
    setup (not part of the C code), one full Green-Jacobi solve of load 0 to 1e-8 and five
    Green iterations; the 32 x 32 configuration (16 modes |k| <= 4, contrast 1e4, rho^2,
    eps_xx, tolerance 1e-6) solved in full with both preconditioners."""
    from oracle import assemble, cbase, material, solve as osolve
    from synthetic import smooth_density
    out = {"threads": cbase.threads()}
    rho = smooth_density(SHAPE, MODES, KMAX, SEED)
    E = material.young_from_density(rho, 1e-4, 1.0, EXPONENT)
    t0 = time.perf_counter()
    prob = osolve.setup(SHAPE, E, NU)
    out["t_setup"] = time.perf_counter() - t0
    f = assemble.assemble_rhs(SHAPE, E, prob.C, np.eye(3)[0])
    t0 = time.perf_counter()
    _, it, conv = cbase.pcg(prob, f, TOL, "green_jacobi")
    out["gj_full_solve_s"], out["gj_full_iters"], out["gj_converged"] = time.perf_counter() - t0, it, conv
    t0 = time.perf_counter()
    cbase.pcg(prob, f, 0.0, "green", max_iter=5)
    out["t_iter"] = {"green_jacobi": out["gj_full_solve_s"] / max(it, 1), "green": (time.perf_counter() - t0) / 5}
    small = (32, 32)
    rho32 = smooth_density(small, 16, 4.0, 0)
    E32 = material.young_from_density(rho32, 1e-4, 1.0, 2.0)
    p32 = osolve.setup(small, E32, NU)
    f32 = assemble.assemble_rhs(small, E32, p32.C, np.eye(3)[0])
    out["c1_32"] = {}
    for pc in PRECONDS:
        reps, t0 = 0, time.perf_counter()
        while reps < 3 or time.perf_counter() - t0 < 0.5:
            _, it32, _ = cbase.pcg(p32, f32, 1e-6, pc)
            reps += 1
        out["c1_32"][pc] = {"iters": it32, "s_per_solve": (time.perf_counter() - t0) / reps}
    return out


def run_cpu_openmp_subprocess():
    env = dict(os.environ, OMP_NUM_THREADS=str(os.cpu_count() or 1), OPENBLAS_NUM_THREADS="1")
    code = "import json, bench; print('CPUOMP ' + json.dumps(bench.cpu_openmp_sample()))"
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, stdout=subprocess.PIPE,
                       stderr=subprocess.PIPE, text=True, timeout=900)
    for line in r.stdout.splitlines():
        if line.startswith("CPUOMP "):
            return json.loads(line[len("CPUOMP "):])
    raise RuntimeError("C baseline sample failed: " + r.stderr[-2000:])


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
    ap.add_argument("--legs", default="fp64,mixed",
                    help="precision legs of the 2D sweep (profiling runs); 'none' runs only the 3D legs")
    ap.add_argument("--no-cells", action="store_true", help="skip the small-cell batch leg")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving leg")
    ap.add_argument("--no-bf16", action="store_true", help="skip the BF16-material variant of the mixed leg")
    ap.add_argument("--no-3d", action="store_true", help="skip the 3D legs (128^3 x 6 loads, 512^3)")
    ap.add_argument("--no-cufft", action="store_true", help="skip the cuFFT timing cross-check")
    ap.add_argument("--only-3d", default="", help="run only these 3D legs (comma list of CONFIGS_3D keys)")
    ap.add_argument("--precisions-3d", default="", help="run only these precisions in the 3D legs (profiling runs)")
    ap.add_argument("--no-graphs", action="store_true",
                    help="launch every kernel from the host (profilers cannot see kernels inside conditional graphs)")
    ap.add_argument("--serving-requests", type=int, default=500,
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
    cpu_omp = None
    oracle_ref = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = run_cpu_sample_subprocess()   # before any CUDA call in this process
        cpu_omp = run_cpu_openmp_subprocess()
        import tempfile
        with tempfile.TemporaryDirectory() as td:
            oracle_ref = run_oracle_reference_subprocess(os.path.join(td, "oracle_ref.npz"))

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
                    out = s.solve(eps_d, TOL, pc, want_stress=True)
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
        return {"precision": precision, "ms": ms, "value": value, "times": times, "rec": rec, "prof": prof,
                "launches": launches,
                "graph_replays": replays, "profiled_step_ms": prof_times, "tuning": tuning,
                "clocks": clk}

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
        def pct(vals, q):
            v = sorted(vals)
            return v[min(len(v) - 1, max(0, int(math.ceil(q * len(v))) - 1))]
        lat = [o["latency_s"] for o in outs]
        run = [o["run_s"] for o in outs]
        que = [o["queued_s"] for o in outs]
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
                "p50_latency_s": pct(lat, 0.50), "p99_latency_s": pct(lat, 0.99),
                "p50_run_s": pct(run, 0.50), "p99_run_s": pct(run, 0.99),
                "p50_queue_s": pct(que, 0.50), "p99_queue_s": pct(que, 0.99),
                "mean_queue_s": statistics.mean(que),
                "latency_note": ("latency = submission to result; run = start of the solve to result (without "
                                 "queueing); queue = submission to start"),
                "max_rel_res": max(float(o["rel_res"].max()) for o in outs),
                "all_converged": all(o["status"] == 0 for o in outs),
                "solvers": {k: st[k] for k in ("solvers_created", "solvers_reused", "solvers_evicted", "peak_used")},
                "serial_fp64_first8_solves_per_s": n_ser / t_ser,
                "served_mixed_first8_run_s_sum": served_first,
                "note": "offered load exceeds capacity, so latency percentiles are queue-dominated"}

    def leg_3d(key):
        """One configuration of CONFIGS_3D: per precision a solver on the device-resident
        density, one warm-up solve, one timed solve (CUDA events on the solver's stream, L2
        flushed before), one profiled solve (per-kernel CUDA events) for the roofline."""
        from synthetic import smooth_density_device
        cfg = CONFIGS_3D[key] if key in CONFIGS_3D else PROFILE_CONFIGS_3D[key]
        shape = cfg["shape"]
        rho3 = smooth_density_device(shape, cfg["modes"], cfg["kmax"], SEED)
        rho3_h = rho3.cpu().numpy()
        loads = torch.tensor(cfg["loads"], device="cuda")
        out = {"workload": cfg["workload"], "grid": list(shape), "loads": int(cfg["loads"].shape[0]), "tol": TOL,
               "dof_per_load": 3 * int(np.prod(shape))}
        precs = [p for p in cfg["precisions"] if not args.precisions_3d or p in args.precisions_3d.split(",")]
        for prec in precs:
            bf = prec == "mixed_bf16"
            s3 = Solver(shape, rho3_h, NU, kind="density", e_min=1.0 / cfg["contrast"], e_max=1.0, exponent=3.0,
                        stream=stream.cuda_stream, io="device", max_loads=max(3, len(cfg["loads"])),
                        precision="fp64" if prec == "fp64" else "mixed", material_bf16=bf,
                        graphs=not args.no_graphs, autotune=True)
            s3.solve(loads, TOL, "green_jacobi", want_stress=True)   # warm-up
            flush.fill_(1.0)
            barrier()
            n0 = s3.launch_count
            clocks = ClockSampler(smi_id)
            clocks.start()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            res = s3.solve(loads, TOL, "green_jacobi", want_stress=True)
            e1.record(stream)
            barrier()
            clk = clocks.stop()
            ms = e0.elapsed_time(e1)
            launches = s3.launch_count - n0
            iters = [int(v) for v in res["iters"].cpu().tolist()]
            rec = {"time_to_tol_ms": ms, "solves_per_s": len(iters) / (ms / 1e3), "iters": iters,
                   "refine_steps": [int(v) for v in res["refine_steps"].cpu().tolist()],
                   "rel_res": [float(v) for v in res["rel_res"].cpu().tolist()],
                   "converged": int(res["status"]) == 0, "gpu_launches": launches, "clocks": clk,
                   "workspace_gb": s3.workspace_bytes / 1e9, "tuning": s3.tuning,
                   "dtype": "f64" if prec == "fp64" else ("f32 inner PCG, bf16 material copy, f64 scalars, residual "
                                                          "and solution" if bf else
                                                          "f32 inner PCG, f64 scalars, residual and solution")}
            s3.set_profiling(True)
            flush.fill_(1.0)
            barrier()
            s3.solve(loads, TOL, "green_jacobi", want_stress=True)
            barrier()
            prof = s3.profile()
            s3.set_profiling(False)
            rec["kernels_ms_total"] = {k: round(v[1], 3) for k, v in prof.items()}
            rec["roofline"] = roofline(prof, sum(iters), shape, prec == "fp64", f"{key}_{prec}",
                                       material_bytes=2 if bf else None)
            s3.close()
            del res
            torch.cuda.empty_cache()
            out[prec] = rec
        if "fp64" in out:
            for prec in precs:
                if prec != "fp64":
                    out[prec]["speedup_vs_fp64"] = out["fp64"]["time_to_tol_ms"] / out[prec]["time_to_tol_ms"]
        del rho3, loads
        torch.cuda.empty_cache()
        return out

    def err_vs_oracle(precision, material_bf16, keys):
        """Relative L2 error of u and max relative error of C_hom of this precision's GPU solve
        (Green-Jacobi to 1e-8, every load of the case) against the oracle's 1e-13 solution,
        per ERR_CASES instance; worst load reported."""
        if oracle_ref is None:
            return None
        out = {}
        for key in keys:
            c = ERR_CASES[key]
            rho_c = smooth_density(c["shape"], c["modes"], c["kmax"], SEED)
            sc = Solver(c["shape"], rho_c, NU, kind="density", e_min=1.0 / c["contrast"], e_max=1.0,
                        exponent=c["exponent"], max_loads=max(c["nloads"], 3), precision=precision,
                        material_bf16=material_bf16, stream=stream.cuda_stream)
            res = sc.solve(np.eye(c["nloads"]), TOL, "green_jacobi")
            sc.close()
            u_ref, ch_ref = oracle_ref[key + "_u"], oracle_ref[key + "_C_hom"]
            du = max(float(np.linalg.norm(res["u"][g] - u_ref[g]) / np.linalg.norm(u_ref[g]))
                     for g in range(c["nloads"]))
            dc = float(np.abs(res["C_hom"] - ch_ref).max() / np.abs(ch_ref).max())
            out[key] = {"u_rel_l2": du, "C_hom_rel": dc, "rel_res_max": float(res["rel_res"].max()),
                        "tol": TOL, "grid": list(c["shape"]), "contrast": c["contrast"], "loads": c["nloads"]}
        return out

    def fp64_probe_leg():
        """The measured FP64 FMA rate beside the derived peak of the FP64 rooflines: the
        probe library (paper_2508_02613_gb300/probe/fp64_fma.cu, built by build()) runs 8
        blocks of 256 threads per SM, each thread 8 independent FMA chains of 16384 steps,
        timed with CUDA events after one warm-up launch; an FMA counts as two flops. It runs
        in a process of its own: the probe library links its own CUDA runtime, and a second
        runtime instance in this process broke CUDA graph teardown in the request server's
        worker threads (a crash inside cuGraphDestroy)."""
        blocks, threads, iters, chains = 152 * 8, 256, 16384, 8
        code = ("import ctypes, sys; lib = ctypes.CDLL(sys.argv[1]); ms = ctypes.c_float(0.0); "
                "st = lib.jfft_probe_fp64_fma(int(sys.argv[2]), int(sys.argv[3]), int(sys.argv[4]), ctypes.byref(ms)); "
                "print(st, ms.value)")
        lib = os.path.join(ROOT, "paper_2508_02613_gb300", "probe", "libjfft_probe.so")
        try:
            r = subprocess.run([sys.executable, "-c", code, lib, str(blocks), str(threads), str(iters)],
                               capture_output=True, text=True, timeout=300,
                               env=dict(os.environ, CUDA_VISIBLE_DEVICES=os.environ.get("CUDA_VISIBLE_DEVICES", str(local))))
            st, ms = r.stdout.split()[:2]
            st, ms = int(st), float(ms)
        except (subprocess.SubprocessError, ValueError, OSError) as e:
            return {"error": f"probe did not run: {type(e).__name__}"}
        if st != 0:
            return {"error": f"cudaError {st}"}
        tflops = blocks * threads * chains * iters * 2 / (ms / 1e3) / 1e12
        return {"tflops": tflops, "ms": ms, "derived_peak_tflops": FP64_PEAK_TFLOPS,
                "ratio_to_derived": tflops / FP64_PEAK_TFLOPS,
                "shape": f"{blocks} x {threads} threads, {chains} chains x {iters} FMAs each"}

    def cufft_leg():
        """Timing cross-check only; cuFFT (through torch.fft) is on no path of the solver. The
        forward real 2D transform and its inverse of the fields one 1024^2 preconditioner
        application transforms (3 loads x 2 components), beside the transform passes of this
        library's Green-Jacobi preconditioner on the same number of fields (its per-kernel CUDA
        events during jfft_apply_precond: J^1/2 scaling, forward transform, symbol block
        multiply, inverse transform, J^1/2 scaling and r.z), FP64 and FP32; L2 flushed before
        every repetition."""
        out = {"fields": f"{N_LOADS} loads x 2 components, {SHAPE[0]}x{SHAPE[1]}", "reps": 10}
        gen = torch.Generator(device="cuda")
        gen.manual_seed(7)
        for prec, dt in (("fp64", torch.float64), ("mixed", torch.float32)):
            x = torch.randn((N_LOADS, 2) + SHAPE, dtype=dt, device="cuda", generator=gen)
            pair = lambda: torch.fft.irfftn(torch.fft.rfftn(x, dim=(-2, -1)), s=SHAPE, dim=(-2, -1))  # noqa: E731
            for _ in range(3):
                pair()
            ts = []
            for _ in range(out["reps"]):
                flush.fill_(1.0)
                barrier()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                pair()
                e1.record(stream)
                barrier()
                ts.append(e0.elapsed_time(e1))
            sp = Solver(SHAPE, rho_h, NU, kind="density", e_min=1e-4, e_max=1.0, exponent=EXPONENT,
                        stream=stream.cuda_stream, io="device", max_loads=N_LOADS, precision=prec)
            r = torch.randn((N_LOADS, 2) + SHAPE, dtype=torch.float64, device="cuda", generator=gen)
            for _ in range(3):
                sp.apply_precond("green_jacobi", r)
            sp.set_profiling(True)
            for _ in range(out["reps"]):
                flush.fill_(1.0)
                barrier()
                sp.apply_precond("green_jacobi", r)
            prof = sp.profile()
            sp.set_profiling(False)
            sp.close()
            passes = {k: v[1] / out["reps"] for k, v in prof.items() if k.startswith("fft_")}
            out[prec] = {"cufft_r2c_c2r_ms": statistics.median(ts), "preconditioner_passes_ms": sum(passes.values()),
                         "passes_ms": {k: round(v, 4) for k, v in passes.items()}}
        return out

    legs = args.legs.split(",")
    if "none" in legs:
        # profiling runs of the 3D legs alone: no 2D sweep, one JSON line with those legs
        out3 = {key: leg_3d(key) for key in (args.only_3d.split(",") if args.only_3d else CONFIGS_3D)}
        if rank == 0:
            print(json.dumps({"configs_3d": out3, "note": "3D legs only (--legs none); no headline value"}))
        return 0
    fp64 = run_leg("fp64") if "fp64" in legs else None
    mixed = run_leg("mixed") if "mixed" in legs else None
    bf16 = run_leg("mixed", material_bf16=True, light=True) if ("mixed" in legs and not args.no_bf16) else None
    if fp64 is None:   # profiling run of the mixed leg only: report it in the fp64 slots too
        fp64 = mixed
    ms, value, launches = fp64["ms"], fp64["value"], fp64["launches"]
    iters = {k: v["iters"] for k, v in fp64["rec"].items()}
    prof = fp64["prof"]
    n_units_fp64 = sum(sum(r["iters"]) for r in fp64["rec"].values()) * PROFILED_STEPS
    roof = roofline(prof, n_units_fp64, SHAPE, fp64["precision"] == "fp64", "2d_1024_sweep")
    # the same for every modelled kernel of the leg (the dominant one is `roofline`)
    roof_all = [{k: r[k] for k in ("kernel", "share", "bound", "achieved", "unit", "frac", "traffic")}
                for r in roofline(prof, n_units_fp64, SHAPE, fp64["precision"] == "fp64", "2d_1024_sweep",
                                  every=True)]

    # ---- e2e through the C ABI with host buffers (FP64, the value's configuration)
    e2e = None
    if not args.no_e2e:
        # the options of the timed FP64 leg (plan-time autotuner included), with host buffers
        sh = Solver(SHAPE, rho_h, NU, kind="density", e_min=1.0 / CONTRASTS[0], e_max=1.0, exponent=EXPONENT,
                    stream=stream.cuda_stream, io="host", max_loads=N_LOADS, pinned=True, autotune=True)
        rho_pin = torch.empty(SHAPE, dtype=torch.float64, pin_memory=True).numpy()
        rho_pin[...] = rho_h
        h2d = d2h = 0

        def step_host():
            nonlocal h2d, d2h
            for c in CONTRASTS:
                sh.set_material(rho_pin, e_min=1.0 / c)
                h2d += rho_pin.nbytes
                for pc in PRECONDS:
                    out = sh.solve(eps_h, TOL, pc, want_stress=True)
                    h2d += eps_h.nbytes
                    d2h += (out["u"].nbytes + out["stress"].nbytes + out["C_hom"].nbytes + out["iters"].nbytes
                            + out["rel_res"].nbytes + out["refine_steps"].nbytes)

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

    legs_3d = {}
    if not args.no_3d:
        for key in (args.only_3d.split(",") if args.only_3d else CONFIGS_3D):
            legs_3d[key] = leg_3d(key)
            for prec in legs_3d[key]:
                if prec in ("mixed", "mixed_bf16"):
                    legs_3d[key][prec]["err_vs_oracle"] = err_vs_oracle("mixed", prec == "mixed_bf16", ("3d_16",))
    cufft_line = cufft_leg() if not args.no_cufft else None
    fp64_probe_line = fp64_probe_leg()
    cells_line = cells_leg() if not args.no_cells else None
    serving_line = serving_leg() if not args.no_serving else None

    mixed_line = None if mixed is None else {
        "value": mixed["value"], "unit": "solves/s", "ms_per_step": mixed["ms"], "speedup_vs_fp64": fp64["ms"] / mixed["ms"],
        "dtype": "f32 inner PCG (operator, FFT, preconditioner, vectors) + f64 scalars, residual and solution",
        "roofline": roofline(mixed["prof"], sum(sum(r["iters"]) for r in mixed["rec"].values()) * PROFILED_STEPS,
                             SHAPE, False, "2d_1024_sweep_mixed"),
        "roofline_kernels": [{k: r[k] for k in ("kernel", "share", "bound", "achieved", "unit", "frac", "traffic")}
                             for r in roofline(mixed["prof"], sum(sum(r["iters"]) for r in mixed["rec"].values())
                                               * PROFILED_STEPS, SHAPE, False, "2d_1024_sweep_mixed", every=True)],
        "clocks": mixed["clocks"], "gpu_launches": mixed["launches"] // args.steps,
        "time_to_tol_ms": {f"{pc}@{c:g}": round(v["ms"], 3) for (c, pc), v in mixed["rec"].items()},
        "iters": {f"{pc}@{c:g}": v["iters"] for (c, pc), v in mixed["rec"].items()},
        "refine_steps": {f"{pc}@{c:g}": v["refine"] for (c, pc), v in mixed["rec"].items()},
        "rel_res_max": max(max(v["rel_res"]) for v in mixed["rec"].values()),
        "kernels_ms_total": {k: round(v[1], 3) for k, v in mixed["prof"].items()},
        "graph_replays": mixed["graph_replays"],
        "tuning": mixed["tuning"],
        "profiled_step_ms": mixed["profiled_step_ms"],
    }
    if mixed_line is not None:
        mixed_line["err_vs_oracle"] = err_vs_oracle("mixed", False, ("2d_32", "2d_256"))
    if mixed_line is not None and bf16 is not None:
        mixed_line["material_bf16"] = {
            "value": bf16["value"], "unit": "solves/s", "ms_per_step": bf16["ms"],
            "speedup_vs_fp32_material": mixed["ms"] / bf16["ms"], "speedup_vs_fp64": fp64["ms"] / bf16["ms"],
            "note": "mixed precision with the FP32 operator reading E from a BF16 copy (options.material_bf16)",
            "time_to_tol_ms": {f"{pc}@{c:g}": round(v["ms"], 3) for (c, pc), v in bf16["rec"].items()},
            "iters": {f"{pc}@{c:g}": v["iters"] for (c, pc), v in bf16["rec"].items()},
            "rel_res_max": max(max(v["rel_res"]) for v in bf16["rec"].values()),
            "err_vs_oracle": err_vs_oracle("mixed", True, ("2d_32", "2d_256"))}
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

    if serving_line is not None and oracle_ref is not None:
        # the served requests run the mixed-precision solver: its error on the 2D and 3D recipes
        serving_line["err_vs_oracle"] = err_vs_oracle("mixed", False, ("2d_32", "2d_256", "3d_16"))

    cpu_omp_line = None
    if cpu_omp is not None:
        step_s = len(CONTRASTS) * cpu_omp["t_setup"] + sum(
            n * cpu_omp["t_iter"][pc] for (c, pc), its in iters.items() for n in its)
        cpu_omp_line = {
            "value": solves_per_step / step_s, "unit": "solves/s", "cores": cpu_omp["threads"], "kind": "c_openmp",
            "sample": ("oracle/cbase (matrix-free Q1 operator, textbook radix-2 FFT, OpenMP, FP64): one full "
                       "Green-Jacobi solve at 1024x1024 (contrast 1e4, load 0, tol 1e-8) and 5 Green iterations, "
                       "the Python oracle's setup per contrast; scaled to this step's 18 solves with the GPU "
                       "run's iteration counts"),
            "gj_full_solve_1024_s": cpu_omp["gj_full_solve_s"], "gj_full_solve_1024_iters": cpu_omp["gj_full_iters"],
            "s_per_iter_1024": cpu_omp["t_iter"], "setup_s_1024": cpu_omp["t_setup"],
            "small_32x32_full_solves": cpu_omp["c1_32"], "cpu": cpu_model()}

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
            "roofline": roof, "roofline_kernels": roof_all, "cpu_baseline": cpu_line,
            "cpu_openmp_baseline": cpu_omp_line, "e2e": e2e,
            "gpu_launches": launches // args.steps,
            "clocks": clk, "fp64_fma_probe": fp64_probe_line, "mixed": mixed_line, "configs_3d": legs_3d,
            "cufft_crosscheck": cufft_line,
            "small_cells": cells_line,
            "serving": serving_line,
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
