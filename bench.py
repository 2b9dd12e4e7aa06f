"""Benchmark of the coupled conservative Allen-Cahn LBM step on GB300.

Workload (default): 512^3 cells, triply periodic, D3Q15 phase field + D3Q27
hydrodynamics, FP32, 400 non-overlapping bubbles with diameters ~ U[16, 32]
(seed 6144), density ratio 1000, viscosity ratio 100, sigma = 1e-4, xi = 5,
M = 0.02, gravity with Eo = 10 at D = 24.  One step = one coupled time step of
every cell (one launch of the fused kernel).

Prints one JSON line:
  value        MLUPS (cells x steps / s / 1e6), state resident in HBM, CUDA events
               on the library's stream, max over ranks;
  e2e          the same metric through the C ABI with pinned host buffers:
               upload of phi0, initialisation, K steps, download of phi, u, p and
               the diagnostics, all inside the timed region;
  roofline     algorithmic bytes per launch / mean launch time vs the measured HBM
               copy bandwidth, and (pattern_ceiling) vs the bandwidth the step's
               AA streaming pattern reaches without arithmetic (pattern_probe);
  cpu_baseline the FP64 oracle on the host cores on a bounded sample.
``--impl reference`` times the FP64 oracle instead (the reference arm).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "coupled phase-field+hydro MLUPS and % HBM roofline; FP16-store vs FP32 at stated err"
UNIT = "MLUPS"
# algorithmic bytes per cell update of the one-pass fused kernel: read + write the
# 15 h and q g populations (rest populations FP32, moving ones in the storage
# format), read phi once, write phi once
STORE_BYTES = {"fp32": 4, "fp16": 2, "bf16": 2}


def bytes_per_cell(q: int, precision: str = "fp32", q_phase: int = 15) -> int:
    b = STORE_BYTES[precision]
    return (4 + (q_phase - 1) * b + 4 + (q - 1) * b) * 2 + 4 + 4
FALLBACK_HBM_GBS = 6800.0


def roofline_mlups(peak_gbs: float, bytes_per_cell_: float) -> float:
    """The memory-bound ceiling of a step (Section 5.1, eq:roofline): the copy
    bandwidth divided by the bytes moved per cell, in MLUPS."""
    return peak_gbs * 1e3 / bytes_per_cell_


def env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def workload(name: str, size: int = 512, generate: bool = True):
    """(Problem, phi0, description) of a benchmark workload; with generate=False
    only the box and lattices (phi0 None), for the description of a run."""
    if name == "roofline":
        count = max(1, round(400 * (size / 512) ** 3))
        desc = (f"roofline: {size}^3 triply periodic, D3Q15+D3Q27, FP32, {count} bubbles D~U[16,32] seed 6144, "
                "rho ratio 1000, mu ratio 100, sigma 1e-4, xi 5, M 0.02, gravity Eo=10 at D=24")
        if not generate:
            return W.Problem(size, size, size, q_hydro=27), None, desc
        prob, phi0, bubbles = W.roofline(n=size, count=count)
        return prob, phi0, desc
    if name == "rising_bubble":
        if not generate:
            prob, phi0 = W.Problem(128, 512, 128, wall=(1, 1, 1), q_hydro=27), None
        else:
            prob, phi0 = W.rising_bubble()
        desc = ("rising bubble: 128x512x128 walled, D3Q15+D3Q27, FP32, D=32 at (64,64,64), Eo 10, Mo 1e-3, "
                "rho ratio 1000, mu ratio 100")
        return prob, phi0, desc
    raise ValueError(name)


def apply_pair(args, prob, phi0, desc):
    """The main step on another lattice pair of Section 5.1: the same box and
    physics with D3Q{qp} + D3Q{q}, or (9+9) the two-dimensional box of as many
    cells (16 size x 32 size x 1, circles of radius 12 on a pitch-64 lattice)."""
    if args.pair == "15+27":
        return prob, phi0, desc
    qp, q = (int(v) for v in args.pair.split("+"))
    if qp == 9:
        prob, phi0 = W.roofline2d(16 * args.size, 32 * args.size)
        return prob, phi0, (f"roofline2d: {prob.nx}x{prob.ny}x1 periodic, D2Q9+D2Q9, FP32, light circles R 12 on a "
                            "pitch-64 lattice, rho ratio 1000, mu ratio 100, sigma 1e-4, xi 5, M 0.02, gravity Eo=10 at D=24")
    prob.q_phase, prob.q_hydro = qp, q
    return prob, phi0, desc.replace("D3Q15+D3Q27", f"D3Q{qp}+D3Q{q}")


def step_kernel_name(args, prob) -> str:
    """The kernel one step launches: the two-cells-per-thread fused step where it
    applies and is chosen (every storage format by default: nx even, D3Q19 /
    D3Q27 hydrodynamics with the D3Q15 phase lattice, or in FP32 with the D3Q19
    / D3Q27 phase lattices, and the D2Q9 pair), else the one-cell fused step."""
    qp = getattr(prob, "q_phase", 15)
    lattices = ((qp == 15 and prob.q_hydro in (19, 27))
                or (args.precision == "fp32" and ((qp in (19, 27) and prob.q_hydro in (19, 27)) or qp == 9)))
    pair = args.form in ("fused", "pair") and prob.nx % 2 == 0 and lattices
    name = "pair_step_kernel" if pair else "fused_step_kernel"
    d = "D2Q" if qp == 9 else "D3Q"
    return f"{name}<{args.precision}, hydro {d}{prob.q_hydro}, phase {d}{qp}>"


def measured_hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            v = float(json.load(f)["hbm_gbs"])
        return v, "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def kernel_source_hash() -> str:
    """Hash of the fused step's sources (both fused kernels) with comments and
    blank space removed (a change of comments leaves the recorded counters
    valid)."""
    h = hashlib.sha256()
    for f in ("lbm_step.cu", "lbm_pair.cu", "lbm_pair_launch.cuh", "lbm_pair_fp32.cu", "lbm_pair_fp16.cu",
              "lbm_pair_bf16.cu", "lbm_pair_wide.cu", "lbm_pair_impl.cuh", "lbm_step_impl.cuh", "lbm_device.cuh",
              "lbm_internal.h"):
        with open(os.path.join(ROOT, "paper_2012_06144_gb300", "csrc", f)) as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]


def recorded_traffic(workload_name: str, cells: int):
    """DRAM bytes per launch of the fused kernel from the committed ncu summary,
    only if it was taken on the current kernel source and the same box."""
    path = os.path.join(ROOT, "profiles", "pair_step_kernel_roofline512_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except Exception:
        return None
    if (rec.get("source_hash") != kernel_source_hash() or rec.get("workload") != workload_name
            or rec.get("cells") != cells):
        return None
    return rec.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.t.join(timeout=2)
        return False

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(seconds_budget: float = 20.0):
    """The FP64 oracle as it stands, on the host cores, on a bounded sample of the
    workload's physics: 128^3 triply periodic with bubbles seeded as in the
    512^3 workload (scaled count), 2 warm-up steps, then as many steps as fit."""
    import oracle

    oracle.build()
    n = 128
    prob, phi0, _ = W.roofline(n=n, count=max(1, round(400 * (n / 512) ** 3)))
    st = oracle.State(oracle.make_problem(prob), phi0)
    st.run(2)
    steps, t0 = 0, time.perf_counter()
    while steps < 20 and (time.perf_counter() - t0) < seconds_budget:
        st.run(1)
        steps += 1
    dt = time.perf_counter() - t0
    return {"value": n ** 3 * steps / dt / 1e6, "unit": UNIT, "cores": oracle.get_threads(), "kind": "oracle",
            "sample": f"{n}^3 triply periodic, {steps} steps after 2 warm-up, same physics and bubble recipe "
                      f"({prob.q_hydro}-velocity hydro lattice), FP64, OpenMP"}


def run_config(args, desc, N, q, precision, world, q_phase=15):
    """The `config` object of the JSON line (the same on both arms)."""
    lat = "D2Q9+D2Q9" if q_phase == 9 else f"D3Q{q_phase}+D3Q{q}"
    return {"workload": desc, "cells": N, "lattices": lat,
            "storage": f"{precision} populations (FP32 rest), in-place AA",
            "l2": f"state {N * (bytes_per_cell(q, precision, q_phase) // 2) / 1e9:.1f} GB per GPU >> 129 MB L2, "
                  "no flush needed",
            "parallelism": f"replicas x{world}"}


def run_reference(args):
    """The reference arm: the FP64 oracle timed on the host cores.  Each step is one
    oracle time step of a bounded 32^3 sample of the workload (same physics and
    bubble recipe, scaled), so K steps finish in a few minutes."""
    rank = env_int("RANK", 0)
    if rank != 0:
        return
    import oracle

    oracle.build()
    full, _, full_desc = workload(args.workload, args.size, generate=False)
    n = 32
    prob, phi0, _ = W.roofline(n=n, count=max(1, round(400 * (n / 512) ** 3)))
    st = oracle.State(oracle.make_problem(prob), phi0)
    st.run(args.warmup)
    t0 = time.perf_counter()
    st.run(args.steps)
    dt = time.perf_counter() - t0
    value = n ** 3 * args.steps / dt / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / max(args.steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": run_config(args, full_desc, full.ncells, full.q_hydro, "fp32", args.gpus),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.get_threads(), "kind": "oracle",
                         "sample": f"{n}^3 triply periodic sample of the same physics and bubble recipe, each "
                                   f"step one FP64 oracle time step; {args.steps} steps after {args.warmup} warm-up"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def time_steps(sim, stream, steps: int) -> float:
    """Milliseconds for `steps` launches on the library's stream (CUDA events)."""
    import torch

    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    sim.step(steps)
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b)


def recorded_precision_errors():
    """The storage formats' errors against the FP64 oracle, as measured by
    tests/test_gpu_precision.py::test_precision_bubble_errors on a GB300 and
    committed (64^3 walled rising bubble, 1000 steps); only if taken on the
    current kernel source."""
    path = os.path.join(ROOT, "profiles", "precision_errors_bubble64.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except Exception:
        return {"record": None, "why": "no committed record"}
    if rec.get("source_hash") != kernel_source_hash():
        return {"record": None, "why": "recorded on another kernel source", "recorded_hash": rec.get("source_hash")}
    return dict(rec, record="profiles/precision_errors_bubble64.json")


def precision_forms(args, stream, peak):
    """FP32, FP16 and BF16 population storage timed on one box and GPU: the
    rising-bubble parameters on a 512^3 box walled on every face (D = 32 at
    (256, 64, 256)), with each form's measured error against the FP64 oracle
    (phi L-infinity, bubble centroid, rise velocity, mass drift on the 64^3
    walled rising bubble after 1000 steps, from the committed record)."""
    import torch

    from paper_2012_06144_gb300 import lbm

    prob, phi0 = W.precision_timing(args.size)
    phi0_dev = torch.from_numpy(phi0).cuda()
    out = {"workload": f"{args.size}^3 walled rising bubble, D3Q15+D3Q27, D=32 at ({args.size // 2}, 64, "
                       f"{args.size // 2}), Eo 10, Mo 1e-3, t_ref 2000, rho ratio 1000, mu ratio 100"}
    steps = min(args.steps, 500)
    for prec in ("fp32", "fp16", "bf16"):
        sim = lbm.Simulation.from_problem(prob, precision=prec, stream=stream)
        sim.init_phase(phi0_dev)
        sim.step(args.warmup)
        sim.synchronize()
        ms = time_steps(sim, stream, steps) / steps
        sim.synchronize()
        bpc = bytes_per_cell(prob.q_hydro, prec)
        out[prec] = {"value": prob.ncells / (ms / 1e3) / 1e6, "unit": UNIT, "ms_per_step": ms, "steps": steps,
                     "bytes_per_cell": bpc, "roofline_frac": prob.ncells * bpc / (ms / 1e3) / 1e9 / peak}
        sim.close()
        del sim
        torch.cuda.empty_cache()
    out["fp16_speedup"] = out["fp32"]["ms_per_step"] / out["fp16"]["ms_per_step"]
    out["bf16_speedup"] = out["fp32"]["ms_per_step"] / out["bf16"]["ms_per_step"]
    out["measured_error"] = recorded_precision_errors()
    del phi0_dev
    torch.cuda.empty_cache()
    return out


def batched_form(args, stream, peak):
    """The batched rising-bubble workload (64 seeded walled problems of four box
    sizes, 42.8 M cells): autotuned, then timed over args.batched_steps steps on
    one GPU (CUDA graphs of 16 steps), next to the same members stepped by one
    launch per member and step."""
    import torch

    from paper_2012_06144_gb300 import lbm

    draws = W.batched(count=args.batched_count)
    batch = lbm.Batch.from_problems([p for p, _, _ in draws], stream=stream)
    for m, (_, phi0, _) in zip(batch.members, draws):
        m.init_phase(phi0)
    cells = batch.cells
    if args.batched_config < 0:
        shape, order, halo, tune_ms = batch.tune(trial_steps=5)
    else:  # a fixed candidate, no tuning (profiling runs)
        shape, order, halo = lbm.batch_candidate(args.batched_config)
        batch.configure(shape, order, halo)
        tune_ms = []
    batch.step(32)
    batch.synchronize()
    steps = args.batched_steps
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    batch.step(steps)
    b.record(stream)
    torch.cuda.synchronize()
    batch.synchronize()  # raises if any member produced a non-finite value
    ms = a.elapsed_time(b) / steps
    # the same members, one launch per member and step (no batching)
    solo_steps = min(steps, 320)
    a.record(stream)
    for _ in range(solo_steps):
        for m in batch.members:
            m.step(1)
    b.record(stream)
    torch.cuda.synchronize()
    batch.synchronize()
    solo_ms = a.elapsed_time(b) / solo_steps
    bpc = bytes_per_cell(27, "fp32")
    out = {"members": len(batch), "cells": cells, "steps": steps, "value": cells / (ms / 1e3) / 1e6, "unit": UNIT,
           "ms_per_step": ms, "roofline_frac": cells * bpc / (ms / 1e3) / 1e9 / peak,
           "tuned": {"tile": lbm.batch_tile_name(shape), "order": order, "halo": halo,
                     "candidates_ms_per_step": {
                         "{}/{}/{}".format(c[2], lbm.batch_tile_name(c[0]), c[1]): float(v)
                         for i, v in enumerate(tune_ms) for c in [lbm.batch_candidate(i)]}},
           "per_member_launches": {"value": cells / (solo_ms / 1e3) / 1e6, "ms_per_step": solo_ms,
                                   "steps": solo_steps},
           "gpu_launches_per_step": (len(batch) + 63) // 64,
           "workload": f"{len(batch)} walled rising bubbles, sizes among 32^3, 48x96x48, 64x128x64, 96x192x96, D = nx/4 at "
                       "y = 2D, rho ratio 100/1000 (10 fails the s_nu bound), Eo ~ U[1,50], seed 6144"}
    batch.close()
    del batch
    torch.cuda.empty_cache()
    return out


def pattern_ceiling(size: int, achieved: float):
    """The bandwidth of the step's data movement without its arithmetic, from the
    stand-alone pattern_probe program: the two-cell step's accesses in FP32 under
    both AA layouts (one lattice natural, the other swapped), next to a plain
    copy, the one-cell AA pattern and the other streaming schemes.  frac = the
    kernel's achieved (algorithmic) GB/s over that ceiling."""
    from paper_2012_06144_gb300 import _build

    if size < 32 or size > 512 or size & (size - 1):
        return None
    try:
        r = subprocess.run([_build.PROBE, str(size)], capture_output=True, text=True, timeout=300)
        probe = json.loads(r.stdout.strip().splitlines()[-1])
    except Exception as exc:  # reported, not fatal: the ceiling is context for the roofline
        return {"error": str(exc)[:200]}
    # the two-cell step alternates its two AA layouts: the ceiling of a step pair is
    # the harmonic mean of the two layouts' bandwidths
    if "pair32_g_natural" in probe and "pair32_g_swapped" in probe:
        gbs = 2.0 / (1.0 / probe["pair32_g_natural"] + 1.0 / probe["pair32_g_swapped"])
        return {"pattern": "the two-cell step's accesses (two cells per thread, aligned pairs where the AA "
                           "layout allows, FP32, no arithmetic), both AA layouts",
                "gbs": gbs, "frac": achieved / gbs, "aa_one_cell_gbs": probe["aa_mix"], "probe": probe}
    return {"pattern": "AA: one lattice natural, the other swapped (42 FP32 planes, no arithmetic)",
            "gbs": probe["aa_mix"], "frac": achieved / probe["aa_mix"], "probe": probe}


def pattern_ceiling_16bit(probe, forms):
    """The bandwidth of the two-cell step's data movement with 16-bit moving
    populations and no arithmetic (pattern_probe's pair16 modes, one per AA
    layout; a step alternates them, so the ceiling is their harmonic mean), and
    the 16-bit forms' achieved (algorithmic) GB/s over it."""
    try:
        nat, sw = probe["pair16_g_natural"], probe["pair16_g_swapped"]
    except (TypeError, KeyError):
        return None
    gbs = 2.0 / (1.0 / nat + 1.0 / sw)
    out = {"pattern": "two cells per thread, 16-bit moving populations (one scalar access per cell for the "
                      "swapped lattice's x-moving populations), periodic box, no arithmetic",
           "gbs": gbs, "g_natural": nat, "g_swapped": sw}
    for k in ("fp16", "bf16"):
        f = forms.get(k)
        if isinstance(f, dict) and "value" in f:
            out[k + "_frac"] = f["value"] * 1e6 * f["bytes_per_cell"] / 1e9 / gbs
    return out


def unfused_bytes_per_cell(q: int) -> int:
    """Algorithmic bytes of one unfused step per cell (FP32): hydro collision
    2q + 1 + 3, phase collision 15 + 15 + 1 + 3 + 1, streaming 2 x 15 and 2 x q."""
    return 4 * ((2 * q + 4) + 35 + 30 + 2 * q)


def unfused_form(args, prob, phi0_dev, stream, peak, fused_ms):
    """The unfused baseline (Algorithm 1's passes: a collision and a streaming
    kernel per lattice over two grids) on the same workload and GPU, next to the
    fused step it is the baseline of."""
    import torch

    from paper_2012_06144_gb300 import lbm

    d, prm = lbm.from_problem(prob)
    prm.kernel_form = lbm.LBM_FORM_UNFUSED
    sim = lbm.Simulation(d, prm, stream=stream)
    sim.init_phase(phi0_dev)
    sim.step(args.warmup // 10 + 3)
    sim.synchronize()
    steps = min(args.steps, 200)
    ms = time_steps(sim, stream, steps) / steps
    sim.synchronize()
    bpc = unfused_bytes_per_cell(prob.q_hydro)
    out = {"value": prob.ncells / (ms / 1e3) / 1e6, "unit": UNIT, "ms_per_step": ms, "steps": steps,
           "kernels_per_step": 4, "bytes_per_cell": bpc,
           "roofline_frac": prob.ncells * bpc / (ms / 1e3) / 1e9 / peak,
           "fused_speedup": ms / fused_ms}
    sim.close()
    del sim
    torch.cuda.empty_cache()
    return out


def stencil_pairs(args, prob, phi0_dev, stream, peak):
    """The stencil pairs of Section 5.1 (phase-field lattice, hydrodynamic lattice)
    on the same workload and GPU, FP32: MLUPS and the fraction of the HBM roof of
    each pair's own bytes per cell, (q_phase + q_hydro) x 8 + 8."""
    import torch

    from paper_2012_06144_gb300 import lbm

    out = {}
    steps = min(args.steps, 200)
    for qp, q in ((15, 19), (15, 27), (19, 19), (27, 27)):
        d, prm = lbm.from_problem(prob)
        d.q_phase, d.q_hydro = qp, q
        sim = lbm.Simulation(d, prm, stream=stream)
        sim.init_phase(phi0_dev)
        sim.step(args.warmup // 10 + 3)
        sim.synchronize()
        ms = time_steps(sim, stream, steps) / steps
        sim.synchronize()
        bpc = (qp + q) * 8 + 8
        out[f"D3Q{qp}+D3Q{q}"] = {"value": prob.ncells / (ms / 1e3) / 1e6, "unit": UNIT, "ms_per_step": ms,
                                  "bytes_per_cell": bpc, "roofline_frac": prob.ncells * bpc / (ms / 1e3) / 1e9 / peak}
        sim.close()
        del sim
        torch.cuda.empty_cache()
    # the two-dimensional pair on a box of as many cells (16 n x 32 n x 1)
    p2, phi2 = W.roofline2d(16 * args.size, 32 * args.size)
    sim = lbm.Simulation.from_problem(p2, stream=stream)
    sim.init_phase(phi2)
    sim.step(args.warmup // 10 + 3)
    sim.synchronize()
    ms = time_steps(sim, stream, steps) / steps
    sim.synchronize()
    bpc = (9 + 9) * 8 + 8
    out["D2Q9+D2Q9"] = {"value": p2.ncells / (ms / 1e3) / 1e6, "unit": UNIT, "ms_per_step": ms, "bytes_per_cell": bpc,
                        "roofline_frac": p2.ncells * bpc / (ms / 1e3) / 1e9 / peak,
                        "box": f"{p2.nx}x{p2.ny}x1 periodic, circles R 12 on a pitch-64 lattice"}
    sim.close()
    del sim
    torch.cuda.empty_cache()
    return out


def rising_bubble_form(args, stream):
    """The walled 128x512x128 rising bubble (D = 32, Eo 10, Mo 1e-3, t_ref 2000)
    for args.rising_steps steps: light-phase centroid and rise velocity recorded
    every 100 steps, terminal velocity over the last reference time, drag
    coefficient and the empirical correlation (Section 6.1)."""
    import torch

    from paper_2012_06144_gb300 import lbm, observables as O

    prob, phi0 = W.rising_bubble()
    sim = lbm.Simulation.from_problem(prob, stream=stream)
    sim.init_phase(phi0)
    t0 = time.perf_counter()
    rec = O.track(sim, steps=args.rising_steps, every=100)
    sim.synchronize()
    wall = time.perf_counter() - t0
    out = O.summary(prob, rec, 32.0, window=1.0)
    t, c, v, _, _ = rec.arrays()
    k = np.linspace(0, len(t) - 1, 11).astype(int)
    out.update({"steps": args.rising_steps, "mlups_with_reductions": prob.ncells * args.rising_steps / wall / 1e6,
                "series_every_tenth": {"t_star": (t[k] / out["t_ref"]).tolist(), "y_c": c[k, 1].tolist(),
                                       "u_y": v[k, 1].tolist()}})
    sim.close()
    del sim
    torch.cuda.empty_cache()
    return out


def max_over_ranks(x: float, world: int, device=None) -> float:
    """Largest value of x over all ranks (the slowest rank's time)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_mlups(world: int, cells: int, steps: int, seconds: float) -> float:
    """Whole-job throughput: every rank advances its own replica of `cells` cells."""
    return world * cells * steps / seconds / 1e6


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=200)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="roofline", choices=["roofline", "rising_bubble"])
    ap.add_argument("--size", type=int, default=512, help="edge of the roofline box (512 = the benchmark)")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp16", "bf16"],
                    help="population storage format (arithmetic is FP32)")
    ap.add_argument("--form", default="fused", choices=["fused", "cell", "pair"],
                    help="fused-step variant of the main step (fused: the library's choice per storage format)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-precision", action="store_true", help="skip the FP16/BF16 storage forms")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched rising-bubble workload")
    ap.add_argument("--batched-steps", type=int, default=5000, help="timed steps of the batched workload")
    ap.add_argument("--batched-count", type=int, default=64, help="members of the batched workload (64 = the benchmark)")
    ap.add_argument("--batched-config", type=int, default=-1,
                    help="tuner candidate of the batched workload (-1: autotune)")
    ap.add_argument("--pair", default="15+27", choices=["15+27", "15+19", "19+19", "27+27", "19+27", "27+19", "9+9"],
                    help="phase + hydrodynamic lattice of the main timed step (9+9: the 2-D box of as many cells)")
    ap.add_argument("--no-rising", action="store_true", help="skip the rising-bubble observables")
    ap.add_argument("--no-unfused", action="store_true", help="skip the unfused baseline")
    ap.add_argument("--no-pairs", action="store_true", help="skip the other stencil pairs")
    ap.add_argument("--no-pattern", action="store_true", help="skip the streaming-pattern bandwidth ceiling")
    ap.add_argument("--rising-steps", type=int, default=10000, help="steps of the rising-bubble run")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    import torch.distributed as dist

    world = env_int("WORLD_SIZE", 1)
    rank = env_int("RANK", 0)
    local = env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    import __graft_entry__

    if rank == 0:
        __graft_entry__.build()
    barrier()
    from paper_2012_06144_gb300 import lbm

    prob, phi0, desc = workload(args.workload, args.size)
    prob, phi0, desc = apply_pair(args, prob, phi0, desc)
    if args.pair != "15+27" and args.precision != "fp32":
        raise SystemExit("other lattice pairs run with FP32 storage")
    N = prob.ncells
    q, qp = prob.q_hydro, prob.q_phase
    headline = args.pair == "15+27" and args.precision == "fp32" and args.workload == "roofline" and args.form == "fused"
    stream = torch.cuda.Stream()
    sim = lbm.Simulation.from_problem(prob, precision=args.precision, form=args.form, stream=stream)
    phi0_dev = torch.from_numpy(phi0).cuda()
    torch.cuda.synchronize()
    sim.init_phase(phi0_dev)
    sim.step(args.warmup)
    sim.synchronize()

    # ---- device-resident timing: one event pair around every launch on the library's stream
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    t_all0, t_all1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        t_all0.record(stream)
        for k in range(args.steps):
            starts[k].record(stream)
            sim.step(1)
            ends[k].record(stream)
        t_all1.record(stream)
        torch.cuda.synchronize()
    barrier()
    sim.synchronize()
    total_ms = max_over_ranks(t_all0.elapsed_time(t_all1), world, "cuda")
    launch_ms = float(np.mean([s.elapsed_time(e) for s, e in zip(starts, ends)]))
    value = job_mlups(world, N, args.steps, total_ms / 1e3)

    # ---- end to end through the C ABI with pinned host buffers
    e2e = None
    if not args.no_e2e:
        host_phi0 = torch.from_numpy(phi0).pin_memory()
        host_phi = torch.empty(prob.shape, dtype=torch.float32).pin_memory()
        host_u = torch.empty((3,) + prob.shape, dtype=torch.float32).pin_memory()
        host_p = torch.empty(prob.shape, dtype=torch.float32).pin_memory()
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lbm.lbm_init_phase(sim.handle, host_phi0.data_ptr(), 0)
        lbm.lbm_step(sim.handle, args.steps)
        diag = lbm.lbm_reduce(sim.handle)
        lbm.lbm_get_fields(sim.handle, host_phi.data_ptr(), host_u.data_ptr(), host_p.data_ptr(), 0)
        dt = max_over_ranks(time.perf_counter() - t0, world, "cuda")
        barrier()
        e2e = {"value": job_mlups(world, N, args.steps, dt), "unit": UNIT,
               "h2d_bytes_per_step": N * 4 / args.steps,
               "d2h_bytes_per_step": (5 * N * 4 + 8 * lbm.LBM_DIAG_COUNT) / args.steps,
               "mass_drift": float(diag[0] / float(phi0.astype(np.float64).sum()) - 1.0)}

    peak, peak_kind = measured_hbm_peak()
    algo_bytes = N * bytes_per_cell(q, args.precision, qp)
    achieved = algo_bytes / (launch_ms / 1e3) / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "roof_mlups": roofline_mlups(peak, bytes_per_cell(q, args.precision, qp)),
            "traffic": recorded_traffic(args.workload, N) if headline else None, "peak_kind": peak_kind,
            "kernel": step_kernel_name(args, prob),
            "algorithmic_bytes_per_cell": bytes_per_cell(q, args.precision, qp),
            "launch_ms": launch_ms}

    sim.close()
    if rank == 0 and not args.no_pattern and headline:
        torch.cuda.empty_cache()
        roof["pattern_ceiling"] = pattern_ceiling(args.size, achieved)
    forms = None
    if rank == 0 and not args.no_precision and headline:
        forms = precision_forms(args, stream, peak)
        if forms and isinstance(roof.get("pattern_ceiling"), dict):
            forms["pattern_ceiling"] = pattern_ceiling_16bit(roof["pattern_ceiling"].get("probe"), forms)
    batched = None
    if rank == 0 and not args.no_batched and headline:
        batched = batched_form(args, stream, peak)
    unfused = None
    if rank == 0 and not args.no_unfused and headline:
        unfused = unfused_form(args, prob, phi0_dev, stream, peak, launch_ms)
    pairs = None
    if rank == 0 and not args.no_pairs and headline:
        pairs = stencil_pairs(args, prob, phi0_dev, stream, peak)
    rising = None
    if rank == 0 and not args.no_rising and headline:
        rising = rising_bubble_form(args, stream)

    if rank == 0:
        cpu = None if args.no_cpu_baseline else cpu_baseline()
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": run_config(args, desc, N, q, args.precision, world, qp),
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks.summary(),
            "gpu_launches": args.steps, "precision_forms": forms, "batched_form": batched,
            "rising_bubble": rising, "unfused_form": unfused, "stencil_pairs": pairs,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
