"""Benchmark of the RRMHD lattice Boltzmann step (arXiv:1508.03452) on GB300.

Workload (one "step" = one lattice Boltzmann time step of every run): the
resistive current sheet on a 1024 x 1024 periodic lattice, B_y = 0.1 x the
periodic double tanh of width 8 cells, n = p = 1, u = 0, three runs with sigma =
10, 100, 1000, float32 populations (the configuration the headline MLUPS metric
is quoted on). Inputs are synthetic (seeded analytic fields); the state of one
run (1.2 GB read + written per step) is far larger than L2, so no flush is done.

Arms:
  default            the CUDA library (C ABI through the Python binding)
  --impl reference   the FP64 CPU oracle on the host cores, each step a bounded
                     sample (a 1024 x 32 strip of the sigma = 100 run)

The default arm also reports, under "learned_seed", the same workload with the
recovery seeded by the learned network (trained on the GPU, before that leg's
timed region, from samples of the method's own current-sheet and
Kelvin-Helmholtz runs): its MLUPS and eigen-solve iterations per cell beside
the plain path's, and both float32 arms' errors against the float64 GPU build;
and, under "batched_sweep", the 64-run uneven-grid Kelvin-Helmholtz sweep in
one handle: one launch per run per step against the autotuned schedule
replayed from CUDA graphs; and, under "flux_rope_3d", the driven 3-D flux rope
(256^3, open faces, the lowest layers driven) with the plain and the learned
seed.

Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS/GPU and HBM-roofline %, mixed+learned vs plain FP32 at matched error"
UNIT = "MLUPS"
SIGMAS = (10.0, 100.0, 1000.0)
NX = NY = 1024
# algorithmic bytes per cell update of the fused step: 63 populations + 12
# primitives, each read once and written once
BYTES_PER_CELL = {"fp64": 2 * (63 + 12) * 8, "fp32": 2 * (63 + 12) * 4, "fp16": 2 * (38 * 2 + 25 * 4 + 12 * 4)}
PROFILE = os.path.join(ROOT, "profiles", "step_kernel_current_sheet_1024.md")
KERNEL_SOURCES = ["step_impl.cuh", "lattice.cuh", "common.cuh", "mlp.cuh", "tma.cuh"]
GROUPS = {"n": (0,), "p": (1,), "eps": (2,), "u": (3, 4, 5), "E": (6, 7, 8), "B": (9, 10, 11)}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x: float, dist=None, device="cpu") -> float:
    """The largest of the ranks' values (the job is as slow as its slowest rank)."""
    if dist is None:
        return float(x)
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(world: int, cells_per_rank: int, steps: int, seconds: float) -> float:
    """Cell updates of all ranks per second, in millions (weak scaling: every
    rank runs the same workload)."""
    return world * cells_per_rank * steps / seconds / 1e6


def code_only(src: str) -> str:
    """C++/CUDA source without its comments, trailing blanks and empty lines:
    what the compiler sees (the sources hold no string literal with a comment
    marker)."""
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    lines = (re.sub(r"//.*", "", line).rstrip() for line in src.splitlines())
    return "\n".join(line for line in lines if line)


def kernel_sha() -> str:
    """Identity of the step kernel's code (comments excluded) and of the nvcc
    flags it is compiled with (include paths excluded), which the committed
    ncu summary records beside the counters it took."""
    from paper_1508_03452_gb300 import build as B

    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1508_03452_gb300", "csrc", name)) as f:
            h.update(code_only(f.read()).encode())
    h.update(" ".join(B.ARCH + [f for f in B.NVCC_FLAGS if not f.startswith("-I")]).encode())
    return h.hexdigest()[:16]


def profiled_traffic(precision: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel sources."""
    try:
        text = open(PROFILE).read()
    except OSError:
        return None
    m_sha = re.search(r"kernel_sources_sha:\s*([0-9a-f]+)", text)
    m_b = re.search(rf"dram_bytes_per_launch_{precision}:\s*([0-9.eE+]+)", text)
    if not m_sha or not m_b or m_sha.group(1) != kernel_sha():
        return None
    return float(m_b.group(1))


def profiled_instructions(precision: str):
    """Warp instructions per cell of the step kernel from the committed ncu
    summary, if it was taken on the current kernel sources."""
    try:
        text = open(PROFILE).read()
    except OSError:
        return None
    m_sha = re.search(r"kernel_sources_sha:\s*([0-9a-f]+)", text)
    m_i = re.search(rf"warp_instructions_per_cell_{precision}:\s*([0-9.eE+]+)", text)
    if not m_sha or not m_i or m_sha.group(1) != kernel_sha():
        return None
    return float(m_i.group(1))


def issue_ceiling(instr_per_cell, sms: int, sm_mhz: float):
    """Cell updates per second, in millions, if every scheduler issued every
    cycle: one thread per cell, so a warp instruction serves 32 cells; four
    schedulers per SM."""
    if not instr_per_cell or not sms or not sm_mhz:
        return None
    return sms * 4 * sm_mhz * 1e6 * 32 / instr_per_cell / 1e6


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        return None


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index, self.proc, self.path, self.skip = index, None, None, 0

    def __enter__(self):
        try:
            import tempfile

            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            # the timed region starts once the sampler is running
            t0 = time.time()
            while time.time() - t0 < 5.0 and self.proc.poll() is None and os.path.getsize(self.path) == 0:
                time.sleep(0.02)
            self.skip = sum(1 for _ in open(self.path))
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return None
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for k, line in enumerate(open(self.path)):
            if k < self.skip:  # taken before the timed region
                continue
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


def _oracle_strip_mlups(seconds: float, threads: int):
    import oracle as O
    from paper_1508_03452_gb300 import workloads as W

    ny = 32
    F = W.current_sheet(NX, ny, 1, delta=8.0)
    s = O.Sim(O.make_params(NX, ny, 1, sigma=100.0, threads=threads))
    s.init(F.n, F.p, F.u, F.B)
    s.step(1)
    t0 = time.perf_counter()
    steps = 0
    while True:
        s.step(1)
        steps += 1
        if time.perf_counter() - t0 >= seconds:
            break
    el = time.perf_counter() - t0
    return NX * ny * steps / el / 1e6, steps, el


def _oracle_config_mlups(threads: int):
    """The oracle on the other workloads, bounded: config 1 in full (the 64^2
    Alfven wave, sigma = 1e6, 500 steps), config 3 on a 2048 x 16 periodic strip
    of the 2048^2 Kelvin-Helmholtz layers (20 steps), config 5 on a 32^3 flux rope
    (open faces, driven bottom; 10 steps)."""
    import oracle as O
    from paper_1508_03452_gb300 import workloads as W

    out = {}
    cases = [
        ("config1_alfven_64x64_full", W.alfven_wave(64, 64, 1), dict(sigma=1e6), 500),
        ("config3_kh_2048x16_strip",
         W.kelvin_helmholtz(2048, 16, 1, V=0.3, ratio=10.0, B0=0.1, a=2.0, noise=1e-3, seed=3), dict(sigma=1e3), 20),
        ("config5_flux_rope_32^3", W.flux_rope(32, 32, 32),
         dict(sigma=500.0, bc=(O.OPEN,) * 4 + (O.DRIVEN, O.OPEN), drive_u0=0.05, drive_layers=W.drive_layers_for(32)),
         10),
    ]
    for name, F, kw, steps in cases:
        s = O.Sim(O.make_params(F.nx, F.ny, F.nz, threads=threads, **kw))
        s.init(F.n, F.p, F.u, F.B)
        t0 = time.perf_counter()
        s.step(steps)
        el = time.perf_counter() - t0
        out[name] = {"value": F.nx * F.ny * F.nz * steps / el / 1e6, "unit": UNIT, "steps": steps, "seconds": el}
    return out


def cpu_baseline_sample(seconds: float = 12.0, threads: int | None = None):
    """The oracle as it stands on the host cores: the sigma = 100 current sheet,
    full 1024-wide rows, a strip of 32 rows (periodic), stepped for ~`seconds`
    on all cores, and for a quarter of that on one thread; bounded samples of
    the other workloads beside it."""
    threads = threads or os.cpu_count() or 1
    v, steps, el = _oracle_strip_mlups(seconds, threads)
    v1, steps1, el1 = _oracle_strip_mlups(seconds / 4, 1)
    return {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"current sheet sigma=100, {NX}x32 periodic strip of the 1024x1024 workload, {steps} steps, "
                      f"{el:.1f} s, FP64 C oracle with OpenMP",
            "single_thread": {"value": v1, "unit": UNIT, "steps": steps1, "seconds": el1},
            "other_workloads": _oracle_config_mlups(threads)}


def run_reference(args, world, rank):
    if rank != 0:
        return
    import oracle as O
    from paper_1508_03452_gb300 import workloads as W

    threads = os.cpu_count() or 1
    ny = 32
    F = W.current_sheet(NX, ny, 1, delta=8.0)
    s = O.Sim(O.make_params(NX, ny, 1, sigma=100.0, threads=threads))
    s.init(F.n, F.p, F.u, F.B)
    for _ in range(args.warmup):
        s.step(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s.step(1)
    el = time.perf_counter() - t0
    value = NX * ny * args.steps / el / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "current_sheet", "grid": [NX, ny, 1], "sigma": 100.0,
                   "note": "bounded sample of the 1024x1024 workload: a 1024x32 periodic strip per step"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"{NX}x{ny} strip of the sigma=100 current sheet, {args.steps} steps"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def hist_quantile(hist, q):
    """Iteration count at quantile q of a recovery histogram (bin k = k + 1
    iterations; the last bin is open-ended and reported as its lower edge)."""
    import numpy as np
    c = np.cumsum(hist)
    if c[-1] == 0:
        return None
    return int(np.searchsorted(c, q * c[-1]) + 1)


def rel_errors(m, ref):
    import numpy as np
    return {k: float(np.linalg.norm(m[list(r)] - ref[list(r)]) / max(np.linalg.norm(ref[list(r)]), 1e-300))
            for k, r in GROUPS.items()}


def learned_seed_leg(args, stream, plain_moments, plain_iters, steps_total):
    """The same workload with the recovery seeded by the learned network:
    samples from the method's own current-sheet and Kelvin-Helmholtz runs,
    training on the GPU, then the timed steps. Errors of both float32 arms
    are taken against a float64 GPU run of the sigma = 100 run."""
    import numpy as np
    import torch

    from paper_1508_03452_gb300 import lbrmhd as L
    from paper_1508_03452_gb300 import workloads as W

    prec = {"fp32": L.FP32, "fp16": L.FP16_DEV, "fp64": L.FP64}[args.precision]
    t0 = time.perf_counter()
    cases = [(W.current_sheet(256, 64, 1, delta=8.0), 100.0)] + [
        (W.kelvin_helmholtz(256, 128, 1, V=0.2, ratio=10.0, B0=0.1, a=2.0, noise=1e-3, seed=s), 1e3) for s in (11, 12)]
    chunks = []
    for F, sigma in cases:
        s = L.Solver(L.make_params(F.nx, F.ny, 1, sigma=sigma, precision=prec, recovery=L.RECOVERY_COLD),
                     stream=stream)
        s.init_fields(0, F.n, F.p, F.u, F.B)
        buf = torch.full((F.N, L.MLP_ROW), float("nan"), dtype=torch.float32, device="cuda")
        s.set_mlp_samples(0, buf)
        for t in range(40):
            s.step(1)
            if t % 4 == 3:
                chunks.append(buf.clone())
        s.close()
    data = torch.cat(chunks)
    data = data[torch.isfinite(data).all(1)].contiguous()
    P = torch.tensor(W.mlp_init_params(1), device="cuda")
    adam = torch.zeros(2 * L.MLP_NPARAM, device="cuda")
    train_steps = 3000
    losses = L.mlp_train(P, adam, data, train_steps, 1024, 1e-3, seed=7).cpu().numpy()
    train_s = time.perf_counter() - t0

    F = W.current_sheet(NX, NY, 1, delta=8.0)
    N = NX * NY

    def learned_run(precision):
        solver = L.Solver([L.make_params(NX, NY, 1, sigma=sg, precision=precision, recovery=L.RECOVERY_MLP)
                           for sg in SIGMAS], stream=stream)
        solver.set_mlp_weights(P)
        for r in range(len(SIGMAS)):
            solver.init_fields(r, F.n, F.p, F.u, F.B)
        solver.step(steps_total - args.steps)  # the plain leg's warm-up, so that the states compare
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        solver.step(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        stats = [solver.stats(r) for r in range(len(SIGMAS))]
        hist = sum(solver.iteration_histogram(r) for r in range(len(SIGMAS)))
        m = solver.moments(1)
        solver.close()
        return ms, stats, hist, m

    ms, stats, hist, m_mlp = learned_run(prec)
    # mixed precision + learned seed: float16-deviation storage of f, g
    ms_mx, stats_mx, hist_mx, m_mx = learned_run(L.FP16_DEV)
    ref = L.Solver(L.make_params(NX, NY, 1, sigma=SIGMAS[1], precision=L.FP64), stream=stream)
    ref.init_fields(0, F.n, F.p, F.u, F.B)
    ref.step(steps_total)
    m64 = ref.moments(0)
    ref.close()
    cells = len(SIGMAS) * N
    return P, {
        "value": cells * args.steps / (ms * 1e-3) / 1e6, "unit": UNIT,
        "iters_per_cell": sum(s["iter_total"] for s in stats) / (cells * steps_total),
        "iters_p99": hist_quantile(hist, 0.99),
        "plain_iters_per_cell": plain_iters,
        "failures": sum(s["recover_fail"] for s in stats),
        "mixed_fp16dev": {"value": cells * args.steps / (ms_mx * 1e-3) / 1e6, "unit": UNIT,
                          "iters_per_cell": sum(s["iter_total"] for s in stats_mx) / (cells * steps_total),
                          "iters_p99": hist_quantile(hist_mx, 0.99),
                          "failures": sum(s["recover_fail"] for s in stats_mx),
                          "err_vs_fp64": rel_errors(m_mx, m64)},
        "err_vs_fp64": rel_errors(m_mlp, m64), "plain_err_vs_fp64": rel_errors(plain_moments, m64),
        "error_run": f"sigma={SIGMAS[1]}, {steps_total} steps, relative L2 per field against the float64 GPU build",
        "train": {"samples": int(data.shape[0]), "adam_steps": train_steps, "batch": 1024,
                  "loss_first": float(losses[:10].mean()), "loss_last": float(losses[-100:].mean()),
                  "seconds_incl_sampling": train_s},
    }


def batched_sweep_leg(args, stream, steps=10):
    """The batched sweep: 64 independent Kelvin-Helmholtz runs of uneven square
    grids (sides 256..1024 step 128, sigma log-uniform [10, 1e4], V in [0.1,
    0.5] c, density ratio {1, 3, 10}; seeded) in one handle, timed with one
    launch per run per step on one stream, with the autotuned schedule
    replayed from CUDA graphs, and with the persistent schedule (all steps in
    one cooperative launch). The runs take the Gauss-law charge and alpha =
    0.02, the options under which the scheme carries flowing magnetised
    plasma furthest; the leg is marked invalid if any recovery failed in it."""
    import torch

    from paper_1508_03452_gb300 import lbrmhd as L
    from paper_1508_03452_gb300 import workloads as W

    prec = {"fp32": L.FP32, "fp16": L.FP16_DEV, "fp64": L.FP64}[args.precision]
    specs = W.kh_sweep(64)
    solver = L.Solver([L.make_params(sp.nx, sp.ny, 1, sigma=sp.sigma, precision=prec, alpha=0.02,
                                     flags=L.FLAG_GAUSS_CHARGE) for sp in specs], stream=stream)
    for r, sp in enumerate(specs):
        F = W.kelvin_helmholtz(sp.nx, sp.ny, 1, V=sp.V, ratio=sp.ratio, B0=0.1, noise=1e-3, seed=sp.seed)
        solver.init_fields(r, F.n, F.p, F.u, F.B)
    cells = sum(sp.nx * sp.ny for sp in specs)

    def timed(k):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        solver.step(k)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    solver.step(3)
    ms_plain = timed(steps)
    best, tune_ms = solver.autotune(3)
    graph_steps = 10
    sched = L.make_schedule(best.kind, best.bx, best.waves, best.order, best.streams, graph_steps)
    solver.set_schedule(sched)
    solver.step(graph_steps)  # captures the graphs
    ms_tuned = timed(steps)
    solver.set_schedule(L.make_schedule(L.SCHED_PERSISTENT, 128, 1, 0, 1, 0))
    ms_persist = timed(steps)
    status = solver.status()
    per_run_fail = [solver.stats(r)["recover_fail"] for r in range(len(specs))]
    fails = sum(per_run_fail)
    solver.close()
    stable = stable_sweep(args, stream, steps)
    return {
        "workload": "kh_sweep_64_runs_sides_256_1024", "runs": len(specs), "cells_per_step": cells, "steps": steps,
        "value": cells * steps / (ms_tuned * 1e-3) / 1e6, "unit": UNIT,
        "per_run_one_stream_mlups": cells * steps / (ms_plain * 1e-3) / 1e6,
        "persistent_mlups": cells * steps / (ms_persist * 1e-3) / 1e6,
        "schedule": sched.as_dict(), "autotune_ms_per_step": tune_ms, "recover_fail": fails,
        "status_bits": status["bits"], "valid": fails == 0 and status["bits"] == 0,
        "runs_with_failures": sum(1 for f in per_run_fail if f),
        "options": "Gauss-law charge (LBRMHD_FLAG_GAUSS_CHARGE), alpha = 0.02",
        "stable_range": stable,
    }


def stable_sweep(args, stream, steps):
    """The same 64 uneven grids and conductivities with the shear drawn inside
    the scheme's stable range (V uniform in [0.05, 0.15] c, uniform density;
    Gauss-law charge, alpha = 0.02): the autotuned schedule from graphs."""
    import numpy as np
    import torch

    from paper_1508_03452_gb300 import lbrmhd as L
    from paper_1508_03452_gb300 import workloads as W

    prec = {"fp32": L.FP32, "fp16": L.FP16_DEV, "fp64": L.FP64}[args.precision]
    specs = W.kh_sweep(64)
    rng = np.random.Generator(np.random.PCG64(2015))
    Vs = rng.uniform(0.05, 0.15, len(specs))
    solver = L.Solver([L.make_params(sp.nx, sp.ny, 1, sigma=sp.sigma, precision=prec, alpha=0.02,
                                     flags=L.FLAG_GAUSS_CHARGE) for sp in specs], stream=stream)
    for r, (sp, V) in enumerate(zip(specs, Vs)):
        F = W.kelvin_helmholtz(sp.nx, sp.ny, 1, V=float(V), ratio=1.0, B0=0.1, noise=1e-3, seed=sp.seed)
        solver.init_fields(r, F.n, F.p, F.u, F.B)
    cells = sum(sp.nx * sp.ny for sp in specs)
    solver.step(3)
    best, _ = solver.autotune(3)
    solver.set_schedule(L.make_schedule(best.kind, best.bx, best.waves, best.order, best.streams, 10))
    solver.step(10)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    solver.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    fails = sum(solver.stats(r)["recover_fail"] for r in range(len(specs)))
    status = solver.status()
    solver.close()
    return {"value": cells * steps / (e0.elapsed_time(e1) * 1e-3) / 1e6, "unit": UNIT, "V_range": [0.05, 0.15],
            "density_ratio": 1.0, "recover_fail": fails, "valid": fails == 0 and status["bits"] == 0,
            "schedule": best.as_dict()}


def kh_2048_leg(args, stream, steps=10):
    """Config 3: Kelvin-Helmholtz shear layers on a 2048^2 periodic lattice
    (V = 0.3 c, density ratio 10, B0 = 0.1, sigma = 1e3, seeded noise 1e-3),
    float32 against float16-deviation storage (float32 arithmetic), each timed
    over `steps` steps after 3 warm-up steps, with both errors against a
    float64 GPU run of the same 13 steps."""
    import torch

    from paper_1508_03452_gb300 import lbrmhd as L
    from paper_1508_03452_gb300 import workloads as W

    n = 2048
    F = W.kelvin_helmholtz(n, n, 1, V=0.3, ratio=10.0, B0=0.1, a=2.0, noise=1e-3, seed=3)
    out = {"workload": "kh_2048x2048_V0.3_ratio10_sigma1e3", "grid": [n, n, 1], "steps": steps}
    moms = {}
    for name, prec in (("fp32", L.FP32), ("fp16_dev", L.FP16_DEV), ("fp64", L.FP64)):
        s = L.Solver(L.make_params(n, n, 1, sigma=1e3, precision=prec), stream=stream)
        s.init_fields(0, F.n, F.p, F.u, F.B)
        s.step(3)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        st = s.stats()
        moms[name] = s.moments()
        tiled = s.status()["tiled_runs"]
        s.close()
        out[name] = {"value": n * n * steps / (e0.elapsed_time(e1) * 1e-3) / 1e6, "unit": UNIT,
                     "iters_per_cell": st["iter_total"] / (n * n * (steps + 3)), "failures": st["recover_fail"],
                     "tile_kernel": bool(tiled)}
    for name in ("fp32", "fp16_dev"):
        out[name]["err_vs_fp64"] = rel_errors(moms[name], moms["fp64"])
    return out


def flux_rope_case(n, prec, recovery):
    from paper_1508_03452_gb300 import lbrmhd as L
    from paper_1508_03452_gb300 import workloads as W

    F = W.flux_rope(n, n, n)
    bc = (L.OPEN,) * 4 + (L.DRIVEN, L.OPEN)  # open faces, driven bottom (z = 0)
    P = L.make_params(n, n, n, bc=bc, sigma=500.0, drive_u0=0.05, drive_layers=W.drive_layers_for(n),
                      precision=prec, recovery=recovery)
    return F, P


RECONNECTION_CASES = [(0.2, 20.0), (0.2, 30.0), (0.2, 50.0), (0.2, 70.0), (0.2, 100.0), (0.4, 100.0)]
RECONNECTION_TIMES = [0.4, 1.2, 2.4, 4.8, 9.6, 23.2]


def reconnection_leg(args, stream, n=512, t_end=23.2, every=0.4):
    """Sec. IV's Kelvin-Helmholtz-driven reconnection on the paper's lattice
    (n^2 on [-0.5, 0.5]^2, dx/dt = 2.5 sqrt 2, periodic x, open y, one layer of
    width dx, B0 = 0.06, u_pert = 0.01) for the cases the scheme carries to the
    paper's final time t = 23.2: uniform density (dn = 0), with the Gauss-law
    charge and alpha = 0.02 (the paper's dn = 1.8 and U0 = 0.6 c runs, and its
    own charge moment and alpha = 0.1, break down within t ~ 1). All runs in one
    handle: U0 = 0.2 c at sigma = 20, 30, 50, 70, 100 and U0 = 0.4 c at sigma =
    100. R(t) = (E^z - E^z_0) / B0 at the null point of the 128 rows around the
    layer, every `every` time units; reported: R at a few times, the log-log
    slope of |R| against sigma at each (Sweet-Parker: -1/2), the ratio of the
    two U0 at sigma = 100, recovery failures and the throughput of the leg."""
    import numpy as np
    import torch

    from paper_1508_03452_gb300 import lbrmhd as L
    from paper_1508_03452_gb300 import workloads as W

    prec = {"fp32": L.FP32, "fp16": L.FP16_DEV, "fp64": L.FP64}[args.precision]
    dx = 1.0 / n
    dt = dx / (math.sqrt(2.0) * 2.5)
    total = int(round(t_end / dt))
    chunk = max(1, int(round(every / dt)))
    bc = (L.PERIODIC, L.PERIODIC, L.OPEN, L.OPEN, L.PERIODIC, L.PERIODIC)
    params = [L.make_params(n, n, 1, bc=bc, tau=1.0, sigma=sg, alpha=0.02, c=2.5, dx=dx, precision=prec,
                            flags=L.FLAG_GAUSS_CHARGE) for _, sg in RECONNECTION_CASES]
    s = L.Solver(params, stream=stream)
    for r, (U0, _) in enumerate(RECONNECTION_CASES):
        F = W.kelvin_helmholtz_paper(n, U0=U0, dn=0.0)
        s.init_fields(r, F.n, F.p, F.u, F.B)
    lo, hi = n // 2 - 64, n // 2 + 64
    series = [[] for _ in RECONNECTION_CASES]
    step = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    while step < total:
        k = min(chunk, total - step)
        s.step(k)
        step += k
        for r in range(len(RECONNECTION_CASES)):
            series[r].append((step * dt, s.reconnection_rate(r, lo, hi, 0.06)["R"]))
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    fails = [s.stats(r)["recover_fail"] for r in range(len(RECONNECTION_CASES))]
    s.close()

    def at(r, t):
        return min(series[r], key=lambda p: abs(p[0] - t))[1]

    sig_runs = [r for r, (U0, _) in enumerate(RECONNECTION_CASES) if U0 == 0.2]
    logs = np.log([RECONNECTION_CASES[r][1] for r in sig_runs])
    out = {"workload": f"kh_paper_{n}x{n}_dn0_gauss_charge_alpha0.02", "t_end": t_end, "steps": total,
           "cases": [{"U0": U0, "sigma": sg, "failures": f} for (U0, sg), f in zip(RECONNECTION_CASES, fails)],
           "value": len(RECONNECTION_CASES) * n * n * total / wall / 1e6, "unit": UNIT,
           "timing": "wall clock over the steps and the R(t) calls", "R": {}, "sigma_slope": {},
           "U0_ratio_sigma100": {}}
    r02, r04 = RECONNECTION_CASES.index((0.2, 100.0)), RECONNECTION_CASES.index((0.4, 100.0))
    for t in RECONNECTION_TIMES:
        key = f"{t:g}"
        out["R"][key] = [at(r, t) for r in range(len(RECONNECTION_CASES))]
        mag = np.abs([at(r, t) for r in sig_runs])
        if np.all(np.isfinite(mag)) and np.all(mag > 0):
            out["sigma_slope"][key] = float(np.polyfit(logs, np.log(mag), 1)[0])
        out["U0_ratio_sigma100"][key] = abs(at(r04, t)) / max(abs(at(r02, t)), 1e-300)
    return out


def flux_rope_leg(args, stream, weights, n=256, steps=10):
    """The driven 3-D flux rope (the paper's stellar-flare set-up, sigma = 500,
    open faces, the lowest layers driven at 0.05 c) on an n^3 lattice: plain
    and learned seed (the network of the learned-seed leg), 3 warm-up and
    `steps` timed steps each, one run per handle."""
    import torch

    from paper_1508_03452_gb300 import lbrmhd as L

    prec = {"fp32": L.FP32, "fp16": L.FP16_DEV, "fp64": L.FP64}[args.precision]
    out = {"workload": f"flux_rope_{n}^3_sigma_500_open_driven", "grid": [n, n, n], "steps": steps}
    for name, rec in (("plain", L.RECOVERY_PLAIN), ("learned_seed", L.RECOVERY_MLP)):
        if rec == L.RECOVERY_MLP and weights is None:
            continue
        F, P = flux_rope_case(n, prec, rec)
        s = L.Solver(P, stream=stream)
        if rec == L.RECOVERY_MLP:
            s.set_mlp_weights(weights)
        s.init_fields(0, F.n, F.p, F.u, F.B)
        s.step(3)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        st = s.stats()
        s.close()
        out[name] = {"value": n ** 3 * steps / (e0.elapsed_time(e1) * 1e-3) / 1e6, "unit": UNIT,
                     "iters_per_cell": st["iter_total"] / (n ** 3 * (steps + 3)), "failures": st["recover_fail"]}
    out["paper_forced"] = paper_flare_case(stream, n, steps, prec)
    return out


def paper_flare_case(stream, n, steps, prec):
    """The paper's flare run (Sec. IV): [-3, 3]^2 x [0, 6] on n^3 cells, every
    face open, sigma = 100, dx/dt = 2.5 sqrt 2 (c = 2.5), background field
    rescaled to B0 = 0.06, E and J relaxed with the fields held, then the
    two-vortex photospheric force F0 = 0.05 while max |u| < 0.3 c."""
    import numpy as np
    import torch

    from paper_1508_03452_gb300 import lbrmhd as L
    from paper_1508_03452_gb300 import workloads as W

    F = W.flux_rope(n, n, n, B_bg=0.06)
    c = 2.5
    P = L.make_params(n, n, n, bc=(L.OPEN,) * 6, sigma=100.0, c=c, dx=6.0 / n, drive_layers=W.drive_layers_for(n),
                      drive_f0=0.05, drive_vmax=0.3 * c, precision=prec)
    s = L.Solver(P, stream=stream)
    t0 = time.perf_counter()
    relax_steps, relax_res = s.init_fields_relaxed(0, F.n, F.p, F.u, F.B, max_iters=100, tol=1e-6)
    relax_s = time.perf_counter() - t0
    s.step(3)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    st = s.stats()
    m = s.moments()
    s.close()
    return {"value": n ** 3 * steps / (e0.elapsed_time(e1) * 1e-3) / 1e6, "unit": UNIT,
            "iters_per_cell": st["iter_total"] / (n ** 3 * (steps + 3)), "failures": st["recover_fail"],
            "relax": {"steps": relax_steps, "residual": relax_res, "seconds": relax_s},
            "max_u_over_c": float(np.sqrt((m[3:6] ** 2).sum(0)).max() / c)}


def run_gpu(args, world, rank, local):
    import numpy as np
    import torch

    from paper_1508_03452_gb300 import lbrmhd as L
    from paper_1508_03452_gb300 import workloads as W

    if not torch.cuda.is_available():
        raise SystemExit("bench.py: no CUDA device (the library has no CPU path)")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    prec = {"fp32": L.FP32, "fp16": L.FP16_DEV, "fp64": L.FP64}[args.precision]
    F = W.current_sheet(NX, NY, 1, delta=8.0)
    params = [L.make_params(NX, NY, 1, sigma=s, precision=prec) for s in SIGMAS]
    stream = torch.cuda.current_stream()
    solver = L.Solver(params, stream=stream)
    N = NX * NY
    # device-resident inputs (float64) for the timed device run
    dev = {k: torch.from_numpy(np.ascontiguousarray(v, dtype=np.float64)).cuda() for k, v in
           (("n", F.n), ("p", F.p), ("u", F.u), ("B", F.B))}
    for r in range(len(SIGMAS)):
        solver.init_fields_device(r, dev["n"], dev["p"], dev["u"], dev["B"])
    # the library's launch schedule for this handle: the autotuner's choice
    # (its dry steps leave the state as it was), replayed from 10-step graphs,
    # both set up before the timed region
    graph_steps = 10
    best, _ = solver.autotune(3)
    sched = L.make_schedule(best.kind, best.bx, best.waves, best.order, best.streams, graph_steps)
    solver.set_schedule(sched)
    solver.step(max(args.warmup, graph_steps))
    torch.cuda.synchronize()

    def barrier():
        if dist is not None:
            dist.barrier()

    cells = N * len(SIGMAS)
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        solver.step(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
    ms = max_over_ranks(e0.elapsed_time(e1), dist, "cuda")
    stats = [solver.stats(r) for r in range(len(SIGMAS))]
    steps_total = max(args.warmup, graph_steps) + args.steps
    plain_iters = sum(s["iter_total"] for s in stats) / (len(SIGMAS) * N * steps_total)
    plain_hist = sum(solver.iteration_histogram(r) for r in range(len(SIGMAS)))
    plain_moments = solver.moments(1) if (rank == 0 and not args.no_learned_seed) else None
    status = solver.status()
    kernel_name = "lb::step_tile_kernel" if status["tiled_runs"] == len(SIGMAS) else "lb::step_kernel"
    launches = args.steps * len(SIGMAS)
    value = whole_job_mlups(world, cells, args.steps, ms * 1e-3)
    # roofline of the dominant (only) kernel of the timed region: the fused step
    bpc = BYTES_PER_CELL[args.precision]
    avg_launch_s = ms * 1e-3 / launches
    achieved = bpc * N / avg_launch_s / 1e9
    peaks = measured_peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    traffic = profiled_traffic(args.precision)

    # end to end through the C ABI with host buffers: host -> device inputs,
    # K steps, device -> host moments of every run
    pin = {k: torch.from_numpy(np.ascontiguousarray(v, dtype=np.float64)).pin_memory() for k, v in
           (("n", F.n), ("p", F.p), ("u", F.u), ("B", F.B))}
    out_host = torch.empty(L.NMOMENTS * N, dtype=torch.float64).pin_memory()
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for r in range(len(SIGMAS)):
        solver.init_fields(r, pin["n"].numpy(), pin["p"].numpy(), pin["u"].numpy(), pin["B"].numpy())
    solver.step(args.steps)
    for r in range(len(SIGMAS)):
        solver._check(solver._L.lbrmhd_get_moments(solver._h, r, L._dp(out_host.numpy())))
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    barrier()
    h2d = len(SIGMAS) * N * 8 * (1 + 1 + 3 + 3)
    d2h = len(SIGMAS) * N * 8 * L.NMOMENTS
    e2e_value = whole_job_mlups(world, cells, args.steps, e2e_s)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"fp32": "f32", "fp16": "f16-storage/f32", "fp64": "f64"}[args.precision],
            "data": "synthetic",
            "config": {"workload": "current_sheet_1024x1024_sigma_10_100_1000", "grid": [NX, NY, 1],
                       "runs": len(SIGMAS), "sigma": list(SIGMAS), "precision": args.precision,
                       "boundaries": "periodic", "l2": "no flush: state per run 1.2 GB >> L2",
                       "schedule": sched.as_dict(), "warmup_steps_run": steps_total - args.steps,
                       "parallelism": f"replicas{world}" if world > 1 else "single"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": kernel_name, "bytes_per_cell": bpc,
                         "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)" if peaks else "fallback"},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d / args.steps,
                    "d2h_bytes_per_step": d2h / args.steps},
            "gpu_launches": launches,
            "recovery": {"iters_mean": plain_iters, "iters_p99": hist_quantile(plain_hist, 0.99),
                         "iters_max": max(s["iter_max"] for s in stats),
                         "failures": sum(s["recover_fail"] for s in stats)},
        }
        weights = None
        if plain_moments is not None:
            weights, line["learned_seed"] = learned_seed_leg(args, stream, plain_moments, plain_iters, steps_total)
        if not args.no_sweep:
            line["batched_sweep"] = batched_sweep_leg(args, stream)
        if not args.no_kh2048:
            line["kh_2048"] = kh_2048_leg(args, stream)
        if not args.no_3d:
            line["flux_rope_3d"] = flux_rope_leg(args, stream, weights)
        if not args.no_reconnection:
            line["reconnection"] = reconnection_leg(args, stream)
        clocks = clk.summary()
        if clocks:
            line["clocks"] = clocks
        ipc = profiled_instructions(args.precision)
        sms = torch.cuda.get_device_properties(local).multi_processor_count
        ceil = issue_ceiling(ipc, sms, (clocks or {}).get("sm_max_mhz") or (peaks or {}).get("sm_max_mhz"))
        if ceil:
            # the kernel is issue-bound: its instruction count at full issue against the achieved rate
            line["issue_roofline"] = {"warp_instructions_per_cell": ipc, "sms": sms, "ceiling_mlups": ceil,
                                      "frac": value / ceil, "source": "ncu instruction count in the profile summary"}
        if not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline_sample(args.cpu_seconds)
        print(json.dumps(line), flush=True)
    solver.close()
    if dist is not None:
        dist.destroy_process_group()


def run_profile_kernel(args):
    """Small untimed cases for ncu captures of the library's other kernels
    (--profile-kernel): `tile` the TMA tile kernel on the 1024^2 current sheet
    (LBRMHD_FLAG_TMA_TILES); `batch` and `persistent` 16 Kelvin-Helmholtz runs of
    the batched sweep (sides 256..1024) under the BATCH and PERSISTENT schedules;
    `diag` the conservation diagnostics and `null` the reconnection-rate null
    search of a 1024^2 run; `mlp` the learned seed's training (gradient,
    reduction, Adam) on 2^20 synthetic sample rows; each for `--steps` calls."""
    import numpy as np
    import torch

    from paper_1508_03452_gb300 import lbrmhd as L
    from paper_1508_03452_gb300 import workloads as W

    stream = torch.cuda.current_stream()
    k = args.profile_kernel
    n = args.steps
    if k in ("tile", "diag", "null"):
        F = W.current_sheet(NX, NY, 1, delta=8.0) if k != "null" else W.kelvin_helmholtz(
            NX, NY, 1, V=0.2, ratio=3.0, B0=0.1, a=2.0, noise=1e-3, seed=5)
        flags = L.FLAG_TMA_TILES if k == "tile" else 0
        s = L.Solver(L.make_params(NX, NY, 1, sigma=100.0, precision=L.FP32, flags=flags), stream=stream)
        s.init_fields(0, F.n, F.p, F.u, F.B)
        if k == "tile":
            s.step(n)
        else:
            s.step(2)
            for _ in range(n):
                if k == "diag":
                    s.diagnostics()
                else:
                    s.reconnection_rate(0, NY // 4 - 64, NY // 4 + 64, 0.1)
        out = s.status()
        s.close()
    elif k in ("batch", "persistent"):
        specs = W.kh_sweep(16)
        s = L.Solver([L.make_params(sp.nx, sp.ny, 1, sigma=sp.sigma, precision=L.FP32, alpha=0.02,
                                    flags=L.FLAG_GAUSS_CHARGE) for sp in specs], stream=stream)
        for r, sp in enumerate(specs):
            F = W.kelvin_helmholtz(sp.nx, sp.ny, 1, V=sp.V, ratio=sp.ratio, B0=0.1, noise=1e-3, seed=sp.seed)
            s.init_fields(r, F.n, F.p, F.u, F.B)
        kind = L.SCHED_BATCH if k == "batch" else L.SCHED_PERSISTENT
        s.set_schedule(L.make_schedule(kind, 128, 1, 0, 1, 0))
        s.step(n)
        out = s.status()
        s.close()
    else:  # mlp
        rows = 1 << 20
        g = torch.Generator(device="cuda").manual_seed(5)
        data = torch.rand(rows * L.MLP_ROW, generator=g, device="cuda", dtype=torch.float32) - 0.5
        P = torch.tensor(W.mlp_init_params(1), device="cuda")
        adam = torch.zeros(2 * L.MLP_NPARAM, device="cuda")
        L.mlp_train(P, adam, data, n, 4096, 1e-3, seed=3)
        out = {"rows": rows}
    torch.cuda.synchronize()
    print(json.dumps({"profile_kernel": k, "calls": n, "out": out}), flush=True)


def run_profile_case(args):
    """Small profiling case (no timing): one 1024 x 1024 current-sheet run
    (sigma = 100), or with --profile-3d N the driven N^3 flux rope, in the
    chosen precision, init + `--steps` steps."""
    import torch

    from paper_1508_03452_gb300 import lbrmhd as L
    from paper_1508_03452_gb300 import workloads as W

    prec = {"fp32": L.FP32, "fp16": L.FP16_DEV, "fp64": L.FP64}[args.precision]
    rec = L.RECOVERY_MLP if args.profile_learned else L.RECOVERY_PLAIN
    if args.profile_3d:
        F, P = flux_rope_case(args.profile_3d, prec, rec)
    else:
        F = W.current_sheet(NX, NY, 1, delta=8.0)
        P = L.make_params(NX, NY, 1, sigma=100.0, precision=prec, recovery=rec)
    s = L.Solver(P, stream=torch.cuda.current_stream())
    if args.profile_learned:  # untrained weights: the inference cost, not the seed quality
        s.set_mlp_weights(torch.tensor(W.mlp_init_params(1), device="cuda"))
    s.init_fields(0, F.n, F.p, F.u, F.B)
    s.step(args.steps)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": args.precision, "steps": args.steps, "stats": s.stats()}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp16", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-learned-seed", action="store_true", help="skip the learned-seed comparison leg")
    ap.add_argument("--no-sweep", action="store_true", help="skip the 64-run batched sweep leg")
    ap.add_argument("--no-3d", action="store_true", help="skip the 3-D flux-rope leg")
    ap.add_argument("--no-kh2048", action="store_true", help="skip the 2048^2 Kelvin-Helmholtz leg")
    ap.add_argument("--no-reconnection", action="store_true", help="skip the Kelvin-Helmholtz reconnection-rate leg")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--profile-case", action="store_true", help="untimed 1024^2 single-run case for ncu captures")
    ap.add_argument("--profile-learned", action="store_true", help="--profile-case with the learned-seed kernel")
    ap.add_argument("--profile-3d", type=int, default=0, metavar="N", help="--profile-case on the driven N^3 flux rope")
    ap.add_argument("--profile-kernel", default="", choices=["", "tile", "batch", "persistent", "diag", "null", "mlp"],
                    help="untimed small case for an ncu capture of one of the other kernels")
    args = ap.parse_args()
    world, rank, local = dist_env()
    if args.profile_kernel:
        run_profile_kernel(args)
    elif args.profile_case:
        run_profile_case(args)
    elif args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_gpu(args, world, rank, local)


if __name__ == "__main__":
    main()
