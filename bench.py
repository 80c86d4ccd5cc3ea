"""Benchmark: RANS cell-updates/s of the GB300 step on the 256 x 256 x 64 urban block.

One "step" is one full time step of the hot path: CFL dt, eddy viscosity,
MacCormack advection, diffusion, porosity drag + BCs, pressure right-hand
side, MG-preconditioned CG pressure solve, projection and the k-omega
update, FP32 fields with FP64 reductions.  Inputs are resident in HBM when the
timed region starts.  The workload is the seeded synthetic urban block (40
solid boxes + 60 porous canopies, seed = rank, log-law inflow 3 m/s at 10 m);
its per-step working set (~400 MB) exceeds the 129 MB L2, so no flush is
needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

The line also carries "adjoint": the adjoint/forward time ratio on the
128 x 128 x 48 parametric design workload (see adjoint_leg), with one
iteration of the gradient-descent design loop and its wind-direction
robustness re-runs (see design_loop_leg), and "batched":
32 instances of uneven size and wind direction advanced by the batched
persistent launches, against the same instances stepped one after another
(see batched_leg).

Multi-GPU: replicas only (each rank advances its own independent grid; no
collective in the data path), weak scaling; rank 0 prints one JSON line.
``--impl reference`` times the FP64 CPU oracle on the host cores instead.

Other measurements, each printing its own JSON line instead of the bench
line: ``--large`` (plain FP64 vs FP32 on the 512 x 512 x 128 block, with the
adjoint over the last 100 steps), ``--karman`` (vortex-shedding validation
against the Strouhal relation), ``--mesh`` (mesh resolver throughput) and
``--preconditioners`` (CG iterations and step time per preconditioner).
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

METRIC = "RANS cell-updates/s at 256x256x64 FP32 (% HBM roofline); adjoint/forward time"
UNIT = "cell-updates/s"
NX, NY, NZ = 256, 256, 64


def workload_config(extra=None):
    cfg = {
        "workload": "urban block 256x256x64, h=2 m, 40 solid boxes + 60 porous canopies (seeded), "
                    "log-law inflow 3 m/s at 10 m, FP32 fields + FP64 reductions, MG-preconditioned CG",
        "nx": NX, "ny": NY, "nz": NZ, "cells": NX * NY * NZ,
        "l2": "no flush: per-step working set ~400 MB > 129 MB L2",
    }
    if extra:
        cfg.update(extra)
    return cfg


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_scalar(x: float, op: str) -> float:
    """All-reduce of one number over the ranks of the default process group
    ("max" or "sum"); the identity without one.  The tensor lives on the GPU
    for NCCL and on the host for gloo."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return x
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def weak_scaling_rate(cells_local: float, steps: int, seconds_local: float):
    """Replicas: each rank advances its own grid.  Whole-job rate = cells of
    all ranks x steps / the slowest rank's time.  Returns (rate, slowest)."""
    cells = reduce_scalar(float(cells_local), "sum")
    slowest = reduce_scalar(float(seconds_local), "max")
    return cells * steps / slowest, slowest


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.hw_slowdown",
              "clocks_event_reasons.hw_thermal_slowdown", "clocks_event_reasons.sw_thermal_slowdown",
              "clocks_event_reasons.sw_power_cap"]

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.out = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()
        return False

    def summary(self):
        if not self.out:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# The headers the profiled kernels are compiled from (the multigrid and CG
# kernels, the fused advection and momentum pass, and what they include);
# host-side launch code and other kernels are outside.
DIGEST_HEADERS = ("mg_fused.cuh", "solver_kernels.cuh", "step_kernels.cuh", "uf_device.cuh", "advect_fused.cuh",
                  "momentum_fused.cuh")
# committed ncu summaries with a table of DRAM bytes per launch
TRAFFIC_PROFILES = ("mg_pcg_urban256.md", "advect_momentum_urban256.md")


def source_digest():
    """Digest of the device code of the profiled solver kernels: the code
    of the headers with comments and whitespace removed, so that an edit of
    a comment does not retire a capture of unchanged kernels."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2204_01117_gb300", "csrc")
    for f in sorted(DIGEST_HEADERS):
        with open(os.path.join(csrc, f)) as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)   # block comments
        text = re.sub(r"//[^\n]*", " ", text)                  # line comments
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_label: str):
    """DRAM bytes per launch of a kernel from a committed ncu summary (a
    table row: label | ncu kernel | DRAM bytes | ...), or None when no
    summary has it or the kernel sources changed since its capture."""
    for name in TRAFFIC_PROFILES:
        p = os.path.join(ROOT, "profiles", name)
        if not os.path.exists(p):
            continue
        text = open(p).read()
        m = re.search(r"source digest:\s*`([0-9a-f]+)`", text)
        if not m or m.group(1) != source_digest():
            continue
        for line in text.splitlines():
            cells = [c.strip() for c in line.strip().strip("|").split("|")]
            if len(cells) >= 3 and cells[0] == kernel_label:
                try:
                    return float(cells[2])
                except ValueError:
                    return None
    return None


def dominant_kernel(kernels: dict, prof_iters: int, mean_iters: float):
    """The kernel with the most time in an average timed step, and its share.

    The eagerly profiled step ran prof_iters CG iterations, the timed steps
    mean_iters on average; as in step_traffic, a kernel that launched at
    least prof_iters times runs once per iteration plus its fixed launches,
    so its time per step is its mean launch time x (fixed launches +
    mean_iters).  (Ranking by the profiled step alone would depend on that
    one step's iteration count.)  Returns (label, entry, ms per step, share)."""
    per_step = {}
    for name, k in kernels.items():
        n = int(k["launches"])
        avg = float(k["total_ms"]) / max(n, 1)
        runs = (n - prof_iters + mean_iters) if (prof_iters > 0 and n >= prof_iters) else n
        per_step[name] = avg * runs
    name = max(per_step, key=per_step.get)
    return name, kernels[name], per_step[name], per_step[name] / sum(per_step.values())


def step_traffic(kernels: dict, prof_iters: int, mean_iters: float, ms_per_step: float, peak: float,
                 cells: int) -> dict:
    """Algorithmic bytes of one whole step and their rate over the
    graph-replayed step time, against the HBM peak.

    One counting, per kernel: its bytes per launch (the compulsory reads and
    writes of the launch, from uf_profile_step) times its launches per step.
    The eagerly profiled step ran prof_iters CG iterations; a kernel that
    launched at least that many times runs once per iteration (plus a fixed
    number of set-up launches), the others a fixed number of times per step.
    The per-iteration launches are then taken at mean_iters, the mean CG
    iterations of the timed steps, so bytes and time describe the same steps.
    Never raises: a malformed profile gives {"error": ...}."""
    try:
        fixed = per_iter = 0.0
        for k in kernels.values():
            n, b = int(k["launches"]), float(k["bytes_per_launch"])
            if prof_iters > 0 and n >= prof_iters:
                fixed += b * (n - prof_iters)
                per_iter += b
            else:
                fixed += b * n
        total = fixed + per_iter * mean_iters
        gbs = total / (ms_per_step * 1e-3) / 1e9
        return {"bytes": total, "bytes_per_cell": total / cells, "fixed_bytes_per_cell": fixed / cells,
                "per_cg_iteration_bytes_per_cell": per_iter / cells, "cg_iters_mean": mean_iters,
                "achieved": gbs, "unit": "GB/s", "frac": gbs / peak}
    except Exception as e:   # noqa: BLE001 -- a report field, not a reason to lose the bench line
        return {"error": repr(e)}


# ---------------------------------------------------------------- adjoint leg

def adjoint_leg():
    """Adjoint/forward time on the parametric design workload: 128x128x48,
    12 buildings (H, dx, dy each) mapped to porosity by one-cell logistic
    ramps, 200 steps at the fixed dt = 0.2 s, checkpoints every 20 steps, FP32
    fields.  forward = uf_run + uf_objective; adjoint = uf_adjoint_run (its
    own checkpointed forward sweep, per-segment recompute, reverse sweep),
    both from the same state and timed on the wall clock with the device
    synchronised on both sides, after one untimed call of each."""
    import torch
    from paper_2204_01117_gb300 import layouts, uf
    d = layouts.design_lattice()
    g = uf.Grid(d.nx, d.ny, d.nz, precision="f32", **d.params())
    g.design_to_phi(d.boxes, d.theta, d.width)
    g.init_state()
    x0 = g.state()
    dphi = torch.empty(g.shapes["phi"], dtype=torch.float32, device="cuda")

    def forward():
        g.set_fields(x0)
        torch.cuda.synchronize()
        t = time.perf_counter()
        g.run(d.steps, stats=False)
        J = g.objective()
        torch.cuda.synchronize()
        return time.perf_counter() - t, J

    def adjoint():
        g.set_fields(x0)
        torch.cuda.synchronize()
        t = time.perf_counter()
        J, _ = g.adjoint_run(d.steps, d.ckpt_every, out=dphi)
        torch.cuda.synchronize()
        return time.perf_counter() - t, J

    forward()
    adjoint()
    tf, Jf = forward()
    ta, Ja = adjoint()
    grad = g.design_vjp(d.boxes, d.theta, d.width, dphi)
    design = design_loop_leg(g, d, x0, dphi, tf)
    out = {"workload": f"design lattice {d.nx}x{d.ny}x{d.nz}, h={d.h} m, 12 parametric buildings "
                       f"(36 parameters), {d.steps} steps at fixed dt={d.fixed_dt} s, checkpoints every "
                       f"{d.ckpt_every}, FP32 fields + FP64 reductions",
           "forward_ms": tf * 1e3, "adjoint_ms": ta * 1e3, "ratio": ta / tf,
           "J": Jf, "J_matches_forward": bool(Ja == Jf),
           "grad_norm": float(sum(x * x for x in grad)) ** 0.5,
           "workspace_bytes": int(g.lib.uf_adjoint_workspace_bytes(g._h, d.steps, d.ckpt_every)),
           "design_loop": design}
    g.free_adjoint_workspace()
    g.close()
    return out


def design_loop_leg(g, d, x0, dphi, forward_s):
    """One iteration of the gradient-descent design loop of Sec. 6 on the
    same workload, with the region-average objective L = sum_i (ubar_i -
    u_t)^2 over the six pedestrian-level target regions (u_t = 0.55 m/s):
    design map + uf_adjoint_run_ex + design VJP, wall clock, device
    synchronised on both sides, after one untimed iteration.  The paper's
    forward-difference gradient needs (parameters + 1) forward runs per
    iteration; that cost is given as the measured forward time times 37.
    Then the +-10 degree robustness re-runs: the three wind directions of
    the design advanced by one batch against three single grids in turn,
    each timed over the 200 steps with CUDA events."""
    import numpy as np
    import torch
    from paper_2204_01117_gb300 import uf
    obj = {"kind": "regions", "regions": d.regions, "u_t": d.u_t}

    def iteration():
        torch.cuda.synchronize()
        t = time.perf_counter()
        g.design_to_phi(d.boxes, d.theta, d.width)
        g.set_fields(x0)
        L, _ = g.adjoint_run(d.steps, d.ckpt_every, out=dphi, objective=obj)
        grad = g.design_vjp(d.boxes, d.theta, d.width, dphi)
        torch.cuda.synchronize()
        return time.perf_counter() - t, L, grad

    iteration()
    ti, L, grad = iteration()
    nparam = d.theta.size
    phi = g.design_to_phi(d.boxes, d.theta, d.width, set_porosity=False)
    winds = (-10.0, 0.0, 10.0)
    params = [dict(d.params(), nx=d.nx, ny=d.ny, nz=d.nz, wind_dir_deg=w) for w in winds]
    b = uf.Batch(params, precision="f32")
    for gb in b.grids:
        gb.set_porosity(phi)
        gb.init_state()
    b.run(3, stats=False)
    for gb in b.grids:
        gb.init_state()

    def timed(run, stream):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        run()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    t_batch = timed(lambda: b.run(d.steps, stats=False), b.stream)
    L_batch = [gb.objective_ex(obj) for gb in b.grids]
    b.close()
    solos = []
    for p in params:
        q = dict(p)
        nx, ny, nz = q.pop("nx"), q.pop("ny"), q.pop("nz")
        s = uf.Grid(nx, ny, nz, precision="f32", stream=g.stream, **q)
        s.set_porosity(phi)
        s.init_state()
        s.run(3, stats=False)
        s.init_state()
        solos.append(s)
    t_seq = timed(lambda: [s.run(d.steps, stats=False) for s in solos], g.stream)
    L_seq = [s.objective_ex(obj) for s in solos]
    for s in solos:
        s.close()
    return {"objective": "region average, 6 pedestrian-level regions z in [0, 3] m, u_t = 0.55 m/s",
            "parameters": nparam, "L": L, "grad_norm": float(np.linalg.norm(grad)),
            "iteration_ms": ti * 1e3,
            "forward_difference_iteration_ms": (nparam + 1) * forward_s * 1e3,
            "speedup_vs_forward_differences": (nparam + 1) * forward_s / ti,
            "robustness": {"winds_deg": list(winds), "L": L_batch, "batched_ms": t_batch,
                           "sequential_ms": t_seq, "batch_equals_solo": L_batch == L_seq}}


# ---------------------------------------------------------------- batched leg

def batched_leg(steps: int = 10, peak: float = 6790.0, peak_kind: str = "measured"):
    """Batched vs sequential single-grid throughput on 32 instances of uneven
    size (nx, ny in 96..256, nz in 32..64), seeded urban layouts scaled by
    area, wind direction uniform in [0, 360) and speed in [2, 8] m/s, FP32.
    The batch is autotuned per size class first; the sequential run is the
    plain single-grid step of each instance in turn (default tuning) on one
    stream.  Both are timed with CUDA events over `steps` steps after 3
    warm-up steps; the roofline comes from one eagerly launched batched step
    (per-launch CUDA events)."""
    import numpy as np
    import torch
    from paper_2204_01117_gb300 import layouts, uf
    insts = layouts.batch_instances(32, seed=0)
    params = [dict(nx=sc.nx, ny=sc.ny, nz=sc.nz, **sc.params()) for sc in insts]
    b = uf.Batch(params, precision="f32")
    for sc, g in zip(insts, b.grids):
        g.set_porosity(sc.phi.astype(np.float32))
        g.init_state()
    classes = b.autotune(reps=2)
    cells = b.cells

    def timed(stream, fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    b.run(3, stats=False)
    ms_b = timed(b.stream, lambda: b.run(steps, stats=False))
    st = b.run(1)
    fixed, per_iter = b.launch_counts()
    prof = b.profile_step()
    inst_cells = [sc.nx * sc.ny * sc.nz for sc in insts]
    # whole batched step with the single-grid counting: the CG-loop launches of
    # the profiled step ran as often as its slowest instance needed (the others
    # skip their items), so they are taken at the cell-weighted mean of the
    # instances' own iteration counts
    prof_iters = int(prof.get("b_cg_dir_q", {}).get("launches", 0))
    mean_iters = sum(c * x.cg_iters for c, x in zip(inst_cells, st)) / float(sum(inst_cells))
    step_bytes = step_traffic(prof, prof_iters, mean_iters, ms_b / steps, peak, cells)
    dom_name, dom, _, dom_share = dominant_kernel(prof, prof_iters, mean_iters)
    avg_ms = dom["total_ms"] / dom["launches"]
    achieved = dom["bytes_per_launch"] / (avg_ms * 1e-3) / 1e9
    b.close()
    del b
    torch.cuda.empty_cache()

    s = torch.cuda.Stream()
    solos = []
    for sc, p in zip(insts, params):
        q = dict(p)
        nx, ny, nz = q.pop("nx"), q.pop("ny"), q.pop("nz")
        g = uf.Grid(nx, ny, nz, precision="f32", stream=s, **q)
        g.set_porosity(sc.phi.astype(np.float32))
        g.init_state()
        g.run(3, stats=False)
        solos.append(g)

    def run_solos():
        for g in solos:
            g.run(steps, stats=False)

    ms_s = timed(s, run_solos)
    for g in solos:
        g.close()
    del solos
    torch.cuda.empty_cache()
    return {
        "workload": "32 instances, nx, ny in 96..256 (multiples of 16), nz in 32..64 (multiples of 8), "
                    "seeded urban layouts scaled by area, wind direction U[0,360) deg, speed U[2,8] m/s, FP32 "
                    "fields + FP64 reductions; 300-step runs, timed over " + str(steps) + " steps",
        "instances": len(insts), "cells": cells, "size_classes": classes,
        "batched": {"value": cells * steps / (ms_b * 1e-3), "unit": UNIT, "ms_per_step": ms_b / steps,
                    "cg_iters_min_max": [min(x.cg_iters for x in st), max(x.cg_iters for x in st)],
                    "launches_fixed_per_iter": [fixed, per_iter]},
        "sequential_single_grid": {"value": cells * steps / (ms_s * 1e-3), "unit": UNIT, "ms_per_step": ms_s / steps},
        "speedup": ms_s / ms_b,
        "roofline": {"bound": "hbm", "kernel": dom_name, "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_source": f"hbm_gbs of {peak_kind}",
                     "step": step_bytes,
                     "kernel_share_of_step": dom_share,
                     "bytes_per_launch": dom["bytes_per_launch"], "avg_launch_us": avg_ms * 1e3},
    }


# ------------------------------------------------------ preconditioner table

def preconditioner_table(steps: int = 10):
    """CG iterations and step time on the 256x256x64 urban block for each
    solver configuration: MG (three smoothers), the paper's AI1 / AI2, Jacobi
    and plain CG under the residual stop rule (||r|| <= 1e-7 ||b||), and AI1 /
    AI2 under the paper's rule (r.z <= 1e-5 ||b||^2, App. A.3), with the
    divergence left after a step.  Each is timed with CUDA events over
    `steps` steps after 3 warm-up steps from the same initial projection."""
    import numpy as np
    import torch
    from paper_2204_01117_gb300 import layouts, uf
    sc = layouts.urban_block(NX, NY, NZ, seed=0)
    cases = [("mg", dict(precond="mg", mg_smoother="cheby")),
             ("mg-constant-transfers", dict(precond="mg", mg_smoother="cheby", mg_transfer="constant")),
             ("mg-jacobi", dict(precond="mg", mg_smoother="jacobi")),
             ("mg-rbgs", dict(precond="mg", mg_smoother="rbgs")), ("ai2", dict(precond="ai2")),
             ("ai1", dict(precond="ai1")), ("jacobi", dict(precond="jacobi")), ("none", dict(precond="none")),
             ("ai2-paper-rule", dict(precond="ai2", cg_stop_rule="paper")),
             ("ai1-paper-rule", dict(precond="ai1", cg_stop_rule="paper"))]
    rows = []
    for name, kw in cases:
        g = uf.Grid(sc.nx, sc.ny, sc.nz, precision="f32", cg_max_iter=5000, **kw, **sc.params())
        g.set_porosity(sc.phi.astype(np.float32))
        g.init_state()
        g.run(3, stats=False)
        st0 = g.step()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(g.stream)
        g.run(steps, stats=False)
        e1.record(g.stream)
        torch.cuda.synchronize()
        st1 = g.step()
        its = (st1.cg_iters_total - st0.cg_iters_total - st1.cg_iters) / steps
        rows.append({"solver": name, "ms_per_step": e0.elapsed_time(e1) / steps, "cg_iters_per_step": its,
                     "divergence": g.divergence()})
        g.close()
    return {"workload": "urban block 256x256x64 FP32, " + str(steps) + " timed steps after 3", "rows": rows}


# ------------------------------------------------------------- large workload

def large_scenario(grid):
    """The 512 x 512 x 128 urban block (1 m cells, 400 boxes of height
    5-120 m, 800 canopies, log law 5 m/s at 10 m), or the same recipe on a
    smaller grid with the object counts scaled by area (for profiling)."""
    from paper_2204_01117_gb300 import layouts
    nx, ny, nz = grid
    if (nx, ny, nz) == (512, 512, 128):
        return layouts.config("urban512")
    area = nx * ny / (512 * 512)
    return layouts.urban_block(nx, ny, nz, h=1.0, n_boxes=max(1, round(400 * area)),
                               n_trees=max(1, round(800 * area)), height=(5.0, min(120.0, 0.9 * nz)), u_ref=5.0)


def fp64_flops_per_cell(kernel_label: str):
    """FP64 operations per finest-level cell of a kernel (an FMA counts two)
    from the committed ncu summary, or None when it is missing or the kernel
    sources changed since."""
    p = os.path.join(ROOT, "profiles", "mg_fp64_urban512.md")
    if not os.path.exists(p):
        return None
    text = open(p).read()
    m = re.search(r"source digest:\s*`([0-9a-f]+)`", text)
    if not m or m.group(1) != source_digest():
        return None
    for line in text.splitlines():
        cells = [c.strip() for c in line.strip().strip("|").split("|")]
        if len(cells) >= 3 and cells[0] == kernel_label:
            try:
                return float(cells[2])
            except ValueError:
                return None
    return None


def run_large(args):
    """Plain FP64 against FP32 + FP64 reductions on the large urban block:
    one FP64 initial state, copied into both grids; `steps` steps of each
    with the CFL time step (the first 3 untimed, the rest timed with CUDA
    events); relative L2 difference of every field and the divergence at the
    end; per-kernel CUDA-event rooflines of one eager step of each; then the
    adjoint of the comfort objective over the last `adjoint_steps` steps of
    the FP32 run, from its state at step steps - adjoint_steps, with the
    fixed time step of the run's first step (a fixed dt is needed for the
    adjoint) and checkpoints every 10 steps, against the forward time of the
    same steps."""
    import numpy as np
    import torch
    from paper_2204_01117_gb300 import uf
    torch.cuda.set_device(0)
    uf.build()
    uf.load()
    grid = tuple(int(x) for x in args.large_grid.split("x"))
    steps = max(8, args.steps if args.steps is not None else 1000)
    adj_steps = min(100, steps // 2)
    t_gen = time.perf_counter()
    sc = large_scenario(grid)
    t_gen = time.perf_counter() - t_gen
    g64 = uf.Grid(sc.nx, sc.ny, sc.nz, precision="f64", **sc.params())
    g64.set_porosity(sc.phi)
    g64.init_state()
    x0 = g64.state()
    g32 = uf.Grid(sc.nx, sc.ny, sc.nz, precision="f32", **sc.params())
    g32.set_porosity(sc.phi.astype(np.float32))
    g32.set_fields(x0)
    del x0
    warm = 3
    first = g32.step()
    its0 = {id(g32): g32.run(warm - 1).cg_iters_total, id(g64): g64.run(warm).cg_iters_total}
    snap_at = steps - adj_steps

    mean_its = {}

    def timed(g, n, snapshot=None):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ms, done, snap, last = 0.0, 0, None, None
        for chunk in ([snapshot - warm, n - snapshot] if snapshot else [n - warm]):
            torch.cuda.synchronize()
            e0.record(g.stream)
            last = g.run(chunk)
            e1.record(g.stream)
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
            done += chunk
            if snapshot and snap is None:
                snap = g.state()
        mean_its[id(g)] = (last.cg_iters_total - its0[id(g)]) / done
        return ms, done, snap

    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    with ClockSampler(vis.split(",")[0].strip() if vis else "0") as clk:
        ms32, n32, snap = timed(g32, steps, snapshot=snap_at if not args.no_adjoint else None)
        ms64, n64, _ = timed(g64, steps)
    err = {}
    for f in ("u", "v", "w", "p", "k", "omega"):
        a = g32.get_state(f).astype(np.float64)
        r = g64.get_state(f)
        err[f] = float(np.linalg.norm(a - r) / max(np.linalg.norm(r), 1e-300))
    div32, div64 = g32.divergence(), g64.divergence()
    peaks, peak_kind = measured_peaks()
    peak = float(peaks.get("hbm_gbs", 6800.0))
    fp64_peak = 152 * 2 * 2 * 2070e6          # SMs x FP64 FMA/clk/SM x 2 flops x max SM clock

    def roofline(g, fp64=False):
        pst, kernels = g.profile_step()
        name, k, _, share = dominant_kernel(kernels, pst.cg_iters, mean_its[id(g)])
        avg_s = k["total_ms"] / k["launches"] * 1e-3
        out = {"bound": "hbm", "kernel": name, "achieved": k["bytes_per_launch"] / avg_s / 1e9, "peak": peak,
               "unit": "GB/s", "peak_source": f"hbm_gbs of {peak_kind}",
               "kernel_share_of_step": share, "avg_launch_us": avg_s * 1e6,
               "cg_iters_mean": mean_its[id(g)]}
        out["frac"] = out["achieved"] / peak
        if fp64:
            fpc = fp64_flops_per_cell(name)
            out["fp64_alu"] = None if fpc is None else {
                "achieved": fpc * sc.cells / avg_s / 1e12, "peak": fp64_peak / 1e12, "unit": "TFLOP/s",
                "frac": fpc * sc.cells / avg_s / fp64_peak, "flops_per_cell": fpc,
                "peak_source": "152 SMs x 2 FP64 FMA/clk x 2 x 2070 MHz"}
        return out

    line = {
        "metric": f"RANS cell-updates/s at {sc.nx}x{sc.ny}x{sc.nz}: plain FP64 vs FP32 + FP64 reductions",
        "value": sc.cells * n32 / (ms32 * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": steps, "warmup": warm,
        "ms_per_step": ms32 / n32, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"urban block {sc.nx}x{sc.ny}x{sc.nz}, h=1 m, {sc.name}, log-law inflow 5 m/s at "
                               f"10 m, CFL dt, MG-preconditioned CG; both runs from one FP64 initial state",
                   "cells": sc.cells, "layout_seconds": t_gen,
                   "l2": "no flush: per-step working set > 129 MB L2"},
        "fp32": {"value": sc.cells * n32 / (ms32 * 1e-3), "ms_per_step": ms32 / n32, "roofline": roofline(g32),
                 "divergence": div32},
        "fp64": {"value": sc.cells * n64 / (ms64 * 1e-3), "ms_per_step": ms64 / n64,
                 "roofline": roofline(g64, fp64=True), "divergence": div64},
        "fp32_vs_fp64_rel_l2": err,
        "clocks": clk.summary(),
    }
    g64.close()
    del g64
    torch.cuda.empty_cache()
    if not args.no_adjoint:
        ga = uf.Grid(sc.nx, sc.ny, sc.nz, precision="f32", fixed_dt=first.dt, **sc.params())
        ga.set_porosity(sc.phi.astype(np.float32))
        ga.set_fields(snap)
        ga.run(1, stats=False)
        ga.set_fields(snap)
        torch.cuda.synchronize()
        t = time.perf_counter()
        ga.run(adj_steps, stats=False)
        J = ga.objective()
        torch.cuda.synchronize()
        tf = time.perf_counter() - t
        ga.set_fields(snap)
        dphi = torch.empty(ga.shapes["phi"], dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        t = time.perf_counter()
        Ja, _ = ga.adjoint_run(adj_steps, 10, out=dphi)
        torch.cuda.synchronize()
        ta = time.perf_counter() - t
        line["adjoint"] = {"steps": adj_steps, "ckpt_every": 10, "fixed_dt": first.dt, "forward_ms": tf * 1e3,
                           "adjoint_ms": ta * 1e3, "ratio": ta / tf, "J": J, "J_matches_forward": bool(Ja == J),
                           "dJ_dphi_norm": float(torch.linalg.vector_norm(dphi.double()).item()),
                           "workspace_bytes": int(ga.lib.uf_adjoint_workspace_bytes(ga._h, adj_steps, 10))}
        ga.free_adjoint_workspace()
        ga.close()
    g32.close()
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------ mesh resolver

def run_mesh(args):
    """The mesh resolver (Sec. 3) on a 256 x 256 x 64 mesh city of 2 m cells:
    40 prism buildings and 60 ellipsoidal canopies (seed 0), 4^3 sample
    points per cell, FP64 decisions.  Timed with CUDA events over 3 calls
    after one untimed call (each call uploads the mesh, resolves every cell
    and writes the grid's porosity).  The ray-triangle tests are counted on
    the host (sample points in each object's box x its triangles); each test
    is 52 FP64 operations, against the FP64 pipe's 152 SMs x 2 FMA/clock x
    2 x 2070 MHz."""
    import numpy as np
    import torch
    from paper_2204_01117_gb300 import layouts, uf
    torch.cuda.set_device(0)
    uf.build()
    uf.load()
    nx, ny, nz, h, sub = 256, 256, 64, 2.0, 4
    tris, objs = layouts.mesh_city(nx, ny, nz, h, n_buildings=40, n_trees=60, seed=0)
    off = (np.arange(sub) + 0.5) / sub
    xs = ((np.arange(nx)[:, None] + off) * h).ravel()
    ys = ((np.arange(ny)[:, None] + off) * h).ravel()
    zs = ((np.arange(nz)[:, None] + off) * h).ravel()
    tests = 0
    for first, count, _ in objs:
        t = tris[first:first + count].reshape(-1, 3)
        lo, hi = t.min(axis=0), t.max(axis=0)
        n = (((xs >= lo[0]) & (xs <= hi[0])).sum() * ((ys >= lo[1]) & (ys <= hi[1])).sum()
             * ((zs >= lo[2]) & (zs <= hi[2])).sum())
        tests += int(n) * count
    g = uf.Grid(nx, ny, nz, h=h, precision="f32")
    g.mesh_to_phi(tris, objs, sub=sub)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 3
    torch.cuda.synchronize()
    e0.record(g.stream)
    for _ in range(reps):
        g.mesh_to_phi(tris, objs, sub=sub)
    e1.record(g.stream)
    torch.cuda.synchronize()
    sec = e0.elapsed_time(e1) * 1e-3 / reps
    peak = 152 * 2 * 2 * 2070e6
    line = {"metric": "mesh resolver cells/s (even-odd ray tests, 4^3 points per cell)", "value": nx * ny * nz / sec,
            "unit": "cells/s", "ms_per_call": sec * 1e3, "n_gpus": 1, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"mesh city {nx}x{ny}x{nz}, h={h} m, 40 prism buildings + 60 canopies "
                                   f"({len(tris)} triangles), seed 0", "sub": sub},
            "ray_triangle_tests": tests, "tests_per_s": tests / sec,
            "roofline": {"bound": "alu", "achieved": tests * 52 / sec / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s",
                         "frac": tests * 52 / sec / peak,
                         "peak_source": "152 SMs x 2 FP64 FMA/clk x 2 x 2070 MHz"}}
    g.close()
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------- vortex shedding

def run_karman(args):
    """The supplement's solver validation: flow past a 0.046 m cylinder on
    512 x 768 cells of 2 mm, inflow 2-20 m/s; the shedding frequency from a
    wake probe against St = 0.198 (1 - 19.7/Re).  Each speed runs at the
    supplement's fixed dt = 1e-4 s and at the dt of cell Courant number 1."""
    import torch
    from paper_2204_01117_gb300 import uf, validation
    torch.cuda.set_device(0)
    uf.build()
    uf.load()
    rows = []
    t0 = time.perf_counter()
    for U in (2.0, 5.0, 10.0, 20.0):
        for mode, kw in (("dt=1e-4 s", dict()), ("Courant 1", dict(cfl=1.0))):
            r = validation.shedding_run(U, **kw)
            r["mode"] = mode
            r["St_error"] = r["St"] / r["St_formula"] - 1.0
            rows.append(r)
    line = {"metric": "Strouhal number of the vortex street vs St = 0.198 (1 - 19.7/Re)",
            "unit": "relative error", "impl": "ours", "n_gpus": 1, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "cylinder D = 0.046 m, 512 x 768 x 1 cells of 2 mm, inflow 2-20 m/s through y-, "
                                   "outflow y+, slip x sides and z; probe 3 D downstream on the axis",
                       "seconds": time.perf_counter() - t0},
            "rows": rows}
    print(json.dumps(line), flush=True)
    return 0


def run_karman_study(args):
    """Where the Strouhal error at small Courant numbers comes from: the
    cylinder at U = 2 m/s (Re = 6.1e3) with the time step swept at 2 mm
    cells (Courant number U dt / h from 0.1, the supplement's dt = 1e-4 s,
    to 1) and on cells 1.5 times finer (4/3 mm: the same physical channel
    and cylinder, 768 x 1152 cells) at the same Courant number 0.1, at the
    same dt = 1e-4 s and at Courant number 1.  Scheme error of the semi-Lagrangian step shrinks
    under refinement at a fixed Courant number; a modelling error would not."""
    import torch
    from paper_2204_01117_gb300 import uf, validation
    torch.cuda.set_device(0)
    uf.build()
    uf.load()
    U = 2.0
    h2 = 2e-3 / 1.5   # 4/3 mm: the finest grid within the reduction buffer's 4096 x-y tiles
    cases = [(2e-3, 512, 768, 1e-4), (2e-3, 512, 768, 2e-4), (2e-3, 512, 768, 5e-4), (2e-3, 512, 768, 1e-3),
             (h2, 768, 1152, 0.1 * h2 / U), (h2, 768, 1152, 1e-4), (h2, 768, 1152, h2 / U)]
    rows = []
    t0 = time.perf_counter()
    for h, nx, ny, dt in cases:
        r = validation.shedding_run(U, dt=dt, nx=nx, ny=ny, h=h)
        r["h"] = h
        r["St_error"] = r["St"] / r["St_formula"] - 1.0
        rows.append(r)
        print(json.dumps({"row": r}), file=sys.stderr, flush=True)
    line = {"metric": "Strouhal number of the vortex street vs St = 0.198 (1 - 19.7/Re): time-step and grid study",
            "unit": "relative error", "impl": "ours", "n_gpus": 1, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "cylinder D = 0.046 m in a 1.024 x 1.536 m channel, U = 2 m/s, 2 mm and 4/3 mm "
                                   "cells, probe 3 D downstream on the axis",
                       "seconds": time.perf_counter() - t0},
            "rows": rows}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- oracle arm

def oracle_sample(max_seconds: float = 150.0, steps_wanted: int = 1):
    """Times the FP64 oracle (as it stands) on the full workload: untimed
    initial projection, then timed oracle steps until `steps_wanted` or the
    time cap.  Returns (cell-updates/s, cores, sample description, steps)."""
    import oracle
    from paper_2204_01117_gb300 import layouts
    oracle.build()
    sc = layouts.urban_block(NX, NY, NZ, seed=0)
    o = oracle.Oracle(sc.nx, sc.ny, sc.nz, **sc.params())
    o.set("phi", sc.phi)
    o.init()
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    t0 = time.perf_counter()
    done = 0
    while done < max(1, steps_wanted):
        o.step()
        done += 1
        if time.perf_counter() - t0 > max_seconds:
            break
    dt = time.perf_counter() - t0
    rate = sc.cells * done / dt
    sample = (f"{done} FP64 oracle step(s) of the full 256x256x64 workload after its own initial "
              f"projection (untimed); CG to ||r||/||b|| <= 1e-13; OpenMP threads={cores}")
    return rate, cores, sample, done, dt


def cpu_model() -> str:
    """The host CPU as /proc/cpuinfo names it (x86: model name; Arm: the
    implementer and part numbers), else the machine type."""
    import platform
    try:
        info = open("/proc/cpuinfo").read()
        m = re.search(r"^model name\s*:\s*(.+)$", info, re.M)
        if m:
            return m.group(1).strip()
        imp = re.search(r"^CPU implementer\s*:\s*(\S+)", info, re.M)
        part = re.search(r"^CPU part\s*:\s*(\S+)", info, re.M)
        if imp and part:
            return f"{platform.machine()} implementer {imp.group(1)} part {part.group(1)}"
    except OSError:
        pass
    return platform.machine()


def oracle_single_box_run():
    """The FP64 oracle on the single-box case (64 x 32 x 16, 100 steps after
    its initial projection); prints one JSON line.  Run in a child process
    so that OMP_NUM_THREADS takes effect."""
    import oracle
    from paper_2204_01117_gb300 import layouts
    oracle.build()
    sc = layouts.single_box()
    o = oracle.Oracle(sc.nx, sc.ny, sc.nz, **sc.params())
    o.set("phi", sc.phi)
    o.init()
    t0 = time.perf_counter()
    o.run(100)
    dt = time.perf_counter() - t0
    print(json.dumps({"value": sc.cells * 100 / dt, "seconds": dt,
                      "threads": int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))}), flush=True)
    return 0


def oracle_thread_scaling():
    """The single-box oracle run with 1 thread and with every core, each in
    a child process."""
    out = {}
    for n in (1, os.cpu_count() or 1):
        env = dict(os.environ, OMP_NUM_THREADS=str(n))
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-single-box"], env=env,
                           capture_output=True, text=True, timeout=600)
        if r.returncode != 0:
            return {"error": r.stderr.strip().splitlines()[-1:] or ["failed"]}
        out[f"threads_{n}"] = json.loads(r.stdout.strip().splitlines()[-1])
    return out


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return 0
    rate, cores, sample, done, dt = oracle_sample(max_seconds=150.0, steps_wanted=max(1, min(args.steps, 3)))
    line = {
        "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus, "steps": done,
        "warmup": 0, "ms_per_step": dt / done * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": workload_config(),
        "cpu_baseline": {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU arm

def run_ours(args):
    import numpy as np
    import torch

    from paper_2204_01117_gb300 import layouts, uf

    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist
    uf.build()
    uf.load()
    sc = layouts.urban_block(NX, NY, NZ, seed=rank)
    g = uf.Grid(sc.nx, sc.ny, sc.nz, precision="f32", **sc.params())
    g.set_porosity(sc.phi.astype(np.float32))
    g.init_state()
    for _ in range(max(args.warmup, 3)):
        g.step(stats=False)
    st0 = g.step()
    fixed, per_iter = g.launch_counts()

    s = g.stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    smi_index = vis.split(",")[local].strip() if vis else str(local)
    with ClockSampler(smi_index) as clk:
        e0.record(s)
        for _ in range(args.steps):
            g.step(stats=False)
        e1.record(s)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    st1 = g.step()
    iters_timed = st1.cg_iters_total - st0.cg_iters_total - st1.cg_iters
    launches = args.steps * fixed + iters_timed * per_iter
    value, slowest_s = weak_scaling_rate(sc.cells, args.steps, ms * 1e-3)
    ms = slowest_s * 1e3

    # -- end to end through the C ABI with pinned host buffers ------------
    names = ("u", "v", "w", "p", "k", "omega")
    host_in = {n: torch.from_numpy(g.get_state(n)).pin_memory() for n in names}
    host_out = {n: torch.empty_like(host_in[n]).pin_memory() for n in names}
    h2d = sum(t.numel() * 4 for t in host_in.values())
    d2h = sum(t.numel() * 4 for t in host_out.values())
    e2e_steps = max(3, min(args.steps, 10))
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        g.put_fields(host_in)      # one contiguous copy per field, repacked on the device
        g.step(stats=False)
        g.take_fields(host_out)    # one synchronisation per step
    torch.cuda.synchronize()
    e2e_value, e2e_s = weak_scaling_rate(sc.cells, e2e_steps, time.perf_counter() - t0)

    # -- per-kernel CUDA-event timing of one eagerly launched step ----------
    pst, kernels = g.profile_step()
    dom_name, dom, _, dom_share = dominant_kernel(kernels, pst.cg_iters, iters_timed / args.steps)
    avg_ms = dom["total_ms"] / dom["launches"]
    achieved = dom["bytes_per_launch"] / (avg_ms * 1e-3) / 1e9
    peaks, peak_kind = measured_peaks()
    peak = float(peaks.get("hbm_gbs", 6800.0))
    traffic = ncu_traffic(dom_name)

    if rank != 0:
        if pg:
            pg.barrier()
            pg.destroy_process_group()
        return 0
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config({"parallelism": f"replicas x{world}", "cg_iters_last_step": st1.cg_iters,
                                   "precond": "MG V-cycle (2+2 Chebyshev-weighted Jacobi)", "cg_tol": 1e-7}),
        "roofline": {"bound": "hbm", "kernel": dom_name, "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                     "peak_source": f"hbm_gbs of {peak_kind}",
                     "kernel_share_of_step": dom_share,
                     "bytes_per_launch": dom["bytes_per_launch"], "avg_launch_us": avg_ms * 1e3,
                     "step": step_traffic(kernels, pst.cg_iters, iters_timed / args.steps, ms / args.steps, peak,
                                          sc.cells)},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "steps": e2e_steps},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
    }
    # the finest-level CG kernel, the bandwidth-bound one, when another kernel
    # (the issue-bound fused advection) leads the step
    cg = kernels.get("mg_down_cg_L0")
    if cg and dom_name != "mg_down_cg_L0":
        cg_ms = cg["total_ms"] / cg["launches"]
        cg_gbs = cg["bytes_per_launch"] / (cg_ms * 1e-3) / 1e9
        line["roofline_solver"] = {"bound": "hbm", "kernel": "mg_down_cg_L0", "achieved": cg_gbs, "peak": peak,
                                   "unit": "GB/s", "frac": cg_gbs / peak, "traffic": ncu_traffic("mg_down_cg_L0"),
                                   "peak_source": f"hbm_gbs of {peak_kind}",
                                   "bytes_per_launch": cg["bytes_per_launch"], "avg_launch_us": cg_ms * 1e3}
    if not args.no_adjoint:
        line["adjoint"] = adjoint_leg()
    if not args.no_batched:
        line["batched"] = batched_leg(peak=peak, peak_kind=peak_kind)
    if not args.no_cpu_baseline and world == 1:
        rate, cores, sample, done, dt = oracle_sample(max_seconds=60.0, steps_wanted=1)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                                "cpu_model": cpu_model(),
                                "single_box_100_steps": oracle_thread_scaling()}
    print(json.dumps(line), flush=True)
    if pg:
        pg.barrier()
        pg.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None, help="timed steps (default 50; 1000 with --large)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip the oracle timing leg")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint/forward timing leg")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched 32-instance leg")
    ap.add_argument("--preconditioners", action="store_true",
                    help="print the solver comparison table (CG iterations, step time) instead of the bench line")
    ap.add_argument("--large", action="store_true",
                    help="print the plain-FP64 vs FP32 comparison on the 512x512x128 block instead of the bench line")
    ap.add_argument("--large-grid", default="512x512x128", help="grid of --large (NXxNYxNZ)")
    ap.add_argument("--karman", action="store_true",
                    help="print the vortex-shedding validation table instead of the bench line")
    ap.add_argument("--karman-study", action="store_true",
                    help="print the time-step and grid study of the vortex-shedding frequency at 2 m/s")
    ap.add_argument("--oracle-single-box", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--mesh", action="store_true",
                    help="print the mesh resolver's throughput instead of the bench line")
    args = ap.parse_args()
    if args.oracle_single_box:
        return oracle_single_box_run()
    if args.mesh:
        return run_mesh(args)
    if args.large:
        return run_large(args)
    if args.karman:
        return run_karman(args)
    if args.karman_study:
        return run_karman_study(args)
    if args.steps is None:
        args.steps = 50
    if args.preconditioners:
        import torch
        torch.cuda.set_device(0)
        from paper_2204_01117_gb300 import uf
        uf.build()
        uf.load()
        print(json.dumps(preconditioner_table()), flush=True)
        return 0
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
