"""Benchmark of the fused hydro stage update on GB300.

Headline workload: the strong spherical blast on a 512^3 mesh (gamma = 1.4,
ambient rho = 1 with seeded +-1 % noise, p = 1e-5, total energy 1 spread over
the cells within four cells of the centre, reflecting walls, CFL 0.3), FP32
bulk with FP64 conserved-total reductions, 200 steps from t = 0.  A step is
one pass of the whole path: the CFL time step from the fused signal-rate
reduction, both Runge-Kutta stages, and the FP64 conserved totals of the new
state.  The state (2.7 GB in FP32) is far larger than the 129 MB L2.  The
FP64 plain path runs the same configuration; the 256^3 periodic smooth flow
(gamma = 5/3, CFL 0.4) is a secondary line, as are the second scheme, the
radiation operators, the batched launch and the adjoint.

metric: cell-updates per RK stage per second = cells * 2 * steps / time.

Prints one JSON line.  Multi-GPU (torchrun): the blast is decomposed into z
slabs, one per rank, with a ghost exchange per stage and a max-reduction of
the signal rate per step over NCCL (strong scaling: the whole 512^3 mesh at
every N); timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "cell-updates/s per RK stage (FP32 fused vs FP64 plain) and % HBM roofline"
UNIT = "cell-updates/s"
N_SIDE = 512
GAMMA = 1.4
CFL = 0.3
STEPS = 200
WORKLOAD = ("3D strong spherical blast 512^3, gamma=1.4, ambient rho=1 with seeded +-1% noise, "
            "p=1e-5, energy 1.0 within 4 cells of the centre, reflecting walls, CFL 0.3, "
            "200 steps; FP32 bulk with FP64 conserved-total reductions")
SMOOTH_N = 256
SMOOTH_GAMMA = 5.0 / 3.0
SMOOTH_CFL = 0.4
SMOOTH_WORKLOAD = ("3D periodic smooth flow 256^3, gamma=5/3, entropy wave + 8 seeded acoustic "
                   "modes (amplitude 1e-3), CFL 0.4")
BYTES_PER_CELL_STAGE = {4: 50.0, 8: 100.0}     # algorithmic: (5+5 + 10+5)/2 values
L2_BYTES = 129 * 2 ** 20


# The sources the profiled stage kernel is compiled and launched from.
STAGE_KERNEL_SOURCES = ("devattr.h", "hydro_math.cuh", "kernels_impl.cuh", "launch.h",
                        "stage_f32.cu", "stage_kernel.cuh", "stage_tma.cuh", "stage_ws.cuh",
                        "tma.cuh", "vec2.cuh")
# the committed ncu summaries of the stage kernel, by tile height
STAGE_PROFILES = {8: os.path.join("profiles", "stage_ws_kernel_blast3d_256.md"),
                  16: os.path.join("profiles", "stage_ws_kernel_ty16_blast3d_256.md")}


def kernel_sources_digest():
    """sha256 over the stage kernel's sources, to tell whether a profile still applies."""
    import hashlib
    root = os.path.join(ROOT, "paper_2509_08971_gb300", "csrc")
    h = hashlib.sha256()
    for f in STAGE_KERNEL_SOURCES:
        h.update(f.encode())
        with open(os.path.join(root, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def profiled(key, ty=8):
    """A figure of the committed ncu summary of the stage kernel with tiles
    of height ty ("traffic-bytes-per-cell-stage": DRAM bytes read + written
    per cell, mean of the two stage launches; "instructions-per-cell-stage":
    warp-instruction issue slots x 32 per cell, mean of the two), or None
    when there is none or the kernel's sources changed since the capture."""
    if ty not in STAGE_PROFILES:
        return None
    path = os.path.join(ROOT, STAGE_PROFILES[ty])
    try:
        rec = {}
        with open(path) as fh:
            for line in fh:
                if ":" in line and line.split(":", 1)[0] in ("sources-sha256", key):
                    k, v = line.split(":", 1)
                    rec[k.strip()] = v.strip()
        if rec.get("sources-sha256") != kernel_sources_digest():
            return None
        return float(rec[key])
    except (OSError, KeyError, ValueError):
        return None


def profiled_traffic(cells, ty=8):
    """DRAM bytes per stage launch on `cells` cells: the profiled per-cell
    figure (captured on a 256^3 case of the same kernel) times the cells; the
    kernel streams each plane once, so its traffic grows with the cells."""
    b = profiled("traffic-bytes-per-cell-stage", ty)
    return None if b is None else b * cells


SCHEDULERS = 152 * 4       # GB300: 152 SMs, four warp schedulers each


def issue_roofline(cells, stage_ms, sm_mhz, ty=8):
    """The stage kernel against the SMs' instruction issue rate: warp
    instructions per second (profiled thread instructions per cell-stage x
    cells / 32 / launch time) over one warp instruction per scheduler per
    clock at the median SM clock sampled during the timed steps."""
    ipc = profiled("instructions-per-cell-stage", ty)
    if ipc is None or not sm_mhz:
        return None
    achieved = ipc * cells / 32.0 / (stage_ms * 1e-3)
    peak = SCHEDULERS * sm_mhz * 1e6
    return {"bound": "issue", "achieved": achieved, "peak": peak,
            "unit": "warp-instructions/s", "frac": achieved / peak,
            "instructions_per_cell_stage": ipc,
            "source": "ncu smsp__inst_executed of the profiled stage launches; SM clock sampled "
                      "by nvidia-smi during the timed steps"}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu = gpu_id
        self.proc = None
        self.lines: list[str] = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.06)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.thread.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for name, flag in zip(names, parts[5:9]):
                if flag.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


class nvtx_range:
    """Names a region of launches for profilers (ncu --nvtx --nvtx-include
    "<name>/"); a no-op where torch has no NVTX support."""

    def __init__(self, name):
        self.name = name

    def __enter__(self):
        try:
            import torch
            torch.cuda.nvtx.range_push(self.name)
            self.on = True
        except Exception:
            self.on = False
        return self

    def __exit__(self, *exc):
        if self.on:
            import torch
            torch.cuda.nvtx.range_pop()
        return False


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x, world, device=None):
    """The largest of each rank's value (the job's time is its slowest rank)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(world, cells_per_rank, stages, ms):
    """Cell-updates per second of the whole job: every rank advances its own
    replica, so the job's work is world x the per-rank work over the max time."""
    return world * cells_per_rank * stages / (ms * 1e-3)


def cpu_threads():
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()


def blast_slab(planes):
    """The middle `planes` z planes of the 512^3 blast (seed 0): the same cells,
    noise and energy density as the full state, the blast inside."""
    import hydro_inputs as H
    k0 = (N_SIDE - planes) // 2
    return H.blast_3d(N_SIDE, seed=0, gamma=GAMMA, planes=(k0, k0 + planes))


def time_oracle(U, steps, threads, bc, gamma, cfl):
    """The oracle as it stands (FP64 C, OpenMP over cells) on state U.
    Returns (cell-stages/s, seconds, threads used)."""
    import oracle
    oracle.set_threads(threads)
    used = oracle.get_threads()
    shape = U.shape[1:]
    g = oracle.Grid(shape, gamma, bc)
    t0 = time.perf_counter()
    g.run(U, steps, cfl)
    sec = time.perf_counter() - t0
    cells = shape[0] * shape[1] * shape[2]
    return cells * 2 * steps / sec, sec, used


def time_oracle_riemann():
    """Configuration 1 in full: the seeded two-state problem (seed 0) on 400
    cells, outflow, CFL 0.4, run to t = 0.15 by the oracle on one thread.
    Returns (cell-stages/s, seconds, steps)."""
    import hydro_inputs as H
    import oracle
    oracle.set_threads(1)
    pb = H.riemann_1d(0)
    U = pb.U(400)
    g = oracle.Grid((1, 1, 400), pb.gamma, oracle.BC_OUTFLOW)
    t0 = time.perf_counter()
    _, _, dts = g.run(U, 10 ** 6, 0.4, 0.15)
    sec = time.perf_counter() - t0
    return 400 * 2 * len(dts) / sec, sec, len(dts)


REF_PLANES = 8          # z planes of the blast per reference step


def run_reference(args, world, rank):
    """Reference arm: the FP64 CPU oracle on the host cores, each step a
    bounded sample of the workload: the middle 8 z planes of the 512^3 blast
    (512 x 512 x 8 cells, reflecting walls, CFL 0.3), the same per-cell
    arithmetic at 1/64 of the cells."""
    if rank != 0:
        return
    import oracle
    U = blast_slab(REF_PLANES)
    threads = cpu_threads()
    if args.warmup:
        time_oracle(U, args.warmup, threads, oracle.BC_REFLECT, GAMMA, CFL)
    rate, sec, used = time_oracle(U, args.steps, threads, oracle.BC_REFLECT, GAMMA, CFL)
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec / max(args.steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD,
                   "sample": f"the middle {REF_PLANES} z planes of the 512^3 blast per step",
                   "cells_per_step": REF_PLANES * N_SIDE * N_SIDE},
        "cpu_baseline": {"value": rate, "unit": UNIT, "cores": used, "kind": "oracle",
                         "sample": f"{args.steps} RK2 steps of a 512x512x{REF_PLANES} slab "
                                   "of the blast"},
        "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


FIELDS = ("rho", "rho_u", "rho_v", "rho_w", "E")


def _field_errors(a, b):
    """Relative L1 per field, sum|a-b| / sum|b| (fields that are zero in the
    reference report the absolute L1 per cell instead)."""
    a = np.asarray(a, dtype=np.float64).reshape(5, -1)
    b = np.asarray(b, dtype=np.float64).reshape(5, -1)
    out = {}
    for f, name in enumerate(FIELDS):
        den = np.sum(np.abs(b[f]))
        num = np.sum(np.abs(a[f] - b[f]))
        out[name] = float(num / den) if den > 0 else float(num / b.shape[1])
    return out


def precision_report():
    """FP32 against FP64 per field and per configuration (one JSON line)."""
    import torch
    import hydro_inputs as H
    import oracle
    import paper_2509_08971_gb300 as hh
    rep = {"report": "precision", "metric": "relative L1 per field, FP32 GPU vs FP64 reference"}
    # configuration 1: seeded Riemann problems (400 cells, outflow, CFL 0.4, t = 0.15)
    worst = {k: 0.0 for k in FIELDS}
    for seed in range(8):
        pb = H.riemann_1d(seed)
        U = pb.U(400)
        ref, t_ref, _ = oracle.Grid((1, 1, 400), pb.gamma, oracle.BC_OUTFLOW).run(U, 10 ** 6, 0.4, 0.15)
        m = hh.HardHydro((1, 1, 400), pb.gamma, hh.HARD_BC_OUTFLOW)
        Ud = torch.tensor(U, dtype=torch.float32, device="cuda")
        m.advance(Ud, 10 ** 4, 0.4, t_end=0.15, t=torch.zeros((), dtype=torch.float64, device="cuda"))
        for k, v in _field_errors(Ud.cpu().numpy(), ref).items():
            worst[k] = max(worst[k], v)
    rep["riemann_1d_400_fp32_vs_oracle"] = worst
    # configuration 2: smooth 3D flow, 100 steps
    n = 64
    U = H.smooth_3d(n, seed=0, gamma=SMOOTH_GAMMA)
    ref, _, _ = oracle.Grid((n, n, n), SMOOTH_GAMMA, oracle.BC_PERIODIC).run(U, 100, SMOOTH_CFL)
    m = hh.HardHydro((n, n, n), SMOOTH_GAMMA, 0)
    Ud = torch.tensor(U, dtype=torch.float32, device="cuda")
    m.advance(Ud, 100, SMOOTH_CFL)
    rep["smooth_3d_64_fp32_vs_oracle"] = _field_errors(Ud.cpu().numpy(), ref)
    n = 256
    U = H.smooth_3d(n, seed=0, gamma=SMOOTH_GAMMA)
    m64 = hh.HardHydro((n, n, n), SMOOTH_GAMMA, 0, dtype=torch.float64)
    V = torch.tensor(U, dtype=torch.float64, device="cuda")
    m64.advance(V, 100, SMOOTH_CFL)
    m32 = hh.HardHydro((n, n, n), SMOOTH_GAMMA, 0)
    Ud = torch.tensor(U, dtype=torch.float32, device="cuda")
    m32.advance(Ud, 100, SMOOTH_CFL)
    rep["smooth_3d_256_fp32_vs_fp64_gpu"] = _field_errors(Ud.cpu().numpy(), V.cpu().numpy())
    del V, Ud, m64, m32
    # configuration 3: spherical blast 512^3, reflecting walls, CFL 0.3
    n = 512
    Ub = H.blast_3d(n, seed=0, dtype=np.float32)
    m32 = hh.HardHydro((n, n, n), 1.4, hh.HARD_BC_REFLECT)
    Ud = torch.tensor(Ub, device="cuda")
    t = torch.zeros((), dtype=torch.float64, device="cuda")
    tl = None
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    _, _, tl = m32.advance(Ud, 200, 0.3, t=t, log_totals=True)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    tot = tl.cpu().numpy()
    rep["blast_512_fp32_200_steps"] = {
        "cell_updates_per_s_per_stage": n ** 3 * 2 * 200 / (ms * 1e-3), "ms": ms,
        "t_final": float(t), "status": hh.hard_hydro_strerror(m32.get_error()),
        "mass_drift_rel": float(abs(tot[-1, 0] - tot[0, 0]) / tot[0, 0]),
        "energy_drift_rel": float(abs(tot[-1, 4] - tot[0, 4]) / tot[0, 4])}
    del Ud
    # 20 steps in FP32 and FP64 from the same input
    Ud = torch.tensor(Ub, device="cuda")
    m32.advance(Ud, 20, 0.3)
    V = torch.tensor(Ub, dtype=torch.float64, device="cuda")
    m64 = hh.HardHydro((n, n, n), 1.4, hh.HARD_BC_REFLECT, dtype=torch.float64)
    m64.advance(V, 20, 0.3)
    rep["blast_512_fp32_vs_fp64_gpu_20_steps"] = _field_errors(Ud.cpu().numpy(), V.cpu().numpy())
    del Ud, V, m64, m32
    # configuration 5: shear layer 256^2, 200 steps
    n = 256
    U = H.shear_2d(n, seed=0, gamma=1.4)
    ref, _, dts = oracle.Grid((1, n, n), 1.4, oracle.BC_PERIODIC).run(U, 200, SMOOTH_CFL)
    m = hh.HardHydro((1, n, n), 1.4, 0)
    Ud = torch.tensor(U, dtype=torch.float32, device="cuda")
    for dt in dts:
        Ud = m.step(Ud, dt)
    rep["shear_2d_256_fp32_vs_oracle"] = _field_errors(Ud.cpu().numpy(), ref)
    print(json.dumps(rep), flush=True)


def stage_roofline(m, U, hbm, peak_kind, kernel_name, reps=20, ty=8):
    """Mean CUDA-event time of the stage-1 and stage-2 launches of handle m on
    state U (inputs larger than L2), against the HBM roofline at the
    algorithmic 50 B per FP32 cell-stage."""
    import torch
    stream = torch.cuda.current_stream()
    cells = U[0].numel()
    U1, U2 = torch.empty_like(U), torch.empty_like(U)
    dt = m.cfl_dt(U, CFL)
    for _ in range(3):
        m.stage(1, None, U, dt, out=U1)
        m.stage(2, U, U1, dt, out=U2)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        m.stage(1, None, U, dt, out=U1)
        m.stage(2, U, U1, dt, out=U2)
    e1.record(stream)
    torch.cuda.synchronize()
    stage_ms = e0.elapsed_time(e1) / (2 * reps)
    alg = BYTES_PER_CELL_STAGE[4] * cells
    achieved = alg / (stage_ms * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": achieved / hbm, "traffic": profiled_traffic(cells, ty), "peak_kind": peak_kind,
            "kernel": kernel_name, "algorithmic_bytes_per_launch": alg, "launch_ms": stage_ms}


def run_sharded(args, world, rank, local):
    """N > 1: the headline workload (the whole 512^3 blast) decomposed into z
    slabs, one per GPU (paper_2509_08971_gb300.slab): per stage a ghost
    exchange of two planes with each neighbour over NCCL, per step one
    all-reduce (max) of the signal rate.  Strong scaling: the job's work is
    the whole mesh whatever N is."""
    import torch
    import torch.distributed as dist
    import hydro_inputs as H
    import paper_2509_08971_gb300 as hh
    from paper_2509_08971_gb300 import autotune, slab

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
    n = args.n
    shape = (n, n, n)
    cells = n ** 3
    L = slab.SlabLayout(n, rank, world, bc_z=(hh.HARD_BC_REFLECT, hh.HARD_BC_REFLECT))
    m = slab.slab_handle(shape, L, GAMMA, [hh.HARD_BC_REFLECT] * 6, dtype=torch.float32)
    backend = slab.CudaSlabBackend(m, L)
    stepper = slab.SlabStepper(backend, slab.HaloExchange(L))
    Ub = H.blast_3d(n, seed=0, gamma=GAMMA, dtype=np.float32, planes=(L.z0, L.z1))
    U0 = torch.tensor(Ub, device=dev)
    U = U0.clone()
    U1 = torch.empty_like(U)
    stepper.exchange(U)                                  # valid ghosts for the tile tuner
    tuned = autotune.tune(m, U, kernel=hh.HARD_KERNEL_FUSED, reps=5)
    stepper.advance(U, U1, max(args.warmup, 3), CFL)
    U.copy_(U0)
    backend.t.zero_()
    barrier()
    stream = torch.cuda.current_stream()
    props = torch.cuda.get_device_properties(dev)
    gpu_id = f"GPU-{props.uuid}" if getattr(props, "uuid", None) else str(dev.index)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(gpu_id) as clk:
        barrier()
        ev0.record(stream)
        stepper.advance(U, U1, args.steps, CFL)
        ev1.record(stream)
        barrier()
    ms = max_over_ranks(ev0.elapsed_time(ev1), world, dev)
    value = cells * 2 * args.steps / (ms * 1e-3)
    status = m.get_error()
    clocks = clk.summary()
    hbm, peak_kind = peaks()
    # this rank's stage kernel on its slab (ghosts from the last exchange)
    stepper.exchange(U)
    roofline = stage_roofline(m, U, hbm, peak_kind,
                              "stage_ws_kernel<32,%d,*> z-chunk %d on a %d-plane slab" % (
                                  tuned["info"][1], tuned["info"][2], L.planes))
    # end to end: the slab from pinned host memory, the steps, the slab back
    Uh = torch.tensor(Ub).pin_memory()
    Uo = torch.empty_like(Uh).pin_memory()
    barrier()
    t0 = time.perf_counter()
    U.copy_(Uh, non_blocking=True)
    backend.t.zero_()
    stepper.advance(U, U1, args.steps, CFL)
    Uo.copy_(U, non_blocking=True)
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world, dev)
    # the batched configuration: the 4096 independent problems split over the
    # ranks by longest-processing-time first, no exchange
    spec = H.batch_spec(4096, seed=0)
    mine = slab.lpt_partition([int(c) for c in spec.cells], world)[rank]
    B = hh.HardBatch([spec.nx[q] for q in mine], [spec.ny[q] for q in mine],
                     [spec.gamma[q] for q in mine] if hasattr(spec.gamma, "__len__") else spec.gamma,
                     hh.HARD_BC_OUTFLOW)
    packed0 = B.pack([H.batch_problem_U(spec, q) for q in mine])
    B.tune(packed0, 0.4)
    P = packed0.clone()
    tb = torch.zeros(len(mine), dtype=torch.float64, device=dev)
    graph = B.capture(P, 50, 0.4, tb)
    P.copy_(packed0)
    tb.zero_()
    barrier()
    b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    b0.record(stream)
    graph.replay()
    b1.record(stream)
    barrier()
    bms = max_over_ranks(b0.elapsed_time(b1), world, dev)
    batched = {"workload": "4096 problems: half 1D n~U{64..4096}, half 2D side~U{32..256}, "
                           "two-state / four-quadrant, gamma 1.4, outflow, CFL 0.4, 50 steps; "
                           f"split over {world} ranks by longest processing time first",
               "value": int(spec.cells.sum()) * 2 * 50 / (bms * 1e-3), "unit": UNIT,
               "problems_per_rank": len(mine), "ms": bms,
               "status": hh.hard_hydro_strerror(B.get_error())}
    del P, packed0, B, graph
    # per step: stage 1, stage 2, the two rate/dt kernels and two plane packs
    # (device copies) per rank; the first step adds the rate kernel
    launches = world * (2 + 4 * args.steps)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "global_cells": cells, "cells_per_gpu": L.planes * n * n,
                   "parallelism": f"z-slabs x{world}: NCCL ghost exchange (2 planes x 5 fields "
                                  "per neighbour per stage) + one all-reduce (max) of the rate "
                                  "per step",
                   "l2": "slab states > 129 MB L2", "tile": {"chosen": tuned["info"]}},
        "roofline": roofline,
        "batched": batched,
        "e2e": {"value": cells * 2 * args.steps / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": world * Uh.numel() * 4 / args.steps,
                "d2h_bytes_per_step": world * Uo.numel() * 4 / args.steps,
                "call": "each rank: its slab from pinned host memory, the decomposed steps, "
                        "the slab back"},
        "gpu_launches": launches,
        "clocks": clocks,
        "status": hh.hard_hydro_strerror(status),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=STEPS)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--f64-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--headline-only", action="store_true",
                    help="time the headline workload only (profiling runs)")
    ap.add_argument("--tile", type=int, default=-1,
                    help="headline stage tile (default: the autotuner's choice)")
    ap.add_argument("--n", type=int, default=N_SIDE,
                    help="mesh side of the headline workload (profiling runs only)")
    ap.add_argument("--shard", action="store_true",
                    help="run the z-slab decomposed path also at N = 1 (checks only)")
    ap.add_argument("--report", choices=["precision"], default=None,
                    help="print a per-field FP32-vs-FP64 error report instead of the bench line")
    args = ap.parse_args()
    world, rank, local = dist_setup()
    if args.report == "precision":
        precision_report()
        return
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    if world > 1 or args.shard:
        run_sharded(args, world, rank, local)
        return

    import torch
    import torch.distributed as dist
    import hydro_inputs as H
    import paper_2509_08971_gb300 as hh
    from paper_2509_08971_gb300 import autotune

    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def rank_max(x):
        return max_over_ranks(x, world, dev)

    stream = torch.cuda.current_stream()
    hbm, peak_kind = peaks()
    n = args.n
    shape = (n, n, n)
    cells = n ** 3
    t_dev = torch.zeros((), dtype=torch.float64, device=dev)

    def advance(m, Ud, k, tlog):
        hh.check(hh.hard_hydro_advance(m.h, Ud.data_ptr(), k, CFL, 0.0, t_dev.data_ptr(), None,
                                       tlog.data_ptr(), stream.cuda_stream), "advance")

    # ---------------- headline: 512^3 blast, FP32 fused, FP64 totals ----------------
    Ub = H.blast_3d(n, seed=rank, gamma=GAMMA, dtype=np.float32)
    U0 = torch.tensor(Ub, device=dev)                    # the initial state, kept for resets
    m32 = hh.HardHydro(shape, GAMMA, hh.HARD_BC_REFLECT, dtype=torch.float32,
                       kernel=hh.HARD_KERNEL_FUSED)
    U = U0.clone()
    if args.tile >= 0:                                   # a fixed tile (profiling runs)
        m32.set_kernel(hh.HARD_KERNEL_FUSED, args.tile)
        tuned = {"tile": args.tile, "info": list(m32.tile_info(args.tile)), "ms": {}}
    else:
        tuned = autotune.tune(m32, U, kernel=hh.HARD_KERNEL_FUSED, reps=5)   # outside the timed region
    tot_log = torch.zeros((max(args.steps, args.warmup, 3), 5), dtype=torch.float64, device=dev)
    advance(m32, U, max(args.warmup, 3), tot_log)
    U.copy_(U0)                                          # the timed steps start at t = 0
    t_dev.zero_()
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    props = torch.cuda.get_device_properties(dev)
    gpu_id = f"GPU-{props.uuid}" if getattr(props, "uuid", None) else str(dev.index)
    with ClockSampler(gpu_id) as clk:
        barrier()
        with nvtx_range("headline_steps"):
            ev0.record(stream)
            advance(m32, U, args.steps, tot_log)
            ev1.record(stream)
            barrier()
    ms = rank_max(ev0.elapsed_time(ev1))
    value = whole_job_value(world, cells, 2 * args.steps, ms)
    status = m32.get_error()
    clocks = clk.summary()
    tot = tot_log[:args.steps].cpu().numpy()
    drift = {"mass_rel": float(abs(tot[-1, 0] - tot[0, 0]) / abs(tot[0, 0])),
             "energy_rel": float(abs(tot[-1, 4] - tot[0, 4]) / abs(tot[0, 4])),
             "t_final": float(t_dev)}
    # kernels of this library launched in the timed region: the signal rate
    # and the first step's dt, then per step stage 1, stage 2 and one
    # finalize launch (the step's totals and the next step's dt)
    launches = 2 + 3 * args.steps
    kname = "stage_ws_kernel<32,%d,*> z-chunk %d (mean of stage 1 and stage 2)" % (
        tuned["info"][1], tuned["info"][2])
    roofline = stage_roofline(m32, U, hbm, peak_kind, kname, ty=tuned["info"][1])
    # the same bytes over half the whole step's time: a floor for the stage
    # launches as they run in the step (stage 2 with its rate and totals
    # epilogue, the finalize launch and the gaps between launches charged to
    # them); launch_ms above times the stage launches alone
    step_half = ms / args.steps / 2
    roofline["in_step"] = {"ms_per_launch": step_half,
                           "achieved": roofline["algorithmic_bytes_per_launch"] / (step_half * 1e-3)
                           / 1e9,
                           "frac": roofline["algorithmic_bytes_per_launch"] / (step_half * 1e-3)
                           / 1e9 / hbm}
    issue = issue_roofline(cells, roofline["launch_ms"], clocks.get("sm_mhz"), tuned["info"][1])
    if args.headline_only:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "ms_per_step": ms / args.steps,
                              "roofline": roofline, "status": hh.hard_hydro_strerror(status)}))
        return

    # ---------------- the same workload end to end through the C ABI, host buffers ----------------
    Uh = torch.tensor(Ub).pin_memory()
    Uo = torch.empty_like(Uh).pin_memory()
    Ud = torch.empty(Uh.shape, dtype=Uh.dtype, device=dev)
    ev2 = torch.cuda.Event(enable_timing=True)

    def copy_gbs():
        # one copy of the state each way between the pinned buffers and the
        # device, on their own (the host's pinned-memory copy rate varies:
        # after other large jobs on the machine it was seen to start several
        # times slower and recover within seconds)
        barrier()
        ev0.record(stream)
        Ud.copy_(Uh, non_blocking=True)
        ev1.record(stream)
        Uo.copy_(Ud, non_blocking=True)
        ev2.record(stream)
        barrier()
        return {"h2d": Uh.numel() * 4 / ev0.elapsed_time(ev1) / 1e6,
                "d2h": Uo.numel() * 4 / ev1.elapsed_time(ev2) / 1e6}

    copy_before = copy_gbs()
    m32.advance_host(Uh, 1, CFL, out=Uo)                 # warm the handle's device buffer
    barrier()
    e2e_runs, e2e_dev = [], []                           # three timed calls, the median reported
    with ClockSampler(gpu_id) as clk_e2e:
        time.sleep(0.3)                                  # the sampler is up before the first call
        for _ in range(3):
            barrier()
            t0 = time.perf_counter()
            ev0.record(stream)
            m32.advance_host(Uh, args.steps, CFL, out=Uo)
            ev1.record(stream)
            barrier()
            e2e_runs.append(rank_max(time.perf_counter() - t0))
            e2e_dev.append(ev0.elapsed_time(ev1))
    e2e_s = sorted(e2e_runs)[1]
    copy_after = copy_gbs()
    e2e = {"value": whole_job_value(world, cells, 2 * args.steps, e2e_s * 1e3), "unit": UNIT,
           "h2d_bytes_per_step": Uh.numel() * 4 / args.steps,
           "d2h_bytes_per_step": Uo.numel() * 4 / args.steps,
           "call": f"hard_hydro_advance_host: one call of {args.steps} steps of the blast from "
                   "t = 0, pinned host buffers, both copies in the timed region; the median of "
                   "three calls",
           "seconds_per_call": e2e_runs,
           "device_ms_per_call": e2e_dev,               # the stream's span: copies and steps
           "pinned_copy_gbs": {"before": copy_before, "after": copy_after},
           "clocks": clk_e2e.summary()}
    del Uh, Uo, Ud, U, U0, m32

    # ---------------- FP64 plain on the same workload ----------------
    m64 = hh.HardHydro(shape, GAMMA, hh.HARD_BC_REFLECT, dtype=torch.float64,
                       kernel=hh.HARD_KERNEL_PLAIN)
    V0 = torch.tensor(H.blast_3d(n, seed=rank, gamma=GAMMA), dtype=torch.float64, device=dev)
    V = V0.clone()
    k64 = max(1, args.f64_steps)
    tl64 = torch.zeros((max(k64, 3), 5), dtype=torch.float64, device=dev)
    advance(m64, V, 3, tl64)
    V.copy_(V0)
    t_dev.zero_()
    barrier()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    advance(m64, V, k64, tl64)
    f1.record(stream)
    barrier()
    ms64 = rank_max(f0.elapsed_time(f1))
    value64 = whole_job_value(world, cells, 2 * k64, ms64)
    fp64 = {"value": value64, "unit": UNIT, "steps": k64, "ms_per_step": ms64 / k64,
            "kernel": "stage_kernel<double,...> (plain loads)", "fp32_fused_speedup": value / value64,
            "status": hh.hard_hydro_strerror(m64.get_error())}
    del V, V0, m64

    # ---------------- secondary: 256^3 periodic smooth flow, FP32 fused ----------------
    n2 = SMOOTH_N
    shape2 = (n2, n2, n2)
    cells2 = n2 ** 3
    U64 = H.smooth_3d(n2, seed=rank, gamma=SMOOTH_GAMMA)
    ms2 = hh.HardHydro(shape2, SMOOTH_GAMMA, hh.HARD_BC_PERIODIC, dtype=torch.float32)
    Us = torch.tensor(U64, dtype=torch.float32, device=dev)
    tuned2 = autotune.tune(ms2, Us, kernel=hh.HARD_KERNEL_FUSED, reps=5)

    def advance2(m, Ud, k, tlog):
        hh.check(hh.hard_hydro_advance(m.h, Ud.data_ptr(), k, SMOOTH_CFL, 0.0, t_dev.data_ptr(),
                                       None, tlog.data_ptr(), stream.cuda_stream), "advance")

    ks = max(20, args.steps)
    tl2 = torch.zeros((ks, 5), dtype=torch.float64, device=dev)
    advance2(ms2, Us, 3, tl2)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    advance2(ms2, Us, ks, tl2)
    e1.record(stream)
    barrier()
    mss = rank_max(e0.elapsed_time(e1))
    smooth = {"workload": SMOOTH_WORKLOAD, "value": whole_job_value(world, cells2, 2 * ks, mss),
              "unit": UNIT, "steps": ks, "ms_per_step": mss / ks,
              "tile": {"chosen": tuned2["info"], "ms_per_stage": tuned2["ms"]},
              "roofline": stage_roofline(ms2, Us, hbm, peak_kind,
                                         "stage_ws_kernel<32,%d,*> z-chunk %d" % (
                                             tuned2["info"][1], tuned2["info"][2]),
                                         ty=tuned2["info"][1]),
              "status": hh.hard_hydro_strerror(ms2.get_error())}
    alg_bytes2 = BYTES_PER_CELL_STAGE[4] * cells2

    # ---------------- second scheme: WENO5-Z + HLL, FP32, 256^3 smooth flow ----------------
    mw = hh.HardHydro(shape2, SMOOTH_GAMMA, hh.HARD_BC_PERIODIC, dtype=torch.float32,
                      scheme=hh.HARD_SCHEME_WENO5Z_HLL)
    Uw = torch.tensor(U64, dtype=torch.float32, device=dev)
    kw = max(2, min(args.steps, 200) // 4)
    advance2(mw, Uw, 3, tl2)
    barrier()
    e0.record(stream)
    advance2(mw, Uw, kw, tl2)
    e1.record(stream)
    barrier()
    msw = rank_max(e0.elapsed_time(e1))
    W1, W2 = torch.empty_like(Uw), torch.empty_like(Uw)
    dtw = mw.cfl_dt(Uw, SMOOTH_CFL)
    for _ in range(2):
        mw.stage(1, None, Uw, dtw, out=W1)
        mw.stage(2, Uw, W1, dtw, out=W2)
    barrier()
    e0.record(stream)
    for _ in range(10):
        mw.stage(1, None, Uw, dtw, out=W1)
        mw.stage(2, Uw, W1, dtw, out=W2)
    e1.record(stream)
    barrier()
    wstage_ms = e0.elapsed_time(e1) / 20
    w_achieved = alg_bytes2 / (wstage_ms * 1e-3) / 1e9
    weno = {"workload": SMOOTH_WORKLOAD.replace("CFL 0.4", "CFL 0.4, WENO5-Z + HLL"),
            "value": whole_job_value(world, cells2, 2 * kw, msw), "unit": UNIT, "steps": kw,
            "ms_per_step": msw / kw, "status": hh.hard_hydro_strerror(mw.get_error()),
            "roofline": {"bound": "hbm", "achieved": w_achieved, "peak": hbm, "unit": "GB/s",
                         "frac": w_achieved / hbm, "traffic": None, "peak_kind": peak_kind,
                         "kernel": "weno_x_kernel + weno_march_kernel (y') + weno_march_kernel "
                                   "(z', combine): one stage's three sweeps, z/y chunks of 64 "
                                   "(mean of stage 1 and stage 2)",
                         "algorithmic_bytes_per_launch": alg_bytes2, "launch_ms": wstage_ms}}
    del mw, Uw, W1, W2

    # ---------------- radiative heating / cooling exchange, FP32 ----------------
    pbr = H.cooling()
    Ur, Err = pbr.state(shape2, seed=rank, spread=0.5)
    mr = hh.HardHydro(shape2, pbr.gamma, hh.HARD_BC_PERIODIC, dtype=torch.float32)
    Urd = torch.tensor(Ur, dtype=torch.float32, device=dev)
    Erd = torch.tensor(Err, dtype=torch.float32, device=dev)
    del Ur, Err
    dt_rad = 1e-12                                  # every launch solves a fresh implicit step
    for _ in range(3):
        mr.rad_exchange(Urd, Erd, dt_rad, *pbr.params)
    barrier()
    e0.record(stream)
    for _ in range(20):
        mr.rad_exchange(Urd, Erd, dt_rad, *pbr.params)
    e1.record(stream)
    barrier()
    rad_ms = e0.elapsed_time(e1) / 20
    rad_bytes = 8 * 4 * cells2                      # reads rho, 3 momenta, E_total, E; writes 2
    rad_achieved = rad_bytes / (rad_ms * 1e-3) / 1e9
    rad = {"workload": "256^3 radiative heating/cooling exchange (Sec. 3.2 cooling case, "
                       "seeded +-50% spread in rho, T_f, T_r; moving fluid), FP32, dt 1e-12 s, "
                       "state 403 MB > L2",
           "value": whole_job_value(world, cells2, 1, rank_max(rad_ms)), "unit": UNIT,
           "launch_ms": rad_ms, "status": hh.hard_hydro_strerror(mr.get_error()),
           "roofline": {"bound": "hbm", "achieved": rad_achieved, "peak": hbm, "unit": "GB/s",
                        "frac": rad_achieved / hbm, "traffic": None, "peak_kind": peak_kind,
                        "kernel": "rad_exchange_kernel<float>",
                        "algorithmic_bytes_per_launch": rad_bytes}}
    del mr, Urd, Erd

    # ---------------- radiation energy advection (WENO5-Z + Rusanov), FP32 ----------------
    Ea = torch.tensor(1.0 + 0.5 * np.random.default_rng(200 + rank).random(shape2),
                      dtype=torch.float32, device=dev)
    dt_adv = ms2.cfl_dt(Us, SMOOTH_CFL)
    for _ in range(2):
        ms2.advect_E(Us, Ea, dt_adv)
    barrier()
    e0.record(stream)
    for _ in range(5):
        ms2.advect_E(Us, Ea, dt_adv)
    e1.record(stream)
    barrier()
    adv_ms = e0.elapsed_time(e1) / 5
    # per Heun step: two stages, each reading E, rho and the three momenta and
    # writing E (24 B/cell), the second also reading E^n (4 B/cell)
    adv_bytes = (24.0 + 28.0) * cells2
    adv_achieved = adv_bytes / (adv_ms * 1e-3) / 1e9
    advect = {"workload": f"{n2}^3 periodic radiation energy advection by the smooth-flow "
                          "velocity field, E ~ 1 + 0.5 U[0,1) (seeded), Heun step, FP32",
              "value": whole_job_value(world, cells2, 2, rank_max(adv_ms)), "unit": UNIT,
              "ms_per_step": adv_ms,
              "roofline": {"bound": "hbm", "achieved": adv_achieved, "peak": hbm, "unit": "GB/s",
                           "frac": adv_achieved / hbm, "traffic": None, "peak_kind": peak_kind,
                           "kernel": "advect_x_kernel + advect_march_kernel (y') + "
                                     "advect_march_kernel (z', Heun stage): three sweeps per stage",
                           "algorithmic_bytes_per_step": adv_bytes}}
    del Ea, ms2, Us

    # ---------------- flux-limited radiation diffusion (multigrid), FP32 ----------------
    mf = hh.HardHydro(shape2, SMOOTH_GAMMA, hh.HARD_BC_PERIODIC, dtype=torch.float32)
    gf = np.random.default_rng(100 + rank)
    Uf = torch.zeros((5,) + shape2, dtype=torch.float32, device=dev)
    Uf[0] = torch.tensor(1.0 + 0.5 * gf.random(shape2), dtype=torch.float32, device=dev)
    Ef0 = torch.tensor(1.0 + 0.5 * gf.random(shape2), dtype=torch.float32, device=dev)
    Ef = Ef0.clone()
    dt_fld = 100.0 * (1.0 / n2) ** 2 * 3            # diffusion number ~ 100 (c = kappa = 1)
    mf.fld_step(Uf, Ef, dt_fld, 1.0, 1.0, rtol=1e-5, max_cycles=40)      # builds the levels
    Ef.copy_(Ef0)
    barrier()
    with nvtx_range("fld_step"):
        e0.record(stream)
        cyc_f, res_f = mf.fld_step(Uf, Ef, dt_fld, 1.0, 1.0, rtol=1e-5, max_cycles=40)
        e1.record(stream)
    barrier()
    fld_ms = e0.elapsed_time(e1)
    # bytes per V-cycle: per level, two pre- and two post-smoothing red-black
    # sweeps (24 B/cell each: x read twice, b and D, x written), the fused
    # residual-restriction (11: x and D of every cell, b of the colour-0
    # cells it evaluates, the coarse b and x), prolongation (12): 119 B/cell,
    # x 8/7 over the levels (the per-cycle convergence check not counted)
    fld_bytes = 119.0 * 8.0 / 7.0 * cells2 * cyc_f
    fld_achieved = fld_bytes / (fld_ms * 1e-3) / 1e9
    fld = {"workload": f"{n2}^3 periodic implicit flux-limited diffusion step, c = kappa = 1, "
                       "rho, E ~ 1 + 0.5 U[0,1) (seeded), diffusion number ~100, "
                       "V-cycles to a 1e-5 relative residual, FP32",
           "value": whole_job_value(world, cells2, cyc_f, rank_max(fld_ms)),
           "unit": "cell-V-cycles/s", "cycles": cyc_f, "rel_residual": res_f, "ms": fld_ms,
           "roofline": {"bound": "hbm", "achieved": fld_achieved, "peak": hbm, "unit": "GB/s",
                        "frac": fld_achieved / hbm, "traffic": None, "peak_kind": peak_kind,
                        "kernel": "V-cycle (smooth/residual/restrict/prolong kernels)",
                        "algorithmic_bytes_per_cycle": fld_bytes / max(cyc_f, 1)}}
    del mf, Uf, Ef, Ef0

    # ---------------- batched: 4096 independent 1D/2D problems ----------------
    spec = H.batch_spec(4096, seed=rank)
    B = hh.HardBatch(spec.nx, spec.ny, spec.gamma, hh.HARD_BC_OUTFLOW)
    packed0 = B.pack([H.batch_problem_U(spec, q) for q in range(spec.nprob)])
    bcells = int(spec.cells.sum())
    btune = B.tune(packed0, SMOOTH_CFL)                     # tile choice, untimed
    P = packed0.clone()
    tb = torch.zeros(spec.nprob, dtype=torch.float64, device=dev)
    graph = B.capture(P, 50, SMOOTH_CFL, tb)                # one persistent launch, captured
    P.copy_(packed0)
    tb.zero_()
    barrier()
    b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    b0.record(stream)
    graph.replay()
    b1.record(stream)
    barrier()
    bms = rank_max(b0.elapsed_time(b1))
    batched = {"workload": "4096 problems: half 1D n~U{64..4096}, half 2D side~U{32..256}, "
                           "two-state / four-quadrant, gamma 1.4, outflow, CFL 0.4, 50 steps",
               "value": whole_job_value(world, bcells, 2 * 50, bms), "unit": UNIT, "cells": bcells,
               "ms": bms, "tile": btune["tile"], "tile_ms_5_steps": btune["ms"],
               "graph_captured": True, "status": hh.hard_hydro_strerror(B.get_error())}
    del P, packed0, B, graph

    # ---------------- adjoint cost: 2D shear layer 256^2, FP32 ----------------
    na = 256
    ma = hh.HardHydro((1, na, na), 1.4, hh.HARD_BC_PERIODIC, dtype=torch.float32)
    Ua = torch.tensor(H.shear_2d(na, seed=rank, gamma=1.4), dtype=torch.float32, device=dev)
    dta = ma.cfl_dt(Ua, SMOOTH_CFL)
    Ga = torch.randn_like(Ua)
    gga = torch.zeros((), dtype=torch.float64, device=dev)
    Va, Ha = torch.empty_like(Ua), torch.empty_like(Ua)
    for _ in range(5):
        ma.step(Ua, dta, out=Va)
        ma.step_backward(Ua, Ga, dta, gga, out=Ha)
    reps_a = 200

    def timed(fn):
        # the best of three windows: these launches are short enough that a
        # host-side stall in one window would dominate it
        best = None
        for _ in range(3):
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a0.record(stream)
            for _ in range(reps_a):
                fn()
            a1.record(stream)
            torch.cuda.synchronize()
            t = a0.elapsed_time(a1) / reps_a
            best = t if best is None else min(best, t)
        return best

    fwd_ms = timed(lambda: ma.step(Ua, dta, out=Va))
    bwd_ms = timed(lambda: ma.step_backward(Ua, Ga, dta, gga, out=Ha))

    def graph_timed(fn, k=50):
        # GPU cost of a step without the per-call host overhead: k steps
        # captured in one CUDA graph, the best of three replays
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            for _ in range(k):
                fn()
        g.replay()
        best = None
        for _ in range(3):
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a0.record()
            g.replay()
            a1.record()
            torch.cuda.synchronize()
            t = a0.elapsed_time(a1) / k
            best = t if best is None else min(best, t)
        del g
        return best

    fwd_g = graph_timed(lambda: ma.step(Ua, dta, out=Va))
    bwd_g = graph_timed(lambda: ma.step_backward(Ua, Ga, dta, gga, out=Ha))
    adjoint = {"workload": "2D periodic shear layer 256^2, gamma 1.4, FP32",
               "forward_step_ms": fwd_g, "backward_step_ms": bwd_g, "ratio": bwd_g / fwd_g,
               "timing": "50 steps captured in one CUDA graph, replayed (GPU cost per step)",
               "eager_forward_step_ms": fwd_ms, "eager_backward_step_ms": bwd_ms,
               "eager_ratio": bwd_ms / fwd_ms,
               "backward_includes": "stage-1 recompute + stage-2 and stage-1 VJP"}
    del ma, Ua, Ga, Va, Ha

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "cells_per_gpu": cells, "global_cells": world * cells,
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "l2": "state 2.7 GB > 129 MB L2 (no flush needed)", "kernel": "fused",
                   "tile": {"chosen": tuned["info"], "ms_per_stage": tuned["ms"]},
                   "step": "CFL rate + stage 1 + stage 2 + FP64 totals",
                   "conservation": drift},
        "roofline": roofline, "issue_roofline": issue,
        "fp64_plain": fp64,
        "smooth_3d_256": smooth,
        "weno5z_hll": weno,
        "rad_exchange": rad,
        "radiation_advection": advect,
        "fld_multigrid": fld,
        "batched": batched,
        "adjoint": adjoint,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clocks,
        "status": hh.hard_hydro_strerror(status),
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        threads = cpu_threads()
        planes = 64
        rate, sec, used = time_oracle(blast_slab(planes), 2, threads, oracle.BC_REFLECT, GAMMA, CFL)
        line["cpu_baseline"] = {
            "value": rate, "unit": UNIT, "cores": used, "kind": "oracle",
            "sample": f"2 RK2 steps of the middle {planes} z planes of the 512^3 blast "
                      f"(512x512x{planes} cells, reflecting walls, CFL 0.3; {sec:.1f} s)"}
        rate1, sec1, _ = time_oracle(blast_slab(4), 1, 1, oracle.BC_REFLECT, GAMMA, CFL)
        line["cpu_baseline"]["single_thread"] = {
            "value": rate1, "unit": UNIT, "cores": 1,
            "sample": f"1 RK2 step of the middle 4 z planes of the blast ({sec1:.1f} s)"}
        for n, steps in ((128, 3), (256, 1)):
            Us = H.smooth_3d(n, seed=0, gamma=SMOOTH_GAMMA)
            rs, ssec, used_s = time_oracle(Us, steps, threads, oracle.BC_PERIODIC, SMOOTH_GAMMA,
                                           SMOOTH_CFL)
            line["cpu_baseline"][f"smooth_3d_{n}"] = {
                "value": rs, "unit": UNIT, "cores": used_s,
                "sample": f"configuration 2 at {n}^3: {steps} RK2 step(s) of the periodic smooth "
                          f"flow ({ssec:.1f} s)"}
            del Us
        rr, rsec, rsteps = time_oracle_riemann()
        line["cpu_baseline"]["riemann_1d_400"] = {
            "value": rr, "unit": UNIT, "cores": 1,
            "sample": f"configuration 1 in full: 400 cells to t = 0.15, {rsteps} steps "
                      f"({1e3 * rsec:.1f} ms)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
