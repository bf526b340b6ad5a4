"""Benchmark: cell-RK-stage updates/s of the FP64 MEG6 + HLLC + alpha-damping
right-hand side with SSP-RK3 on one B300, plus the roofline of the dominant
kernel (the interface-flux kernel) and of the whole step, and the CPU oracle as
the baseline.

Workloads (--workload):
  tgv (default)  3D viscous Taylor-Green vortex, Re = 1600, M = 0.1, Pr = 0.71,
                 on a 128^3 periodic [0, 2 pi]^3 mesh with a 0.1 h sinusoidal
                 node perturbation, CFL 0.2 (dt computed on the device every step).
  jet            480 x 170 x 170 (13.9 M cells) jet-like box: uniform in x on
                 [0, 20 D], stretched (ratio 1.02) away from the axis, quiescent
                 ambient, sonic top-hat inflow with a 1 % random velocity
                 perturbation drawn per step (counter-based hash of seed, step,
                 cell), Sutherland viscosity, Re_D = 1e5, sponge, fixed dt = 2e-3.
A step is one full SSP-RK3 step (three right-hand sides, stage combinations and,
for tgv, the time step); the working sets (~3 GB, ~20 GB) are far larger than
L2, so no flush is needed between steps.

The default run (tgv, FP64, 128^3, one GPU) also measures, beside the headline and
under the same rules: "mixed" (the same workload on the mixed-precision path, with
its state against the FP64 path's after the same steps), "jet" (the 480 x 170 x 170
jet-like box, FP64) and "serving" (a bounded 32-job sample of the serving stream,
per-job FP64 against the continuous-batching server); --no-extras skips them.  The
arithmetic roofline's peak is the FMA throughput measured on the same GPU first
(gbr_alu_peak), with the unit-count figure and the nominal one beside it.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--workload tgv|jet]
Under torchrun (N > 1) each rank advances its own copy of the workload (the
jobs are independent: replicas, weak scaling); rank 0 prints one JSON line.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_CELLS_EDGE = 128
CFL = 0.2
JET_DT = 2e-3
JET_SEED = 2303
METRIC = "cell-RK-stage updates/s"
# Arithmetic peaks of this ALU-bound path.  The roofline's denominator is the FMA throughput
# measured live on the GPU that runs the kernels (gbr_alu_peak, before the timed region); beside it
# the figures derived from unit counts and the maximum SM clock, and the nominal FP64 figure:
# FP64 148 SMs x 2 DFMA/clk x 2 flop x 2.032 GHz = 1.203 TFLOP/s (nominal 1.25),
# FP32 148 SMs x 128 FFMA/clk x 2 flop x 2.032 GHz = 77.0 TFLOP/s.
SM_MAX_GHZ = 2.032
FP64_DERIVED_TFLOPS = 148 * 2 * 2 * SM_MAX_GHZ / 1e3
FP32_DERIVED_TFLOPS = 148 * 128 * 2 * SM_MAX_GHZ / 1e3
FP64_NOMINAL_TFLOPS = 1.25


def measured_hbm_gbs():
    """HBM copy bandwidth measured on this machine (MEASURED_PEAKS.json), else the recipe's fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6400.0, "fallback"


HBM_PEAK_GBS, HBM_PEAK_KIND = measured_hbm_gbs()
# minimum HBM traffic of a 3D FP64 cell-stage: state and cell geometry, stage average
BYTES_PER_CELL_STAGE_3D = 186.7
# DRAM bytes (read + write) per interface of the 3D viscous interface kernel, from one ncu
# capture of a launch of the current kernels (dram__bytes_read.sum + dram__bytes_write.sum):
# FP64, 385.2 MB for the 893,952 interfaces of a 96^3 y-sweep; FP32 (mixed path), 327.9 MB for
# the 2,113,536 of a 128^3 z-sweep.  Traffic grows in proportion to the interfaces of a launch.
FACE_DRAM_BYTES_PER_INTERFACE = 385.20e6 / 893952
FACE_DRAM_BYTES_PER_INTERFACE_F32 = 327.90e6 / 2113536
# FP64 operations (DFMA + DMUL + DADD thread-instructions) the FP64 interface kernel executes per
# interface, from the same capture (smsp__sass_thread_inst_executed_op_{dfma,dmul,dadd}_pred_on:
# 200.9 + 93.6 + 58.8): below the algorithmic flop count because the mesh-only interface geometry
# is stored once per mesh and the algebra is restructured.  Each occupies one FP64 pipe slot, so
# the pipe's rate is half the measured FMA peak in flop/s.
FACE_FP64_OPS_PER_INTERFACE = 353.3
# Warp instructions the FP32 interface kernel issues per interface, from the 128^3 z-sweep capture
# (smsp__inst_executed.sum 89.5 M for 2,113,536 interfaces; the x-sweep issues ~5 % more).  The
# kernel is bound by instruction issue rather than HBM: each SM sub-partition issues one warp
# instruction per clock, 4 per SM.
FACE_F32_WARP_INSTR_PER_INTERFACE = 89.5e6 / 2113536
ISSUE_PEAK_WARP_INSTR_PER_S = 148 * 4 * SM_MAX_GHZ * 1e9


def load_flops():
    with open(os.path.join(ROOT, "tests", "golden", "flop_counts.json")) as f:
        return json.load(f)


def face_alg_bytes(wl):
    """Algorithmic HBM bytes per interface of one sweep: every array element the interface kernel
    needs, read once (the cells of a sweep are shared by its interfaces), and the flux written once."""
    nd = 3
    nv = nd + 2
    visc = wl.case.get("reynolds", 0.0) > 0.0
    er = 4 if wl.precision == "mixed" else 8
    # primitives and P' along the sweep, and P'' (the FP32 kernel forms P'' from P and P' itself)
    cells = er * (nv + nv + (0 if wl.precision == "mixed" else nv))
    if visc:
        cells += er * (1 + 1 + (nd - 1) * (nd + 1))               # T, T', tangential [u, T]' of two directions
    # interface metrics: FP64, or the FP32 copies the mixed path reads; the FP64 kernel also reads
    # the stored interface geometry (unit normal, |n^|^2, 1/|n^|, |n^|, 1/|n^|^2, viscous m_e)
    metrics = er * (nd + (nd * nd if visc else 0) + (1 if wl.case.get("moving", 0) else 0))
    if wl.precision != "mixed":
        metrics += er * (7 + (3 if visc else 0))
    return cells + metrics + er * nv


class Workload:
    """Inputs and per-step driving of one benchmark workload."""

    def __init__(self, kind, edge=N_CELLS_EDGE, precision="fp64", scheme="meg6"):
        from paper_2303_10785_b300 import inputs as I

        self.kind = kind
        self.precision = precision
        self.scheme = scheme
        self.inflow = self.sponge = None
        if kind == "tgv":
            n = (edge,) * 3
            self.case = I.case_params(3, n, reynolds=1600.0, prandtl=0.71)
            self.nodes = I.nodes_tgv_3d(edge, 0.1)
            xc = I.centroids(self.nodes, n, (1, 1, 1))
            self.q = I.prim_to_cons(I.tgv_prim(*xc, mach=0.1), self.case["gamma"])
            self.name = f"tgv3d_viscous_{edge}^3_perturbed"
            self.flops_key = "tgv3d_viscous"
            self.config = {"cells": edge ** 3, "cfl": CFL, "reynolds": 1600.0, "mach": 0.1}
        else:
            n = (480, 170, 170)
            self.case, self.nodes, self.q, self.inflow, sigma, qamb = I.jet_case(n)
            self.sponge = (sigma, qamb)
            self.name = "jet3d_viscous_480x170x170_stretched"
            self.flops_key = "jet3d_viscous"
            self.config = {"cells": n[0] * n[1] * n[2], "dt": JET_DT, "reynolds_d": 1e5, "sutherland": True,
                           "inflow_perturbation": "1 % velocity, SplitMix64(seed, step, cell, component)"}
        self.case = dict(self.case, precision=precision, gradient_scheme=scheme)
        if precision != "fp64":
            self.name += "_" + precision
        if scheme != "meg6":
            self.name += "_" + scheme
        self.n = n
        self.cells = n[0] * n[1] * n[2]
        self.faces_per_rhs = sum((n[0] + (d == 0)) * (n[1] + (d == 1)) * (n[2] + (d == 2)) for d in range(3))
        self.planes = None

    def attach(self, solver, n_steps):
        """Boundary data on the solver; for the jet, the inflow planes of n_steps steps on the device."""
        if self.inflow is None:
            return
        import torch

        from paper_2303_10785_b300 import inputs as I

        solver.set_sponge(*self.sponge)
        planes = np.stack([I.jet_inflow_step(self.inflow, JET_SEED, s) for s in range(n_steps)])
        self.planes = torch.from_numpy(planes).to(solver.device)
        torch.cuda.synchronize(solver.device)

    def step(self, solver, i):
        """One SSP-RK3 step number i (all work queued on the solver's stream)."""
        if self.planes is not None:
            solver.set_inflow(self.planes[i % self.planes.shape[0]])
            solver.rk_step(-JET_DT)
        else:
            solver.rk_step(CFL)

    def oracle_sample(self, small=False):
        """A bounded sample of the workload for the CPU oracle: (case, nodes, q, inflow, sponge, cells, text).
        small: the sample a single thread times (a 64^3 Taylor-Green vortex of the same recipe, or the
        first 10 x-cells of the jet)."""
        from paper_2303_10785_b300 import inputs as I

        if self.kind == "tgv":
            if small:
                e = 64
                n = (e,) * 3
                case = dict(self.case, n=n)
                nodes = I.nodes_tgv_3d(e, 0.1)
                xc = I.centroids(nodes, n, (1, 1, 1))
                q = I.prim_to_cons(I.tgv_prim(*xc, mach=0.1), self.case["gamma"])
                return case, nodes, q, None, None, e ** 3, "the same Taylor-Green recipe on 64^3"
            return self.case, self.nodes, self.q, None, None, self.cells, f"the full {self.n[0]}^3 workload"
        m = (10, 170, 170) if small else (40, 170, 170)
        case, nodes, q, inflow, sigma, qamb = I.jet_case(m, Lx=20.0 * m[0] / 480)
        return (case, nodes, q, I.jet_inflow_step(inflow, JET_SEED, 0), (sigma, qamb), m[0] * m[1] * m[2],
                f"the first {m[0]} of the 480 x-cells of the jet grid (full 170 x 170 cross-section, inflow, sponge)")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "", 1).isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "", 1).isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[3 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def dist_max(value, device=None):
    """Max of a float over the ranks of the default process group (the value itself alone).
    The jobs of the ranks are independent (replicas or shards of the serving stream): this
    timing reduction is the only collective."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def shard(items, rank, world):
    """The items of one rank: every world-th item from position rank (a partition of the list)."""
    return list(items[rank::world])


def merge_serving(records):
    """Whole-job serving statistics from per-rank records {"lat": [s...], "work": W, "makespan": s}:
    time-to-N-steps percentiles over every rank's jobs, throughput = all work / slowest makespan."""
    lat = np.concatenate([np.asarray(r["lat"], dtype=np.float64) for r in records])
    work = float(sum(r["work"] for r in records))
    span = max(r["makespan"] for r in records)
    return {"jobs": int(lat.size), "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "makespan_s": span, "cell_rk_stage_updates_per_s": work / max(span, 1e-9)}


def gather_objects(obj):
    """Every rank's object, in rank order (the object itself alone)."""
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [obj]
    out = [None] * dist.get_world_size()
    dist.all_gather_object(out, obj)
    return out


def _oracle_stage(orc, q):
    """One SSP-RK3 stage of the oracle: a right-hand side and the first stage combination."""
    return q + 1e-3 * orc.rhs(q)


def _oracle_for(wl, small=False):
    import oracle as O

    case, nodes, q, inflow, sponge, cells, text = wl.oracle_sample(small)
    orc = O.Oracle(case, nodes)
    if inflow is not None:
        orc.set_inflow(inflow)
        orc.set_sponge(*sponge)
    return orc, q, cells, text


def cpu_baseline(wl, seconds=10.0, max_samples=40):
    """The oracle as it stands on the host cores: RK stages of a bounded sample of the workload,
    repeated until about `seconds` of CPU work (at least two)."""
    import oracle as O

    orc, q, cells, text = _oracle_for(wl)
    samples = 0
    t0 = time.perf_counter()
    while samples < 2 or (time.perf_counter() - t0 < seconds and samples < max_samples):
        _oracle_stage(orc, q)
        samples += 1
    el = time.perf_counter() - t0
    cores = O.threads()
    out = {"value": cells * samples / el, "unit": METRIC, "cores": cores, "kind": "oracle",
           "sample": f"{samples} RK stage(s) (right-hand side + stage combination) of {text}, "
                     f"geometry set-up excluded, {el:.1f} s"}
    # the same oracle on one thread, on a smaller sample of the workload (one stage)
    O.set_threads(1)
    try:
        orc1, q1, cells1, text1 = _oracle_for(wl, small=True)
        t0 = time.perf_counter()
        _oracle_stage(orc1, q1)
        el1 = time.perf_counter() - t0
        out["value_1_thread"] = cells1 / el1
        out["sample_1_thread"] = f"1 RK stage of {text1} on 1 thread, {el1:.1f} s"
    finally:
        O.set_threads(cores)
    return out


def config_of(wl, world):
    """The workload description both arms report (identical for the GPU and the reference arm)."""
    return dict({"workload": wl.name}, **wl.config, precision=wl.precision, gradients=wl.scheme,
                parallelism=f"replicas{world}", l2="working set >> 126 MB L2, no flush")


def run_reference(args, wl):
    """Reference arm: the CPU oracle as it stands, one RK stage of the workload's sample per step."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle as O

    orc, q, cells, text = _oracle_for(wl)
    for _ in range(args.warmup):
        _oracle_stage(orc, q)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        _oracle_stage(orc, q)
    el = time.perf_counter() - t0
    value = cells * args.steps / el
    sample = f"{args.steps} RK stage(s) of {text} on the host cores (one stage per step)"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_of(wl, args.gpus),
        "cpu_baseline": {"value": value, "unit": METRIC, "cores": O.threads(), "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def measure_peaks():
    """FP64 and FP32 FMA throughput of this GPU (TFLOP/s), measured by the library's probe."""
    from paper_2303_10785_b300 import gbr

    f64, ms64 = gbr.alu_peak("fp64")
    f32, ms32 = gbr.alu_peak("mixed")
    return {"fp64_tflops": f64, "fp32_tflops": f32, "probe_ms": {"fp64": ms64, "fp32": ms32},
            "fp64_derived_tflops": FP64_DERIVED_TFLOPS, "fp32_derived_tflops": FP32_DERIVED_TFLOPS,
            "fp64_nominal_tflops": FP64_NOMINAL_TFLOPS}


def measure(wl, dev, steps, warmup, e2e_steps, peaks, world, local, keep_state=False):
    """Time `steps` SSP-RK3 steps of `wl` device-resident (after `warmup` steps), then `e2e_steps`
    steps end to end through the C ABI from pinned host memory; the interface kernel's roofline
    and the whole step's.  Returns a dict (the final device-resident state under "state" if asked)."""
    import torch

    from paper_2303_10785_b300 import gbr

    solver = gbr.Solver(wl.case, wl.nodes, device=dev)
    stream = solver.stream
    cells = wl.cells
    wl.attach(solver, warmup + steps + 2 + e2e_steps)

    def barrier():
        if world > 1:
            import torch.distributed as dist

            dist.barrier()

    # ---- device-resident throughput
    solver.set_state(wl.q)
    step = 0
    for _ in range(warmup):
        wl.step(solver, step)
        step += 1
    solver.sync()
    solver.profile(True)
    barrier()
    torch.cuda.synchronize(dev)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clocks:
        ev0.record(stream)
        for _ in range(steps):
            wl.step(solver, step)
            step += 1
        ev1.record(stream)
        torch.cuda.synchronize(dev)
    barrier()
    ms = ev0.elapsed_time(ev1)
    face_ms, face_launches, launches = solver.profile(False)
    solver.sync()
    ms = dist_max(ms, dev)
    value = world * 3 * cells * steps / (ms / 1e3)
    out = {"value": value, "ms": ms, "launches": launches, "clocks": clocks.summary(),
           "workspace_bytes": solver.workspace_bytes}
    if keep_state:
        out["state"] = solver.get_state()

    # ---- end to end through the C ABI with pinned host buffers (copies inside the timed region)
    out["e2e"] = None
    if e2e_steps:
        h_in = torch.from_numpy(np.ascontiguousarray(wl.q)).pin_memory()
        h_out = torch.empty_like(h_in).pin_memory()

        # every step: the state uploaded from pinned host memory, one SSP-RK3 step, the new state
        # downloaded to pinned host memory -- through the pipelined transfers of the C ABI, so the
        # upload of the next state and the download of the last overlap the step in between
        for _ in range(2):
            solver.set_state_async(h_in)
            wl.step(solver, step)
            step += 1
            solver.get_state_async(h_out)
        solver.sync()
        barrier()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            solver.set_state_async(h_in)
            wl.step(solver, step)
            step += 1
            solver.get_state_async(h_out)
        solver.sync()
        e2e_s = dist_max(time.perf_counter() - t0, dev)
        nbytes = int(wl.q.size * 8)
        out["e2e"] = {"value": world * 3 * cells * e2e_steps / e2e_s, "unit": METRIC, "h2d_bytes_per_step": nbytes,
                      "d2h_bytes_per_step": nbytes, "steps": e2e_steps}
    solver.close()

    # ---- roofline of the interface-flux kernel and of the whole step
    counts = load_flops()[wl.flops_key]
    fl = counts["face_flops_per_face"]
    faces_per_launch = wl.faces_per_rhs / 3.0
    avg_launch_s = (face_ms / 1e3) / max(face_launches, 1)
    mixed = wl.precision == "mixed"
    fp_peak = peaks["fp32_tflops"] if mixed else peaks["fp64_tflops"]
    fp_derived = FP32_DERIVED_TFLOPS if mixed else FP64_DERIVED_TFLOPS
    alg_bytes = face_alg_bytes(wl)
    t_alu = fl / (fp_peak * 1e12)
    t_hbm = alg_bytes / (HBM_PEAK_GBS * 1e9)
    common = {"kernel": "k_face<3,visc>", "flops_per_face": fl, "alg_bytes_per_face": alg_bytes,
              "faces_per_launch": faces_per_launch, "avg_launch_ms": avg_launch_s * 1e3,
              "face_share_of_step": face_ms / ms if ms > 0 else None}
    if t_alu >= t_hbm:
        achieved = fl * faces_per_launch / avg_launch_s / 1e12
        roofline = dict({"bound": "alu", "achieved": achieved, "peak": fp_peak, "unit": "TFLOP/s",
                         "frac": achieved / fp_peak}, **common)
        roofline["peak_note"] = ((
            "FP32" if mixed else "FP64") + " FMA throughput measured on this GPU by gbr_alu_peak (of measured)")
        roofline["peak_derived"] = fp_derived
        roofline["frac_of_derived"] = achieved / fp_derived
        if not mixed:
            roofline["peak_nominal"] = FP64_NOMINAL_TFLOPS
            # the executed FP64 operations against the FP64 pipe's rate (one operation per slot)
            pipe_rate = FACE_FP64_OPS_PER_INTERFACE * faces_per_launch / avg_launch_s
            roofline["fp64_ops_per_face_executed"] = FACE_FP64_OPS_PER_INTERFACE
            roofline["pipe_frac"] = pipe_rate / (fp_peak * 1e12 / 2.0)
            roofline["frac_note"] = (
                "achieved counts the method's flops per interface as the oracle performs them; the "
                "kernel executes fewer FP64 operations (mesh-only interface geometry stored once, "
                "restructured algebra), so frac can exceed 1; pipe_frac is the executed FP64 "
                "operations over the FP64 pipe's measured rate")
    else:
        achieved = alg_bytes * faces_per_launch / avg_launch_s / 1e9
        roofline = dict({"bound": "hbm", "achieved": achieved, "peak": HBM_PEAK_GBS, "unit": "GB/s",
                         "frac": achieved / HBM_PEAK_GBS}, **common)
        roofline["peak_note"] = f"HBM copy bandwidth, {HBM_PEAK_KIND} (MEASURED_PEAKS.json)"
        if mixed:
            # the instructions the kernel issues against the GPU's issue rate at the maximum clock
            issue_rate = FACE_F32_WARP_INSTR_PER_INTERFACE * faces_per_launch / avg_launch_s
            roofline["warp_instr_per_face_executed"] = FACE_F32_WARP_INSTR_PER_INTERFACE
            roofline["issue_frac"] = issue_rate / ISSUE_PEAK_WARP_INSTR_PER_S
            roofline["frac_note"] = (
                "the FP32 interface kernel is bound by instruction issue, not HBM (ncu: ~65 % of the "
                "issue slots busy, DRAM at ~35 %); issue_frac is its executed warp instructions over "
                "148 SMs x 4 issues per clock at the maximum SM clock")
    if mixed:
        roofline["traffic"] = FACE_DRAM_BYTES_PER_INTERFACE_F32 * faces_per_launch
        roofline["traffic_note"] = "bytes per launch, scaled from a 128^3 ncu capture by interfaces"
    else:
        roofline["traffic"] = FACE_DRAM_BYTES_PER_INTERFACE * faces_per_launch
        roofline["traffic_note"] = "bytes per launch, scaled from a 96^3 ncu capture by interfaces"
    f_cell = counts["step_flops_per_cell_stage"]
    per_gpu = value / world
    t_flop = f_cell / (fp_peak * 1e12)
    t_byte = BYTES_PER_CELL_STAGE_3D / (HBM_PEAK_GBS * 1e9)
    out["roofline"] = roofline
    out["step_roofline"] = {"flops_per_cell_stage": f_cell, "bytes_per_cell_stage": BYTES_PER_CELL_STAGE_3D,
                            "bound": "alu" if t_flop >= t_byte else "hbm",
                            "achieved_tflops": f_cell * per_gpu / 1e12, "frac": max(t_flop, t_byte) * per_gpu,
                            "fp_peak_tflops": fp_peak, "hbm_peak_gbs": HBM_PEAK_GBS,
                            "frac_note": "flops per cell-stage as the counting oracle performs them; the "
                                         "kernels execute fewer (stored mesh-only terms, restructured "
                                         "algebra), so frac can exceed 1"}
    return out


def sub_record(wl, r, steps):
    """A workload measured beside the headline: its value, step time, end-to-end value and rooflines."""
    return {"workload": wl.name, "config": wl.config, "precision": wl.precision, "value": r["value"],
            "unit": METRIC, "steps": steps, "ms_per_step": r["ms"] / steps, "e2e": r["e2e"],
            "gpu_launches": r["launches"], "roofline": r["roofline"], "step_roofline": r["step_roofline"],
            "clocks": r["clocks"]}


def run_gpu(args, wl):
    import torch

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    peaks = measure_peaks()
    # the end-to-end loop runs as many steps as the device-resident one (its pipeline fill and drain,
    # one upload and one download that no step hides, are then spread as over a run)
    e2e_steps = 0 if args.no_e2e else max(1, args.steps)
    extras = world == 1 and not args.no_extras and wl.kind == "tgv" and wl.precision == "fp64" \
        and wl.scheme == "meg6" and args.edge == N_CELLS_EDGE
    r = measure(wl, dev, args.steps, args.warmup, e2e_steps, peaks, world, local, keep_state=extras)
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": r["value"], "unit": METRIC, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r["ms"] / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64" if wl.precision == "mixed" else "f64", "data": "synthetic",
        "config": config_of(wl, world),
        "workspace_gb": r["workspace_bytes"] / 1e9,
        "e2e": r["e2e"], "gpu_launches": r["launches"], "roofline": r["roofline"],
        "step_roofline": r["step_roofline"], "clocks": r["clocks"], "alu_peaks": peaks,
    }
    if extras:
        # the same 128^3 Taylor-Green vortex on the mixed-precision path, and its state after the same
        # number of steps against the FP64 path's (the tests bound both against the FP64 oracle)
        wm = Workload("tgv", args.edge, "mixed", "meg6")
        rm = measure(wm, dev, args.steps, args.warmup, e2e_steps, peaks, world, local, keep_state=True)
        rec = sub_record(wm, rm, args.steps)
        a, b = rm.pop("state"), r.pop("state")
        nv = b.shape[0]
        scale = np.abs(b).reshape(nv, -1).max(axis=1)
        scale[1:nv - 1] = scale[1:nv - 1].max()
        rec["linf_vs_fp64_path"] = float((np.abs(a - b).reshape(nv, -1).max(axis=1) / scale).max())
        rec["linf_note"] = (f"state after {args.warmup + args.steps} CFL {CFL} steps against the FP64 path's, "
                            "max |diff| / max |Q| per component")
        rec["speedup_vs_fp64"] = rm["value"] / r["value"]
        line["mixed"] = rec
        # the 13.9 M-cell jet (FP64), the paper's largest grid shape, with its own rooflines
        wj = Workload("jet")
        js = min(args.steps, 10)
        rj = measure(wj, dev, js, 3, min(e2e_steps, js), peaks, world, local)
        line["jet"] = sub_record(wj, rj, js)
        # a bounded sample of the serving stream: per-job FP64 against the continuous-batching server
        line["serving"] = serving_sample(args, local)
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl)
    print(json.dumps(line), flush=True)


def serve_stream(specs, load, pool_gb, slots, chunk, local):
    """Serve one stream three ways: (1) the plain FP64 per-job form (one job at a time through
    gbr_rk_step), (2) the continuous-batching server with each job in its own precision and (3) the
    server with every job in mixed precision.  Arrivals at `load` x the measured FP64 per-job
    capacity (0: a burst, every job at t = 0).  Returns the three jobs lists and their statistics."""
    import torch

    from paper_2303_10785_b300 import inputs as I
    from paper_2303_10785_b300 import serving

    def jobs_at(rate, precision=None):
        out = []
        for sp in specs:
            case, nodes, q, cfl = I.serving_job_inputs(sp, precision)
            out.append(serving.Job(sp["id"], case, nodes, q, sp["steps"], cfl, sp["arrival"] / rate))
        return out

    # FP64 per-job capacity on a sample of the stream's jobs (a few steps each, after a warm-up step)
    sample = [sp for sp in specs[:: max(1, len(specs) // 8)]]
    work = secs = 0.0
    stream = torch.cuda.current_stream()
    for sp in sample:
        case, nodes, q, cfl = I.serving_job_inputs(sp, "fp64")
        job = serving.Job(sp["id"], case, nodes, q, 4, cfl)
        s = job.make_solver(stream)
        s.rk_step(cfl)
        s.sync()
        t0 = time.perf_counter()
        for _ in range(job.steps):
            s.rk_step(cfl)
        s.sync()
        secs += time.perf_counter() - t0
        work += job.work
        s.close()
    capacity = work / secs
    mean_work = float(np.mean([I.serving_job_work(sp) for sp in specs]))
    rate = load * capacity / mean_work if load > 0 else float("inf")

    base = jobs_at(rate, "fp64")
    serving.run_serial(base)
    st_base = serving.latency_stats(base)
    pool = int(pool_gb * 1e9)
    srv = serving.Server(pool, max_active=slots, chunk_steps=chunk)
    mix = jobs_at(rate)
    with ClockSampler(local) as clocks:
        srv.run(mix)
    st_mix = serving.latency_stats(mix)
    info = srv.batch.info()
    tuning = srv.batch.tuning()
    peak = {"active": srv.peak_active, "pool_bytes": srv.peak_pool}
    srv.close()
    srv = serving.Server(pool, max_active=slots, chunk_steps=chunk)
    allmix = jobs_at(rate, "mixed")
    srv.run(allmix)
    st_allmix = serving.latency_stats(allmix)
    launches_allmix = srv.batch.info()["launches"]
    srv.close()
    errors = [j.error for j in mix + base + allmix if j.error]
    return {"base": base, "mix": mix, "allmix": allmix, "st_base": st_base, "st_mix": st_mix,
            "st_allmix": st_allmix, "capacity": capacity, "rate": rate, "tuning": tuning, "peak": peak,
            "errors": errors, "launches": info["launches"] + launches_allmix, "clocks": clocks.summary()}


def serving_summary(r, st_base, st_mix, st_allmix):
    return {"batched_mixed": st_mix, "batched_all_mixed": st_allmix, "per_job_fp64": st_base,
            "fp64_capacity_per_job": r["capacity"],
            "all_mixed_throughput_ratio": st_allmix["cell_rk_stage_updates_per_s"]
            / st_base["cell_rk_stage_updates_per_s"],
            "arrival_rate_jobs_per_s": r["rate"] if r["rate"] != float("inf") else "burst",
            "throughput_ratio": st_mix["cell_rk_stage_updates_per_s"] / st_base["cell_rk_stage_updates_per_s"],
            "peak": r["peak"], "tuning": r["tuning"], "errors": r["errors"]}


def serving_sample(args, local):
    """The default line's serving record: a bounded sample of the serving stream (32 jobs, 2D edges
    32-256, 3D edges 32-64, 50-150 steps, half of them mixed precision) arriving at once, served per
    job in FP64 and by the continuous-batching server; the full stream is --workload serving."""
    from paper_2303_10785_b300 import inputs as I

    jobs = 32
    specs = I.serving_stream(jobs, seed=args.seed, rate=1.0, edge2d=(32, 256), edge3d=(32, 64), steps=(50, 150))
    r = serve_stream(specs, 0.0, 16.0, 32, 8, local)
    out = serving_summary(r, r["st_base"], r["st_mix"], r["st_allmix"])
    out["stream"] = (f"{jobs} jobs, burst, 2D edge 32-256 (vortex, Sod slab), 3D edge 32-64 (Taylor-Green), "
                     "50-150 steps, FP64 or mixed per job (seed %d)" % args.seed)
    out["gpu_launches"] = r["launches"]
    out["clocks"] = r["clocks"]
    return out


def run_serving(args):
    """The serving stream: jobs of mixed kinds, sizes and precisions with Poisson arrivals at an
    offered load of `--load` x the measured FP64 per-job capacity, served (1) by the plain FP64
    per-job form, (2) by the continuous-batching server with each job in its own precision (the
    line's value) and (3) by the server with every job in mixed precision; aggregate
    cell-RK-stage updates/s and time-to-N-steps p50/p99 of each."""
    import torch

    from paper_2303_10785_b300 import inputs as I

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    # each rank serves its own stream of --jobs jobs (independent jobs: weak scaling)
    specs = I.serving_stream(args.jobs, seed=args.seed + rank, rate=1.0)
    r = serve_stream(specs, args.load, args.pool_gb, args.slots, args.chunk, local)
    st_base, st_mix, st_allmix, errors = r["st_base"], r["st_mix"], r["st_allmix"], r["errors"]

    def record(jobs, st):
        done = [j for j in jobs if j.finished is not None and j.error is None]
        return {"lat": [j.finished - j.arrival for j in done], "work": float(sum(j.work for j in done)),
                "makespan": st["makespan_s"]}

    recs = gather_objects({"mix": record(r["mix"], st_mix), "base": record(r["base"], st_base),
                           "allmix": record(r["allmix"], st_allmix), "errors": errors, "launches": r["launches"]})
    if world > 1:
        st_mix = merge_serving([x["mix"] for x in recs])
        st_base = merge_serving([x["base"] for x in recs])
        st_allmix = merge_serving([x["allmix"] for x in recs])
        errors = [e for x in recs for e in x["errors"]]
    if rank != 0:
        return
    summ = serving_summary(dict(r, errors=errors), st_base, st_mix, st_allmix)
    line = {
        "metric": METRIC, "value": st_mix["cell_rk_stage_updates_per_s"], "unit": METRIC, "n_gpus": world,
        "steps": None, "warmup": None, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64 and f32+f64 per job", "data": "synthetic",
        "config": {"workload": f"serving_stream_{args.jobs}_jobs_per_gpu", "seed": args.seed, "offered_load": args.load,
                   "pool_gb": args.pool_gb, "slots": args.slots, "chunk_steps": args.chunk,
                   "l2": "working sets of the large jobs >> 126 MB L2, no flush"},
        "serving": summ, "gpu_launches": sum(x["launches"] for x in recs), "clocks": r["clocks"],
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None, help="timed steps (default 60 for tgv, 20 for jet)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gbr", choices=["gbr", "reference"])
    ap.add_argument("--workload", default="tgv", choices=["tgv", "jet", "serving"])
    ap.add_argument("--jobs", type=int, default=64, help="serving: jobs in the stream")
    ap.add_argument("--seed", type=int, default=0, help="serving: stream seed")
    ap.add_argument("--load", type=float, default=1.2,
                    help="serving: offered load / FP64 per-job capacity (0: every job arrives at once)")
    ap.add_argument("--pool-gb", type=float, default=64.0, help="serving: device pool for job workspaces")
    ap.add_argument("--slots", type=int, default=64, help="serving: batch slots")
    ap.add_argument("--chunk", type=int, default=8, help="serving: steps between looks at the queue")
    ap.add_argument("--scheme", default="meg6", choices=["meg6", "mig4"],
                    help="gradients: explicit E6 (MEG6) or implicit IG4 line solves (MIG4)")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"],
                    help="mixed: FP32 reconstruction and fluxes, FP64 state, metrics, GCL and RK accumulation")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="default run only: skip the mixed-precision, jet and serving records beside the headline")
    ap.add_argument("--edge", type=int, default=N_CELLS_EDGE, help="tgv cells per edge (profiling runs use smaller grids)")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = 60 if args.workload == "tgv" else 20
    if args.warmup < 3:
        args.warmup = 3
    if args.workload == "serving":
        if args.impl != "reference":
            run_serving(args)
        elif dist_env()[1] == 0:
            print(json.dumps({"impl": "reference", "unavailable": "the serving stream has no CPU reference arm: "
                              "the oracle evaluates one grid at a time"}), flush=True)
        return
    wl = Workload(args.workload, args.edge, args.precision, args.scheme)
    if args.impl == "reference":
        run_reference(args, wl)
    else:
        run_gpu(args, wl)


if __name__ == "__main__":
    main()
