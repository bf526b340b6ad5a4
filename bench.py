"""Benchmark: cell-RK-stage updates/s of the FP64 MEG6 + HLLC + alpha-damping
right-hand side with SSP-RK3 on one B300, plus the roofline of the dominant
kernel (the interface-flux kernel) and the CPU oracle as the baseline.

Workload: 3D viscous Taylor-Green vortex, Re = 1600, M = 0.1, Pr = 0.71, on a
128^3 periodic [0, 2 pi]^3 mesh with a 0.1 h sinusoidal node perturbation, CFL
0.2 (dt computed on the device every step).  A step is one full SSP-RK3 step
(three right-hand sides, time step, stage combinations); the working set
(~3 GB) is far larger than L2, so no flush is needed between steps.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
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
WORKLOAD = "tgv3d_viscous_128^3_perturbed"
METRIC = "cell-RK-stage updates/s"
# FP64 peak used as the roofline denominator of this ALU-bound path: 148 SMs x
# 2 DFMA/clk/SM x 2 flop x 2.032 GHz = 1.20 TFLOP/s nominal at the maximum SM
# clock (the pool's FP64 figure is 1.25 TFLOP/s; derivation in the design doc).
FP64_PEAK_TFLOPS = 1.25


def load_flops():
    with open(os.path.join(ROOT, "tests", "golden", "flop_counts.json")) as f:
        return json.load(f)


def workload():
    from paper_2303_10785_b300 import inputs as I

    n = N_CELLS_EDGE
    case = I.case_params(3, (n, n, n), reynolds=1600.0, prandtl=0.71)
    nodes = I.nodes_tgv_3d(n, 0.1)
    xc = I.centroids(nodes, (n, n, n), (1, 1, 1))
    q = I.prim_to_cons(I.tgv_prim(*xc, mach=0.1), case["gamma"])
    return case, nodes, q


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


def _oracle_stage(orc, q):
    """One SSP-RK3 stage of the oracle: a right-hand side and the first stage combination."""
    return q + 1e-3 * orc.rhs(q)


def cpu_baseline(samples=1):
    """The oracle as it stands on the host cores: right-hand sides of the full 128^3 workload."""
    import oracle as O

    case, nodes, q = workload()
    orc = O.Oracle(case, nodes)
    t0 = time.perf_counter()
    for _ in range(samples):
        _oracle_stage(orc, q)
    el = time.perf_counter() - t0
    cells = N_CELLS_EDGE ** 3
    return {"value": cells * samples / el, "unit": METRIC, "cores": O.threads(), "kind": "oracle",
            "sample": f"{samples} RK stage(s) (right-hand side + stage combination) of the full 128^3 "
                      f"workload, geometry set-up excluded, {el:.1f} s"}


def run_reference(args):
    """Reference arm: the CPU oracle as it stands, one RK stage of the full workload per step."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle as O

    case, nodes, q = workload()
    orc = O.Oracle(case, nodes)
    for _ in range(args.warmup):
        _oracle_stage(orc, q)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        _oracle_stage(orc, q)
    el = time.perf_counter() - t0
    value = N_CELLS_EDGE ** 3 * args.steps / el
    sample = f"{args.steps} RK stage(s) of the full 128^3 workload on the host cores (one stage per step)"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "cells": N_CELLS_EDGE ** 3, "cfl": CFL, "reynolds": 1600.0},
        "cpu_baseline": {"value": value, "unit": METRIC, "cores": O.threads(), "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_gpu(args):
    import torch

    from paper_2303_10785_b300 import gbr

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    case, nodes, q = workload()
    solver = gbr.Solver(case, nodes, device=dev)
    stream = solver.stream
    cells = N_CELLS_EDGE ** 3

    def barrier():
        if world > 1:
            import torch.distributed as dist

            dist.barrier()

    # ---- device-resident throughput
    solver.set_state(q)
    for _ in range(args.warmup):
        solver.rk_step(CFL)
    solver.sync()
    solver.profile(True)
    barrier()
    torch.cuda.synchronize(dev)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clocks:
        ev0.record(stream)
        for _ in range(args.steps):
            solver.rk_step(CFL)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
    barrier()
    ms = ev0.elapsed_time(ev1)
    face_ms, face_launches, launches = solver.profile(False)
    solver.sync()
    if world > 1:
        import torch.distributed as dist

        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = world * 3 * cells * args.steps / (ms / 1e3)

    # ---- end to end through the C ABI with pinned host buffers (copies inside the timed region)
    e2e = None
    if not args.no_e2e:
        h_in = torch.from_numpy(np.ascontiguousarray(q)).pin_memory()
        h_out = torch.empty_like(h_in).pin_memory()
        import ctypes

        L = solver.L
        for _ in range(2):
            solver._check(L.gbr_set_state(solver.h, ctypes.c_void_p(h_in.data_ptr()), 0))
            solver.rk_step(CFL)
            solver._check(L.gbr_get_state(solver.h, ctypes.c_void_p(h_out.data_ptr()), 0))
        barrier()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        e2e_steps = max(1, min(args.steps, 10))
        for _ in range(e2e_steps):
            solver._check(L.gbr_set_state(solver.h, ctypes.c_void_p(h_in.data_ptr()), 0))
            solver.rk_step(CFL)
            solver._check(L.gbr_get_state(solver.h, ctypes.c_void_p(h_out.data_ptr()), 0))
        solver.sync()
        e2e_s = time.perf_counter() - t0
        if world > 1:
            import torch.distributed as dist

            t = torch.tensor([e2e_s], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_s = float(t.item())
        nbytes = int(q.size * 8)
        e2e = {"value": world * 3 * cells * e2e_steps / e2e_s, "unit": METRIC, "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": nbytes, "steps": e2e_steps}

    # ---- roofline of the interface-flux kernel (FP64 ALU bound)
    fl = load_flops()["tgv3d_viscous"]["face_flops_per_face"]
    faces_per_launch = (N_CELLS_EDGE + 1) * N_CELLS_EDGE * N_CELLS_EDGE
    avg_launch_s = (face_ms / 1e3) / max(face_launches, 1)
    achieved = fl * faces_per_launch / avg_launch_s / 1e12
    roofline = {"kernel": "k_face<3,visc>", "bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None,
                "flops_per_face": fl, "faces_per_launch": faces_per_launch, "avg_launch_ms": avg_launch_s * 1e3,
                "face_share_of_step": face_ms / ms if ms > 0 else None,
                "peak_note": "FP64 derived from the pool's unit counts and clock (nominal 1.25 TFLOP/s)"}
    if rank != 0:
        solver.close()
        return
    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "cells": cells, "cfl": CFL, "reynolds": 1600.0, "mach": 0.1,
                   "parallelism": f"replicas{world}", "l2": "working set ~3 GB >> 126 MB L2, no flush"},
        "e2e": e2e, "gpu_launches": launches, "roofline": roofline, "clocks": clocks.summary(),
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(2)
    print(json.dumps(line), flush=True)
    solver.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gbr", choices=["gbr", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--edge", type=int, default=128, help="cells per edge (profiling runs use smaller grids)")
    args = ap.parse_args()
    global N_CELLS_EDGE, WORKLOAD
    if args.edge != N_CELLS_EDGE:
        N_CELLS_EDGE = args.edge
        WORKLOAD = f"tgv3d_viscous_{args.edge}^3_perturbed"
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
