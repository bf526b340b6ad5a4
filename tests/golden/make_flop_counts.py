"""Writes flop_counts.json: algorithmic FP64 operation counts of the method per
cell-stage and per interface, from the oracle's counting build (add/sub, mul,
div and sqrt count 1 each; an fma is a mul plus an add).  Calls only oracle/.

Interface counts are taken on the benchmark workloads' types: the viscous
Taylor-Green vortex on the 0.1 h perturbed periodic mesh (t = 0 state, 48^3),
the jet-like case on the full 170 x 170 cross-section of its stretched grid
(first 12 x cells, quiescent start, inflow and sponge set) and the 2D vortex at
64^2.  The oracle evaluates gradients on its whole padded box, so the gradient
work per cell is taken from the line operators instead (E6 and the second
derivative per point, as the difference of two line lengths) times the fields
and directions one cell needs.  The stage combination and the time step are
counted on the oracle's SSP-RK3 step and time-step functions.  The per
cell-stage total is
  interfaces/cell x per interface + gradients + primitives + residual
  + stage combination (+ time step / 3 when the step is CFL-controlled)."""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from paper_2303_10785_b300 import inputs as I  # noqa: E402


def per_point(kind):
    """Operations per point of a periodic line operator (difference of two lengths)."""
    a = O.flop_counts(lambda: O.op1d(kind, np.sin(0.1 * np.arange(200)), counting=True))["all"]["flops"]
    b = O.flop_counts(lambda: O.op1d(kind, np.sin(0.1 * np.arange(100)), counting=True))["all"]["flops"]
    return (a - b) / 100.0


def count(case, nodes, q, inflow=None, sponge=None, cfl_controlled=True):
    orc = O.Oracle(case, nodes, counting=True)
    if inflow is not None:
        orc.set_inflow(inflow)
    if sponge is not None:
        orc.set_sponge(*sponge)
    c = O.flop_counts(lambda: orc.rhs(q))
    nd = case["ndim"]
    n = case["n"][:nd]
    cells = 1
    for v in n:
        cells *= v
    faces = 0
    for d in range(nd):
        f = 1
        for e in range(nd):
            f *= n[e] + (1 if e == d else 0)
        faces += f
    e6 = per_point("e6")
    second = per_point("second") - e6
    viscous = case.get("reynolds", 0.0) > 0.0
    nv = nd + 2
    grad = (nv + (1 if viscous else 0)) * nd * e6 + nv * nd * second
    step = O.flop_counts(lambda: orc.rk3(q, 1e-4))
    stage = (step["misc"]["flops"]) / (3.0 * cells)
    dt = O.flop_counts(lambda: orc.dt(q, 0.2))["all"]["flops"] / cells
    face = c["face"]["flops"] / faces
    total = (faces / cells) * face + grad + c["prim"]["flops"] / cells + c["res"]["flops"] / cells + stage
    if cfl_controlled:
        total += dt / 3.0
    return {
        "cells": cells,
        "faces": faces,
        "face_flops_per_face": face,
        "face_ops_per_face": {k: c["face"][k] / faces for k in ("add", "mul", "div", "sqrt")},
        "prim_flops_per_cell": c["prim"]["flops"] / cells,
        "res_flops_per_cell": c["res"]["flops"] / cells,
        "all_flops_per_cell": c["all"]["flops"] / cells,
        "e6_flops_per_point": e6,
        "second_derivative_flops_per_point": second,
        "grad_flops_per_cell": grad,
        "stage_flops_per_cell": stage,
        "dt_flops_per_cell": dt,
        "cfl_controlled": cfl_controlled,
        "step_flops_per_cell_stage": total,
    }


def main():
    out = {}
    n = 48
    case = I.case_params(3, (n, n, n), reynolds=1600.0)
    nodes = I.nodes_tgv_3d(n, 0.1)
    xc = I.centroids(nodes, (n, n, n), (1, 1, 1))
    out["tgv3d_viscous"] = count(case, nodes, I.prim_to_cons(I.tgv_prim(*xc), 1.4))
    case, nodes, q, inflow, sigma, qamb = I.jet_case(n=(12, 170, 170), Lx=0.5)
    out["jet3d_viscous"] = count(case, nodes, q, inflow, (sigma, qamb), cfl_controlled=False)
    n = 64
    case = I.case_params(2, (n, n))
    nodes = I.nodes_wavy_2d(n)
    xc = I.centroids(nodes, (n, n), (1, 1))
    out["vortex2d_inviscid"] = count(case, nodes, I.prim_to_cons(I.vortex_prim(xc[0], xc[1]), 1.4))
    with open(os.path.join(HERE, "flop_counts.json"), "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
