"""Writes flop_counts.json: algorithmic FP64 operation counts of the method per
cell-stage and per interface, from the oracle's counting build (add/sub, mul,
div and sqrt count 1 each; an fma is a mul plus an add).  Calls only oracle/.

The counts are taken on the benchmark workload type (viscous Taylor-Green
vortex on the 0.1 h perturbed periodic mesh, t = 0 state) at 48^3 and on the
2D vortex at 64^2.  Per-cell figures of the gradient phase are not used for the
roofline (the oracle evaluates gradients on its whole padded box)."""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from paper_2303_10785_b300 import inputs as I  # noqa: E402


def count(case, nodes, q):
    orc = O.Oracle(case, nodes, counting=True)
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
    return {
        "cells": cells,
        "faces": faces,
        "face_flops_per_face": c["face"]["flops"] / faces,
        "face_ops_per_face": {k: c["face"][k] / faces for k in ("add", "mul", "div", "sqrt")},
        "prim_flops_per_cell": c["prim"]["flops"] / cells,
        "res_flops_per_cell": c["res"]["flops"] / cells,
        "all_flops_per_cell": c["all"]["flops"] / cells,
    }


def main():
    out = {}
    n = 48
    case = I.case_params(3, (n, n, n), reynolds=1600.0)
    nodes = I.nodes_tgv_3d(n, 0.1)
    xc = I.centroids(nodes, (n, n, n), (1, 1, 1))
    out["tgv3d_viscous"] = count(case, nodes, I.prim_to_cons(I.tgv_prim(*xc), 1.4))
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
