"""Shared helpers for the tests (no numerical method here)."""
import numpy as np

from paper_2303_10785_b300 import inputs as I


def cancellation_scale(orc, q):
    """Per conserved component: max over cells of J * sum_d (|G_{+1/2}| + |G_{-1/2}|)."""
    nd = orc.nd
    _, det = orc.cell_metrics()
    acc = np.zeros(q.shape)
    for d in range(nd):
        g = np.abs(orc.face_flux(q, d))
        ax = g.ndim - 1 - d
        lo = np.take(g, np.arange(0, g.shape[ax] - 1), axis=ax)
        hi = np.take(g, np.arange(1, g.shape[ax]), axis=ax)
        acc += lo + hi
    return np.max((acc / det).reshape(q.shape[0], -1), axis=1)


def rel_err(a, b, scale=None):
    """Per component max|a - b| / scale (default: max|b| per component)."""
    a = np.asarray(a)
    b = np.asarray(b)
    nv = a.shape[0]
    diff = np.abs(a - b).reshape(nv, -1).max(axis=1)
    if scale is None:
        scale = np.abs(b).reshape(nv, -1).max(axis=1)
    return diff / np.maximum(scale, 1e-300)


def uniform_flow_case(nd, n, **kw):
    case = I.case_params(nd, n, **kw)
    P = I.uniform_prim(tuple(reversed(n)), nd, gamma=case["gamma"], mach=0.5)
    return case, I.prim_to_cons(P, case["gamma"])
