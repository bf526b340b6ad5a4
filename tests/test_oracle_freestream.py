"""Oracle pins: freestream preservation on static and deforming meshes (Sec. 8.1.1, Sec. 8.2.1).

The paper reports machine-zero y/z-velocity errors with the conservative
(freestream-preserving) metrics and 1e-3 (sinusoidal) / 1e-1 (random)
errors with the non-conservative metrics of App. D.  The non-FP runs here are
the negative control: the same oracle with only the metric scheme switched.
"""
import numpy as np
import pytest

import oracle as O
from paper_2303_10785_b300 import inputs as I
from _util import cancellation_scale, uniform_flow_case


def _run(orc, q, steps, cfl=0.4):
    for _ in range(steps):
        q = orc.rk3(q, orc.dt(q, cfl))
    return q


@pytest.mark.parametrize("grid", ["sinusoidal", "random"])
def test_static_freestream_3d(grid):
    n = (20, 20, 20)
    nodes = I.nodes_sinusoidal_3d(20) if grid == "sinusoidal" else I.nodes_random(n, (4.0, 4.0, 4.0), frac=0.2)
    case, Q = uniform_flow_case(3, n)
    fp = O.Oracle(case, nodes)
    scale = cancellation_scale(fp, Q)
    L = fp.rhs(Q)
    assert (np.abs(L).reshape(5, -1).max(axis=1) / scale).max() < 1e-13
    q = _run(fp, Q, 4)
    assert np.abs(q[2] / q[0]).max() < 1e-13 and np.abs(q[3] / q[0]).max() < 1e-13

    nonfp = O.Oracle(dict(case, metric_scheme=1), nodes)
    Ln = nonfp.rhs(Q)
    assert (np.abs(Ln).reshape(5, -1).max(axis=1) / scale).max() > 1e-6
    qn = _run(nonfp, Q, 4)
    assert np.sqrt(np.mean((qn[2] / qn[0]) ** 2)) > 1e-5


def test_static_freestream_2d_wavy():
    case, Q = uniform_flow_case(2, (64, 64))
    orc = O.Oracle(case, I.nodes_wavy_2d(64))
    scale = cancellation_scale(orc, Q)
    assert (np.abs(orc.rhs(Q)).reshape(4, -1).max(axis=1) / scale).max() < 1e-13
    q = _run(orc, Q, 5)
    assert np.abs(q[2] / q[0]).max() < 1e-13


def _stage_geometry(m, t, dt):
    ts = (t, t + dt, t + 0.5 * dt)
    return [m.nodes(s) for s in ts], [m.velocity(s) for s in ts]


@pytest.mark.parametrize("scheme,expect_fp", [(0, True), (1, False)])
def test_deforming_freestream_3d(scheme, expect_fp):
    m = I.motion_deforming_3d(n=16, L=12.0)
    case, Q = uniform_flow_case(3, (16, 16, 16), metric_scheme=scheme)
    orc = O.Oracle(case, m.nodes(0.0), m.velocity(0.0))
    t, dt = 0.0, 0.01
    q = Q.copy()
    for _ in range(5):
        sn, sv = _stage_geometry(m, t, dt)
        q = orc.rk3(q, dt, sn, sv)
        t += dt
    err = max(np.abs(q[2] / q[0]).max(), np.abs(q[3] / q[0]).max(), np.abs(q[1] / q[0] - 1.0).max())
    if expect_fp:
        assert err < 1e-13
    else:
        assert err > 1e-6


def test_deforming_freestream_2d():
    m = I.motion_dynamic_2d(n=32, L=10.0, amp=0.3)
    case, Q = uniform_flow_case(2, (32, 32))
    orc = O.Oracle(case, m.nodes(0.0), m.velocity(0.0))
    assert np.abs(orc.gcl()).max() > 1e-3  # the mesh really deforms
    t, dt = 0.0, 0.02
    q = Q.copy()
    for _ in range(5):
        sn, sv = _stage_geometry(m, t, dt)
        q = orc.rk3(q, dt, sn, sv)
        t += dt
    assert np.abs(q[2] / q[0]).max() < 1e-13 and np.abs(q - Q).max() < 1e-12
