"""Three-dimensional parity over 100 SSP-RK3 steps (App. B): the CUDA path against the oracle.

The smooth-case bar is 1e-10 of max |Q| per component after 100 steps (the momentum
components share the momentum-vector scale).  Two 3D cases:

* the viscous Taylor-Green vortex (Re = 1600, M = 0.1, constant mu) on the 0.1 h sinusoidally
  perturbed periodic mesh of the 3D workload, 32^3 cells, CFL 0.2 with the time step computed on
  each side every step (they must agree to round-off as well);
* a viscous flow on the deforming mesh of Sec. 8.2.1 (16^3 cells, every node oscillating by
  1.5 cell widths), the geometry, time metrics and GCL term recomputed at every stage time,
  fixed dt = 0.01 for 100 steps (one full period of the motion).

Each case is also run on the mixed-precision path (FP32 state increments and fluxes, FP64
metrics/GCL/RK accumulation) against the same FP64 oracle states: L-infinity within 1e-5.
"""
import numpy as np
import pytest

import oracle as O
from paper_2303_10785_b300 import gbr
from paper_2303_10785_b300 import inputs as I

pytestmark = pytest.mark.gpu

GAMMA = 1.4


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    __graft_entry__.build()


def component_scale(b):
    nv = b.shape[0]
    sc = np.abs(b).reshape(nv, -1).max(axis=1)
    sc[1:nv - 1] = sc[1:nv - 1].max()
    return sc


def rel_state(a, b):
    nv = a.shape[0]
    return (np.abs(a - b).reshape(nv, -1).max(axis=1) / component_scale(b)).max()


@pytest.fixture(scope="module")
def tgv32():
    n = 32
    case = I.case_params(3, (n, n, n), reynolds=1600.0)
    nodes = I.nodes_tgv_3d(n, 0.1)
    xc = I.centroids(nodes, (n, n, n), (1, 1, 1))
    q0 = I.prim_to_cons(I.tgv_prim(*xc, mach=0.1), GAMMA)
    orc = O.Oracle(case, nodes)
    qo, dts = q0.copy(), []
    for _ in range(100):
        dts.append(orc.dt(qo, 0.2))
        qo = orc.rk3(qo, dts[-1])
    return case, nodes, q0, qo, dts


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_hundred_steps_viscous_tgv_perturbed_mesh(tgv32, precision):
    case, nodes, q0, qo, dts = tgv32
    s = gbr.Solver(dict(case, precision=precision), nodes)
    s.set_state(q0)
    for _ in range(100):
        s.rk_step(0.2)
    s.sync()
    t, dt = s.time()
    err = rel_state(s.get_state(), qo)
    s.close()
    if precision == "fp64":
        assert abs(dt - dts[-1]) <= 1e-12 * dts[-1]
        assert abs(t - sum(dts)) <= 1e-12 * sum(dts)
        assert err < 1e-10, err
    else:
        assert abs(dt - dts[-1]) <= 1e-5 * dts[-1]
        assert err < 1e-5, err


@pytest.fixture(scope="module")
def deforming16():
    n, L, dt = 16, 12.0, 0.01
    m = I.motion_deforming_3d(n=n, L=L)
    case = I.case_params(3, (n, n, n), moving=1, reynolds=500.0)
    nodes, vel = m.nodes(0.0), m.velocity(0.0)
    xc = I.centroids(nodes, (n, n, n), (1, 1, 1))
    k = 2 * np.pi / L
    q0 = I.prim_to_cons(I.tgv_prim(xc[0] * k, xc[1] * k, xc[2] * k, mach=0.3), GAMMA)
    orc = O.Oracle(case, nodes, vel)
    qo, t = q0.copy(), 0.0
    for _ in range(100):
        ts = (t, t + dt, t + 0.5 * dt)
        qo = orc.rk3(qo, dt, [m.nodes(x) for x in ts], [m.velocity(x) for x in ts])
        t += dt
    return case, m, q0, qo, dt, t


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_hundred_steps_deforming_mesh_3d(deforming16, precision):
    case, m, q0, qo, dt, t_end = deforming16
    s = gbr.Solver(dict(case, precision=precision), m.nodes(0.0), m.velocity(0.0))
    s.set_motion(m, 0.0)
    s.set_state(q0)
    for _ in range(100):
        s.rk_step(-dt)
    s.sync()
    t, _ = s.time()
    err = rel_state(s.get_state(), qo)
    s.close()
    assert abs(t - t_end) < 1e-12
    assert err < (1e-10 if precision == "fp64" else 1e-5), err
