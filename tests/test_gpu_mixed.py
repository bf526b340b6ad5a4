"""GPU: the mixed-precision path (gbr_params.precision = GBR_PREC_MIXED) against the FP64 oracle.

The mixed path computes primitives, gradients, the characteristic reconstruction,
the limiter and the HLLC and viscous fluxes in FP32 and keeps the state, the
metrics, 1/J, the GCL term, the flux divergence and the RK accumulation in FP64.
Its results therefore differ from the FP64 oracle by FP32 round-off, not by the
scheme.  Two choices keep that round-off independent of the Mach number M: the FP32 primitives
hold p - p_ref (p_ref a pressure of the initial state, so that FP32 does not spend its
digits on the O(1/M^2) mean pressure), and the HLLC star correction S (Q*K - QK) is
formed with (S* - U) factored out (no difference of two O(rho) states multiplied by S ~ c).
Without them the error grows like 1/M.  Tolerances:
* right-hand sides: 2e-6 of the cancellation scale -- about 30 FP32 ulps;
  the largest observed is ~2e-7, the same from M = 0.02 to M = 0.5;
* states after many steps: L-infinity 1e-5 relative to max |Q| per component;
* freestream: right-hand side 1e-6 of the cancellation scale, velocity 1e-6 of
  the freestream speed after steps on a deforming mesh.
"""
import numpy as np
import pytest

import oracle as O
from paper_2303_10785_b300 import gbr
from paper_2303_10785_b300 import inputs as I
from _util import cancellation_scale
from test_gpu_parity import CASES, GAMMA, case_jet, rel_state

pytestmark = pytest.mark.gpu

RHS_TOL = 2e-6
STATE_TOL = 1e-5
FREESTREAM_TOL = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    __graft_entry__.build()


def mixed(case):
    return dict(case, precision="mixed")


def pair(case, nodes, vel, extra=None):
    orc = O.Oracle(case, nodes, vel)
    s = gbr.Solver(mixed(case), nodes, vel)
    if extra:
        for obj in (orc, s):
            obj.set_inflow(extra["inflow"])
            obj.set_sponge(extra["sigma"], extra["qamb"])
    return orc, s


@pytest.mark.parametrize("name", sorted(CASES))
def test_mixed_rhs_matches_fp64_oracle(name):
    case, nodes, vel, q = CASES[name]()
    orc, s = pair(case, nodes, vel)
    s.set_state(q)
    Lg = s.rhs().cpu().numpy()
    Lo = orc.rhs(q)
    scale = cancellation_scale(orc, q)
    err = (np.abs(Lg - Lo).reshape(q.shape[0], -1).max(axis=1) / scale).max()
    assert err < RHS_TOL, err
    # and it is not the FP64 path: FP32 round-off is visible
    assert err > 1e-12
    s.close()


@pytest.mark.parametrize("mach", [0.02, 0.1, 0.3])
def test_mixed_rhs_error_does_not_grow_at_low_mach(mach):
    # viscous Taylor-Green vortex on a randomly perturbed mesh: the FP32 error relative to the
    # cancellation scale stays at a few ulps as M falls (it grew like 1/M with absolute FP32
    # pressures or a star correction formed as a difference of states)
    n = (20, 18, 16)
    case = I.case_params(3, n, reynolds=1600.0)
    nodes = I.nodes_random(n, (2 * np.pi,) * 3, frac=0.15)
    xc = I.centroids(nodes, n, (1, 1, 1))
    q = I.prim_to_cons(I.tgv_prim(*xc, mach=mach), GAMMA)
    orc, s = pair(case, nodes, None)
    s.set_state(q)
    Lg = s.rhs().cpu().numpy()
    scale = cancellation_scale(orc, q)
    err = (np.abs(Lg - orc.rhs(q)).reshape(5, -1).max(axis=1) / scale).max()
    assert err < RHS_TOL, err
    s.close()


@pytest.mark.parametrize("n", [(20, 18, 16), (21, 18, 16), (22, 17, 15)])
def test_mixed_rhs_both_first_derivative_forms(n):
    # the FP32 first derivatives take four x-cells per thread where the padded rows (n_x + 12
    # cells) are 16-byte aligned, and one cell per thread elsewhere: both against the oracle
    case = I.case_params(3, n, reynolds=1600.0)
    nodes = I.nodes_random(n, (2 * np.pi,) * 3, frac=0.15)
    xc = I.centroids(nodes, n, (1, 1, 1))
    q = I.prim_to_cons(I.tgv_prim(*xc, mach=0.1), GAMMA)
    orc, s = pair(case, nodes, None)
    s.set_state(q)
    Lg = s.rhs().cpu().numpy()
    scale = cancellation_scale(orc, q)
    err = (np.abs(Lg - orc.rhs(q)).reshape(5, -1).max(axis=1) / scale).max()
    assert err < RHS_TOL, err
    s.close()


def test_mixed_workspace_is_smaller_than_fp64():
    case, nodes, vel, q = CASES["3d_tgv"]()
    s64 = gbr.Solver(case, nodes, vel)
    s32 = gbr.Solver(mixed(case), nodes, vel)
    assert s32.workspace_bytes < s64.workspace_bytes
    s64.close()
    s32.close()


def test_mixed_vortex_twenty_steps_wavy_mesh():
    # the 64^2 vortex on the wavy periodic mesh, CFL 0.4, 20 steps (the small 2D workload)
    case, nodes, vel, q = CASES["2d_vortex"]()
    orc, s = pair(case, nodes, vel)
    s.set_state(q)
    qo = q.copy()
    for _ in range(20):
        qo = orc.rk3(qo, orc.dt(qo, 0.4))
        s.rk_step(0.4)
    s.sync()
    assert rel_state(s.get_state(), qo) < STATE_TOL
    s.close()


def test_mixed_viscous_taylor_green_steps():
    n = 32
    case = I.case_params(3, (n, n, n), reynolds=1600.0)
    nodes = I.nodes_tgv_3d(n, 0.1)
    xc = I.centroids(nodes, (n, n, n), (1, 1, 1))
    q = I.prim_to_cons(I.tgv_prim(*xc, mach=0.1), GAMMA)
    orc, s = pair(case, nodes, None)
    s.set_state(q)
    qo = q.copy()
    for _ in range(10):
        qo = orc.rk3(qo, orc.dt(qo, 0.2))
        s.rk_step(0.2)
    s.sync()
    assert rel_state(s.get_state(), qo) < STATE_TOL
    s.close()


def test_mixed_moving_mesh_steps():
    m = I.motion_dynamic_2d(n=64, L=10.0, amp=0.1)
    case = I.case_params(2, (64, 64), moving=1)
    nodes, vel = m.nodes(0.0), m.velocity(0.0)
    xc = I.centroids(nodes, (64, 64), (1, 1))
    q = I.prim_to_cons(I.vortex_prim(xc[0], xc[1]), GAMMA)
    orc, s = pair(case, nodes, vel)
    s.set_motion(m, 0.0)
    s.set_state(q)
    t, dt = 0.0, 0.01
    qo = q.copy()
    for _ in range(20):
        ts = (t, t + dt, t + 0.5 * dt)
        qo = orc.rk3(qo, dt, [m.nodes(x) for x in ts], [m.velocity(x) for x in ts])
        s.rk_step(-dt)
        t += dt
    s.sync()
    assert rel_state(s.get_state(), qo) < STATE_TOL
    s.close()


def test_mixed_jet_steps_with_inflow_and_sponge():
    case, nodes, vel, q, extra = case_jet()
    orc, s = pair(case, nodes, vel, extra)
    s.set_state(q)
    qo = q.copy()
    for _ in range(3):
        qo = orc.rk3(qo, 2e-3)
        s.rk_step(-2e-3)
    s.sync()
    assert rel_state(s.get_state(), qo) < STATE_TOL
    s.close()


def test_mixed_freestream_static_and_moving():
    n = (20, 20, 20)
    case = I.case_params(3, n)
    nodes = I.nodes_random(n, (4.0, 4.0, 4.0), frac=0.2)
    q = I.prim_to_cons(I.uniform_prim((20, 20, 20), 3), GAMMA)
    orc, s = pair(case, nodes, None)
    s.set_state(q)
    scale = cancellation_scale(orc, q)
    L = s.rhs().cpu().numpy()
    assert (np.abs(L).reshape(5, -1).max(axis=1) / scale).max() < FREESTREAM_TOL
    s.close()
    # deforming mesh: the uniform flow u = (1, 0, 0) stays uniform
    m = I.motion_deforming_3d(n=16, L=12.0)
    case = mixed(I.case_params(3, (16, 16, 16), moving=1))
    q = I.prim_to_cons(I.uniform_prim((16, 16, 16), 3), GAMMA)
    s = gbr.Solver(case, m.nodes(0.0), m.velocity(0.0))
    s.set_motion(m, 0.0)
    s.set_state(q)
    for _ in range(5):
        s.rk_step(-0.01)
    s.sync()
    qg = s.get_state()
    vel = qg[1:4] / qg[0]
    assert np.abs(vel[1:]).max() < FREESTREAM_TOL and np.abs(vel[0] - 1.0).max() < FREESTREAM_TOL
    s.close()
