"""GPU: the workloads at their full sizes, checked against the oracle where it finishes in
seconds to a minute, else through properties that hold at any size.

* 2D dynamic mesh: 256^2 periodic mesh deformed in time as x = xi + 0.1 sin(2 pi t/T)
  sin(2 pi xi/L) sin(2 pi eta/L) (and y likewise), GCL metric terms recomputed every stage, the
  isentropic vortex for 500 SSP-RK3 steps, FP64 and mixed precision against one oracle run
  (FP64: maximum difference after 100 steps, L1 and maximum after 500).
* Jet: the 480 x 170 x 170 stretched jet grid with inflow, sponge and Sutherland viscosity; the
  right-hand side of a perturbed state on the GPU against the oracle's right-hand side on the first
  40 x-cells of the same grid (identical nodes; cells whose stencils do not reach the cut); and 100
  steps from the quiescent state on the FP64 and the mixed path, the mixed state within its
  tolerance of the FP64 one.
* Taylor-Green vortex: 128^3, 200 steps at CFL 0.2 on the 0.1 h perturbed mesh and on the
  unperturbed one: mass, momentum and energy totals conserved to round-off on both (~1e-14), and
  the two kinetic-energy histories agree to the scheme's truncation error (3.5e-10 relative at
  step 200); the mixed path follows the FP64 path within its tolerance.  And the right-hand side
  of the perturbed case 20 steps in, every cell, against the oracle's (MEG6 and MIG4, FP64 and
  mixed).
"""
import numpy as np
import pytest

import oracle as O
from paper_2303_10785_b300 import gbr
from paper_2303_10785_b300 import inputs as I
from _util import cancellation_scale
from test_gpu_parity import GAMMA, component_scale, rel_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    __graft_entry__.build()


def test_dynamic_mesh_256_five_hundred_steps_fp64_and_mixed():
    # FP64: within 1e-10 after 100 steps; later, single cells where the App. E test resolves at
    # round-off differ by up to ~1e-9 (measured 1.2e-9 at step 475) while the L1
    # difference stays at round-off (4.6e-13 at step 500).  Mixed: within 1e-5 throughout.
    n, dt, steps = 256, 0.004, 500
    m = I.motion_dynamic_2d(n=n, L=10.0, amp=0.1)
    case = I.case_params(2, (n, n), moving=1)
    nodes, vel = m.nodes(0.0), m.velocity(0.0)
    xc = I.centroids(nodes, (n, n), (1, 1))
    q = I.prim_to_cons(I.vortex_prim(xc[0], xc[1]), GAMMA)
    solvers = {}
    for prec in ("fp64", "mixed"):
        s = gbr.Solver(dict(case, precision=prec), nodes, vel)
        s.set_motion(m, 0.0)
        s.set_state(q)
        solvers[prec] = s
    orc = O.Oracle(case, nodes, vel)
    qo, t = q.copy(), 0.0
    for i in range(steps):
        ts = (t, t + dt, t + 0.5 * dt)
        qo = orc.rk3(qo, dt, [m.nodes(x) for x in ts], [m.velocity(x) for x in ts])
        t += dt
        for s in solvers.values():
            s.rk_step(-dt)
        if i + 1 == 100:
            e64 = rel_state(solvers["fp64"].get_state(), qo)
            print("dynamic 256^2 100 steps: fp64", e64)
            assert e64 < 1e-10
    q64 = solvers["fp64"].get_state()
    d = np.abs(q64 - qo).reshape(4, -1)
    sc = component_scale(qo)
    l1 = (d.mean(axis=1) / sc).max()
    e64 = (d.max(axis=1) / sc).max()
    e32 = rel_state(solvers["mixed"].get_state(), qo)
    print("dynamic 256^2 500 steps: fp64 max", e64, "L1", l1, "mixed", e32)
    assert l1 < 1e-11 and e64 < 1e-8
    assert e32 < 1e-5
    for s in solvers.values():
        assert abs(s.time()[0] - t) < 1e-12
        s.close()


def _jet_state(n, xc):
    # the quiescent jet state with smooth perturbations everywhere (a non-trivial right-hand side)
    nk, nj, ni = xc[0].shape
    P = np.zeros((5, nk, nj, ni))
    w = np.sin(0.7 * xc[0]) * np.cos(0.9 * xc[1]) * np.sin(1.1 * xc[2] + 0.3)
    P[0] = 1.0 + 0.05 * w
    P[1] = 0.3 * np.exp(-(xc[1] ** 2 + xc[2] ** 2)) + 0.02 * w
    P[2] = 0.02 * np.cos(0.8 * xc[0]) * w
    P[3] = -0.02 * w
    P[4] = 1.0 + 0.03 * w
    return I.prim_to_cons(P, GAMMA)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_full_jet_rhs_matches_oracle_on_the_inflow_block(precision):
    n = (480, 170, 170)
    case, nodes, _, inflow, sigma, qamb = I.jet_case(n)
    xc = I.centroids(nodes, n, (0, 0, 0))
    q = _jet_state(n, xc)
    s = gbr.Solver(dict(case, precision=precision), nodes)
    s.set_inflow(inflow)
    s.set_sponge(sigma, qamb)
    s.set_state(q)
    Lg = s.rhs().cpu().numpy()
    s.close()
    m = 40
    case_m, nodes_m, _, inflow_m, _, _ = I.jet_case((m, n[1], n[2]), Lx=20.0 * m / n[0])
    orc = O.Oracle(case_m, nodes_m)
    orc.set_inflow(inflow_m)
    orc.set_sponge(np.ascontiguousarray(sigma[:, :, :m]), qamb)
    qm = np.ascontiguousarray(q[:, :, :, :m])
    Lo = orc.rhs(qm)
    keep = 24  # cells whose metric and reconstruction stencils stay inside the first 40
    scale = cancellation_scale(orc, qm)
    err = (np.abs(Lg[:, :, :, :keep] - Lo[:, :, :, :keep]).reshape(5, -1).max(axis=1) / scale).max()
    print("jet", precision, err)
    assert err < (1e-12 if precision == "fp64" else 2e-6)


@pytest.mark.parametrize("scheme", ["meg6", "mig4"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_taylor_green_128_rhs_matches_oracle_after_twenty_steps(precision, scheme):
    # the bench's workload itself: 128^3 on the 0.1 h perturbed mesh, every cell of the
    # right-hand side of a state 20 CFL 0.2 steps in (the limiter active) against the oracle's
    n = 128
    case = I.case_params(3, (n, n, n), reynolds=1600.0)
    if scheme == "mig4":
        case = dict(case, gradient_scheme="mig4")
    nodes = I.nodes_tgv_3d(n, 0.1)
    xc = I.centroids(nodes, (n, n, n), (1, 1, 1))
    q = I.prim_to_cons(I.tgv_prim(*xc, mach=0.1), GAMMA)
    s = gbr.Solver(dict(case, precision=precision), nodes)
    s.set_state(q)
    for _ in range(20):
        s.rk_step(0.2)
    qs = s.get_state()
    Lg = s.rhs().cpu().numpy()
    s.close()
    orc = O.Oracle(case, nodes)
    Lo = orc.rhs(qs)
    err = (np.abs(Lg - Lo).reshape(5, -1).max(axis=1) / cancellation_scale(orc, qs)).max()
    print("tgv 128^3", scheme, precision, err)
    assert err < (1e-12 if precision == "fp64" else 2e-6)


def test_full_jet_mixed_follows_fp64_for_a_hundred_steps():
    # the 13.9 M-cell jet from its quiescent state with the inflow and the sponge, 100 steps at
    # the bench's fixed time step on the FP64 and on the mixed path: the jet enters, both stay
    # finite, and the mixed state stays within its tolerance of the FP64 state
    n, steps, dt = (480, 170, 170), 100, 2e-3
    case, nodes, q, inflow, sigma, qamb = I.jet_case(n)
    out = {}
    for precision in ("fp64", "mixed"):
        s = gbr.Solver(dict(case, precision=precision), nodes)
        s.set_inflow(inflow)
        s.set_sponge(sigma, qamb)
        s.set_state(q)
        for _ in range(steps):
            s.rk_step(-dt)
        out[precision] = s.get_state()
        s.close()
    qd, qm = out["fp64"], out["mixed"]
    assert np.isfinite(qd).all() and np.isfinite(qm).all()
    assert np.abs(qd - q).max() > 1e-2  # the jet has entered the box
    err = rel_state(qm, qd)
    print("jet mixed vs fp64 after", steps, "steps", err)
    assert err < 1e-5


def _totals(q, det):
    """Totals of the conserved variables and, per component, the scale they are compared at (the
    momentum components share that of the momentum vector: w of the TGV starts at zero)."""
    ref = np.abs(q * det).reshape(q.shape[0], -1).sum(axis=1)
    ref[1:-1] = ref[1:-1].max()
    return (q * det).reshape(q.shape[0], -1).sum(axis=1), ref


def test_taylor_green_128_two_hundred_steps_perturbed_and_unperturbed():
    n, steps = 128, 200
    case = I.case_params(3, (n, n, n), reynolds=1600.0)
    out = {}
    for name, amp in (("perturbed", 0.1), ("unperturbed", 0.0)):
        nodes = I.nodes_tgv_3d(n, amp)
        xc = I.centroids(nodes, (n, n, n), (1, 1, 1))
        q = I.prim_to_cons(I.tgv_prim(*xc), GAMMA)
        orc = O.Oracle(case, nodes)  # cell volumes J^-1 of the discrete metrics
        _, det = orc.cell_metrics()
        s = gbr.Solver(case, nodes)
        s.set_state(q)
        tot0, ref = _totals(q, det)
        ek = []
        for i in range(steps):
            s.rk_step(0.2)
            if (i + 1) % 50 == 0:
                qs = s.get_state()
                ek.append((s.time()[0], float((0.5 * (qs[1] ** 2 + qs[2] ** 2 + qs[3] ** 2) / qs[0] * det).sum() / det.sum())))
        qn = s.get_state()
        tot, _ = _totals(qn, det)
        drift = np.abs(tot - tot0) / ref
        print(name, "conservation drift", drift, "ek", ek)
        assert drift.max() < 1e-12
        out[name] = (ek, qn)
        s.close()
        if name == "perturbed":
            sm = gbr.Solver(dict(case, precision="mixed"), nodes)
            sm.set_state(q)
            for _ in range(steps):
                sm.rk_step(0.2)
            e32 = rel_state(sm.get_state(), qn)
            print("mixed vs fp64 after 200 steps", e32)
            assert e32 < 1e-5
            sm.close()
    (ek_p, _), (ek_u, _) = out["perturbed"], out["unperturbed"]
    for (tp, ep), (tu, eu) in zip(ek_p, ek_u):
        print("t", tp, tu, "ek", ep, eu, "rel", abs(ep - eu) / eu)
        assert abs(ep - eu) < 1e-8 * eu  # measured 3.5e-10 at step 200
