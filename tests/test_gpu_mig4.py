"""GPU: MIG4 gradients (gbr_params.gradient_scheme = GBR_GRAD_MIG4) against the MIG4 oracle.

The CUDA path solves each grid line's tridiagonal IG4 system with factors computed once per
direction (cyclic by Sherman-Morrison on periodic axes, explicit end rows on open axes); the
oracle builds and solves each line's system on its own.  The MIG4 metrics are built from IG4
too (Sec. 7 step 2): one line solve per geometry line, on periodic axes over the unwrapped line
extended 64 cells beyond each side.  Same tolerances as the MEG6 parity tests: metrics within
1e-13 of their scale, right-hand sides within 1e-12 of the cancellation scale, states within
1e-12 after a step; the mixed path within its own FP32 tolerance."""
import numpy as np
import pytest

import oracle as O
from paper_2303_10785_b300 import gbr
from _util import cancellation_scale
from test_gpu_parity import CASES, case_jet, rel_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    __graft_entry__.build()


def mig4(case, **kw):
    return dict(case, gradient_scheme="mig4", **kw)


def rhs_err(orc, s, q):
    Lg = s.rhs().cpu().numpy()
    Lo = orc.rhs(q)
    return (np.abs(Lg - Lo).reshape(q.shape[0], -1).max(axis=1) / cancellation_scale(orc, q)).max()


@pytest.mark.parametrize("name", ["3d_tgv", "2d_moving", "3d_moving_viscous", "2d_vortex"])
def test_mig4_metrics_match_oracle(name):
    """Cell, interface and time metrics of MIG4 grids (IG4-based operators) against the oracle's."""
    case, nodes, vel, q = CASES[name]()
    orc = O.Oracle(mig4(case), nodes, vel)
    s = gbr.Solver(mig4(case), nodes, vel)
    nd = case["ndim"]
    mh_o, det_o = orc.cell_metrics()
    mh_g = s.field(gbr.GBR_FIELD_CELL_METRICS)
    det_g = s.field(gbr.GBR_FIELD_CELL_DET)
    assert np.abs(det_g - det_o).max() < 1e-13 * np.abs(det_o).max()
    h = np.abs(det_o).max() ** (1.0 / nd)
    mscale = max(np.abs(mh_o).max(), np.abs(nodes).max() * h ** (nd - 1))
    assert np.abs(mh_g - mh_o).max() < 1e-13 * mscale
    for d in range(nd):
        fh_o, fu_o, ft_o = orc.face_metrics(d)
        assert np.abs(s.field(gbr.GBR_FIELD_FACE_HAT, d) - fh_o).max() < 1e-13 * mscale
        if case["reynolds"] > 0:
            assert np.abs(s.field(gbr.GBR_FIELD_FACE_UNHAT, d) - fu_o).max() < 1e-12 * np.abs(fu_o).max()
        if vel is not None:
            assert np.abs(s.field(gbr.GBR_FIELD_FACE_TIME, d) - ft_o).max() < 1e-12 * np.abs(ft_o).max()
    if vel is not None:
        assert np.abs(s.field(gbr.GBR_FIELD_GCL) - orc.gcl()).max() < 1e-11 * np.abs(orc.gcl()).max()
    # and they are not the E6-based metrics
    _, meg6_det = O.Oracle(case, nodes, vel).cell_metrics()
    assert np.abs(meg6_det - det_g).max() > 1e3 * 1e-13 * np.abs(det_o).max()
    s.close()


@pytest.mark.parametrize("name", sorted(CASES))
def test_mig4_rhs_matches_oracle(name):
    case, nodes, vel, q = CASES[name]()
    orc = O.Oracle(mig4(case), nodes, vel)
    s = gbr.Solver(mig4(case), nodes, vel)
    s.set_state(q)
    assert rhs_err(orc, s, q) < 1e-12
    # and the gradients are not the E6 ones
    meg6 = O.Oracle(case, nodes, vel)
    assert np.abs(meg6.rhs(q) - s.rhs().cpu().numpy()).max() > 1e-9
    s.close()


def test_mig4_open_axes_jet_step_matches_oracle():
    case, nodes, vel, q, extra = case_jet()
    orc = O.Oracle(mig4(case), nodes, vel)
    s = gbr.Solver(mig4(case), nodes, vel)
    for obj in (orc, s):
        obj.set_inflow(extra["inflow"])
        obj.set_sponge(extra["sigma"], extra["qamb"])
    s.set_state(q)
    assert rhs_err(orc, s, q) < 1e-12
    qo = orc.rk3(q, 2e-3)
    s.rk_step(-2e-3)
    s.sync()
    assert rel_state(s.get_state(), qo) < 1e-12
    s.close()


def test_mig4_vortex_steps_match_oracle():
    case, nodes, vel, q = CASES["2d_vortex"]()
    orc = O.Oracle(mig4(case), nodes, vel)
    s = gbr.Solver(mig4(case), nodes, vel)
    s.set_state(q)
    qo = q.copy()
    for _ in range(10):
        qo = orc.rk3(qo, orc.dt(qo, 0.4))
        s.rk_step(0.4)
    s.sync()
    assert rel_state(s.get_state(), qo) < 1e-11
    s.close()


@pytest.mark.parametrize("name", ["3d_tgv", "3d_inviscid_ragged", "2d_vortex"])
def test_mig4_mixed_precision_rhs(name):
    # 3d_tgv and 2d_vortex: y/z lines by TMA tiles (rows of 52 and 76 floats, multiples of 16
    # bytes); 3d_inviscid_ragged: rows of 49 floats, the staged plain-copy kernel
    case, nodes, vel, q = CASES[name]()
    orc = O.Oracle(mig4(case), nodes, vel)
    s = gbr.Solver(mig4(case, precision="mixed"), nodes, vel)
    s.set_state(q)
    assert rhs_err(orc, s, q) < 2e-5
    s.close()


def test_mig4_member_of_a_batch_matches_oracle():
    """A MIG4 member stepped in a batch beside a MEG6 member (its own IG4 line solves inside the
    batched step) against the MIG4 oracle after 5 steps of the 64^2 vortex."""
    case, nodes, vel, q = CASES["2d_vortex"]()
    orc = O.Oracle(mig4(case), nodes, vel)
    s = gbr.Solver(mig4(case), nodes, vel)
    other = gbr.Solver(case, nodes, vel)
    s.set_state(q)
    other.set_state(q)
    b = gbr.Batch(2)
    b.add(s, 0.4)
    b.add(other, 0.4)
    b.step(5)
    b.sync()
    qo = q.copy()
    for _ in range(5):
        qo = orc.rk3(qo, orc.dt(qo, 0.4))
    assert rel_state(s.get_state(), qo) < 1e-10
    b.close()
    s.close()
    other.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_mig4_long_lines_take_the_per_line_kernel(precision):
    # x-lines of 800 cells do not fit the staged kernel's shared memory in FP64 (32 lines x 813
    # doubles > 200 KB) and run one thread per line in global memory; the y-lines are staged.
    # FP32 rows of 800 cells still fit.  Both precisions must match the oracle.
    from paper_2303_10785_b300 import inputs as I

    n = (800, 12)
    case = mig4(I.case_params(2, n), precision=precision)
    nodes = I.nodes_uniform(n, (40.0, 0.6))
    xc = I.centroids(nodes, n, (1, 1))
    kx, ky = 2 * np.pi / 40.0 * 3, 2 * np.pi / 0.6
    wave = np.sin(kx * xc[0]) * np.cos(ky * xc[1])
    P = np.stack([1.0 + 0.1 * wave, 0.5 + 0.05 * wave, 0.1 * np.cos(kx * xc[0]), 1.0 / (1.4 * 0.25) + 0.2 * wave])
    q = I.prim_to_cons(P, 1.4)
    orc = O.Oracle(dict(case, precision="fp64"), nodes)
    s = gbr.Solver(case, nodes)
    s.set_state(q)
    assert rhs_err(orc, s, q) < (1e-12 if precision == "fp64" else 2e-6)
    s.close()


def test_mig4_mixed_open_axes_jet_rhs():
    case, nodes, vel, q, extra = case_jet()
    orc = O.Oracle(mig4(case), nodes, vel)
    s = gbr.Solver(mig4(case, precision="mixed"), nodes, vel)
    for obj in (orc, s):
        obj.set_inflow(extra["inflow"])
        obj.set_sponge(extra["sigma"], extra["qamb"])
    s.set_state(q)
    assert rhs_err(orc, s, q) < 2e-5
    s.close()


def test_bounded_wait_timeout_is_reported_and_context_stays_usable():
    # the line solves' wait for a tile copy is bounded: when it runs out the block flags a sticky
    # error and leaves; this runs that path on purpose (a wait that nothing completes)
    case, nodes, vel, q = CASES["3d_tgv"]()
    s = gbr.Solver(mig4(case), nodes, vel)
    s.set_state(q)
    with pytest.raises(gbr.GbrError):
        s.check_bounded_wait(0)
    s.check_bounded_wait(64)
    with pytest.raises(gbr.GbrError) as err:
        s.sync()
    assert err.value.status == gbr.GBR_ETIMEOUT
    orc = O.Oracle(mig4(case), nodes, vel)
    assert rhs_err(orc, s, q) < 1e-12  # the context still computes
    s.close()
