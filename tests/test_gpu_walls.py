"""GPU: wall-bounded grids without ghost nodes (App. C metrics) and slip walls
 against the oracle: metrics, right-hand sides (1e-12 of the cancellation scale),
steps (1e-12), the mixed path (2e-5), and a batch member equal to the same grid alone."""
import numpy as np
import pytest

import oracle as O
from paper_2303_10785_b300 import gbr
from paper_2303_10785_b300 import inputs as I
from _util import cancellation_scale
from test_gpu_parity import rel_state

pytestmark = pytest.mark.gpu
W = gbr.GBR_BC_WALL
GAMMA = 1.4


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    __graft_entry__.build()


def smooth(xc, yc, Lx, Ly, u0=0.2):
    rho = 1.0 + 0.2 * np.cos(np.pi * xc / Lx) * np.cos(2 * np.pi * yc / Ly)
    u = u0 + 0.3 * np.sin(np.pi * xc / Lx) * np.cos(2 * np.pi * yc / Ly)
    v = 0.4 + 0.2 * np.cos(np.pi * xc / Lx) * np.sin(2 * np.pi * yc / Ly)
    p = 1.0 / (GAMMA * 0.25) + 0.3 * np.cos(2 * np.pi * xc / Lx)
    return np.stack([rho, u, v, p])


def channel_2d():
    n = (26, 20)
    nodes = I.nodes_channel(n, (2.0, 1.5), amp=0.04)
    case = I.case_params(2, n, periodic=(0, 1), bc=((W, W), (1, 1), (1, 1)), ghost_nodes=0)
    xc = I.centroids(nodes, n, (0, 1), G=0)
    return case, nodes, I.prim_to_cons(smooth(xc[0], xc[1], 2.0, 1.5), GAMMA)


def box_2d_viscous():
    n = (22, 18)

    def f(i, j):
        X, Y = i * 2.0 / n[0], j * 1.5 / n[1]
        s = 0.05 * np.sin(np.pi * X / 2.0) * np.sin(np.pi * Y / 1.5)
        return X + s, Y + s

    nodes = I.nodes_from_functions(n, (0, 0), 0, f)
    case = I.case_params(2, n, periodic=(0, 0), bc=((W, W), (W, 1), (1, 1)), ghost_nodes=0, reynolds=200.0)
    xc = I.centroids(nodes, n, (0, 0), G=0)
    return case, nodes, I.prim_to_cons(smooth(xc[0], xc[1], 2.0, 1.5), GAMMA)


def channel_3d_viscous():
    n = (16, 14, 13)
    nodes = I.nodes_channel(n, (2.0, 1.5, 1.5), amp=0.03)
    case = I.case_params(3, n, periodic=(0, 1, 1), bc=((W, W), (1, 1), (1, 1)), ghost_nodes=0, reynolds=500.0)
    xc = I.centroids(nodes, n, (0, 1, 1), G=0)
    P = smooth(xc[0], xc[1], 2.0, 1.5)
    P = np.stack([P[0], P[1], P[2], 0.1 + 0 * P[0], P[3]])
    return case, nodes, I.prim_to_cons(P, GAMMA)


CASES = {"channel_2d": channel_2d, "box_2d_viscous": box_2d_viscous, "channel_3d_viscous": channel_3d_viscous}


@pytest.mark.parametrize("name", sorted(CASES))
def test_walls_metrics_rhs_and_steps_match_oracle(name):
    case, nodes, q = CASES[name]()
    orc = O.Oracle(case, nodes)
    s = gbr.Solver(case, nodes)
    # interface metrics of every direction, wall interfaces included; 3D hat metrics are differences
    # of products (coordinate x metric derivative), so round-off scales with |x| h^(nd-1); the App. C
    # chain at the walls (one-sided derivatives of one-sided derivatives, coefficient sums up to 4)
    # rounds differently from the oracle's order by up to a few 1e-13 of that scale
    nd = case["ndim"]
    mh_o, det_o = orc.cell_metrics()
    h = np.abs(det_o).max() ** (1.0 / nd)
    mscale = max(np.abs(mh_o).max(), np.abs(nodes).max() * h ** (nd - 1))
    assert np.abs(s.field(gbr.GBR_FIELD_CELL_DET) - det_o).max() < 1e-13 * np.abs(det_o).max()
    for d in range(nd):
        fo, _, _ = orc.face_metrics(d)
        fg = s.field(gbr.GBR_FIELD_FACE_HAT, d)
        assert np.abs(fg - fo).max() < 5e-13 * mscale
    s.set_state(q)
    Lg = s.rhs().cpu().numpy()
    Lo = orc.rhs(q)
    scale = cancellation_scale(orc, q)
    assert (np.abs(Lg - Lo).reshape(q.shape[0], -1).max(axis=1) / scale).max() < 1e-12
    qo = q.copy()
    for _ in range(3):
        qo = orc.rk3(qo, orc.dt(qo, 0.4))
        s.rk_step(0.4)
    s.sync()
    assert rel_state(s.get_state(), qo) < 1e-12
    s.close()


def test_walls_mixed_precision_rhs():
    case, nodes, q = channel_3d_viscous()
    orc = O.Oracle(case, nodes)
    s = gbr.Solver(dict(case, precision="mixed"), nodes)
    s.set_state(q)
    Lg = s.rhs().cpu().numpy()
    scale = cancellation_scale(orc, q)
    assert (np.abs(Lg - orc.rhs(q)).reshape(q.shape[0], -1).max(axis=1) / scale).max() < 2e-5
    s.close()


def test_walled_grid_in_a_batch_equals_alone():
    case, nodes, q = channel_2d()
    alone = gbr.Solver(case, nodes)
    alone.set_state(q)
    for _ in range(4):
        alone.rk_step(0.4)
    alone.sync()
    b = gbr.Batch(2)
    s = gbr.Solver(case, nodes)
    s.set_state(q)
    b.add(s, 0.4)
    b.step(4)
    b.sync()
    assert np.array_equal(s.get_state(), alone.get_state())
    b.close()
    s.close()
    alone.close()
