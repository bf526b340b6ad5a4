"""Oracle pins of wall-bounded grids: App. C metrics (no ghost nodes) and the slip
wall.

* The App. C derivative is exact for linear data and second order at the walls (App. C calls its
  formulas low order); affine grids get exact metrics.
* The one-sided operators are the same in every line and D = delta o I holds with the same I, so
  the metric identities -- and freestream preservation with zero-gradient ends -- survive.
* Method of images: on a uniform grid, a channel between slip walls is exactly the half of a
  periodic domain of twice the width holding the mirrored state (density and pressure even,
  wall-normal velocity odd), so the right-hand sides must agree.
* A slip wall passes no mass and no energy: the wall-face mass flux vanishes and the totals of
  mass and energy stay constant over steps.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2303_10785_b300 import inputs as I
from _util import cancellation_scale

GAMMA = 1.4
WALLS = 3  # ORC_BC_WALL


def channel_case(n, walls=True, **kw):
    nd = len(n)
    bc = ((WALLS, WALLS) if walls else (1, 1), (1, 1), (1, 1))
    return I.case_params(nd, n, periodic=(0,) + (1,) * (nd - 1), bc=bc, ghost_nodes=0, **kw)


def test_wall_derivative_linear_exact_second_order():
    x = np.arange(24.0)
    assert np.abs(O.op1d("D_walls", 3.0 - 2.0 * x) + 2.0).max() < 1e-13
    errs = []
    for n in (32, 64, 128):
        h = 1.0 / n
        xc = (np.arange(n) + 0.5) * h
        errs.append(np.abs(O.op1d("D_walls", np.sin(3 * xc)) / h - 3 * np.cos(3 * xc)).max())
    assert math.log2(errs[0] / errs[1]) > 1.9 and math.log2(errs[1] / errs[2]) > 1.9


def test_affine_walled_grid_has_exact_metrics():
    n = (16, 12)
    nodes = I.nodes_channel(n, (2.0, 1.5), amp=0.0)
    orc = O.Oracle(channel_case(n), nodes)
    mh, det = orc.cell_metrics()
    h = (2.0 / 16, 1.5 / 12)
    assert np.abs(det - h[0] * h[1]).max() < 1e-15
    assert np.abs(mh[0][0] - h[1]).max() < 1e-15 and np.abs(mh[1][1] - h[0]).max() < 1e-15
    assert np.abs(mh[0][1]).max() < 1e-15 and np.abs(mh[1][0]).max() < 1e-15


@pytest.mark.parametrize("nd", [2, 3])
def test_freestream_preserved_with_app_c_metrics(nd):
    n = (16, 12) if nd == 2 else (16, 12, 10)
    L = (2.0, 1.5) if nd == 2 else (2.0, 1.5, 1.2)
    nodes = I.nodes_channel(n, L, amp=0.04)
    orc = O.Oracle(channel_case(n, walls=False), nodes)
    vel = (0.5, 1.0) if nd == 2 else (0.5, 1.0, 0.2)
    q = I.prim_to_cons(I.uniform_prim(tuple(reversed(n)), nd, vel=vel), GAMMA)
    scale = cancellation_scale(orc, q)
    assert (np.abs(orc.rhs(q)).reshape(nd + 2, -1).max(axis=1) / scale).max() < 1e-13


def _smooth_state(xc, yc, Lx, Ly):
    rho = 1.0 + 0.2 * np.cos(np.pi * xc / Lx) * np.cos(2 * np.pi * yc / Ly)
    u = 0.3 * np.sin(np.pi * xc / Lx) * np.cos(2 * np.pi * yc / Ly)  # odd about the walls
    v = 0.4 + 0.2 * np.cos(np.pi * xc / Lx) * np.sin(2 * np.pi * yc / Ly)
    p = 1.0 / (GAMMA * 0.25) + 0.3 * np.cos(2 * np.pi * xc / Lx)
    return np.stack([rho, u, v, p])


def test_slip_walls_equal_the_mirrored_periodic_domain():
    nx, ny, Lx, Ly = 24, 16, 2.0, 1.5
    wall_nodes = I.nodes_channel((nx, ny), (Lx, Ly), amp=0.0)
    walls = O.Oracle(channel_case((nx, ny)), wall_nodes)
    xc = I.centroids(wall_nodes, (nx, ny), (0, 1), G=0)
    qw = I.prim_to_cons(_smooth_state(xc[0], xc[1], Lx, Ly), GAMMA)
    # the doubled periodic domain [-Lx, Lx) with the even/odd extension
    per_nodes = I.nodes_uniform((2 * nx, ny), (2 * Lx, Ly), origin=(-Lx, 0.0))
    per = O.Oracle(I.case_params(2, (2 * nx, ny)), per_nodes)
    xp = I.centroids(per_nodes, (2 * nx, ny), (1, 1))
    Pp = _smooth_state(np.abs(xp[0]), xp[1], Lx, Ly)
    Pp[1] = np.where(xp[0] < 0, -Pp[1], Pp[1])
    qp = I.prim_to_cons(Pp, GAMMA)
    assert np.abs(qp[:, :, nx:] - qw).max() < 1e-14
    Lw = walls.rhs(qw)
    Lp = per.rhs(qp)[:, :, nx:]
    scale = cancellation_scale(per, qp)
    assert (np.abs(Lw - Lp).reshape(4, -1).max(axis=1) / scale).max() < 1e-13


def test_slip_walls_pass_no_mass_and_no_energy():
    n, Lx, Ly = (20, 16), 2.0, 1.5
    nodes = I.nodes_channel(n, (Lx, Ly), amp=0.04)
    orc = O.Oracle(channel_case(n), nodes)
    xc = I.centroids(nodes, n, (0, 1), G=0)
    P = _smooth_state(xc[0], xc[1], Lx, Ly)
    P[1] += 0.2  # flow into the left wall and away from the right one
    q = I.prim_to_cons(P, GAMMA)
    g = orc.face_flux(q, 0)  # x-direction interfaces: index 0 and n_x are the walls
    fscale = np.abs(g).max()
    assert np.abs(g[0][:, 0]).max() < 1e-14 * fscale and np.abs(g[0][:, -1]).max() < 1e-14 * fscale
    assert np.abs(g[3][:, 0]).max() < 1e-14 * fscale and np.abs(g[3][:, -1]).max() < 1e-14 * fscale
    _, det = orc.cell_metrics()
    tot0 = (q * det).sum(axis=(1, 2))
    qq = q.copy()
    for _ in range(5):
        qq = orc.rk3(qq, orc.dt(qq, 0.4))
    tot = (qq * det).sum(axis=(1, 2))
    ref = np.abs(q * det).sum(axis=(1, 2))
    assert abs(tot[0] - tot0[0]) < 1e-13 * ref[0] and abs(tot[3] - tot0[3]) < 1e-13 * ref[3]
    # on the straight grid the walls' face normals are exact (affine metrics): no force along them
    nodes = I.nodes_channel(n, (Lx, Ly), amp=0.0)
    orc = O.Oracle(channel_case(n), nodes)
    xc = I.centroids(nodes, n, (0, 1), G=0)
    P = _smooth_state(xc[0], xc[1], Lx, Ly)
    P[1] += 0.2
    q = I.prim_to_cons(P, GAMMA)
    _, det = orc.cell_metrics()
    tot0 = (q * det).sum(axis=(1, 2))
    qq = q.copy()
    for _ in range(5):
        qq = orc.rk3(qq, orc.dt(qq, 0.4))
    tot = (qq * det).sum(axis=(1, 2))
    assert abs(tot[2] - tot0[2]) < 1e-13 * np.abs(q * det).sum(axis=(1, 2))[2]


def test_walls_rejected_on_too_short_axes_and_with_motion():
    n = (8, 12)
    nodes = I.nodes_channel(n, (1.0, 1.5))
    with pytest.raises(ValueError):
        O.Oracle(channel_case(n), nodes)
