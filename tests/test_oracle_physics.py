"""Oracle pins against closed forms and textbook solutions.

* Cartesian reduction: on a uniform mesh the curvilinear scheme equals a
  separately written 1D Cartesian MEG6 + textbook HLLC sweep.
* Discrete conservation on periodic static meshes (Sec. 3).
* Design order: 4th order for a linear entropy wave with the limiter switched
  off (Sec. 5.1) and for the alpha-damping viscous term (Sec. 5.2) on uniform
  meshes; at least 2nd order on the wavy mesh, where the interface flux is the
  product of a reconstructed state and a separately interpolated metric (each
  a flux-difference value exact only for linear data, Sec. 7 step 3), which
  costs an O(h^2) cross term.  The Taylor-Green initial energy decay rate
  -(3/4)/Re, and a Sod slab against the exact Riemann solution.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2303_10785_b300 import inputs as I
from _textbook import char_matrices_x, exact_riemann, toro_hllc_x

GAMMA = 1.4


def cartesian_meg6_flux_x(P, gamma=GAMMA):
    """Face fluxes F_{i+1/2} (index i) of a periodic 1D line of 3D primitive states P[5, n]."""
    n = P.shape[1]
    r = lambda a, s: np.roll(a, -s, axis=1)  # r(a, s)[i] = a[i + s]
    d1 = 0.75 * (r(P, 1) - r(P, -1)) - 0.15 * (r(P, 2) - r(P, -2)) + (r(P, 3) - r(P, -3)) / 60.0
    d2 = 2 * (r(P, 1) - 2 * P + r(P, -1)) - 0.5 * (r(d1, 1) - r(d1, -1))
    F = np.zeros((5, n))
    for i in range(n):
        cells = [(i + m) % n for m in (-1, 0, 1, 2)]
        Lm, Rm = char_matrices_x(0.5 * (P[0, i] + P[0, (i + 1) % n]), 0.5 * (P[4, i] + P[4, (i + 1) % n]), gamma)
        W = Lm @ P[:, cells]
        W2 = Lm @ d2[:, cells]
        W1 = Lm @ d1[:, [i, (i + 1) % n]]
        WL = np.empty(5)
        WR = np.empty(5)
        for s in range(5):
            wl = W[s, 1] + 0.5 * W1[s, 0] + W2[s, 1] / 12.0
            WL[s] = O.mp_limit(wl, W[s, 0], W[s, 1], W[s, 2], W2[s, 0], W2[s, 1], W2[s, 2])
            # right state: the left-biased state of the mirrored line (x -> -x flips W')
            rv, rv2 = W[s, ::-1], W2[s, ::-1]
            wr = rv[1] + 0.5 * (-W1[s, 1]) + rv2[1] / 12.0
            WR[s] = O.mp_limit(wr, rv[0], rv[1], rv[2], rv2[0], rv2[1], rv2[2])
        F[:, i] = toro_hllc_x(Rm @ WL, Rm @ WR, gamma)
    return F


@pytest.mark.parametrize("nd", [2, 3])
def test_cartesian_reduction(nd):
    nx, h = 24, 0.25
    n = (nx, 6, 6)[:nd]
    orc = O.Oracle(I.case_params(nd, n), I.nodes_uniform(n, tuple(m * h for m in n)))
    x = (np.arange(nx) + 0.5) * h
    k = 2 * np.pi / (nx * h)
    line = np.stack([1 + 0.2 * np.sin(k * x) + 0.1 * (x > 3.0), 0.3 + 0.1 * np.cos(k * x), 0.2 + 0 * x,
                     (-0.1 if nd == 3 else 0.0) + 0 * x, 1 + 0.1 * np.sin(2 * k * x)])
    F = cartesian_meg6_flux_x(line)
    ref = -(F - np.roll(F, 1, axis=1)) / h
    keep = [0, 1, 2, 3, 4] if nd == 3 else [0, 1, 2, 4]
    P = np.broadcast_to(line[keep].reshape((len(keep),) + (1,) * (nd - 1) + (nx,)), (len(keep),) + tuple(reversed(n)))
    L = orc.rhs(I.prim_to_cons(np.ascontiguousarray(P), GAMMA))
    for c, cc in enumerate(keep):
        got = L[c].reshape(-1, nx)
        assert np.abs(got - ref[cc][None, :]).max() < 1e-12 * np.abs(ref[cc]).max() + 1e-13


def test_discrete_conservation_static_periodic():
    nodes = I.nodes_wavy_2d(32)
    orc = O.Oracle(I.case_params(2, (32, 32)), nodes)
    xc = I.centroids(nodes, (32, 32), (1, 1))
    Q = I.prim_to_cons(I.vortex_prim(xc[0], xc[1]), GAMMA)
    res = orc.residual(Q)
    assert np.all(np.abs(res.sum(axis=(1, 2))) < 1e-13 * np.abs(res).sum(axis=(1, 2)))
    _, det = orc.cell_metrics()
    total0 = (Q * det).sum(axis=(1, 2))
    q = Q.copy()
    for _ in range(5):
        q = orc.rk3(q, orc.dt(q, 0.4))
    total = (q * det).sum(axis=(1, 2))
    assert np.all(np.abs(total - total0) < 1e-13 * np.abs(Q * det).sum(axis=(1, 2)))


def _mesh(n, wavy, L=10.0):
    return I.nodes_wavy_2d(n, L=L) if wavy else I.nodes_uniform((n, n), (L, L))


def _entropy_wave_rhs_error(n, wavy):
    """Max error of dQ/dt for rho = 1 + 0.2 sin(k (x + y)) advected by (1, 0.5), limiter off."""
    L = 10.0
    nodes = _mesh(n, wavy, L)
    orc = O.Oracle(I.case_params(2, (n, n), mp_eps=1e300), nodes)
    xc = I.centroids(nodes, (n, n), (1, 1))
    k = 2 * np.pi / L
    rho = 1 + 0.2 * np.sin(k * (xc[0] + xc[1]))
    P = np.stack([rho, 1 + 0 * rho, 0.5 + 0 * rho, 1.0 / (GAMMA * 0.25) + 0 * rho])
    Lq = orc.rhs(I.prim_to_cons(P, GAMMA))
    exact = -1.5 * 0.2 * k * np.cos(k * (xc[0] + xc[1]))
    return np.abs(Lq[0] - exact).max()


def test_design_order_linear_entropy_wave():
    eu = [_entropy_wave_rhs_error(n, False) for n in (32, 64)]
    assert math.log2(eu[0] / eu[1]) > 3.8  # Sec. 5.1: fourth order
    ew = [_entropy_wave_rhs_error(n, True) for n in (32, 64)]
    assert math.log2(ew[0] / ew[1]) > 1.8


def test_entropy_wave_time_accuracy():
    # one full SSP-RK3 integration on the uniform mesh with dt ~ h^(4/3): error falls at 4th order
    def err(n):
        L = 10.0
        nodes = _mesh(n, False, L)
        orc = O.Oracle(I.case_params(2, (n, n), mp_eps=1e300), nodes)
        xc = I.centroids(nodes, (n, n), (1, 1))

        def prim(t):
            rho = 1 + 0.2 * np.sin(2 * np.pi * (xc[0] + xc[1] - 1.5 * t) / L)
            return np.stack([rho, 1 + 0 * rho, 0.5 + 0 * rho, 1.0 / (GAMMA * 0.25) + 0 * rho])

        q = I.prim_to_cons(prim(0.0), GAMMA)
        tf, h = 0.5, L / n
        steps = int(math.ceil(tf / (0.5 * h ** (4.0 / 3.0) / 3.0)))
        for _ in range(steps):
            q = orc.rk3(q, tf / steps)
        return np.abs(q[0] - prim(tf)[0]).max()

    assert math.log2(err(16) / err(32)) > 3.5


def _viscous_shear_error(n, wavy):
    L = 10.0
    nodes = _mesh(n, wavy, L)
    visc = O.Oracle(I.case_params(2, (n, n), reynolds=100.0), nodes)
    inv = O.Oracle(I.case_params(2, (n, n)), nodes)
    xc = I.centroids(nodes, (n, n), (1, 1))
    k = 2 * np.pi / L
    u = np.sin(k * xc[1])
    Q = I.prim_to_cons(np.stack([1 + 0 * u, u, 0 * u, 1.0 / (GAMMA * 0.25) + 0 * u]), GAMMA)
    dL = visc.rhs(Q) - inv.rhs(Q)
    mu = 1.0 / 100.0
    ex_mom = -mu * k * k * u  # mu d2u/dy2
    ex_en = mu * (k * k * np.cos(k * xc[1]) ** 2 - k * k * u * u)  # d/dy(mu u du/dy)
    return np.abs(dL[1] - ex_mom).max(), np.abs(dL[3] - ex_en).max()


def test_design_order_alpha_damping_viscous_term():
    m32, e32 = _viscous_shear_error(32, False)
    m64, e64 = _viscous_shear_error(64, False)
    assert math.log2(m32 / m64) > 3.8 and math.log2(e32 / e64) > 3.8  # Sec. 5.2: fourth order
    w64, _ = _viscous_shear_error(64, True)
    w128, _ = _viscous_shear_error(128, True)
    assert math.log2(w64 / w128) > 1.8


@pytest.mark.parametrize("perturbed", [False, True])
def test_taylor_green_initial_dissipation_rate(perturbed):
    n, Re = 32, 1600.0
    nodes = I.nodes_tgv_3d(n, amp_frac=0.1) if perturbed else I.nodes_uniform((n, n, n), (2 * np.pi,) * 3)
    orc = O.Oracle(I.case_params(3, (n, n, n), reynolds=Re), nodes)
    xc = I.centroids(nodes, (n, n, n), (1, 1, 1))
    Q = I.prim_to_cons(I.tgv_prim(*xc, mach=0.1), GAMMA)
    L = orc.rhs(Q)
    _, det = orc.cell_metrics()
    u = Q[1:4] / Q[0]
    dke = np.sum(det * (np.sum(u * L[1:4], axis=0) - 0.5 * np.sum(u * u, axis=0) * L[0])) / np.sum(det)
    assert dke == pytest.approx(-0.75 / Re, rel=1e-2)


def _sod_l1(ny):
    nx, Ly = 6, 1.0
    nodes = I.nodes_skewed_2d((nx, ny), (Ly * nx / ny, Ly), skew_deg=20.0, jitter=0.1)
    orc = O.Oracle(I.case_params(2, (nx, ny)), nodes)
    xc = I.centroids(nodes, (nx, ny), (1, 1))
    rho, p = I.sod_slab_prim(xc[1], L=Ly)
    z = np.zeros_like(rho)
    q = I.prim_to_cons(np.stack([rho, z, z, p]), GAMMA)  # slab varies along y
    t, tf = 0.0, 0.1
    while t < tf - 1e-14:
        dt = min(orc.dt(q, 0.4), tf - t)
        q = orc.rk3(q, dt)
        t += dt
    s = np.mod(xc[1], Ly)
    ex1 = exact_riemann(0.125, 0.0, 0.1, 1.0, 0.0, 1.0, GAMMA, ((s - 0.25) / tf).ravel())[0].reshape(s.shape)
    ex2 = exact_riemann(1.0, 0.0, 1.0, 0.125, 0.0, 0.1, GAMMA, ((s - 0.75) / tf).ravel())[0].reshape(s.shape)
    ex = np.where(s < 0.5, ex1, ex2)
    _, det = orc.cell_metrics()
    return np.sum(np.abs(q[0] - ex) * det) / np.sum(np.abs(ex) * det)


def test_sod_slab_on_skewed_mesh_converges_to_exact_solution():
    e1, e2 = _sod_l1(100), _sod_l1(200)
    assert e1 < 0.05
    assert e2 < 0.75 * e1
