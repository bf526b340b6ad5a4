"""Oracle pins for the CFL time step (App. B), heat conduction (Sec. 2, Sec. 5.2) and
Sutherland's law (Sec. 2), each against a closed form computed here without the oracle.

* Time step.  On an affine grid x = A xi (A constant, any shear and stretching) the
  unhatted metrics are the rows of A^-1 exactly, so App. B's step is, per cell,
  CFL / max_e(|U_e| + c ||row_e(A^-1)||) with U_e = row_e(A^-1) . (u - x_t), and the
  viscous bound 1 / (nu_eff ||row_e(A^-1)||^2), nu_eff = max(4/3, gamma/Pr) mu(T) / rho
  (reading A20 of the undefined alpha and mu of App. B).  States are random per cell;
  the grid translates with a constant velocity in the moving case, so xi_t enters U.
* Heat conduction.  A fluid at rest with uniform pressure and a temperature wave
  T = T0 + a sin(k y) has no inviscid flux divergence beyond round-off, and its viscous
  energy right-hand side is div(kappa grad T) with kappa = mu gamma / ((gamma - 1) Pr):
  -kappa a k^2 sin(k y) for constant mu; with Sutherland's mu(T) the exact divergence is
  formed symbolically (sympy).  Fourth order on a uniform mesh (Sec. 5.2), second on the
  wavy mesh (the interface metric/state product, Sec. 7 step 3), for several gamma and Pr;
  second order with Sutherland's mu, evaluated at a second-order interface temperature.
* Sutherland's law in its textbook dimensional form mu/mu_ref = (T/T_ref)^(3/2) (T_ref + S)/(T + S)
  with air's S = 110.4 K, and its two asymptotes (mu ~ T^(3/2) for T << S, mu ~ T^(1/2) for T >> S).

Each pin was checked once against a plausible mistake planted in the oracle (CPU only,
then reverted); every planted mistake failed the test named beside it:
  hat metric instead of the unhatted one in the time step (no factor J)   -> test_dt_affine_*
  grid velocity dropped from U in the time step                          -> test_dt_translating_grid
  nu_eff without 1/rho                                                   -> test_dt_affine_viscous
  kappa without gamma                                                    -> test_heat_conduction_*
  heat flux with the wrong sign                                          -> test_heat_conduction_*
  Sutherland with theta^(1/2) in place of theta^(3/2)                    -> test_sutherland_*
"""
import math

import numpy as np
import pytest
import sympy as sp

import oracle as O
from paper_2303_10785_b300 import inputs as I

A3 = np.array([[0.31, 0.05, -0.04], [0.02, 0.27, 0.06], [-0.03, 0.04, 0.35]])
A2 = np.array([[0.31, 0.07], [-0.05, 0.26]])


def affine_nodes(A, n):
    """Periodic nodes x_a = sum_d A[a, d] xi_d (xi_d = node index); the period vectors are n_d A[:, d]."""
    nd = len(n)
    return I.nodes_from_functions(tuple(n), (1,) * nd, 0,
                                  lambda *Ix: tuple(sum(A[a, d] * Ix[d] for d in range(nd)) for a in range(nd)))


def random_prim(n, seed, gamma=1.4):
    """rho in [0.5, 1.5], |u_a| <= 0.8, p in [0.6, 1.4] per cell (SplitMix64)."""
    nd = len(n)
    shape = tuple(reversed(n))
    idx = np.arange(int(np.prod(shape)), dtype=np.uint64).reshape(shape)
    rho = 1.0 + 0.5 * I.hash_uniform(seed, 0, idx)
    u = [0.8 * I.hash_uniform(seed, 1 + a, idx) for a in range(nd)]
    p = 1.0 + 0.4 * I.hash_uniform(seed, 9, idx)
    return np.stack([rho] + u + [p])


def sutherland_textbook(T, mu_ref, T_ref, S):
    return mu_ref * (T / T_ref) ** 1.5 * (T_ref + S) / (T + S)


def dt_closed_form(A, P, cfl, gamma, grid_vel=None, mu=None, prandtl=0.71):
    """App. B on an affine grid: unhatted metrics are the rows of A^-1."""
    nd = A.shape[0]
    Ainv = np.linalg.inv(A)
    rho, u, p = P[0], P[1:1 + nd], P[-1]
    c = np.sqrt(gamma * p / rho)
    rel = u - (0.0 if grid_vel is None else np.asarray(grid_vel).reshape((nd,) + (1,) * nd))
    inv_bound = np.inf
    visc_bound = np.inf
    for e in range(nd):
        U = sum(Ainv[e, a] * rel[a] for a in range(nd))
        g2 = float(np.sum(Ainv[e] ** 2))
        inv_bound = min(inv_bound, float(np.min(1.0 / (np.abs(U) + c * math.sqrt(g2)))))
        if mu is not None:
            nu = max(4.0 / 3.0, gamma / prandtl) * mu(p / rho) / rho
            visc_bound = min(visc_bound, float(np.min(1.0 / (nu * g2))))
    return cfl * min(inv_bound, visc_bound), cfl * inv_bound, cfl * visc_bound


@pytest.mark.parametrize("nd", [2, 3])
def test_dt_affine_inviscid(nd):
    A = A3 if nd == 3 else A2
    n = (8, 7, 6)[:nd]
    orc = O.Oracle(I.case_params(nd, n), affine_nodes(A, n))
    P = random_prim(n, seed=11)
    got = orc.dt(I.prim_to_cons(P, 1.4), 0.37)
    want, _, _ = dt_closed_form(A, P, 0.37, 1.4)
    assert got == pytest.approx(want, rel=1e-13)


@pytest.mark.parametrize("nd,sutherland", [(2, False), (3, False), (3, True)])
def test_dt_affine_viscous(nd, sutherland):
    A = A3 if nd == 3 else A2
    n = (8, 7, 6)[:nd]
    re, gamma, pr = 2.0, 1.4, 0.71
    kw = dict(reynolds=re, prandtl=pr)
    if sutherland:
        kw.update(sutherland_s=0.3768, t_ref=1.2)
        mu = lambda T: sutherland_textbook(T, 1.0 / re, 1.2, 0.3768 * 1.2)
    else:
        mu = lambda T: 1.0 / re + 0.0 * T
    orc = O.Oracle(I.case_params(nd, n, **kw), affine_nodes(A, n))
    P = random_prim(n, seed=12)
    got = orc.dt(I.prim_to_cons(P, gamma), 0.4)
    want, inv_b, visc_b = dt_closed_form(A, P, 0.4, gamma, mu=mu, prandtl=pr)
    assert visc_b < inv_b  # the viscous bound decides here, so the test pins it
    assert got == pytest.approx(want, rel=1e-13)
    # and with a high Reynolds number the convective bound decides again
    orc_hi = O.Oracle(I.case_params(nd, n, reynolds=1e4, prandtl=pr), affine_nodes(A, n))
    want_hi, inv_hi, _ = dt_closed_form(A, P, 0.4, gamma, mu=lambda T: 1e-4 + 0.0 * T, prandtl=pr)
    assert want_hi == inv_hi
    assert orc_hi.dt(I.prim_to_cons(P, gamma), 0.4) == pytest.approx(want_hi, rel=1e-13)


@pytest.mark.parametrize("nd", [2, 3])
def test_dt_translating_grid(nd):
    """Sec. 4 time metrics: xi_t = -(x_t . grad xi), so U_e = row_e(A^-1) . (u - V)."""
    A = A3 if nd == 3 else A2
    n = (8, 7, 6)[:nd]
    V = np.array([0.9, -0.6, 0.5])[:nd]
    nodes = affine_nodes(A, n)
    vel = np.ascontiguousarray(np.broadcast_to(V.reshape((nd,) + (1,) * nd), nodes.shape))
    orc = O.Oracle(I.case_params(nd, n), nodes, vel)
    P = random_prim(n, seed=13)
    got = orc.dt(I.prim_to_cons(P, 1.4), 0.3)
    want, _, _ = dt_closed_form(A, P, 0.3, 1.4, grid_vel=V)
    still, _, _ = dt_closed_form(A, P, 0.3, 1.4)
    assert abs(want - still) > 1e-3 * still  # the grid velocity matters for this state
    assert got == pytest.approx(want, rel=1e-13)


def test_sutherland_textbook_values():
    """Sec. 2: Sutherland's law, dimensional, for air (T_ref = 293 K, S = 110.4 K)."""
    T_ref, S, mu_ref = 293.0, 110.4, 1.0 / 250.0
    orc = O.Oracle(I.case_params(2, (6, 6), reynolds=250.0, sutherland_s=S / T_ref, t_ref=T_ref), None)
    assert orc.viscosity(T_ref) == pytest.approx(mu_ref, rel=1e-15)
    for T in (30.0, 150.0, 250.0, 400.0, 1000.0, 3000.0):
        assert orc.viscosity(T) == pytest.approx(sutherland_textbook(T, mu_ref, T_ref, S), rel=1e-14)
    # asymptotes: mu ~ T^(3/2) far below S, mu ~ T^(1/2) far above it
    lo = math.log(orc.viscosity(2e-3) / orc.viscosity(1e-3)) / math.log(2.0)
    hi = math.log(orc.viscosity(2e7) / orc.viscosity(1e7)) / math.log(2.0)
    assert lo == pytest.approx(1.5, abs=1e-4)
    assert hi == pytest.approx(0.5, abs=1e-4)
    # constant viscosity when S <= 0
    orc_c = O.Oracle(I.case_params(2, (6, 6), reynolds=250.0), None)
    assert orc_c.viscosity(17.0) == mu_ref


def _heat_case(n, wavy, gamma, prandtl, sutherland):
    L, T0, a, re = 10.0, 1.0, 0.1, 100.0
    nodes = I.nodes_wavy_2d(n, L=L) if wavy else I.nodes_uniform((n, n), (L, L))
    kw = dict(gamma=gamma, prandtl=prandtl)
    if sutherland:
        kw.update(sutherland_s=0.3768, t_ref=T0)
    visc = O.Oracle(I.case_params(2, (n, n), reynolds=re, **kw), nodes)
    inv = O.Oracle(I.case_params(2, (n, n), **kw), nodes)
    xc = I.centroids(nodes, (n, n), (1, 1))
    k = 2 * np.pi / L
    T = T0 + a * np.sin(k * xc[1])
    p0 = 1.0
    z = 0.0 * T
    Q = I.prim_to_cons(np.stack([p0 / T, z, z, p0 + z]), gamma)
    dL = visc.rhs(Q) - inv.rhs(Q)
    # exact div(kappa(T) grad T) for T = T0 + a sin(k y), kappa = mu(T) gamma / ((gamma - 1) Pr)
    y = sp.symbols("y")
    Ts = T0 + a * sp.sin(k * y)
    th = Ts / T0
    mu = (1 / re) * (th ** sp.Rational(3, 2) * (1 + 0.3768) / (th + 0.3768) if sutherland else 1)
    kappa = mu * gamma / ((gamma - 1) * prandtl)
    exact = sp.lambdify(y, sp.diff(kappa * sp.diff(Ts, y), y), "numpy")(xc[1])
    scale = float(np.abs(exact).max())
    mom = float(np.abs(dL[1:3]).max())
    return float(np.abs(dL[3] - exact).max()) / scale, mom / scale, float(np.abs(dL[0]).max()) / scale


@pytest.mark.parametrize("gamma,prandtl", [(1.4, 0.71), (1.4, 2.0), (5.0 / 3.0, 0.71)])
def test_heat_conduction_uniform_mesh_fourth_order(gamma, prandtl):
    e32, m32, r32 = _heat_case(32, False, gamma, prandtl, False)
    e64, _, _ = _heat_case(64, False, gamma, prandtl, False)
    assert e64 < 1e-4
    assert math.log2(e32 / e64) > 3.8  # Sec. 5.2: fourth order
    assert m32 < 1e-12 and r32 < 1e-12  # no viscous momentum or mass flux at rest


def test_heat_conduction_wavy_mesh_and_sutherland():
    e64, _, _ = _heat_case(64, True, 1.4, 0.71, False)
    e128, _, _ = _heat_case(128, True, 1.4, 0.71, False)
    assert e128 < 2e-3 and math.log2(e64 / e128) > 1.8
    # temperature-dependent kappa(T) through Sutherland's mu at the interface temperature; that
    # temperature is the mean of the alpha-damping states T_i + T'_i/2 and T_{i+1} - T'_{i+1}/2
    # (beta^D = 0), a second-order value (T_face - T''/8), so the divergence is second order here
    s32, _, _ = _heat_case(32, False, 1.4, 0.71, True)
    s64, _, _ = _heat_case(64, False, 1.4, 0.71, True)
    assert s64 < 1e-4 and math.log2(s32 / s64) > 1.8
