"""Oracle pins of the MIG4 gradients (Eq. IG4_grads, alpha = 5/14).

IG4 is the compact implicit scheme
    alpha f'_{i-1} + f'_i + alpha f'_{i+1} = (2 + alpha)/3 (f_{i+1} - f_{i-1}) + (4 alpha - 1)/12 (f_{i+2} - f_{i-2})
(read with differences).  Pinned by what fixes it independently of the oracle's
solver: its exact response to Fourier modes on a periodic line (the modified wavenumber of
the scheme, derived by inserting e^{i theta j}), a dense solve of the circulant system with
numpy, exactness for quadratics on an open line (every row -- the explicit end rows of reading
the end rows and the IG4 rows -- is exact for them), fourth-order convergence, and, for the whole MIG4
right-hand side, freestream preservation and the fourth-order entropy-wave RHS.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2303_10785_b300 import inputs as I
from _util import cancellation_scale, uniform_flow_case

AL = 5.0 / 14.0
C1 = (2.0 + AL) / 3.0
C2 = (4.0 * AL - 1.0) / 12.0
GAMMA = 1.4


@pytest.mark.parametrize("n,k", [(9, 1), (9, 4), (16, 3), (64, 1), (64, 17)])
def test_fourier_modes_exact(n, k):
    th = 2 * np.pi * k / n
    i = np.arange(n)
    g = O.op1d("ig4", np.sin(th * i))
    # inserting f = e^{i theta j}: f' (1 + 2 alpha cos theta) = 2i (C1 sin theta + C2 sin 2 theta) f
    exact = np.cos(th * i) * 2 * (C1 * np.sin(th) + C2 * np.sin(2 * th)) / (1 + 2 * AL * np.cos(th))
    assert np.abs(g - exact).max() < 2e-14 * np.abs(exact).max()


def test_cyclic_solve_equals_dense_solve():
    rng = np.random.default_rng(4)
    for n in (7, 12, 31):
        f = rng.standard_normal(n)
        A = np.eye(n) + AL * (np.roll(np.eye(n), 1, axis=1) + np.roll(np.eye(n), -1, axis=1))
        rhs = C1 * (np.roll(f, -1) - np.roll(f, 1)) + C2 * (np.roll(f, -2) - np.roll(f, 2))
        assert np.abs(np.linalg.solve(A, rhs) - O.op1d("ig4", f)).max() < 1e-13


def test_open_line_exact_for_quadratics():
    x = np.linspace(-1.0, 2.0, 23)
    h = x[1] - x[0]
    f = 0.5 - 1.5 * x + 2.5 * x * x
    assert np.abs(O.op1d("ig4_open", f) / h - (-1.5 + 5.0 * x)).max() < 1e-12


def test_fourth_order_convergence_periodic():
    errs = []
    for n in (32, 64, 128):
        x = 2 * np.pi * np.arange(n) / n
        h = 2 * np.pi / n
        errs.append(np.abs(O.op1d("ig4", np.sin(x) + 0.3 * np.cos(2 * x)) / h - (np.cos(x) - 0.6 * np.sin(2 * x))).max())
    assert math.log2(errs[0] / errs[1]) > 3.9 and math.log2(errs[1] / errs[2]) > 3.9


def test_mig4_differs_from_meg6_and_keeps_the_freestream():
    n = (16, 16, 16)
    nodes = I.nodes_random(n, (4.0, 4.0, 4.0), frac=0.2)
    case, Q = uniform_flow_case(3, n)
    mig4 = O.Oracle(dict(case, gradient_scheme="mig4"), nodes)
    scale = cancellation_scale(mig4, Q)
    assert (np.abs(mig4.rhs(Q)).reshape(5, -1).max(axis=1) / scale).max() < 1e-13
    xc = I.centroids(nodes, n, (1, 1, 1))
    q = I.prim_to_cons(I.tgv_prim(xc[0] * np.pi / 2, xc[1] * np.pi / 2, xc[2] * np.pi / 2, mach=0.3), GAMMA)
    meg6 = O.Oracle(case, nodes)
    d = np.abs(mig4.rhs(q) - meg6.rhs(q)).max()
    assert d > 1e-6


def _entropy_wave_rhs_error(n, scheme):
    L = 10.0
    nodes = I.nodes_uniform((n, n), (L, L))
    orc = O.Oracle(I.case_params(2, (n, n), mp_eps=1e300, gradient_scheme=scheme), nodes)
    xc = I.centroids(nodes, (n, n), (1, 1))
    k = 2 * np.pi / L
    rho = 1 + 0.2 * np.sin(k * (xc[0] + xc[1]))
    P = np.stack([rho, 1 + 0 * rho, 0.5 + 0 * rho, 1.0 / (GAMMA * 0.25) + 0 * rho])
    Lq = orc.rhs(I.prim_to_cons(P, GAMMA))
    return np.abs(Lq[0] + 1.5 * 0.2 * k * np.cos(k * (xc[0] + xc[1]))).max()


def test_mig4_entropy_wave_fourth_order():
    e = [_entropy_wave_rhs_error(n, "mig4") for n in (32, 64)]
    assert math.log2(e[0] / e[1]) > 3.8  # Sec. 5.1: MIG4 is fourth order as well


def test_mig4_open_axes_jet_like_case_runs_and_is_finite():
    n = (24, 14, 12)
    case = I.case_params(3, n, periodic=(0, 0, 0), bc=((2, 1), (1, 1), (1, 1)), reynolds=1e4,
                         gradient_scheme="mig4")
    nodes = I.nodes_jet(*n, Lx=3.0, h0=0.1, ratio=1.05)
    xc = I.centroids(nodes, n, (0, 0, 0))
    inflow = np.ascontiguousarray(I.jet_inflow_prim(xc[1][:, :, 0], xc[2][:, :, 0], delta=0.1))
    P = np.zeros((5, n[2], n[1], n[0]))
    P[0] = 1.0
    P[4] = 1.0
    orc = O.Oracle(case, nodes)
    orc.set_inflow(inflow)
    L = orc.rhs(I.prim_to_cons(P, GAMMA))
    assert np.all(np.isfinite(L))
    # the implicit gradients spread the inflow's influence along x with the decay |r|^k of the
    # inverse of the IG4 matrix, r = (-1 + sqrt(1 - 4 alpha^2)) / (2 alpha) = -0.42: far from the inflow
    # the quiescent state sees only that tail
    near = np.abs(L[:, :, :, :3]).max()
    assert np.abs(L[:, :, :, 14:]).max() < 0.42 ** 8 * near
