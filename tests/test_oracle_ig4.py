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


def _lambda1(th, scheme):
    """f' / f for f = e^{i theta m}: IG4 (Eq. IG4_grads) or E6 (Eq. E6_grads)."""
    if scheme == "mig4":
        return 1j * (2 * C1 * np.sin(th) + 2 * C2 * np.sin(2 * th)) / (1 + 2 * AL * np.cos(th))
    return 1j * (1.5 * np.sin(th) - 0.3 * np.sin(2 * th) + np.sin(3 * th) / 30.0)


def _interface_and_derivative(th, scheme):
    """Transfer functions of Sec. 7 for the cell mode f_m = e^{i theta (m + 1/2)}: the interface
    value I (Eq. FP-interp / interp-formulae, with f'' = 2 (f_{i+1} - 2 f_i + f_{i-1}) - (f'_{i+1} -
    f'_{i-1}) / 2) at i + 1/2 relative to f_i, and D = I_{i+1/2} - I_{i-1/2} (Eq. FP-interp2)
    relative to f_i."""
    l1 = _lambda1(th, scheme)
    l2 = 4 * (np.cos(th) - 1) - 1j * np.sin(th) * l1
    e = np.exp(1j * th)
    icoef = 0.5 * ((1 + e) + 0.5 * l1 * (1 - e) + l2 * (1 + e) / 12.0)
    return icoef, icoef * (1 - 1 / e)


@pytest.mark.parametrize("scheme", ["mig4", "meg6"])
def test_metrics_are_the_schemes_own_operators(scheme):
    """Sec. 7 step 2: the metric derivative and interpolation use the scheme's own gradients (IG4 for
    MIG4, E6 for MEG6).  Grid x = h i, y = h j + B sin(theta i) sin(theta j) (periodic, theta = 2 pi/n):
    the centroid y_c = h (j + 1/2) + B c^2 s_i s_j with c = cos(theta/2), s_m = sin(theta (m + 1/2)), so
    every metric and interface metric is a Fourier mode whose amplitude is the operator's transfer
    function: y_xi = B c^2 Im(tD e^{i theta (i+1/2)}) s_j, y_eta likewise, xi^_x = y_eta,
    eta^_x = -y_xi, xi^_y = 0, eta^_y = h, 1/J = h y_eta, and the interface values along each
    direction through the interpolation's transfer function.  On the periodic axes the MIG4 lines
    are the unwrapped lines (the x and y of this grid grow by n h per period)."""
    n, h, B = 16, 0.3, 0.05
    th = 2 * np.pi / n

    def f(Ii, Jj):
        return h * Ii, h * Jj + B * np.sin(th * Ii) * np.sin(th * Jj)

    nodes = I.nodes_from_functions((n, n), (1, 1), 0, f)
    orc = O.Oracle(I.case_params(2, (n, n), reynolds=100.0, gradient_scheme=scheme), nodes)
    ti, tD = _interface_and_derivative(th, scheme)
    m = np.arange(n)
    c2 = np.cos(th / 2) ** 2
    s = np.sin(th * (m + 0.5))
    dmode = np.imag(tD * np.exp(1j * th * (m + 0.5)))   # D of s_m at cell m
    imode = np.imag(ti * np.exp(1j * th * (m + 0.5)))   # I of s_m at interface m + 1/2
    J_, I_ = np.meshgrid(m, m, indexing="ij")           # [j][i]
    y_xi = B * c2 * dmode[I_] * s[J_]
    y_eta = h + B * c2 * s[I_] * dmode[J_]
    mh, det = orc.cell_metrics()
    tol = 1e-14
    assert np.abs(mh[0, 0] - y_eta).max() < tol and np.abs(mh[0, 1]).max() < tol
    assert np.abs(mh[1, 0] + y_xi).max() < tol and np.abs(mh[1, 1] - h).max() < tol
    assert np.abs(det - h * y_eta).max() < tol
    # interface hat metrics: faces f = 0..n along xi hold i + 1/2 with i = f - 1 (periodic wrap)
    fh0, _, _ = orc.face_metrics(0)
    fh1, _, _ = orc.face_metrics(1)
    fi = (np.arange(n + 1) - 1) % n
    want0 = h + B * c2 * imode[fi][None, :] * dmode[:, None]   # I_xi(y_eta): [j][f]
    want1 = -B * c2 * dmode[None, :] * imode[fi][:, None]      # I_eta(-y_xi): [f][i]
    assert np.abs(fh0[0] - want0).max() < tol and np.abs(fh0[1]).max() < tol
    assert np.abs(fh1[0] - want1).max() < tol and np.abs(fh1[1] - h).max() < tol
    # the other scheme's transfer function is far away at this resolution
    other = "meg6" if scheme == "mig4" else "mig4"
    _, tD_o = _interface_and_derivative(th, other)
    assert abs(tD_o - tD) * B * c2 > 1e3 * tol
