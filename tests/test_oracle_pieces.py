"""Oracle pins: eigenvectors (App. A), HLLC (Sec. 5.1.1) and the improved MP limiter (App. E).

HLLC is pinned against the textbook Cartesian HLLC with Davis wave speeds
(tests/_textbook.py), and against Galilean and rotation invariance.
"""
import numpy as np
import pytest

import oracle as O
from _textbook import toro_hllc_x

GAMMA = 1.4


def _B(nd, n, rho, u, p, gamma=GAMMA):
    """App. A coefficient matrix B_xi with a unit normal (J = 1, xi_x = n)."""
    U = float(np.dot(n[:nd], u[:nd]))
    nv = nd + 2
    B = np.zeros((nv, nv))
    for r in range(nv):
        B[r, r] = U
    for a in range(nd):
        B[0, 1 + a] = rho * n[a]
        B[1 + a, nv - 1] = n[a] / rho
        B[nv - 1, 1 + a] = gamma * p * n[a]
    return B, U


@pytest.mark.parametrize("nd", [2, 3])
def test_eigenvectors_invert_and_diagonalise(nd):
    rng = np.random.default_rng(0)
    for trial in range(20):
        nh = rng.normal(size=3)
        if trial == 0:
            nh = np.array([0.0, 0.0, 1.0]) if nd == 3 else np.array([0.0, 1.0, 0.0])
        if nd == 2:
            nh[2] = 0.0
        scale = 10 ** rng.uniform(-3, 1)
        rho, p = rng.uniform(0.2, 3.0), rng.uniform(0.1, 5.0)
        R, L = O.eigen(nd, nh * scale, rho, p)
        nv = nd + 2
        assert np.abs(R @ L - np.eye(nv)).max() < 1e-13
        assert np.abs(L @ R - np.eye(nv)).max() < 1e-13
        n = nh / np.linalg.norm(nh[:nd])
        u = rng.normal(size=3)
        B, U = _B(nd, n, rho, u, p)
        a = np.sqrt(GAMMA * p / rho)
        lam = np.diag([U - a] + [U] * (nv - 2) + [U + a])
        assert np.abs(B @ R - R @ lam).max() < 1e-12 * max(1.0, np.abs(B).max())


def _random_pair(rng, branch):
    """Left/right primitive states whose HLLC solution falls in the requested branch."""
    shift = {"L": 3.0, "starL": 0.3, "starR": -0.3, "R": -3.0}[branch]
    PL = np.array([rng.uniform(0.5, 2), shift + rng.uniform(-0.2, 0.2), rng.normal(), rng.normal(), rng.uniform(0.5, 2)])
    PR = np.array([rng.uniform(0.5, 2), shift + rng.uniform(-0.2, 0.2), rng.normal(), rng.normal(), rng.uniform(0.5, 2)])
    return PL, PR


@pytest.mark.parametrize("branch", ["L", "starL", "starR", "R"])
def test_hllc_identity_metrics_is_textbook_hllc(branch):
    rng = np.random.default_rng(1)
    for _ in range(20):
        PL, PR = _random_pair(rng, branch)
        F = O.hllc(3, PL, PR, [1.0, 0.0, 0.0], 0.0)
        assert np.allclose(F, toro_hllc_x(PL, PR), rtol=1e-13, atol=1e-13)


def test_hllc_equal_states_give_physical_flux():
    rng = np.random.default_rng(2)
    for _ in range(30):
        P = np.array([rng.uniform(0.5, 2), *rng.normal(size=3), rng.uniform(0.5, 2)])
        nh = rng.normal(size=3)
        nt = rng.normal()
        F = O.hllc(3, P, P, nh, nt)
        rho, u, p = P[0], P[1:4], P[4]
        E = p / (GAMMA - 1) + 0.5 * rho * u @ u
        U = nt + nh @ u
        ref = np.array([rho * U, *(rho * u * U + nh * p), (E + p) * U - nt * p])
        assert np.allclose(F, ref, rtol=1e-13, atol=1e-13)


def test_hllc_rotation_and_scaling():
    rng = np.random.default_rng(3)
    for _ in range(20):
        PL, PR = _random_pair(rng, rng.choice(["L", "starL", "starR", "R"]))
        Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        F0 = toro_hllc_x(PL, PR)
        n = Q @ np.array([1.0, 0.0, 0.0])
        PLr = np.concatenate([[PL[0]], Q @ PL[1:4], [PL[4]]])
        PRr = np.concatenate([[PR[0]], Q @ PR[1:4], [PR[4]]])
        s = 10 ** rng.uniform(-2, 1)
        F = O.hllc(3, PLr, PRr, s * n, 0.0)
        ref = s * np.concatenate([[F0[0]], Q @ F0[1:4], [F0[4]]])
        assert np.allclose(F, ref, rtol=1e-12, atol=1e-12 * s)


def test_hllc_moving_face_is_galilean_transform_of_textbook():
    rng = np.random.default_rng(4)
    for _ in range(40):
        PLg, PRg = _random_pair(rng, rng.choice(["L", "starL", "starR", "R"]))  # grid-frame states
        xt = rng.normal(size=3)  # grid velocity
        Fg = toro_hllc_x(PLg, PRg)
        PL = PLg.copy()
        PL[1:4] += xt
        PR = PRg.copy()
        PR[1:4] += xt
        nh = np.array([1.0, 0.0, 0.0])
        F = O.hllc(3, PL, PR, nh, -nh @ xt)
        ref = np.array([Fg[0], *(Fg[1:4] + xt * Fg[0]), Fg[4] + xt @ Fg[1:4] + 0.5 * (xt @ xt) * Fg[0]])
        assert np.allclose(F, ref, rtol=1e-12, atol=1e-12)


def test_hllc_2d_matches_3d_with_zero_w():
    rng = np.random.default_rng(5)
    for _ in range(20):
        PL, PR = _random_pair(rng, rng.choice(["L", "starL", "starR", "R"]))
        PL[3] = PR[3] = 0.0
        nh = np.array([rng.normal(), rng.normal(), 0.0])
        F3 = O.hllc(3, PL, PR, nh, 0.1)
        F2 = O.hllc(2, PL[[0, 1, 2, 4]], PR[[0, 1, 2, 4]], nh[:2], 0.1)
        assert np.allclose(F2, F3[[0, 1, 2, 4]], rtol=1e-13, atol=1e-13)
        assert abs(F3[3]) < 1e-13


def test_mp_limiter_leaves_constant_and_linear_data():
    for c in (-2.0, 0.0, 3.5):
        assert O.mp_limit(c, c, c, c, 0.0, 0.0, 0.0) == c
    for slope in (-1.0, 0.3, 2.0):
        w = np.array([-1.0, 0.0, 1.0]) * slope + 0.7
        wl = w[1] + 0.5 * slope
        assert O.mp_limit(wl, w[0], w[1], w[2], 0.0, 0.0, 0.0) == pytest.approx(wl, abs=1e-15)


def test_mp_limiter_keeps_smooth_extremum():
    # samples of x^2 at -1, 0, 1 with curvature d = 2: the van Leer value 1/6 must survive
    assert O.mp_limit(1.0 / 6.0, 1.0, 0.0, 1.0, 2.0, 2.0, 2.0) == pytest.approx(1.0 / 6.0)


def test_mp_limiter_monotone_data_stays_between_neighbours():
    rng = np.random.default_rng(6)
    for _ in range(5000):
        w = np.sort(rng.normal(size=3)) * rng.choice([-1.0, 1.0])
        wl = rng.uniform(-3, 3)
        out = O.mp_limit(wl, w[0], w[1], w[2], 0.0, 0.0, 0.0)
        lo, hi = min(w[1], w[2]), max(w[1], w[2])
        assert lo - 1e-12 <= out <= hi + 1e-12


def test_mp_limiter_symmetries():
    rng = np.random.default_rng(7)
    for _ in range(2000):
        a = rng.normal(size=7)
        out = O.mp_limit(*a, eps=0.0)
        assert O.mp_limit(*(-a), eps=0.0) == pytest.approx(-out, abs=1e-12)  # reflection
        s = 10 ** rng.uniform(-2, 2)
        assert O.mp_limit(*(s * a), eps=0.0) == pytest.approx(s * out, rel=1e-12, abs=1e-12 * s)  # scaling
        c = rng.normal()
        b = a.copy()
        b[:4] += c
        assert O.mp_limit(*b, eps=0.0) == pytest.approx(out + c, abs=1e-11)  # translation of values
