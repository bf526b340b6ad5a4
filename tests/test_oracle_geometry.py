"""Oracle pins: conservative metrics, metric identities, Jacobian and the GCL term (Sec. 4, Sec. 7, App. D)."""
import numpy as np
import pytest

import oracle as O
from paper_2303_10785_b300 import inputs as I


def identity_residual(orc):
    """max over components a of |sum_d delta_d (face hat metric fh[d][a])| (Eq. metric-Idty)."""
    nd = orc.nd
    out = []
    for a in range(nd):
        s = 0.0
        for d in range(nd):
            fh, _, _ = orc.face_metrics(d)
            s = s + np.diff(fh[a], axis=nd - 1 - d)
        out.append(np.abs(s).max())
    return max(out)


def test_uniform_grid_metrics_are_exact():
    h = 0.3
    orc = O.Oracle(I.case_params(3, (12, 10, 8)), I.nodes_uniform((12, 10, 8), (12 * h, 10 * h, 8 * h)))
    mh, det = orc.cell_metrics()
    assert np.allclose(det, h ** 3, rtol=1e-13)
    for e in range(3):
        for a in range(3):
            assert np.allclose(mh[e, a], h * h if e == a else 0.0, atol=1e-14)
    orc2 = O.Oracle(I.case_params(2, (12, 10)), I.nodes_uniform((12, 10), (12 * h, 10 * h)))
    mh2, det2 = orc2.cell_metrics()
    assert np.allclose(det2, h * h, rtol=1e-13)
    assert np.allclose(mh2[0, 0], h, rtol=1e-13) and np.allclose(mh2[1, 1], h, rtol=1e-13)
    assert np.abs(mh2[0, 1]).max() < 1e-14 and np.abs(mh2[1, 0]).max() < 1e-14


def test_affine_grid_metrics_are_cofactors():
    # x = A xi for a constant matrix A: the conservative metrics equal the cofactors of A (exact)
    rng = np.random.default_rng(0)
    A = np.eye(3) + 0.2 * rng.normal(size=(3, 3))
    n = (10, 9, 8)
    L = (1.0, 1.2, 0.9)
    nodes = np.einsum("ab,b...->a...", A, I.nodes_uniform(n, L))
    orc = O.Oracle(I.case_params(3, n), np.ascontiguousarray(nodes))
    mh, det = orc.cell_metrics()
    h = np.array(L) / np.array(n)
    M = A * h[None, :]  # d x_a / d xi_d
    assert np.allclose(det, np.linalg.det(M), rtol=1e-12)
    inv = np.linalg.inv(M)  # d xi_e / d x_a
    for e in range(3):
        for a in range(3):
            assert np.allclose(mh[e, a], inv[e, a] * np.linalg.det(M), rtol=1e-11, atol=1e-14)


@pytest.mark.parametrize("grid", ["sinusoidal", "random"])
def test_metric_identities_hold_to_roundoff_and_fail_without_fp(grid):
    n = (20, 20, 20)
    nodes = I.nodes_sinusoidal_3d(20) if grid == "sinusoidal" else I.nodes_random(n, (4.0, 4.0, 4.0), frac=0.2)
    h2 = (4.0 / 20) ** 2
    fp = O.Oracle(I.case_params(3, n), nodes)
    assert identity_residual(fp) < 1e-13 * h2
    nonfp = O.Oracle(I.case_params(3, n, metric_scheme=1), nodes)
    assert identity_residual(nonfp) > 1e-6 * h2


def test_metric_identities_2d_wavy():
    orc = O.Oracle(I.case_params(2, (64, 64)), I.nodes_wavy_2d(64))
    # round-off of D applied to coordinates of size L = 10 is a few 1e-15
    assert identity_residual(orc) < 1e-13


def test_periodic_closure_is_required():
    nodes = I.nodes_uniform((8, 8), (1.0, 1.0))
    nodes[0, 3, -1] += 0.01  # break the constant period vector on one node of the closing face
    with pytest.raises(ValueError):
        O.Oracle(I.case_params(2, (8, 8)), nodes)


def test_time_metrics_of_translation_and_gcl():
    m = I.motion_dynamic_2d(n=32, L=10.0, amp=0.3)
    case = I.case_params(2, (32, 32))
    vel = np.zeros_like(m.velocity(0.2))
    vel[0], vel[1] = 0.7, -0.2
    orc = O.Oracle(case, m.nodes(0.2), vel)
    mh, _ = orc.cell_metrics()
    mt = orc.cell_time_metrics()
    # xi_t = -(x_t xi_x + y_t xi_y) in hat form (Sec. 4)
    for e in range(2):
        assert np.allclose(mt[e], -(0.7 * mh[e, 0] - 0.2 * mh[e, 1]), atol=1e-15)
    # a rigid translation leaves every cell volume unchanged: (1/J)_t = 0 by the metric identity
    assert np.abs(orc.gcl()).max() < 1e-13


@pytest.mark.parametrize("n", [32, 64])
def test_gcl_term_matches_rate_of_change_of_cell_volume(n):
    m = I.motion_dynamic_2d(n=n, L=10.0, amp=0.3)
    case = I.case_params(2, (n, n))
    t0, dl = 0.13, 1e-5
    g = O.Oracle(case, m.nodes(t0), m.velocity(t0)).gcl()
    dp = O.Oracle(case, m.nodes(t0 + dl)).cell_metrics()[1]
    dm = O.Oracle(case, m.nodes(t0 - dl)).cell_metrics()[1]
    ddt = (dp - dm) / (2 * dl)
    assert np.abs(g - ddt).max() < 1e-6 * np.abs(ddt).max()


def test_gcl_3d_deforming_matches_volume_rate():
    m = I.motion_deforming_3d(n=16, L=12.0)
    case = I.case_params(3, (16, 16, 16))
    t0, dl = 0.07, 1e-5
    g = O.Oracle(case, m.nodes(t0), m.velocity(t0)).gcl()
    dp = O.Oracle(case, m.nodes(t0 + dl)).cell_metrics()[1]
    dm = O.Oracle(case, m.nodes(t0 - dl)).cell_metrics()[1]
    ddt = (dp - dm) / (2 * dl)
    assert np.abs(g - ddt).max() < 5e-2 * np.abs(ddt).max()
