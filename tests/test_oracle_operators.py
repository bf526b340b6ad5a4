"""Oracle pins: the one-dimensional operators and the worked coefficients printed in Sec. 7.

The paper prints (Sec. 7, freestream proof) the composite stencil of the
averaged MEG6 interface derivative, 2282, -546, 89, -3, -1 over 2880, and the
leading/trailing terms of the triple composite (xi_x)_{i+1/2} - (xi_x)_{i-1/2}
over 23887872000 = 2880^3.  Reproducing them pins the E6 sign reading, the
1/12 van Leer factor, the proof-sign reading, the assembly of the
conservative metrics (Eq. GCL_metrics) and the interface interpolation.
"""
import numpy as np
import pytest

import oracle as O
from paper_2303_10785_b300 import inputs as I

PRINTED_D = {1: 2282, 2: -546, 3: 89, 4: -3, 5: -1}  # Sec. 7, coefficient of (y_{i+m} - y_{i-m}) / 2880


def test_composite_derivative_stencil_matches_printed_coefficients():
    n = 24
    e = np.zeros(n)
    e[0] = 1.0
    # D applied to an impulse at index 0: out[i] is the coefficient c_{-i} of D f_i = sum_m c_m f_{i+m}
    out = O.op1d("D", e)
    for m, c in PRINTED_D.items():
        assert out[(-m) % n] * 2880 == pytest.approx(c, abs=1e-9)  # c_{+m} multiplies f_{i+m}
        assert out[m % n] * 2880 == pytest.approx(-c, abs=1e-9)
    assert abs(out[0]) < 1e-15
    assert max(abs(out[i]) for i in range(6, n - 5)) < 1e-15
    assert 2880 ** 3 == 23887872000


def _poly_exact_degree(kind, shift, order_of_derivative):
    n = 64
    x = np.arange(n) - n / 2.0
    i = n // 2
    xi = x[i] + shift
    exact = []
    for p in range(0, 9):
        out = O.op1d(kind, x ** p)[i]
        if order_of_derivative == 0:
            ex = xi ** p
        elif order_of_derivative == 1:
            ex = p * xi ** (p - 1) if p > 0 else 0.0
        else:
            ex = p * (p - 1) * xi ** (p - 2) if p > 1 else 0.0
        exact.append(abs(out - ex) <= 1e-9 * max(1.0, abs(ex)))
    deg = 0
    while deg + 1 < len(exact) and exact[deg + 1]:
        deg += 1
    return deg


def test_polynomial_exactness_of_operators():
    # E6 (Eq. E6_grads) is sixth order: exact through degree 6
    assert _poly_exact_degree("e6", 0.0, 1) == 6
    # the gradient-based second derivative is exact through degree 5
    assert _poly_exact_degree("second", 0.0, 2) == 5
    # the averaged interface derivative D (Eq. FP-interp2) is fourth order (Sec. 5.1: fourth-order flux derivatives)
    assert _poly_exact_degree("D", 0.0, 1) == 4
    # App. D E4 is fourth order
    assert _poly_exact_degree("e4", 0.0, 1) == 4
    # the averaged van Leer interface value is a flux-difference value, exact only for linear data
    assert _poly_exact_degree("face", 0.5, 0) == 1


def test_first_and_second_derivative_on_sine():
    n = 40
    x = 2 * np.pi * np.arange(n) / n
    h = 2 * np.pi / n
    assert np.abs(O.op1d("e6", np.sin(x)) / h - np.cos(x)).max() < 2e-5
    assert np.abs(O.op1d("second", np.sin(x)) / h ** 2 + np.sin(x)).max() < 1e-3


def _triple_coefficient(yo, zo):
    """Coefficient of y_{yo} z_{zo} in (xi_x)_{i+1/2} - (xi_x)_{i-1/2} at cell 0, by a mixed difference."""
    n = 16
    pad = 10  # the oracle takes centroids on the extended box [-10, n+10) per axis
    orc = O.Oracle(I.case_params(3, (n, n, n)))
    ax = np.arange(-pad, n + pad, dtype=np.float64)
    Z, Y, X = np.meshgrid(ax, ax, ax, indexing="ij")
    base = np.stack([X, Y, Z])  # unit spacing, unwrapped
    eps = 0.5

    def value(dy, dz):
        xc = base.copy()
        if dy:
            xc[1][yo[2] + pad, yo[1] + pad, yo[0] + pad] += eps
        if dz:
            xc[2][zo[2] + pad, zo[1] + pad, zo[0] + pad] += eps
        orc.set_centroids(np.ascontiguousarray(xc))
        fh, _, _ = orc.face_metrics(0)
        # face index f = i + 1 holds interface i+1/2; cell (0,0,0)
        return fh[0][0, 0, 1] - fh[0][0, 0, 0]

    mixed = value(1, 1) - value(1, 0) - value(0, 1) + value(0, 0)
    return mixed / (eps * eps)


@pytest.mark.parametrize(
    "yo,zo,printed",
    [
        ((-5, -5, -5), (-5, -5, 0), -1),  # -y_{i-5,j-5,k-5} z_{i-5,j-5,k}
        ((-5, -5, -4), (-5, -5, 0), -3),  # -3 y_{i-5,j-5,k-4} z_{i-5,j-5,k}
        ((5, 5, 4), (5, 5, 0), 3),  # +3 y_{i+5,j+5,k+4} z_{i+5,j+5,k}
        ((5, 5, 5), (5, 5, 0), 1),  # +y_{i+5,j+5,k+5} z_{i+5,j+5,k}
    ],
)
def test_triple_composite_terms_match_printed_worked_example(yo, zo, printed):
    c = _triple_coefficient(yo, zo)
    assert c * 23887872000 == pytest.approx(printed, abs=5e-3)
