"""Pins of the oracle's Sec. 3 stencil: Taylor coefficients and the Laplacian.

The oracle solves the Taylor moment system numerically; these tests check it
against things fixed independently of that code:
  * the textbook closed form of the central second-derivative weights,
        c_m = 2 (-1)^(m+1) (R!)^2 / (m^2 (R-m)! (R+m)!),   in exact rationals;
  * the moment identities that define "order 2R";
  * exactness of the Laplacian on every polynomial of total degree <= 9;
  * the exact truncation error on x^10:  2 h^8 sum_m c_m m^10  (a constant);
  * the 25-point star footprint the paper names (nine points per axis).
"""
from fractions import Fraction
from math import factorial

import numpy as np
import pytest


def textbook_coeffs(R):
    """Closed-form central weights (exact rationals), m = 1..R."""
    return [Fraction(2 * (-1) ** (m + 1) * factorial(R) ** 2,
                     m * m * factorial(R - m) * factorial(R + m)) for m in range(1, R + 1)]


@pytest.mark.parametrize("order", [2, 4, 6, 8, 10, 12])
def test_coeffs_match_textbook_closed_form(orc, order):
    R = order // 2
    c = orc.fd_coeffs(order)
    exact = textbook_coeffs(R)
    for m in range(1, R + 1):
        assert c[m] == pytest.approx(float(exact[m - 1]), rel=1e-12, abs=1e-15)
    assert c[0] == pytest.approx(float(-2 * sum(exact)), rel=1e-12)


def test_order8_centre_weight_is_minus_205_over_72(orc):
    # -2 (8/5 - 1/5 + 8/315 - 1/560) = -205/72, from the exact closed form.
    assert -2 * sum(textbook_coeffs(4)) == Fraction(-205, 72)
    assert orc.fd_coeffs(8)[0] == pytest.approx(-205 / 72, rel=1e-13)


@pytest.mark.parametrize("order", [2, 4, 6, 8])
def test_moment_identities(orc, order):
    R = order // 2
    c = orc.fd_coeffs(order)
    m = np.arange(1, R + 1, dtype=np.float64)
    assert np.sum(c[1:] * m ** 2) == pytest.approx(1.0, abs=1e-13)
    for p in range(2, R + 1):
        assert abs(np.sum(c[1:] * m ** (2 * p))) < 1e-9 * np.sum(np.abs(c[1:]) * m ** (2 * p))
    # the next moment does not vanish: the order is exactly 2R
    assert abs(np.sum(c[1:] * m ** (2 * R + 2))) > 1e-3


def test_bad_orders_rejected(orc):
    for order in (0, 1, 3, 7, 18):
        with pytest.raises(ValueError):
            orc.fd_coeffs(order)


def _monomials(deg):
    return [(a, b, c) for a in range(deg + 1) for b in range(deg + 1 - a) for c in range(deg + 1 - a - b)]


def _poly_and_laplacian(shape, h, origin, coeffs):
    nz, ny, nx = shape
    x = (np.arange(nx) - origin[0]) * h[0]
    y = (np.arange(ny) - origin[1]) * h[1]
    z = (np.arange(nz) - origin[2]) * h[2]
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    u = np.zeros(shape)
    lap = np.zeros(shape)
    for (a, b, c), w in coeffs.items():
        u += w * X ** a * Y ** b * Z ** c
        if a >= 2:
            lap += w * a * (a - 1) * X ** (a - 2) * Y ** b * Z ** c
        if b >= 2:
            lap += w * b * (b - 1) * X ** a * Y ** (b - 2) * Z ** c
        if c >= 2:
            lap += w * c * (c - 1) * X ** a * Y ** b * Z ** (c - 2)
    return u, lap


@pytest.mark.parametrize("deg", [2, 5, 8, 9])
def test_laplacian_exact_on_polynomials(orc, deg):
    """Order 8 is exact on every polynomial of total degree <= 9 (odd terms
    cancel by symmetry), with unequal spacings, at points >= 4 cells inside."""
    rng = np.random.default_rng(deg)
    shape = (13, 14, 15)
    h = (0.11, 0.13, 0.09)
    coeffs = {m: rng.uniform(-1, 1) for m in _monomials(deg)}
    u, lap = _poly_and_laplacian(shape, h, (7.3, 6.6, 6.1), coeffs)
    got = orc.laplacian(u, h, 8)
    inner = (slice(4, -4),) * 3
    scale = np.max(np.abs(u)) * 3 * (205 / 72) / min(h) ** 2
    err = np.max(np.abs(got[inner] - lap[inner]))
    assert err < 1e-12 * scale, (deg, err, scale)


def test_laplacian_truncation_error_on_x10(orc):
    """For u = x^10 the order-8 error is exactly 2 h^8 sum_m c_m m^10 = -1152 h^8
    everywhere >= 4 cells inside (the 10th derivative is the constant 10!)."""
    exact = textbook_coeffs(4)
    lead = 2 * sum(c * m ** 10 for m, c in zip(range(1, 5), exact))
    assert lead == -1152
    shape = (9, 9, 13)
    h = (0.25, 1.0, 1.0)
    u, lap = _poly_and_laplacian(shape, h, (6.0, 4.0, 4.0), {(10, 0, 0): 1.0})
    got = orc.laplacian(u, h, 8)
    inner = (slice(4, -4),) * 3
    err = got[inner] - lap[inner]
    assert np.allclose(err, float(lead) * h[0] ** 8, rtol=1e-6, atol=0)


def test_twenty_five_point_star(orc):
    """Sec. 3 names a 25-point stencil, nine points on each axis: the response
    to a unit spike has exactly 25 non-zeros, on the three axis lines."""
    n = 11
    u = np.zeros((n, n, n))
    u[5, 5, 5] = 1.0
    h = (1.0, 2.0, 3.0)
    L = orc.laplacian(u, h, 8)
    nz_idx = np.argwhere(L != 0.0)
    assert len(nz_idx) == 25
    off = nz_idx - 5
    assert np.all(np.sum(off != 0, axis=1) <= 1)            # star: no cross terms
    for ax in range(3):
        assert np.sum(off[:, ax] != 0) == 8                 # 4 each side per axis
    c = orc.fd_coeffs(8)
    assert L[5, 5, 5] == pytest.approx(c[0] * (1 / 1 + 1 / 4 + 1 / 9), rel=1e-14)
    assert L[5, 5, 9] == pytest.approx(c[4] / 1.0, rel=1e-14)   # x offset +4 (hx = 1)
    assert L[1, 5, 5] == pytest.approx(c[4] / 9.0, rel=1e-14)   # z offset -4 (hz = 3)


def test_laplacian_zero_outside_grid(orc):
    """Reading R2: u = 0 beyond the edges, so the operator is symmetric:
    <a, L b> = <L a, b> for arbitrary fields."""
    rng = np.random.default_rng(3)
    a = rng.standard_normal((7, 8, 9))
    b = rng.standard_normal((7, 8, 9))
    h = (1.0, 1.3, 0.8)
    la, lb = orc.laplacian(a, h, 8), orc.laplacian(b, h, 8)
    assert np.sum(a * lb) == pytest.approx(np.sum(la * b), rel=1e-12)
