"""Pins of the optimised-stencil weights (reading R16) and of custom weights
in the oracle's Laplacian and stepper.

* Consistency: sum_m m^2 c_m = 1, so the stencil is exact on quadratics; it
  is not exact on quartics (formal order 2: the accuracy traded for the
  smaller dispersion error).
* Optimality: the weights are a constrained minimum of the stated objective,
  evaluated here with an independent quadrature (Simpson on a different
  grid): every feasible direction increases it.
* Purpose: the largest relative symbol error over the band is several times
  smaller than the Taylor weights'.
* The stepper uses the weights it is given: a standing wave built from the
  eigenvalue of those weights evolves exactly.
"""
import numpy as np
import pytest

from test_oracle_bruteforce import textbook

KMAX = 2 * np.pi / 3   # three points per shortest wavelength


def symbol_rel_err(c, k):
    S = sum(2 * c[m - 1] * (1 - np.cos(m * k)) for m in range(1, len(c) + 1))
    return S / k ** 2 - 1


def objective(c, kmax=KMAX, n=30001):
    k = np.linspace(1e-9, kmax, n)
    e2 = symbol_rel_err(c, k) ** 2
    h = k[1] - k[0]
    return h / 3 * (e2[0] + e2[-1] + 4 * e2[1:-1:2].sum() + 2 * e2[2:-1:2].sum())


@pytest.mark.parametrize("order", [8, 6, 4])
def test_consistency_and_order(orc, order):
    c = orc.optimized_coeffs(order, KMAX)
    R = order // 2
    assert sum(m * m * c[m] for m in range(1, R + 1)) == pytest.approx(1.0, abs=1e-13)
    assert c[0] == pytest.approx(-2 * sum(c[1:]), abs=1e-14)
    # quadratics exact, quartics not
    shape, h = (20, 21, 22), (10.0, 11.0, 9.0)
    nz, ny, nx = shape
    Z, Y, X = np.meshgrid(np.arange(nz) * h[2], np.arange(ny) * h[1], np.arange(nx) * h[0], indexing="ij")
    inner = (slice(R, -R),) * 3
    lap = orc.laplacian(X * X + 3 * Y * Z - Z * Z, h, order, coef=c[1:])
    assert np.max(np.abs(lap[inner] - 0.0)) < 1e-9
    lap4 = orc.laplacian(X ** 4, h, order, coef=c[1:])
    assert np.max(np.abs(lap4[inner] - 12 * X[inner] ** 2)) > 1e-3


def test_constrained_minimum(orc):
    c = orc.optimized_coeffs(8, KMAX)[1:]
    g = np.array([1.0, 4.0, 9.0, 16.0])
    J0 = objective(c)
    rng = np.random.default_rng(1)
    for _ in range(20):
        d = rng.standard_normal(4)
        d -= g * (d @ g) / (g @ g)            # stay on sum m^2 c_m = 1
        d /= np.linalg.norm(d)
        for eps in (1e-3, -1e-3):
            assert objective(c + eps * d) > J0
    # and the Taylor weights are feasible but worse
    assert objective(np.array(textbook(4))) > 10 * J0


def test_dispersion_error_smaller_than_taylor(orc):
    k = np.linspace(1e-6, KMAX, 4001)
    c = orc.optimized_coeffs(8, KMAX)[1:]
    e_opt = np.abs(symbol_rel_err(c, k)).max()
    e_tay = np.abs(symbol_rel_err(textbook(4), k)).max()
    assert e_opt < e_tay / 5, (e_opt, e_tay)


def test_stepper_uses_the_given_weights(orc):
    c = orc.optimized_coeffs(8, KMAX)
    shape, h, v, dt = (34, 36, 38), (10.0, 12.0, 9.0), 2000.0, 0.8e-3
    kv = np.array([2 * np.pi / 97.0, 2 * np.pi / 61.0, 2 * np.pi / 143.0])
    nz, ny, nx = shape
    Z, Y, X = np.meshgrid(np.arange(nz) * h[2], np.arange(ny) * h[1], np.arange(nx) * h[0], indexing="ij")
    phi = np.cos(kv[0] * X + 0.3) * np.cos(kv[1] * Y + 1.1) * np.cos(kv[2] * Z - 0.4)
    K = sum(4 * c[m] * np.sin(m * kv[a] * h[a] / 2) ** 2 / h[a] ** 2 for a in range(3) for m in range(1, 5))
    cwdt = 1 - dt * dt * v * v * K / 2
    n = 4
    vel = np.full(shape, v, np.float32)
    _, _, un = orc.forward(vel, h, dt, n, nbl=0, u_prev0=cwdt * phi, u_cur0=phi, want_state=True, coef=c[1:])
    inner = (slice(16, -16),) * 3
    expect = np.cos(n * np.arccos(cwdt)) * phi
    assert np.max(np.abs(un[inner] - expect[inner])) < 1e-12
    _, _, ut = orc.forward(vel, h, dt, n, nbl=0, u_prev0=cwdt * phi, u_cur0=phi, want_state=True)
    assert np.max(np.abs(ut[inner] - expect[inner])) > 1e-8   # Taylor weights give another result
