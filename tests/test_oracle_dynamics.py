"""Pins of the oracle's time stepping (Eq. 5, Alg. 1, damping reading R3).

* Exact discrete standing wave: phi = prod_a cos(k_a x_a + s_a) satisfies
  L phi = -K phi with K = sum_a sum_m 4 c_m sin^2(m k_a h_a / 2) / h_a^2, so with
  u^0 = phi and u^-1 = cos(w dt) phi, cos(w dt) = 1 - dt^2 v^2 K / 2, Eq. 5
  gives u^n = cos(n w dt) phi exactly wherever the zero boundary has not
  reached yet (4 cells per step).  K uses the textbook coefficients.
* Discrete energy E^{n+1/2} = (u^{n+1}-u^n)^T C^-1 (u^{n+1}-u^n) - u^{n+1 T} L u^n
  (C = dt^2 v^2) is conserved when eta = 0, and with damping its change per step
  is exactly  - sum eta dt (u^{n+1} - u^{n-1})^2 / C.
* 3-D homogeneous Green's function: (1/v^2) p_tt - lap p = delta(x) w(t) has
  p(r, t) = w(t - r/v) / (4 pi r).
"""
from fractions import Fraction
from math import factorial

import numpy as np
import pytest

import workloads as W


def textbook(R):
    return [float(Fraction(2 * (-1) ** (m + 1) * factorial(R) ** 2,
                           m * m * factorial(R - m) * factorial(R + m))) for m in range(1, R + 1)]


def _grid(shape, h):
    nz, ny, nx = shape
    z = np.arange(nz) * h[2]
    y = np.arange(ny) * h[1]
    x = np.arange(nx) * h[0]
    return np.meshgrid(z, y, x, indexing="ij")


@pytest.mark.parametrize("order", [8, 4])
def test_standing_wave_is_exact(orc, order):
    R = order // 2
    shape = (36, 34, 38)
    h = (10.0, 12.0, 9.0)
    v = 2000.0
    dt = 0.9e-3
    k = np.array([2 * np.pi / 97.0, 2 * np.pi / 61.0, 2 * np.pi / 143.0])   # rad/m (x, y, z)
    s = (0.3, 1.1, -0.4)
    Z, Y, X = _grid(shape, h)
    phi = np.cos(k[0] * X + s[0]) * np.cos(k[1] * Y + s[1]) * np.cos(k[2] * Z + s[2])
    c = textbook(R)
    K = sum(4 * c[m - 1] * np.sin(m * k[a] * h[a] / 2) ** 2 / h[a] ** 2
            for a in range(3) for m in range(1, R + 1))
    cwdt = 1 - dt * dt * v * v * K / 2
    wdt = np.arccos(cwdt)
    vel = np.full(shape, v, np.float32)
    nsteps = 4
    _, _, un = orc.forward(vel, h, dt, nsteps, order=order, nbl=0,
                           u_prev0=cwdt * phi, u_cur0=phi, want_state=True)
    m = R * nsteps
    inner = (slice(m, -m),) * 3
    expect = np.cos(nsteps * wdt) * phi
    assert np.max(np.abs(un[inner] - expect[inner])) < 1e-12
    # and the boundary does matter outside the domain of dependence
    assert np.max(np.abs(un - expect)) > 1e-6
    # the discrete frequency approximates the continuous v|k|
    w_cont = v * np.linalg.norm(k)
    assert abs(wdt / dt - w_cont) / w_cont < (3e-3 if order == 8 else 1e-2)


def _energy(orc, h, order, C, u_new, u_old):
    d = u_new - u_old
    return np.sum(d * d / C) - np.sum(u_new * orc.laplacian(u_old, h, order))


def test_energy_conserved_without_damping(orc):
    rng = np.random.default_rng(11)
    shape = (18, 20, 22)
    h = (10.0, 9.0, 11.0)
    vel = rng.uniform(1500.0, 3500.0, shape).astype(np.float32)
    dt = W.cfl_dt(0.35, h, 3500.0)
    C = dt * dt * vel.astype(np.float64) ** 2
    u_m1 = rng.standard_normal(shape)
    u_0 = u_m1 + 0.01 * rng.standard_normal(shape)
    e0 = _energy(orc, h, 8, C, u_0, u_m1)
    assert e0 > 0
    for nt in (1, 37, 400):
        _, up, uc = orc.forward(vel, h, dt, nt, nbl=0, u_prev0=u_m1, u_cur0=u_0, want_state=True)
        e = _energy(orc, h, 8, C, uc, up)
        assert e == pytest.approx(e0, rel=1e-11), nt


def test_energy_decrement_with_damping_is_exact(orc):
    rng = np.random.default_rng(12)
    shape = (16, 17, 18)
    h = (10.0, 10.0, 12.0)
    nbl = 4
    vel = rng.uniform(1500.0, 3000.0, shape).astype(np.float32)
    dt = W.cfl_dt(0.35, h, 3000.0)
    C = dt * dt * vel.astype(np.float64) ** 2
    vmax = float(vel.max())
    ex = orc.damping_profile(shape[2], nbl, h[0], vmax)
    ey = orc.damping_profile(shape[1], nbl, h[1], vmax)
    ez = orc.damping_profile(shape[0], nbl, h[2], vmax)
    eta = ez[:, None, None] + ey[None, :, None] + ex[None, None, :]
    assert eta.max() > 0 and np.count_nonzero(eta == 0) > 0
    u_prev, u_cur = rng.standard_normal(shape), rng.standard_normal(shape)
    e_prev = _energy(orc, h, 8, C, u_cur, u_prev)
    for _ in range(12):
        _, a, b = orc.forward(vel, h, dt, 1, nbl=nbl, u_prev0=u_prev, u_cur0=u_cur, want_state=True)
        assert np.array_equal(a, u_cur)
        u_next = b
        e_next = _energy(orc, h, 8, C, u_next, u_cur)
        dec = -np.sum(eta * dt * (u_next - u_prev) ** 2 / C)
        assert dec < 0
        assert e_next - e_prev == pytest.approx(dec, rel=1e-9, abs=1e-12 * abs(e_prev))
        u_prev, u_cur, e_prev = u_cur, u_next, e_next


def _green_error(orc, dt, n=100, h=10.0, v=1500.0, f=10.0, tmax=0.52):
    """Rel. L2 error of traces against w(t - r/v) / (4 pi r) for six receivers,
    each compared only before the first reflection off the u = 0 walls can
    arrive (image source across each face) and after its wavelet has ended."""
    nt = int(round(tmax / dt))
    vel = np.full((n, n, n), v, np.float32)
    s0 = n // 2
    src = np.array([[s0, s0, s0]], np.int32)
    offs = [(15, 0, 0), (0, -20, 0), (0, 0, 22), (12, 12, 12), (-14, 0, 14), (0, 18, -9)]
    rec = np.array([[s0 + a, s0 + b, s0 + c] for a, b, c in offs], np.int32)
    w = W.ricker(f, dt, nt)
    tr = orc.forward(vel, (h, h, h), dt, nt, nbl=0, src_ijk=src, wavelet=w[None, :], rec_ijk=rec)
    t = (np.arange(nt) + 1) * dt            # traces[n] holds u^{n+1}, time (n+1) dt
    errs = []
    for r_i, (a, b, c) in enumerate(offs):
        pos = np.array([s0 + a, s0 + b, s0 + c], float)
        r = h * np.sqrt(a * a + b * b + c * c)
        t_refl = np.inf
        for ax in range(3):                 # zero cells at index -1 and n on each axis
            for wall in (-1, n):
                img = np.array([s0, s0, s0], float)
                img[ax] = 2 * wall - s0
                t_refl = min(t_refl, h * np.linalg.norm(img - pos) / v)
        assert t_refl > r / v + 2.5 / f     # the whole wavelet fits the window
        keep = t < t_refl - 3 * dt
        tau = t - r / v - 1.5 / f
        arg = (np.pi * f * tau) ** 2
        exact = (1 - 2 * arg) * np.exp(-arg) / (4 * np.pi * r)
        errs.append(np.linalg.norm((tr[:, r_i] - exact)[keep]) / np.linalg.norm(exact[keep]))
    return np.array(errs)


@pytest.mark.slow
def test_green_function_and_convergence(orc):
    e1 = _green_error(orc, 1.0e-3)
    assert np.all(e1 < 0.02), e1
    e2 = _green_error(orc, 2.0e-3)
    # leapfrog in time is second order: halving dt cuts the error about 4x
    assert np.all(e1 < e2 * 0.5), (e1, e2)
