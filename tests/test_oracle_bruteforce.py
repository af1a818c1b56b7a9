"""Brute-force and symmetry pins of the oracle's whole stepper.

The dense stepper here is written independently of the oracle: the Laplacian
is a Kronecker sum of 1-D banded matrices built from the textbook closed-form
weights, the damping enters as diagonal matrices, and the source is put inside
the update's numerator (the oracle adds it after the sweep, Alg. 1 style).
On tiny grids both must agree to FP64 rounding.

Then properties that fix the source/receiver conventions:
  * linearity and superposition in the wavelets;
  * reciprocity  trace(r <- s) = trace(s <- r)  in a heterogeneous damped model,
    which holds exactly because the update is symmetric after scaling by
    (c / (1 + eta dt))^(1/2) with the source injected as c w / (h^3 (1 + eta dt));
  * equal spacings: permuting the axes of the model permutes the result.
"""
from fractions import Fraction
from math import factorial

import numpy as np
import pytest

import workloads as W


def textbook(R):
    return [float(Fraction(2 * (-1) ** (m + 1) * factorial(R) ** 2,
                           m * m * factorial(R - m) * factorial(R + m))) for m in range(1, R + 1)]


def d2_matrix(n, h, R):
    c = textbook(R)
    D = np.zeros((n, n))
    for i in range(n):
        D[i, i] = -2.0 * sum(c) / h ** 2
        for m in range(1, R + 1):
            if i + m < n:
                D[i, i + m] = c[m - 1] / h ** 2
            if i - m >= 0:
                D[i, i - m] = c[m - 1] / h ** 2
    return D


def profile(n, L, h, vmax, refl=1e-3):
    if L == 0:
        return np.zeros(n)
    eta_max = 1.5 * vmax * np.log(1.0 / refl) / (L * h)
    i = np.arange(n)
    d = np.maximum.reduce([L - i, i - (n - 1 - L), np.zeros(n, int)])
    return eta_max * (d / L) ** 2


def dense_forward(p, order=8):
    nz, ny, nx = p.vel.shape
    hx, hy, hz = p.h
    R = order // 2
    Ix, Iy, Iz = np.eye(nx), np.eye(ny), np.eye(nz)
    Lop = (np.kron(np.kron(Iz, Iy), d2_matrix(nx, hx, R))
           + np.kron(np.kron(Iz, d2_matrix(ny, hy, R)), Ix)
           + np.kron(np.kron(d2_matrix(nz, hz, R), Iy), Ix))
    v = p.vel.astype(np.float64).ravel()
    C = p.dt ** 2 * v * v
    vmax = float(p.vel.max())
    ex, ey, ez = (profile(nx, p.nbl, hx, vmax), profile(ny, p.nbl, hy, vmax), profile(nz, p.nbl, hz, vmax))
    e = (ez[:, None, None] + ey[None, :, None] + ex[None, None, :]).ravel() * p.dt
    flat = lambda ijk: (ijk[2] * ny + ijk[1]) * nx + ijk[0]
    N = nx * ny * nz
    u_prev, u = np.zeros(N), np.zeros(N)
    traces = np.zeros((p.nt, len(p.rec_ijk)))
    for n in range(p.nt):
        rhs = 2 * u - (1 - e) * u_prev + C * (Lop @ u)
        for s, ijk in enumerate(p.src_ijk):
            q = flat(ijk)
            rhs[q] += C[q] * float(p.wavelet[s, n]) / (hx * hy * hz)
        u_next = rhs / (1 + e)
        traces[n] = [u_next[flat(ijk)] for ijk in p.rec_ijk]
        u_prev, u = u, u_next
    return traces, u.reshape(nz, ny, nx)


def run(orc, p, **kw):
    return orc.forward(p.vel, p.h, p.dt, p.nt, order=kw.get("order", p.order), nbl=p.nbl,
                       src_ijk=p.src_ijk, wavelet=p.wavelet, rec_ijk=p.rec_ijk, want_state=True)


@pytest.mark.parametrize("shape,nbl,order", [((11, 10, 12), 2, 8), ((9, 9, 9), 0, 8),
                                             ((9, 12, 10), 3, 6), ((8, 7, 9), 1, 4), ((10, 9, 11), 4, 2)])
def test_dense_stepper_agrees(orc, shape, nbl, order):
    p = W.tiny_problem(shape=shape, nt=40, nbl=nbl, nsrc=3, nrec=6, seed=sum(shape) + nbl)
    # put a source and a receiver on a corner and an edge too
    p.src_ijk[0] = [0, 0, 0]
    p.rec_ijk[0] = [shape[2] - 1, shape[1] - 1, shape[0] - 1]
    p.rec_ijk[1] = p.src_ijk[1]
    tr_d, u_d = dense_forward(p, order)
    tr_o, _, u_o = run(orc, p, order=order)
    scale = np.max(np.abs(u_d))
    assert scale > 0
    assert np.max(np.abs(u_o - u_d)) < 1e-12 * scale
    assert np.max(np.abs(tr_o - tr_d)) < 1e-12 * max(np.max(np.abs(tr_d)), 1e-300)


def test_linearity_and_superposition(orc):
    p = W.tiny_problem(shape=(14, 13, 15), nt=60, nbl=3, nsrc=2, nrec=7, seed=5)
    tr, _, u = run(orc, p)
    p2 = W.tiny_problem(shape=(14, 13, 15), nt=60, nbl=3, nsrc=2, nrec=7, seed=5)
    p2.wavelet = (p2.wavelet.astype(np.float64) * 0.5).astype(np.float32)   # exact in FP32
    tr2, _, u2 = run(orc, p2)
    assert np.allclose(tr2, 0.5 * tr, rtol=1e-13, atol=0)
    single = []
    for s in range(2):
        q = W.tiny_problem(shape=(14, 13, 15), nt=60, nbl=3, nsrc=2, nrec=7, seed=5)
        q.wavelet[1 - s] = 0.0
        single.append(run(orc, q)[0])
    assert np.max(np.abs(single[0] + single[1] - tr)) < 1e-13 * np.max(np.abs(tr))


def test_reciprocity_heterogeneous_damped(orc):
    rng = np.random.default_rng(21)
    shape = (20, 18, 22)
    vel = rng.uniform(1600.0, 3200.0, shape).astype(np.float32)
    h = (10.0, 12.0, 9.0)
    dt = W.cfl_dt(0.3, h, 3200.0)
    nt = 150
    w = W.ricker(25.0, dt, nt)[None, :]
    a = np.array([[3, 4, 2]], np.int32)        # inside the damping layer
    b = np.array([[15, 11, 14]], np.int32)     # inner region
    t_ab = orc.forward(vel, h, dt, nt, nbl=5, src_ijk=a, wavelet=w, rec_ijk=b)
    t_ba = orc.forward(vel, h, dt, nt, nbl=5, src_ijk=b, wavelet=w, rec_ijk=a)
    assert np.max(np.abs(t_ab)) > 0
    assert np.max(np.abs(t_ab - t_ba)) < 1e-11 * np.max(np.abs(t_ab))


def test_axis_permutation(orc):
    rng = np.random.default_rng(8)
    shape = (13, 15, 17)                       # (nz, ny, nx)
    vel = rng.uniform(1500.0, 3000.0, shape).astype(np.float32)
    h = (10.0, 10.0, 10.0)
    dt = W.cfl_dt(0.3, h, 3000.0)
    nt = 50
    w = W.ricker(30.0, dt, nt)[None, :]
    src = np.array([[4, 6, 9]], np.int32)
    rec = np.array([[1, 2, 3], [16, 14, 12], [8, 7, 6]], np.int32)
    tr, _, u = orc.forward(vel, h, dt, nt, nbl=3, src_ijk=src, wavelet=w, rec_ijk=rec, want_state=True)
    # swap x and z: array axes (k, j, i) -> (i, j, k), positions (i, j, k) -> (k, j, i)
    vel_t = np.ascontiguousarray(vel.transpose(2, 1, 0))
    tr_t, _, u_t = orc.forward(vel_t, h, dt, nt, nbl=3, src_ijk=src[:, ::-1].copy(), wavelet=w,
                               rec_ijk=rec[:, ::-1].copy(), want_state=True)
    scale = np.max(np.abs(u))
    assert np.max(np.abs(u_t.transpose(2, 1, 0) - u)) < 1e-12 * scale
    assert np.max(np.abs(tr_t - tr)) < 1e-12 * scale
