"""Pins of the oracle's free surface (the paper's surface option, Sec. 3;
reading R15: p = 0 on the plane k = 0 through the odd image u(-m) = -u(m)).

* The odd image makes phi = cos(kx x) cos(ky y) sin(kz z) (z from the
  surface) an exact eigenfunction of the discrete Laplacian right up to the
  surface, with the same eigenvalue K as the full-space standing wave; a
  standing sine wave then evolves as cos(n w dt) phi exactly, surface included.
* With no damping the half-space operator stays symmetric, so the discrete
  energy is conserved.
* A dense stepper written here (odd reflection in the 1-D z matrix, plane 0
  projected to zero, no top layer) agrees with the oracle on tiny grids.
* A point source under the surface radiates w(t - r/v)/(4 pi r) minus its
  image w(t - r'/v)/(4 pi r') (r' from the source mirrored above k = 0).
* The adjoint stays the transpose (dot-product test) and the gradient the
  derivative (central differences) with the surface on.
"""
import numpy as np
import pytest

import workloads as W
from test_oracle_bruteforce import d2_matrix, profile, textbook


def _eigen(shape, h, k, R):
    nz, ny, nx = shape
    Z, Y, X = np.meshgrid(np.arange(nz) * h[2], np.arange(ny) * h[1], np.arange(nx) * h[0], indexing="ij")
    phi = np.cos(k[0] * X + 0.3) * np.cos(k[1] * Y - 0.7) * np.sin(k[2] * Z)
    c = textbook(R)
    K = sum(4 * c[m - 1] * np.sin(m * k[a] * h[a] / 2) ** 2 / h[a] ** 2 for a in range(3) for m in range(1, R + 1))
    return phi, K


def test_odd_image_laplacian_is_exact_at_the_surface(orc):
    shape, h = (20, 22, 24), (10.0, 11.0, 9.0)
    phi, K = _eigen(shape, h, (2 * np.pi / 83.0, 2 * np.pi / 71.0, 2 * np.pi / 57.0), 4)
    lap = orc.laplacian(phi, h, 8, free_surface=True)
    inner = (slice(0, -4), slice(4, -4), slice(4, -4))   # every depth from the surface down
    assert np.max(np.abs(lap[inner] + K * phi[inner])) < 1e-12 * K
    # without the image the surface rows are wrong
    lap0 = orc.laplacian(phi, h, 8)
    assert np.max(np.abs(lap0[:4, 4:-4, 4:-4] + K * phi[:4, 4:-4, 4:-4])) > 1e-6 * K


def test_standing_sine_wave_is_exact_with_free_surface(orc):
    shape, h, v, dt = (34, 36, 38), (10.0, 12.0, 9.0), 2000.0, 0.9e-3
    phi, K = _eigen(shape, h, (2 * np.pi / 97.0, 2 * np.pi / 61.0, 2 * np.pi / 143.0), 4)
    cwdt = 1 - dt * dt * v * v * K / 2
    wdt = np.arccos(cwdt)
    vel = np.full(shape, v, np.float32)
    n = 4
    _, _, un = orc.forward(vel, h, dt, n, nbl=0, u_prev0=cwdt * phi, u_cur0=phi, want_state=True,
                           free_surface=True)
    m = 4 * n
    region = (slice(0, -m), slice(m, -m), slice(m, -m))    # the surface side is exact too
    assert np.max(np.abs(un[region] - np.cos(n * wdt) * phi[region])) < 1e-12
    assert not np.any(un[0])                                 # p = 0 on the surface plane


def test_energy_conserved_with_free_surface(orc):
    rng = np.random.default_rng(12)
    shape, h = (18, 20, 22), (10.0, 9.0, 11.0)
    vel = rng.uniform(1500.0, 3500.0, shape).astype(np.float32)
    dt = W.cfl_dt(0.35, h, 3500.0)
    C = dt * dt * vel.astype(np.float64) ** 2
    u_m1 = rng.standard_normal(shape)
    u_0 = u_m1 + 0.01 * rng.standard_normal(shape)
    u_m1[0] = 0.0
    u_0[0] = 0.0
    C[0] = 1.0   # plane 0 never moves; any positive weight

    def energy(u_new, u_old):
        d = u_new - u_old
        return np.sum(d * d / C) - np.sum(u_new * orc.laplacian(u_old, h, 8, free_surface=True))

    e0 = energy(u_0, u_m1)
    assert e0 > 0
    for nt in (1, 29, 300):
        _, up, uc = orc.forward(vel, h, dt, nt, nbl=0, u_prev0=u_m1, u_cur0=u_0, want_state=True,
                                free_surface=True)
        assert energy(uc, up) == pytest.approx(e0, rel=1e-11), nt


def dense_forward_fs(p, order=8):
    """Independent dense stepper with the free surface (reading R15)."""
    nz, ny, nx = p.vel.shape
    hx, hy, hz = p.h
    R = order // 2
    Dz = d2_matrix(nz, hz, R)
    c = textbook(R)
    for k in range(1, nz):             # odd image: u(k - m) = -u(m - k) for k - m < 0
        for m in range(k + 1, R + 1):
            Dz[k, m - k] -= c[m - 1] / hz ** 2
    Ix, Iy, Iz = np.eye(nx), np.eye(ny), np.eye(nz)
    Lop = (np.kron(np.kron(Iz, Iy), d2_matrix(nx, hx, R)) + np.kron(np.kron(Iz, d2_matrix(ny, hy, R)), Ix)
           + np.kron(np.kron(Dz, Iy), Ix))
    v = p.vel.astype(np.float64).ravel()
    C = p.dt ** 2 * v * v
    vmax = float(p.vel.max())
    ez = profile(nz, p.nbl, hz, vmax)
    ez[: min(p.nbl, nz - 1 - p.nbl)] = 0.0   # no layer under the surface
    ex, ey = profile(nx, p.nbl, hx, vmax), profile(ny, p.nbl, hy, vmax)
    e = (ez[:, None, None] + ey[None, :, None] + ex[None, None, :]).ravel() * p.dt
    surface = np.zeros((nz, ny, nx), bool)
    surface[0] = True
    surface = surface.ravel()
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
        u_next[surface] = 0.0
        traces[n] = [u_next[flat(ijk)] for ijk in p.rec_ijk]
        u_prev, u = u, u_next
    return traces, u.reshape(nz, ny, nx)


@pytest.mark.parametrize("shape,nbl", [((11, 10, 12), 2), ((12, 9, 9), 0), ((10, 8, 9), 3)])
def test_dense_stepper_with_free_surface(orc, shape, nbl):
    p = W.tiny_problem(shape=shape, nt=40, nbl=nbl, nsrc=3, nrec=6, seed=sum(shape) + 7 * nbl)
    p.src_ijk[0] = [1, 2, 0]            # a source on the surface plane (it must vanish)
    p.src_ijk[1] = [3, 3, 1]            # and one just below it
    p.rec_ijk[0] = [2, 2, 0]
    p.rec_ijk[1] = [4, 3, 1]
    tr_d, u_d = dense_forward_fs(p)
    tr_o, _, u_o = orc.forward(p.vel, p.h, p.dt, p.nt, nbl=p.nbl, src_ijk=p.src_ijk, wavelet=p.wavelet,
                               rec_ijk=p.rec_ijk, want_state=True, free_surface=True)
    scale = np.max(np.abs(u_d))
    assert scale > 0
    assert np.max(np.abs(u_o - u_d)) < 1e-12 * scale
    assert np.max(np.abs(tr_o - tr_d)) < 1e-12 * np.max(np.abs(tr_d))
    assert not np.any(tr_o[:, 0])


@pytest.mark.slow
def test_image_source_green_function(orc):
    n, hh, v, f, dt = 100, 10.0, 1500.0, 10.0, 1.0e-3
    nt = 420
    vel = np.full((n, n, n), v, np.float32)
    ks = 14                                        # source 14 cells under the surface
    src = np.array([[50, 50, ks]], np.int32)
    offs = [(15, 0, 0), (0, -12, 6), (0, 0, -8), (10, 10, 10), (-14, 0, -10), (0, 18, 4)]
    rec = np.array([[50 + a, 50 + b, ks + c] for a, b, c in offs], np.int32)
    w = W.ricker(f, dt, nt)
    tr = orc.forward(vel, (hh, hh, hh), dt, nt, nbl=0, src_ijk=src, wavelet=w[None, :], rec_ijk=rec,
                     free_surface=True)
    t = (np.arange(nt) + 1) * dt
    for r_i, (a, b, c) in enumerate(offs):
        pos = np.array([50 + a, 50 + b, ks + c], float)
        r = hh * np.sqrt(a * a + b * b + c * c)
        r_img = hh * np.linalg.norm(pos - np.array([50, 50, -ks], float))
        t_refl = np.inf                            # the zero walls other than the surface
        for ax, walls in ((0, (-1, n)), (1, (-1, n)), (2, (n,))):
            for wall in walls:
                img = np.array([50, 50, ks], float)
                img[ax] = 2 * wall - img[ax]
                t_refl = min(t_refl, hh * np.linalg.norm(img - pos) / v)
        assert t_refl > r_img / v + 2.5 / f
        keep = t < t_refl - 3 * dt

        def ricker(tt):
            arg = (np.pi * f * (tt - 1.5 / f)) ** 2
            return (1 - 2 * arg) * np.exp(-arg)

        exact = ricker(t - r / v) / (4 * np.pi * r) - ricker(t - r_img / v) / (4 * np.pi * r_img)
        err = np.linalg.norm((tr[:, r_i] - exact)[keep]) / np.linalg.norm(exact[keep])
        assert err < 0.01, (r_i, err)


def test_adjoint_dot_product_with_free_surface(orc):
    p = W.tiny_problem(shape=(14, 13, 15), nt=60, nbl=3, nsrc=2, nrec=5, seed=4)
    p.src_ijk[0] = [3, 4, 1]
    p.rec_ijk[0] = [5, 5, 0]
    p.rec_ijk[1] = [6, 2, 1]
    rng = np.random.default_rng(9)
    w = rng.standard_normal((len(p.src_ijk), p.nt)).astype(np.float32)
    r = rng.standard_normal((p.nt, len(p.rec_ijk)))
    Fw = orc.forward(p.vel, p.h, p.dt, p.nt, nbl=p.nbl, src_ijk=p.src_ijk, wavelet=w, rec_ijk=p.rec_ijk,
                     free_surface=True)
    FTr = orc.adjoint(p.vel, p.h, p.dt, p.nt, nbl=p.nbl, src_ijk=p.src_ijk, rec_ijk=p.rec_ijk, resid=r,
                      free_surface=True)
    lhs, rhs = float(np.sum(Fw * r)), float(np.sum(w.astype(np.float64) * FTr))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs), (lhs, rhs)


def test_gradient_finite_differences_with_free_surface(orc):
    p = W.tiny_problem(shape=(14, 15, 16), nt=90, nbl=3, nsrc=1, nrec=6, seed=6)
    p.vel = np.round(p.vel).astype(np.float32)
    p.src_ijk[0] = [8, 7, 2]
    p.rec_ijk[:3] = [[3, 3, 1], [10, 9, 1], [5, 12, 0]]
    kw = dict(nbl=p.nbl, src_ijk=p.src_ijk, wavelet=p.wavelet, rec_ijk=p.rec_ijk, free_surface=True)
    d_obs = orc.forward(np.round(p.vel * 1.03).astype(np.float32), p.h, p.dt, p.nt, **kw)

    def misfit(vel):
        tr = orc.forward(vel, p.h, p.dt, p.nt, **kw)
        return 0.5 * float(np.sum((tr - d_obs) ** 2)), tr

    _, tr = misfit(p.vel)
    g = orc.gradient(p.vel, p.h, p.dt, p.nt, resid=tr - d_obs, **kw)
    assert not np.any(g[0])                       # c on the surface plane moves nothing
    nz, ny, nx = p.vel.shape
    Z, Y, X = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    dv = np.round(np.exp(-((Z - 3.0) ** 2 + (Y - 7.0) ** 2 + (X - 8.0) ** 2) / (2 * 2.5 ** 2)) * 1024) / 1024
    eps = 2.0
    Jp, _ = misfit((p.vel + eps * dv).astype(np.float32))
    Jm, _ = misfit((p.vel - eps * dv).astype(np.float32))
    fd = (Jp - Jm) / (2 * eps)
    an = float(np.sum(g * dv))
    assert an != 0.0
    assert abs(fd - an) <= 2e-5 * abs(an), (fd, an)
