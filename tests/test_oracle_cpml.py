"""Pins of the oracle's CPML stepper (reading R17).

* Without layers it is the plain stepper of Eq. 5.
* A dense stepper written here from the same discrete equations (Kronecker
  first- and second-difference matrices, memory vectors per axis, recursive
  convolutions with b = exp(-(d + alpha) dt), g = d (b - 1)/(d + alpha))
  agrees to FP64 rounding, with and without the free surface.
* Its purpose: waves leave the grid.  Against a run on a grid large enough
  that nothing comes back in the time window, a 10-cell CPML leaves a small
  error at receivers outside the layers, far below the damping layer's
  (reading R3) of the same width.
* A long run after the source stops decays instead of growing.
"""
import numpy as np
import pytest

import workloads as W
from test_oracle_bruteforce import d2_matrix

D1 = [4 / 5, -1 / 5, 4 / 105, -1 / 280]


def d1_matrix(n, h):
    D = np.zeros((n, n))
    for i in range(n):
        for m in range(1, 5):
            if i + m < n:
                D[i, i + m] += D1[m - 1] / h
            if i - m >= 0:
                D[i, i - m] -= D1[m - 1] / h
    return D


def cpml_bg(n, L, h, vmax, refl, f0, dt, top_free=False):
    b, g = np.ones(n), np.zeros(n)
    if L == 0:
        return b, g
    d0 = 3 * vmax * np.log(1 / refl) / (2 * L * h)
    for i in range(n):
        x = max(0 if top_free else L - i, i - (n - 1 - L), 0)
        if x == 0:
            continue
        s = x / L
        d, al = d0 * s * s, np.pi * f0 * (1 - s)
        b[i] = np.exp(-(d + al) * dt)
        g[i] = d * (b[i] - 1) / (d + al)
    return b, g


def dense_cpml(p, f0, free_surface=False):
    nz, ny, nx = p.vel.shape
    hx, hy, hz = p.h
    Ix, Iy, Iz = np.eye(nx), np.eye(ny), np.eye(nz)
    D2z = d2_matrix(nz, hz, 4)
    if free_surface:                       # odd image above k = 0
        c = [8 / 5, -1 / 5, 8 / 315, -1 / 560]
        for k in range(1, nz):
            for m in range(k + 1, 5):
                D2z[k, m - k] -= c[m - 1] / hz ** 2
    D2 = [np.kron(np.kron(Iz, Iy), d2_matrix(nx, hx, 4)), np.kron(np.kron(Iz, d2_matrix(ny, hy, 4)), Ix),
          np.kron(np.kron(D2z, Iy), Ix)]
    D1m = [np.kron(np.kron(Iz, Iy), d1_matrix(nx, hx)), np.kron(np.kron(Iz, d1_matrix(ny, hy)), Ix),
           np.kron(np.kron(d1_matrix(nz, hz), Iy), Ix)]
    vmax = float(p.vel.max())
    prof = [cpml_bg(nx, p.nbl, hx, vmax, p.refl, f0, p.dt), cpml_bg(ny, p.nbl, hy, vmax, p.refl, f0, p.dt),
            cpml_bg(nz, p.nbl, hz, vmax, p.refl, f0, p.dt, top_free=free_surface)]
    K, J, I = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    idx = [I.ravel(), J.ravel(), K.ravel()]
    B = [prof[a][0][idx[a]] for a in range(3)]
    G = [prof[a][1][idx[a]] for a in range(3)]
    v = p.vel.astype(np.float64).ravel()
    C = p.dt ** 2 * v * v
    N = nx * ny * nz
    psi = [np.zeros(N) for _ in range(3)]
    zeta = [np.zeros(N) for _ in range(3)]
    flat = lambda ijk: (ijk[2] * ny + ijk[1]) * nx + ijk[0]
    surface = (K.ravel() == 0) if free_surface else np.zeros(N, bool)
    u_prev, u = np.zeros(N), np.zeros(N)
    traces = np.zeros((p.nt, len(p.rec_ijk)))
    for n in range(p.nt):
        for a in range(3):
            psi[a] = B[a] * psi[a] + G[a] * (D1m[a] @ u)
        total = np.zeros(N)
        for a in range(3):
            d2 = D2[a] @ u
            on = G[a] != 0
            dpsi = D1m[a] @ psi[a]
            zeta[a] = np.where(on, B[a] * zeta[a] + G[a] * (d2 + dpsi), zeta[a])
            total += np.where(on, d2 + dpsi + zeta[a], d2)
        u_next = 2 * u - u_prev + C * total
        for s, ijk in enumerate(p.src_ijk):
            q = flat(ijk)
            u_next[q] += C[q] * float(p.wavelet[s, n]) / (hx * hy * hz)
        u_next[surface] = 0.0
        traces[n] = [u_next[flat(ijk)] for ijk in p.rec_ijk]
        u_prev, u = u, u_next
    return traces, u.reshape(nz, ny, nx)


def test_without_layers_it_is_the_plain_stepper(orc):
    p = W.tiny_problem(shape=(14, 13, 15), nt=50, nbl=0, nsrc=2, nrec=6, seed=5)
    tr_c, u_c = orc.forward_cpml(p.vel, p.h, p.dt, p.nt, nbl=0, src_ijk=p.src_ijk, wavelet=p.wavelet,
                                 rec_ijk=p.rec_ijk, want_state=True)
    tr_o, _, u_o = orc.forward(p.vel, p.h, p.dt, p.nt, nbl=0, src_ijk=p.src_ijk, wavelet=p.wavelet,
                               rec_ijk=p.rec_ijk, want_state=True)
    assert np.max(np.abs(u_c - u_o)) <= 1e-13 * np.max(np.abs(u_o))
    assert np.max(np.abs(tr_c - tr_o)) <= 1e-13 * np.max(np.abs(tr_o))


@pytest.mark.parametrize("shape,nbl,fs", [((12, 10, 11), 3, False), ((11, 12, 10), 2, False), ((12, 11, 13), 3, True)])
def test_dense_stepper_agrees(orc, shape, nbl, fs):
    p = W.tiny_problem(shape=shape, nt=40, nbl=nbl, nsrc=2, nrec=6, seed=sum(shape) + nbl)
    p.src_ijk[0] = [1, 2, 2]               # a source inside a layer
    p.rec_ijk[0] = [shape[2] - 1, 1, shape[0] - 2]
    tr_d, u_d = dense_cpml(p, 30.0, fs)
    tr_o, u_o = orc.forward_cpml(p.vel, p.h, p.dt, p.nt, nbl=p.nbl, f0=30.0, src_ijk=p.src_ijk,
                                 wavelet=p.wavelet, rec_ijk=p.rec_ijk, want_state=True, free_surface=fs)
    scale = np.max(np.abs(u_d))
    assert scale > 0
    assert np.max(np.abs(u_o - u_d)) < 1e-12 * scale
    assert np.max(np.abs(tr_o - tr_d)) < 1e-12 * np.max(np.abs(tr_d))


@pytest.mark.slow
def test_cpml_absorbs_far_better_than_the_damping_layer(orc):
    v, h, f = 2000.0, 10.0, 15.0
    dt = W.cfl_dt(0.35, (h, h, h), v)
    nt, L, n, big = 300, 10, 60, 150
    recs = [(18, 0, 0), (15, 15, 0), (0, 0, 17), (-16, 8, -8)]

    def run(nn, nbl, kind):
        vel = np.full((nn, nn, nn), v, np.float32)
        c = nn // 2
        src = np.array([[c, c, c]], np.int32)
        rec = np.array([[c + a, c + b, c + e] for a, b, e in recs], np.int32)
        w = W.ricker(f, dt, nt)[None, :]
        if kind == "cpml":
            return orc.forward_cpml(vel, (h, h, h), dt, nt, nbl=nbl, f0=f, src_ijk=src, wavelet=w, rec_ijk=rec)
        return orc.forward(vel, (h, h, h), dt, nt, nbl=nbl, src_ijk=src, wavelet=w, rec_ijk=rec)

    ref = run(big, 0, "plain")             # walls 75 cells away: nothing returns within 300 steps
    err = {}
    for kind in ("cpml", "damping"):
        tr = run(n, L, kind)
        err[kind] = max(np.linalg.norm(tr[:, r] - ref[:, r]) / np.linalg.norm(ref[:, r]) for r in range(len(recs)))
    assert err["cpml"] < 0.02, err
    assert err["damping"] > 5 * err["cpml"], err


def test_long_run_decays(orc):
    """A rough random model (strong scattering) keeps losing energy through
    the layers for 3000 steps after the source stops: no late growth."""
    p = W.tiny_problem(shape=(30, 32, 34), nt=3000, nbl=8, nsrc=1, nrec=3, seed=2)
    p.wavelet[:, 200:] = 0.0               # the source stops
    tr = orc.forward_cpml(p.vel, p.h, p.dt, p.nt, nbl=p.nbl, f0=25.0, src_ijk=p.src_ijk, wavelet=p.wavelet,
                          rec_ijk=p.rec_ijk)
    window = [np.abs(tr[a:a + 300]).max() for a in range(0, 3000, 300)]
    assert window[0] > 0
    assert window[-1] < 1e-2 * window[0]
    assert window[-1] < window[5] < window[2]
