"""Pins of the oracle's adjoint and velocity gradient.

* Dot-product test: for the forward map F: wavelets -> traces (linear in the
  wavelet), <F w, r> = <w, F^T r> for random w and r, to FP64 rounding.
* The adjoint equals the explicit transpose of F built column by column on a
  tiny grid (F applied to unit wavelets).
* Gradient: the directional derivative of J(v) = 1/2 |F_v w - d_obs|^2 by
  central differences matches <dJ/dv, dv>, with velocity perturbations that
  are exact in FP32 (integer velocities, +-2 m/s).
"""
import numpy as np
import pytest

import workloads as W


def _setup(seed=3, shape=(14, 13, 15), nt=70, nbl=3, nsrc=2, nrec=5):
    p = W.tiny_problem(shape=shape, nt=nt, nbl=nbl, nsrc=nsrc, nrec=nrec, seed=seed)
    p.src_ijk[0] = [1, 2, 1]           # one source inside a damping layer
    return p


def test_dot_product(orc):
    p = _setup()
    rng = np.random.default_rng(9)
    w = rng.standard_normal((len(p.src_ijk), p.nt)).astype(np.float32)
    r = rng.standard_normal((p.nt, len(p.rec_ijk)))
    Fw = orc.forward(p.vel, p.h, p.dt, p.nt, nbl=p.nbl, src_ijk=p.src_ijk, wavelet=w, rec_ijk=p.rec_ijk)
    FTr = orc.adjoint(p.vel, p.h, p.dt, p.nt, nbl=p.nbl, src_ijk=p.src_ijk, rec_ijk=p.rec_ijk, resid=r)
    lhs = float(np.sum(Fw * r))
    rhs = float(np.sum(w.astype(np.float64) * FTr))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1e-300), (lhs, rhs)


def test_adjoint_is_the_explicit_transpose(orc):
    p = _setup(seed=4, shape=(9, 10, 11), nt=12, nbl=2, nsrc=2, nrec=3)
    ns, nr, nt = len(p.src_ijk), len(p.rec_ijk), p.nt
    F = np.zeros((nt * nr, ns * nt))
    for s in range(ns):
        for n in range(nt):
            w = np.zeros((ns, nt), np.float32)
            w[s, n] = 1.0
            F[:, s * nt + n] = orc.forward(p.vel, p.h, p.dt, nt, nbl=p.nbl, src_ijk=p.src_ijk, wavelet=w,
                                           rec_ijk=p.rec_ijk).ravel()
    rng = np.random.default_rng(1)
    r = rng.standard_normal((nt, nr))
    FTr = orc.adjoint(p.vel, p.h, p.dt, nt, nbl=p.nbl, src_ijk=p.src_ijk, rec_ijk=p.rec_ijk, resid=r)
    assert np.max(np.abs(FTr.ravel() - F.T @ r.ravel())) <= 1e-12 * np.max(np.abs(FTr))


def _misfit(orc, p, vel, d_obs):
    tr = orc.forward(vel, p.h, p.dt, p.nt, nbl=p.nbl, src_ijk=p.src_ijk, wavelet=p.wavelet, rec_ijk=p.rec_ijk)
    return 0.5 * float(np.sum((tr - d_obs) ** 2)), tr


@pytest.mark.parametrize("kind", ["point", "smooth", "source"])
def test_gradient_matches_finite_differences(orc, kind):
    p = _setup(seed=6, shape=(14, 15, 16), nt=90, nbl=3, nsrc=1, nrec=6)
    p.vel = np.round(p.vel).astype(np.float32)          # integer velocities: v +- 2 exact in FP32
    rng = np.random.default_rng(2)
    d_obs = orc.forward(np.round(p.vel * 1.03).astype(np.float32), p.h, p.dt, p.nt, nbl=p.nbl,
                        src_ijk=p.src_ijk, wavelet=p.wavelet, rec_ijk=p.rec_ijk)
    J0, tr = _misfit(orc, p, p.vel, d_obs)
    g = orc.gradient(p.vel, p.h, p.dt, p.nt, nbl=p.nbl, src_ijk=p.src_ijk, wavelet=p.wavelet,
                     rec_ijk=p.rec_ijk, resid=tr - d_obs)
    if kind == "point":
        dv = np.zeros(p.vel.shape)
        dv[7, 7, 8] = 1.0
    elif kind == "source":             # the source term of the gradient lives here
        dv = np.zeros(p.vel.shape)
        i, j, k = p.src_ijk[0]
        dv[k, j, i] = 1.0
    else:
        # a coherent Gaussian bump, quantised to 1/1024 so v +- 2 dv stays exact in FP32
        nz, ny, nx = p.vel.shape
        Z, Y, X = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        r2 = (Z - 6.0) ** 2 + (Y - 7.0) ** 2 + (X - 8.0) ** 2
        dv = np.round(np.exp(-r2 / (2 * 2.5 ** 2)) * 1024) / 1024
    eps = 2.0
    Jp, _ = _misfit(orc, p, (p.vel + eps * dv).astype(np.float32), d_obs)
    Jm, _ = _misfit(orc, p, (p.vel - eps * dv).astype(np.float32), d_obs)
    fd = (Jp - Jm) / (2 * eps)
    an = float(np.sum(g * dv))
    assert an != 0.0
    assert abs(fd - an) <= 2e-5 * abs(an), (fd, an)


def test_zero_residual_gives_zero_gradient(orc):
    p = _setup(seed=2, nt=20)
    g = orc.gradient(p.vel, p.h, p.dt, p.nt, nbl=p.nbl, src_ijk=p.src_ijk, wavelet=p.wavelet,
                     rec_ijk=p.rec_ijk, resid=np.zeros((p.nt, len(p.rec_ijk))))
    assert not np.any(g)
