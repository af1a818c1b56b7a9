"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds no arithmetic of the propagator itself: it only draws the
inputs a user would hand to it — velocity models, the source wavelet and the
source/receiver geometry — in FP64 with ``numpy.random.default_rng(seed)`` and
rounds them once to FP32, so both sides consume identical FP32 values.

The paper uses no public dataset: its only model description is the printout
``vmin 1500 / vmax 4500`` of its example run (Sec. 5.3).  The workloads below
follow that style.  Index convention: arrays are [nz][ny][nx]; positions are
(i, j, k) with k = 0 at the surface.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

__all__ = ["Problem", "ricker", "cfl_dt", "small_homogeneous", "layered_240",
           "smooth_gradient_200", "batched_shots", "fractal_large", "tiny_problem",
           "gardner_density", "layered_240_vd", "tiny_problem_vd", "layered_vd_plain"]


@dataclass
class Problem:
    """One forward-modelling problem: grid, physics and acquisition."""
    name: str
    vel: np.ndarray                 # [nz][ny][nx] float32, m/s
    h: tuple                        # (hx, hy, hz) metres
    dt: float                       # seconds
    nt: int
    nbl: int                        # damping width in cells, all six faces
    src_ijk: np.ndarray             # [nsrc][3] int32
    wavelet: np.ndarray             # [nsrc][nt] float32
    rec_ijk: np.ndarray             # [nrec][3] int32
    order: int = 8
    refl: float = 1e-3
    meta: dict = field(default_factory=dict)
    free_surface: bool = False      # p = 0 on the plane k = 0 (odd image), no top layer
    cpml: bool = False              # the nbl-cell layers are a CPML instead of damping layers
    cpml_f0: float = 0.0            # CPML frequency shift (Hz)
    rho: np.ndarray | None = None   # [nz][ny][nx] float32 kg/m^3: variable-density (staggered) system

    @property
    def shape(self):
        return self.vel.shape

    @property
    def npoints(self) -> int:
        nz, ny, nx = self.vel.shape
        return nx * ny * nz


def ricker(fpeak: float, dt: float, nt: int, t0: float | None = None) -> np.ndarray:
    """Unit-amplitude Ricker wavelet sampled at t_n = n dt, FP64 rounded to FP32.

    w(t) = (1 - 2 pi^2 f^2 tau^2) exp(-pi^2 f^2 tau^2),  tau = t - t0,
    t0 = 1.5 / f by default (so |w(0)| < 1e-8).
    """
    if t0 is None:
        t0 = 1.5 / fpeak
    t = np.arange(nt, dtype=np.float64) * dt - t0
    a = (np.pi * fpeak * t) ** 2
    return ((1.0 - 2.0 * a) * np.exp(-a)).astype(np.float32)


def cfl_dt(cfl: float, h, vmax: float) -> float:
    """dt = CFL * min(h) / vmax (the CFL reading used by the workloads)."""
    return float(cfl) * float(min(h)) / float(vmax)


def _smooth_noise(shape, sigma: float, seed: int, amp: float, dtype=np.float64) -> np.ndarray:
    """White N(0,1) noise, Gaussian-smoothed (sigma in cells), scaled to max |.| = amp.
    dtype sets the precision of the smoothing (FP32 for the large batched set)."""
    from scipy.ndimage import gaussian_filter
    rng = np.random.default_rng(seed)
    n = rng.standard_normal(shape).astype(dtype)
    s = gaussian_filter(n, sigma=sigma, mode="wrap")
    return (s * (amp / np.max(np.abs(s)))).astype(np.float64)


def surface_grid(nx: int, ny: int, k: int = 0, start: int = 0, stride: int = 1,
                 count_x: int | None = None, count_y: int | None = None) -> np.ndarray:
    """Receivers on a regular (i, j) grid in plane k, ordered j-major."""
    ii = np.arange(start, nx, stride)[: count_x]
    jj = np.arange(start, ny, stride)[: count_y]
    J, I = np.meshgrid(jj, ii, indexing="ij")
    out = np.stack([I.ravel(), J.ravel(), np.full(I.size, k)], axis=1)
    return out.astype(np.int32)


def small_homogeneous(nt: int = 100) -> Problem:
    """64^3, h = 10 m, v = 1500 m/s, dt = 1 ms, L = 8, Ricker 15 Hz at the grid
    centre, 16 receivers on a line at k = 4 (i = 2 + 4r, j = 32)."""
    n = 64
    vel = np.full((n, n, n), 1500.0, dtype=np.float32)
    dt = 1e-3
    rec = np.array([[2 + 4 * r, 32, 4] for r in range(16)], dtype=np.int32)
    return Problem("homogeneous-64^3", vel, (10.0, 10.0, 10.0), dt, nt, 8,
                   np.array([[32, 32, 32]], np.int32), ricker(15.0, dt, nt)[None, :], rec,
                   meta={"cfl": 1500.0 * dt / 10.0})


def layered_240(nt: int = 1000, n: int = 240) -> Problem:
    """240^3, h = 10 m, L = 20, four flat layers 1500/2200/3000/4500 m/s with
    interfaces at three sorted depths drawn by seed 1 in [L+10, nz-L-10],
    times (1 + delta), delta a seed-2 white field Gaussian-smoothed (sigma 4
    cells) scaled to max |delta| = 0.05.  dt from CFL 0.4 on the model maximum.
    Ricker 10 Hz at (n/2, n/2, 4); receivers on every (i, j) of plane k = 0."""
    L = 20
    rng = np.random.default_rng(1)
    depths = np.sort(rng.choice(np.arange(L + 10, n - L - 10 + 1), size=3, replace=False))
    layer_v = np.array([1500.0, 2200.0, 3000.0, 4500.0])
    kk = np.arange(n)
    vz = layer_v[np.searchsorted(depths, kk, side="right")]
    vel = np.broadcast_to(vz[:, None, None], (n, n, n)).astype(np.float64)
    vel = vel * (1.0 + _smooth_noise((n, n, n), 4.0, 2, 0.05))
    vel32 = vel.astype(np.float32)
    h = (10.0, 10.0, 10.0)
    dt = cfl_dt(0.4, h, float(vel32.max()))
    src = np.array([[n // 2, n // 2, 4]], np.int32)
    return Problem(f"layered-{n}^3", vel32, h, dt, nt, L, src, ricker(10.0, dt, nt)[None, :],
                   surface_grid(n, n, 0), meta={"cfl": 0.4, "interfaces": depths.tolist()})


def smooth_gradient_200(nt: int = 1000, n: int = 200, anomaly: bool = False) -> Problem:
    """200^3, h = 10 m, L = 20: background linear in depth 1500 -> 4000 m/s times
    (1 + seed-3 smoothed field, sigma 10, max 3%), clipped to [1500, 4000];
    with anomaly=True also times (1 + 0.1 G), G a unit Gaussian bump of sigma
    15 cells at the centre.  Ricker 10 Hz at (n/2, n/2, 4); 64 x 64 receivers at
    k = 0 with i, j = 4 + 3 r."""
    L = 20
    z = np.linspace(0.0, 1.0, n)
    base = 1500.0 + 2500.0 * z
    vel = np.broadcast_to(base[:, None, None], (n, n, n)).astype(np.float64)
    vel = np.clip(vel * (1.0 + _smooth_noise((n, n, n), 10.0, 3, 0.03)), 1500.0, 4000.0)
    if anomaly:
        c = (n - 1) / 2.0
        g = np.arange(n) - c
        r2 = g[:, None, None] ** 2 + g[None, :, None] ** 2 + g[None, None, :] ** 2
        vel = vel * (1.0 + 0.1 * np.exp(-r2 / (2.0 * 15.0 ** 2)))
    vel32 = vel.astype(np.float32)
    h = (10.0, 10.0, 10.0)
    dt = cfl_dt(0.4, h, 4000.0 * 1.1)
    src = np.array([[n // 2, n // 2, 4]], np.int32)
    rec = surface_grid(n, n, 0, start=4, stride=3, count_x=64, count_y=64)
    return Problem(f"gradient-{n}^3" + ("-anomaly" if anomaly else ""), vel32, h, dt, nt, L, src,
                   ricker(10.0, dt, nt)[None, :], rec, meta={"cfl": 0.4})


def batched_shots(nshots: int = 32, nt: int = 800, seed: int = 4) -> list:
    """Shots with uneven grids: nx, ny in U{128..320}, nz in U{128..256} (step 16),
    L = 20, per-shot 3-5 flat layers (seed 4+s) times a +-5% smoothed field
    (smoothing in FP32), Ricker f ~ U[8, 20] Hz at (nx/2, ny/2, 4), receivers
    at k = 0 with stride 4.  Sizes are drawn in order from seed; each shot's
    model only from its own seeds, so the shots are built in parallel."""
    from concurrent.futures import ThreadPoolExecutor
    rng = np.random.default_rng(seed)
    dims = []
    for s in range(nshots):
        nx = int(rng.choice(np.arange(128, 321, 16)))
        ny = int(rng.choice(np.arange(128, 321, 16)))
        nz = int(rng.choice(np.arange(128, 257, 16)))
        dims.append((nx, ny, nz, float(rng.uniform(8.0, 20.0))))

    def build(s):
        nx, ny, nz, f = dims[s]
        r2 = np.random.default_rng(seed + s)
        nl = int(r2.integers(3, 6))
        depths = np.sort(r2.choice(np.arange(30, nz - 30), size=nl - 1, replace=False))
        lv = np.sort(r2.uniform(1500.0, 4500.0, size=nl))
        vz = lv[np.searchsorted(depths, np.arange(nz), side="right")]
        pert = _smooth_noise((nz, ny, nx), 4.0, 1000 + seed + s, 0.05, dtype=np.float32)
        vel32 = (vz[:, None, None] * (1.0 + pert)).astype(np.float32)
        h = (10.0, 10.0, 10.0)
        dt = cfl_dt(0.4, h, float(vel32.max()))
        src = np.array([[nx // 2, ny // 2, 4]], np.int32)
        return Problem(f"shot{s}-{nx}x{ny}x{nz}", vel32, h, dt, nt, 20, src,
                       ricker(f, dt, nt)[None, :], surface_grid(nx, ny, 0, stride=4),
                       meta={"fpeak": f})

    with ThreadPoolExecutor(max_workers=8) as ex:
        return list(ex.map(build, range(nshots)))


def fractal_large(nt: int = 500, shape=(512, 1024, 1024), seed: int = 5, beta: float = 3.0) -> Problem:
    """1024 x 1024 x 512 (nx, ny, nz), h = 12.5 m, L = 32: a Gaussian random field
    with amplitude spectrum |k|^(-beta/2) (FP64 FFT, seed 5) mapped linearly to
    [1500, 5000] m/s.  dt from CFL 0.4.  Ricker 10 Hz at (nx/2, ny/2, 4);
    receivers on every (i, j) of plane k = 0."""
    import scipy.fft as sfft
    nz, ny, nx = shape
    rng = np.random.default_rng(seed)
    spec = sfft.rfftn(rng.standard_normal(shape), workers=-1)
    kz = np.fft.fftfreq(nz)[:, None, None]
    ky = np.fft.fftfreq(ny)[None, :, None]
    kx = np.fft.rfftfreq(nx)[None, None, :]
    kk2 = kz * kz + ky * ky + kx * kx
    kk2[0, 0, 0] = np.inf
    spec *= kk2 ** (-beta / 4.0)          # |k|^(-beta/2)
    del kk2
    f = sfft.irfftn(spec, s=shape, workers=-1)
    del spec
    lo, hi = f.min(), f.max()
    vel32 = (1500.0 + 3500.0 * ((f - lo) / (hi - lo))).astype(np.float32)
    h = (12.5, 12.5, 12.5)
    dt = cfl_dt(0.4, h, 5000.0)
    src = np.array([[nx // 2, ny // 2, 4]], np.int32)
    return Problem(f"fractal-{nx}x{ny}x{nz}", vel32, h, dt, nt, 32, src,
                   ricker(10.0, dt, nt)[None, :], surface_grid(nx, ny, 0), meta={"cfl": 0.4})


def tiny_problem(shape=(11, 10, 12), nt: int = 30, nbl: int = 2, seed: int = 7,
                 h=(10.0, 11.0, 12.0), nsrc: int = 2, nrec: int = 5) -> Problem:
    """Small heterogeneous problem for brute-force checks: v ~ U[1500, 3000]
    per cell (seed), sources and receivers at seeded grid points."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    vel = rng.uniform(1500.0, 3000.0, size=shape).astype(np.float32)
    dt = cfl_dt(0.3, h, 3000.0)
    src = np.stack([rng.integers(0, nx, nsrc), rng.integers(0, ny, nsrc), rng.integers(0, nz, nsrc)], 1)
    rec = np.stack([rng.integers(0, nx, nrec), rng.integers(0, ny, nrec), rng.integers(0, nz, nrec)], 1)
    w = np.stack([ricker(f, dt, nt) for f in rng.uniform(20.0, 40.0, nsrc)]) if nsrc else np.zeros((0, nt), np.float32)
    return Problem(f"tiny-{nx}x{ny}x{nz}", vel, tuple(h), dt, nt, nbl, src.astype(np.int32),
                   w.astype(np.float32), rec.astype(np.int32))


def gardner_density(vel: np.ndarray, seed: int, amp: float = 0.03, sigma: float = 4.0) -> np.ndarray:
    """Density from velocity by Gardner's empirical rule rho = 310 v^0.25
    (kg/m^3, v in m/s; 1930 kg/m^3 at 1500 m/s, 2540 at 4500), times
    (1 + delta), delta a seeded white field Gaussian-smoothed (sigma cells)
    scaled to max |delta| = amp, so density is not a function of velocity.
    FP64, rounded once to FP32."""
    v = vel.astype(np.float64)
    rho = 310.0 * v ** 0.25 * (1.0 + _smooth_noise(vel.shape, sigma, seed, amp))
    return rho.astype(np.float32)


def layered_240_vd(nt: int = 1000, n: int = 240) -> Problem:
    """The layered 240^3 workload with density: Gardner's rule on its velocity
    times a seed-6 smoothed +-3 % field; dt from CFL 0.4 on the model maximum."""
    p = layered_240(nt, n)
    p.rho = gardner_density(p.vel, 6)
    p.name = f"layered-vd-{n}^3"
    return p


def tiny_problem_vd(shape=(11, 10, 12), nt: int = 30, nbl: int = 2, seed: int = 7,
                    h=(10.0, 11.0, 12.0), nsrc: int = 2, nrec: int = 5) -> Problem:
    """tiny_problem with a density drawn per cell from U[1000, 2600] (seed + 1000)."""
    p = tiny_problem(shape, nt, nbl, seed, h, nsrc, nrec)
    rng = np.random.default_rng(seed + 1000)
    p.rho = rng.uniform(1000.0, 2600.0, size=shape).astype(np.float32)
    p.name = p.name.replace("tiny", "tiny-vd")
    return p


def layered_vd_plain(nt: int = 100, n: int = 512) -> Problem:
    """n^3, h = 10 m, L = 20: the four flat layers of layered_240 (interfaces
    drawn by seed 1 in [L+10, n-L-10]) without the smoothed perturbations,
    density by Gardner's rule without perturbation (cheap to build at large
    n).  dt from CFL 0.4; Ricker 10 Hz at (n/2, n/2, 4); receivers on every
    (i, j) of plane k = 0 with stride 4."""
    L = 20
    rng = np.random.default_rng(1)
    depths = np.sort(rng.choice(np.arange(L + 10, n - L - 10 + 1), size=3, replace=False))
    layer_v = np.array([1500.0, 2200.0, 3000.0, 4500.0])
    vz = layer_v[np.searchsorted(depths, np.arange(n), side="right")]
    vel32 = np.ascontiguousarray(np.broadcast_to(vz[:, None, None].astype(np.float32), (n, n, n)))
    rz = (310.0 * vz ** 0.25).astype(np.float32)
    rho32 = np.ascontiguousarray(np.broadcast_to(rz[:, None, None], (n, n, n)))
    h = (10.0, 10.0, 10.0)
    dt = cfl_dt(0.4, h, 4500.0)
    src = np.array([[n // 2, n // 2, 4]], np.int32)
    return Problem(f"layered-vd-plain-{n}^3", vel32, h, dt, nt, L, src, ricker(10.0, dt, nt)[None, :],
                   surface_grid(n, n, 0, stride=4), rho=rho32, meta={"cfl": 0.4, "interfaces": depths.tolist()})
