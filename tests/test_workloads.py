"""The seeded synthetic inputs: each generator produces the sizes, value
ranges, acquisition geometry and wavelet its recipe states, and the same
arrays on every call (CPU only; no oracle arithmetic involved)."""
import numpy as np
import pytest

import workloads as W


def test_ricker_peak_onset_and_spectrum():
    f, dt = 10.0, 1e-3
    w = W.ricker(f, dt, 4096).astype(np.float64)
    assert abs(w[150] - 1.0) < 1e-7                               # t0 = 1.5 / f = 150 samples
    assert np.argmax(w) == 150
    assert abs(w[0]) < 1e-8                                       # negligible onset
    spec = np.abs(np.fft.rfft(w))
    freqs = np.fft.rfftfreq(w.size, dt)
    assert abs(freqs[np.argmax(spec)] - f) <= freqs[1]            # peak frequency f
    assert abs(np.sum(w)) * dt < 1e-6                             # zero mean (no DC)


def test_cfl_dt():
    assert W.cfl_dt(0.4, (10.0, 12.0, 9.0), 4500.0) == pytest.approx(0.4 * 9.0 / 4500.0)


def test_small_homogeneous():
    p = W.small_homogeneous(100)
    assert p.shape == (64, 64, 64) and np.all(p.vel == 1500.0)
    assert p.h == (10.0, 10.0, 10.0) and p.dt == 1e-3 and p.nbl == 8 and p.nt == 100
    assert p.src_ijk.tolist() == [[32, 32, 32]]
    assert p.rec_ijk.tolist() == [[2 + 4 * r, 32, 4] for r in range(16)]
    assert p.wavelet.shape == (1, 100) and np.array_equal(p.wavelet[0], W.ricker(15.0, 1e-3, 100))


def test_layered_240():
    p = W.layered_240(20)
    q = W.layered_240(20)
    assert np.array_equal(p.vel, q.vel) and p.dt == q.dt           # seeded
    n, L = 240, 20
    assert p.shape == (n, n, n) and p.vel.dtype == np.float32 and p.nbl == L
    depths = p.meta["interfaces"]
    assert len(depths) == 3 and depths == sorted(set(depths))
    assert all(L + 10 <= d <= n - L - 10 for d in depths)
    layer_v = np.array([1500.0, 2200.0, 3000.0, 4500.0])
    vz = layer_v[np.searchsorted(depths, np.arange(n), side="right")]
    ratio = p.vel.astype(np.float64) / vz[:, None, None] - 1.0
    assert np.max(np.abs(ratio)) == pytest.approx(0.05, abs=1e-6)   # smoothed field scaled to 5 %
    assert p.dt == pytest.approx(0.4 * 10.0 / float(p.vel.max()))
    assert p.src_ijk.tolist() == [[120, 120, 4]]
    assert p.rec_ijk.shape == (n * n, 3) and np.all(p.rec_ijk[:, 2] == 0)
    assert len({(i, j) for i, j, _ in p.rec_ijk.tolist()}) == n * n


def test_smooth_gradient_200():
    p = W.smooth_gradient_200(10)
    n = 200
    assert p.shape == (n, n, n) and p.nbl == 20
    assert p.vel.min() >= 1500.0 and p.vel.max() <= 4000.0
    # the depth trend: plane means rise from ~1500 to ~4000 m/s
    means = p.vel.mean(axis=(1, 2))
    assert means[0] < 1600.0 and means[-1] > 3800.0 and np.all(np.diff(means[5:-5]) > 0)
    grid = 4 + 3 * np.arange(64)
    assert p.rec_ijk.shape == (64 * 64, 3) and np.all(p.rec_ijk[:, 2] == 0)
    assert set(p.rec_ijk[:, 0].tolist()) == set(grid.tolist()) == set(p.rec_ijk[:, 1].tolist())
    a = W.smooth_gradient_200(10, n=64, anomaly=True)
    b = W.smooth_gradient_200(10, n=64)
    c = 31
    assert a.vel[c, c, c] / b.vel[c, c, c] == pytest.approx(1.1, rel=2e-3)   # centred 10 % bump


def test_batched_shots():
    shots = W.batched_shots(nshots=6, nt=12)
    again = W.batched_shots(nshots=6, nt=12)
    for p, q in zip(shots, again):
        assert np.array_equal(p.vel, q.vel)
    for p in shots:
        nz, ny, nx = p.shape
        assert 128 <= nx <= 320 and 128 <= ny <= 320 and 128 <= nz <= 256
        assert nx % 16 == 0 and ny % 16 == 0 and nz % 16 == 0
        assert p.nbl == 20 and p.nt == 12
        assert 8.0 <= p.meta["fpeak"] <= 20.0
        assert 1500.0 * 0.95 - 1e-3 <= p.vel.min() and p.vel.max() <= 4500.0 * 1.05 + 1e-3
        assert p.src_ijk.tolist() == [[nx // 2, ny // 2, 4]]
        assert np.all(p.rec_ijk[:, 2] == 0) and np.all(p.rec_ijk[:, :2] % 4 == 0)
        assert p.dt == pytest.approx(0.4 * 10.0 / float(p.vel.max()))


def test_fractal_large_recipe_on_a_small_grid():
    p = W.fractal_large(nt=5, shape=(24, 32, 40))
    q = W.fractal_large(nt=5, shape=(24, 32, 40))
    assert np.array_equal(p.vel, q.vel)
    assert p.vel.min() == pytest.approx(1500.0) and p.vel.max() == pytest.approx(5000.0)
    assert p.h == (12.5, 12.5, 12.5) and p.nbl == 32 and p.dt == pytest.approx(0.4 * 12.5 / 5000.0)
    # a red spectrum: most of the variance in the lowest wavenumbers
    f = p.vel.astype(np.float64) - p.vel.mean()
    power = np.abs(np.fft.fftn(f)) ** 2
    k = np.sqrt(sum(np.meshgrid(*[np.fft.fftfreq(n) ** 2 for n in f.shape], indexing="ij")))
    assert power[(k > 0) & (k < 0.1)].sum() > power[k >= 0.25].sum()


def test_gardner_density():
    rng = np.random.default_rng(0)
    vel = rng.uniform(1500.0, 4500.0, (20, 22, 24)).astype(np.float32)
    rho = W.gardner_density(vel, 6)
    base = 310.0 * vel.astype(np.float64) ** 0.25
    dev = rho / base - 1.0
    assert np.max(np.abs(dev)) == pytest.approx(0.03, abs=1e-6)
    assert 310.0 * 1500.0 ** 0.25 == pytest.approx(1930.0, rel=1e-3)
    p = W.layered_vd_plain(nt=5, n=80)
    assert np.allclose(p.rho, 310.0 * p.vel.astype(np.float64) ** 0.25, rtol=1e-6)
