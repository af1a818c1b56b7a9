"""GPU (FP32, C ABI) against the FP64 oracle.

Gates from the propagator's accuracy target: relative L2 error of the
wavefield and of the traces <= 1e-5 after 100 steps and <= 1e-4 after 1000.
Relative L2 = ||gpu - oracle||_2 / ||oracle||_2 over the whole array, in FP64.
Where the 100-step traces hold only numerical precursors (the 64^3 case:
the first arrival reaches the receivers after step 280), their error is
reported relative to max|u| * sqrt(#samples) instead ("below floor").
"""
import numpy as np
import pytest

import paper_2007_06048_gb300 as M
import workloads as W
from _gpu_util import rel_l2, run_gpu, run_oracle, torch_cuda

pytestmark = pytest.mark.gpu


def test_homogeneous_64_100_steps(orc):
    p = W.small_homogeneous(100)
    tr_o, _, u_o = run_oracle(orc, p)
    tr_g, u_g, prop = run_gpu(p)
    assert rel_l2(u_g, u_o) <= 1e-5
    floor = np.abs(u_o).max() * np.sqrt(tr_o.size)
    assert np.linalg.norm(tr_g - tr_o) / floor <= 1e-5
    assert prop.launches >= p.nt


def test_homogeneous_64_1000_steps(orc):
    p = W.small_homogeneous(1000)
    tr_o, _, u_o = run_oracle(orc, p)
    tr_g, u_g, _ = run_gpu(p)
    assert rel_l2(u_g, u_o) <= 1e-4
    assert rel_l2(tr_g, tr_o) <= 1e-4


def test_layered_240_100_steps(orc):
    p = W.layered_240(100)
    tr_o, _, u_o = run_oracle(orc, p)
    tr_g, u_g, _ = run_gpu(p)
    assert rel_l2(u_g, u_o) <= 1e-5
    assert rel_l2(tr_g, tr_o) <= 1e-5


def test_layered_240_1000_steps_full_size(orc):
    """The benchmarked workload itself: 240^3, 1000 steps, 57 600 receivers."""
    p = W.layered_240(1000)
    tr_o, _, u_o = run_oracle(orc, p)
    tr_g, u_g, _ = run_gpu(p)
    assert rel_l2(u_g, u_o) <= 1e-4
    assert rel_l2(tr_g, tr_o) <= 1e-4


# ragged tiles and z ranges, one-point and one-wide grids, and layers that fill
# an axis (2 nbl = n: no inner point along z)
SHAPES = [((9, 9, 9), 0), ((13, 17, 35), 2), ((70, 33, 65), 5), ((5, 40, 3), 1), ((1, 1, 1), 0),
          ((2, 67, 129), 0), ((40, 1, 30), 0), ((37, 45, 131), 9), ((8, 10, 12), 4)]


@pytest.mark.parametrize("shape,nbl", SHAPES, ids=[f"{s}-L{n}" for s, n in SHAPES])
def test_ragged_and_degenerate_shapes(orc, shape, nbl):
    nz, ny, nx = shape
    p = W.tiny_problem(shape=shape, nt=40, nbl=nbl, nsrc=3, nrec=9, seed=nx * 7 + ny * 3 + nz)
    corners = [[0, 0, 0], [nx - 1, ny - 1, nz - 1], [nx - 1, 0, nz - 1], [0, ny - 1, 0]]
    p.src_ijk[0] = corners[1]
    p.src_ijk[1] = p.src_ijk[2]          # two sources on one point add up
    p.rec_ijk[:4] = corners
    p.rec_ijk[4] = p.rec_ijk[5]          # duplicated receiver
    p.rec_ijk[6] = p.src_ijk[0]
    tr_o, _, u_o = run_oracle(orc, p)
    tr_g, u_g, _ = run_gpu(p)
    assert rel_l2(u_g, u_o) <= 1e-5
    assert rel_l2(tr_g, tr_o) <= 1e-5
    assert np.array_equal(tr_g[:, 4], tr_g[:, 5])


def test_zero_steps_and_no_sources_or_receivers(orc):
    torch = torch_cuda()
    p = W.tiny_problem(shape=(12, 11, 10), nt=0, nbl=2, nsrc=0, nrec=0)
    prop = M.Propagator.from_problem(p)
    prop.set_model(torch.from_numpy(p.vel).cuda())
    fin = torch.full(p.vel.shape, 7.0, device="cuda")
    prop.forward(None, None, fin)
    torch.cuda.synchronize()
    assert torch.count_nonzero(fin).item() == 0
    q = W.tiny_problem(shape=(12, 11, 10), nt=20, nbl=2, nsrc=0, nrec=3)
    tr, u, _ = run_gpu(q)
    assert not np.any(tr) and not np.any(u)


def test_host_buffers_match_device_buffers():
    """The end-to-end path: host numpy arrays in and out through the same ABI."""
    torch = torch_cuda()
    p = W.tiny_problem(shape=(30, 28, 70), nt=60, nbl=4, nsrc=2, nrec=11, seed=3)
    tr_d, u_d, _ = run_gpu(p)
    prop = M.Propagator.from_problem(p)
    prop.set_model(np.ascontiguousarray(p.vel))
    tr_h = np.zeros((p.nt, len(p.rec_ijk)), np.float32)
    u_h = np.zeros(p.vel.shape, np.float32)
    prop.forward(np.ascontiguousarray(p.wavelet), tr_h, u_h)
    assert np.array_equal(tr_h, tr_d)
    assert np.array_equal(u_h, u_d)
    pinned_tr = torch.zeros((p.nt, len(p.rec_ijk)), pin_memory=True)
    prop.forward(torch.from_numpy(np.ascontiguousarray(p.wavelet)).pin_memory(), pinned_tr, None)
    assert np.array_equal(pinned_tr.numpy(), tr_d)


@pytest.mark.parametrize("nt", [1, 3, 8, 61])
@pytest.mark.parametrize("kernel", ["tma", "simple", "cpml"])
def test_host_traces_download_in_chunks(nt, kernel):
    """Host traces come down in row chunks while the loop runs (each chunk
    after the step that makes its rows final): every row equals the
    device-buffer run's, for step counts below, at and above the chunk
    count, with both step kernels and with CPML layers."""
    p = W.tiny_problem(shape=(40, 36, 70), nt=nt, nbl=5, nsrc=2, nrec=13, seed=21)
    if kernel == "cpml":
        p.cpml, p.cpml_f0 = True, 12.0
    kern = M.KERNEL_SIMPLE if kernel == "simple" else M.KERNEL_AUTO
    tr_d, _, _ = run_gpu(p, kernel=kern, want_final=False)
    prop = M.Propagator.from_problem(p)
    if kern != M.KERNEL_AUTO:
        prop.set_kernel(kern)
    prop.set_model(np.ascontiguousarray(p.vel))
    for _ in range(2):   # the second call replays the cached graph
        tr_h = np.full((p.nt, len(p.rec_ijk)), np.nan, np.float32)
        prop.forward(np.ascontiguousarray(p.wavelet), tr_h, None)
        assert np.array_equal(tr_h, tr_d)
    prop.close()


def test_standing_wave_fp32():
    """The exact discrete standing wave of Eq. 5 (see the oracle pins), now in
    FP32 on the GPU through set_state / get_state: relative error ~ FP32 eps."""
    shape = (48, 44, 52)
    h = (10.0, 12.0, 9.0)
    v, dt = 2000.0, 0.9e-3
    k = np.array([2 * np.pi / 97.0, 2 * np.pi / 61.0, 2 * np.pi / 143.0])
    nz, ny, nx = shape
    Z, Y, X = np.meshgrid(np.arange(nz) * h[2], np.arange(ny) * h[1], np.arange(nx) * h[0], indexing="ij")
    phi = np.cos(k[0] * X + 0.3) * np.cos(k[1] * Y + 1.1) * np.cos(k[2] * Z - 0.4)
    c = [8 / 5, -1 / 5, 8 / 315, -1 / 560]
    K = sum(4 * c[m - 1] * np.sin(m * k[a] * h[a] / 2) ** 2 / h[a] ** 2 for a in range(3) for m in range(1, 5))
    cwdt = 1 - dt * dt * v * v * K / 2
    nt = 5
    p = W.Problem("standing", np.full(shape, v, np.float32), h, dt, nt, 0, np.zeros((0, 3), np.int32),
                  np.zeros((0, nt), np.float32), np.zeros((0, 3), np.int32))
    _, u, _, (up, uc) = run_gpu(p, state=(cwdt * phi, phi), want_state=True)
    m = 4 * nt
    inner = (slice(m, -m),) * 3
    expect = np.cos(nt * np.arccos(cwdt)) * phi
    assert np.array_equal(u, uc)
    assert np.max(np.abs(u[inner] - expect[inner])) < 2e-5


# P = sum of coef * s^a t^b r^c over centred coordinates s = (i - i_c) / 3
# (t, r alike; off-grid centres): degree up to 8 along each axis, where Sec.
# 3's order-8 second difference is exact (it is exact up to degree 9)
_POLY = [(1.0, 8, 0, 0), (-0.7, 0, 8, 0), (0.4, 0, 0, 8), (1.3, 3, 2, 3), (-0.5, 5, 0, 4), (0.9, 2, 6, 0),
         (0.6, 7, 1, 1), (-0.8, 1, 1, 7), (0.2, 0, 0, 0)]
_TAYLOR8 = (8 / 5, -1 / 5, 8 / 315, -1 / 560)


def _poly_and_laplacian(shape, h, scale=3.0):
    nz, ny, nx = shape
    S = (scale * h[0], scale * h[1], scale * h[2])
    Z, Y, X = np.meshgrid((np.arange(nz) - (nz - 1) / 2 + 0.37) / scale, (np.arange(ny) - (ny - 1) / 2 - 0.21) / scale,
                          (np.arange(nx) - (nx - 1) / 2 + 0.13) / scale, indexing="ij")
    P = np.zeros(shape)
    lap = np.zeros(shape)
    for coef, a, b, c in _POLY:
        P += coef * X ** a * Y ** b * Z ** c
        if a >= 2:
            lap += coef * a * (a - 1) * X ** (a - 2) * Y ** b * Z ** c / S[0] ** 2
        if b >= 2:
            lap += coef * b * (b - 1) * X ** a * Y ** (b - 2) * Z ** c / S[1] ** 2
        if c >= 2:
            lap += coef * c * (c - 1) * X ** a * Y ** b * Z ** (c - 2) / S[2] ** 2
    return P, lap


def _pair_rounding_bound(U, h):
    """2^-24 times the sum over the stencil's pairs of |w| (|u(+m)| + |u(-m)| +
    2|u|): the size of one FP32 rounding of every pair term, per point."""
    U = np.abs(U.astype(np.float64))
    out = np.zeros(U.shape)
    for ax, hh in zip((2, 1, 0), h):
        for m in range(1, 5):
            out += abs(_TAYLOR8[m - 1]) / hh ** 2 * (np.roll(U, -m, axis=ax) + np.roll(U, m, axis=ax) + 2 * U)
    return out * 2.0 ** -24


@pytest.mark.parametrize("kernel", [M.KERNEL_TMA, M.KERNEL_SIMPLE])
def test_polynomial_laplacian_fp32(kernel):
    """The polynomial pin on the GPU: with u^{-1} = 2 u^0 = 2P (exact in FP32)
    one undamped step leaves u^1 = c * L_h P, and L_h is exact on P (degree
    <= 8 per axis; unequal spacings, heterogeneous velocity) at every point 4
    cells inside the grid.  Per point the difference from c * Laplacian(P)
    stays within 8 FP32 roundings of the stencil's pair terms (plus the
    rounding of the product): an order-6 stencil, a dropped m = 4 pair or a
    1 % error in its weight exceed that bound by factors of 10^3 to 10^5."""
    shape, h, dt = (40, 36, 44), (9.0, 12.0, 10.0), 1.0e-3
    rng = np.random.default_rng(31)
    vel = rng.uniform(1500.0, 3000.0, shape).astype(np.float32)
    P, lap = _poly_and_laplacian(shape, h)
    P32 = P.astype(np.float32)
    p = W.Problem("poly", vel, h, dt, 1, 0, np.zeros((0, 3), np.int32), np.zeros((0, 1), np.float32),
                  np.zeros((0, 3), np.int32))
    _, u1, _ = run_gpu(p, kernel=kernel, state=(2 * P32, P32))
    c = (dt * dt) * vel.astype(np.float64) ** 2
    inner = (slice(4, -4),) * 3
    err = np.abs(u1.astype(np.float64) - c * lap)[inner]
    bound = (8 * c * _pair_rounding_bound(P32, h) + 2.0 ** -22 * np.abs(c * lap))[inner]
    assert np.all(err <= bound), float(np.max(err / bound))


def test_error_paths():
    torch = torch_cuda()
    p = W.tiny_problem(shape=(16, 16, 16), nt=10, nbl=2)
    prop = M.Propagator.from_problem(p)
    wav = torch.from_numpy(p.wavelet).cuda()
    tr = torch.zeros((p.nt, len(p.rec_ijk)), device="cuda")
    with pytest.raises(M.MmodError) as ei:
        prop.forward(wav, tr)
    assert ei.value.status == -6                      # no model yet
    bad = p.vel.copy()
    bad[3, 4, 5] = -1.0
    with pytest.raises(M.MmodError) as ei:
        prop.set_model(torch.from_numpy(bad).cuda())
    assert ei.value.status == -1
    bad[3, 4, 5] = np.nan
    with pytest.raises(M.MmodError) as ei:
        prop.set_model(torch.from_numpy(bad).cuda())
    assert ei.value.status == -1
    fast = (p.vel * 10).astype(np.float32)            # breaks the CFL bound
    with pytest.raises(M.MmodError) as ei:
        prop.set_model(torch.from_numpy(fast).cuda())
    assert ei.value.status == -2
    prop.set_model(torch.from_numpy(p.vel).cuda())
    prop.forward(wav, tr)
    with pytest.raises(M.MmodError):
        prop.set_kernel(99)
    torch.cuda.synchronize()


def test_damping_reciprocal_within_one_ulp():
    """The step kernels' 1/(1+e) (approximate reciprocal + one Newton-Raphson
    step) stays within 1 ulp of CUDA's correctly rounded reciprocal."""
    torch_cuda()
    assert M.mmod_check_recip(1 << 22) <= 1


BITWISE = SHAPES + [((64, 64, 64), 8), ((240, 240, 240), 20), ((200, 130, 97), 12)]


@pytest.mark.parametrize("shape,nbl", BITWISE, ids=[f"{s}-L{n}" for s, n in BITWISE])
def test_tma_kernel_is_bitwise_the_plain_kernel(shape, nbl):
    """The pipelined kernel performs the plain kernel's FP32 operations in the
    same order: final wavefield and traces agree bit for bit."""
    nz, ny, nx = shape
    if shape == (240, 240, 240):
        p = W.layered_240(1000)
    else:
        p = W.tiny_problem(shape=shape, nt=50, nbl=nbl, nsrc=3, nrec=17, seed=nx + ny + nz)
        p.src_ijk[0] = [nx - 1, 0, nz // 2]
    tr_s, u_s, _ = run_gpu(p, kernel=M.KERNEL_SIMPLE)
    for v in range(M.mmod_tma_variant_count()):
        tr_t, u_t, prop = run_gpu(p, kernel=M.KERNEL_TMA, variant=v)
        assert np.array_equal(u_s, u_t), M.mmod_tma_variant_name(v)
        assert np.array_equal(tr_s, tr_t), M.mmod_tma_variant_name(v)
    for pdl in (0, 1):   # programmatic dependent launch off / on
        tr_o, u_o, _ = run_gpu(p, kernel=M.KERNEL_TMA, pdl=pdl)
        assert np.array_equal(u_s, u_o), pdl
        assert np.array_equal(tr_s, tr_o), pdl
    # one step kernel per time step plus the final receiver gather and the unpack
    assert prop.launches == p.nt + 2
    assert prop.loop_ms() > 0
