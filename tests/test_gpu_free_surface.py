"""Free surface (p = 0 on k = 0 through the odd image; no top layer) on the
GPU against the FP64 oracle, and bit for bit across the library's kernels.

Tolerances as for the damped forward: relative L2 <= 1e-5 after 100 steps
and <= 1e-4 after 1000 (FP32 stepping against FP64).  Traces far from every
source hold only numerical precursors early on, so their error is measured
against the larger of their own norm and max|u| * sqrt(#samples) (the
wavefield scale, as for the 100-step homogeneous case).
"""
import numpy as np
import pytest

import paper_2007_06048_gb300 as M
import workloads as W
from _gpu_util import rel_l2, run_gpu, run_oracle, torch_cuda

pytestmark = pytest.mark.gpu


def _fs(p):
    p.free_surface = True
    return p


def trace_err(tr_g, tr_o, u_o):
    floor = np.abs(u_o).max() * np.sqrt(tr_o.size)
    return float(np.linalg.norm(tr_g.astype(np.float64) - tr_o) / max(np.linalg.norm(tr_o), floor))


SHAPES = [((40, 36, 70), 4), ((5, 40, 33), 1), ((33, 64, 131), 6), ((9, 20, 9), 0), ((70, 17, 65), 8)]


@pytest.mark.parametrize("shape,nbl", SHAPES, ids=[f"{s}-L{n}" for s, n in SHAPES])
def test_free_surface_matches_oracle(orc, shape, nbl):
    nz, ny, nx = shape
    p = _fs(W.tiny_problem(shape=shape, nt=100, nbl=nbl, nsrc=3, nrec=12, seed=sum(shape) + nbl))
    p.src_ijk[0] = [nx // 2, ny // 2, 0]       # on the surface: injects nothing
    p.src_ijk[1] = [nx // 3, ny // 3, 1]       # just below it
    p.rec_ijk[0] = [nx // 2, ny // 2, 0]       # reads 0
    p.rec_ijk[1] = [nx // 2, ny // 2, 1]
    p.rec_ijk[2] = [nx - 1, 0, min(3, nz - 1)]
    tr_o, _, u_o = run_oracle(orc, p)
    tr_g, u_g, _ = run_gpu(p)
    assert rel_l2(u_g, u_o) <= 1e-5
    assert trace_err(tr_g, tr_o, u_o) <= 1e-5
    assert not np.any(u_g[0]) and not np.any(tr_g[:, 0])


def test_free_surface_layered_240_1000_steps(orc):
    """The benchmarked model with a free surface: receivers one plane under it."""
    p = _fs(W.layered_240(1000))
    p.rec_ijk[:, 2] = 1
    tr_o, _, u_o = run_oracle(orc, p)
    tr_g, u_g, _ = run_gpu(p)
    assert rel_l2(u_g, u_o) <= 1e-4
    assert rel_l2(tr_g, tr_o) <= 1e-4


def test_free_surface_kernels_and_variants_bitwise():
    p = _fs(W.tiny_problem(shape=(60, 50, 90), nt=40, nbl=5, nsrc=2, nrec=20, seed=3))
    p.src_ijk[0] = [40, 20, 2]
    tr_s, u_s, _ = run_gpu(p, kernel=M.KERNEL_SIMPLE)
    for v in range(M.mmod_tma_variant_count()):
        tr_t, u_t, _ = run_gpu(p, kernel=M.KERNEL_TMA, variant=v)
        assert np.array_equal(u_t, u_s) and np.array_equal(tr_t, tr_s), v


def test_free_surface_persistent_and_zlen_bitwise():
    torch = torch_cuda()
    p = _fs(W.tiny_problem(shape=(97, 40, 70), nt=30, nbl=4, nsrc=2, nrec=25, seed=4))
    tr_s, u_s, _ = run_gpu(p)
    for persistent, zlen in ((1, 0), (0, 3), (1, 5), (0, 97)):
        prop = M.Propagator.from_problem(p)
        prop.set_option(M.OPT_PERSISTENT, persistent)
        prop.set_option(M.OPT_ZLEN, zlen)
        prop.set_model(torch.from_numpy(p.vel).cuda())
        wav = torch.from_numpy(p.wavelet).cuda()
        tr = torch.zeros((p.nt, len(p.rec_ijk)), device="cuda")
        fin = torch.zeros(p.vel.shape, device="cuda")
        prop.forward(wav, tr, fin)
        torch.cuda.synchronize()
        assert np.array_equal(tr.cpu().numpy(), tr_s), (persistent, zlen)
        assert np.array_equal(fin.cpu().numpy(), u_s), (persistent, zlen)
        prop.close()


def test_free_surface_standing_sine_wave_fp32():
    """sin(kz z) cos cos is an exact discrete eigenfunction up to the surface:
    the FP32 run follows cos(n w dt) phi to FP32 accuracy there too."""
    shape, h, v, dt, nt = (48, 44, 52), (10.0, 12.0, 9.0), 2000.0, 0.9e-3, 5
    k = np.array([2 * np.pi / 97.0, 2 * np.pi / 61.0, 2 * np.pi / 143.0])
    nz, ny, nx = shape
    Z, Y, X = np.meshgrid(np.arange(nz) * h[2], np.arange(ny) * h[1], np.arange(nx) * h[0], indexing="ij")
    phi = np.cos(k[0] * X + 0.3) * np.cos(k[1] * Y + 1.1) * np.sin(k[2] * Z)
    c = [8 / 5, -1 / 5, 8 / 315, -1 / 560]
    K = sum(4 * c[m - 1] * np.sin(m * k[a] * h[a] / 2) ** 2 / h[a] ** 2 for a in range(3) for m in range(1, 5))
    cwdt = 1 - dt * dt * v * v * K / 2
    p = W.Problem("standing-fs", np.full(shape, v, np.float32), h, dt, nt, 0, np.zeros((0, 3), np.int32),
                  np.zeros((0, nt), np.float32), np.zeros((0, 3), np.int32), free_surface=True)
    _, u, _ = run_gpu(p, state=(cwdt * phi, phi))
    m = 4 * nt
    region = (slice(0, -m), slice(m, -m), slice(m, -m))
    expect = np.cos(nt * np.arccos(cwdt)) * phi
    assert np.max(np.abs(u[region] - expect[region])) < 2e-5
    assert not np.any(u[0])


def test_free_surface_adjoint_and_gradient(orc):
    torch = torch_cuda()
    p = _fs(W.tiny_problem(shape=(24, 26, 70), nt=80, nbl=4, nsrc=2, nrec=30, seed=13))
    p.rec_ijk[:10] = [[3 + 6 * r, 13, r % 2] for r in range(10)]   # receivers at and under the surface
    rng = np.random.default_rng(3)
    resid = rng.standard_normal((p.nt, len(p.rec_ijk))).astype(np.float32)
    prop = M.Propagator.from_problem(p)
    prop.set_model(torch.from_numpy(p.vel).cuda())
    adj = torch.zeros((len(p.src_ijk), p.nt), device="cuda")
    prop.adjoint(torch.from_numpy(resid).cuda(), adj)
    a_o = orc.adjoint(p.vel, p.h, p.dt, p.nt, nbl=p.nbl, src_ijk=p.src_ijk, rec_ijk=p.rec_ijk, resid=resid,
                      free_surface=True)
    assert rel_l2(adj.cpu().numpy(), a_o) <= 1e-5
    g = torch.zeros(p.vel.shape, device="cuda")
    prop.gradient(torch.from_numpy(p.wavelet).cuda(), torch.from_numpy(resid).cuda(), g, 8, M.CKPT_FP32)
    g_o = orc.gradient(p.vel, p.h, p.dt, p.nt, nbl=p.nbl, src_ijk=p.src_ijk, wavelet=p.wavelet,
                       rec_ijk=p.rec_ijk, resid=resid, free_surface=True)
    torch.cuda.synchronize()
    err = rel_l2(g.cpu().numpy(), g_o)
    print(f"free surface, FP32 checkpoints: gradient rel L2 vs FP64 oracle {err:.3e}")
    assert err <= 1e-5
    assert not np.any(g.cpu().numpy()[0])


def test_free_surface_batch_bitwise():
    torch = torch_cuda()
    shots = [_fs(W.tiny_problem(shape=s, nt=40, nbl=L, nsrc=2, nrec=15, seed=i + 60))
             for i, (s, L) in enumerate([((40, 36, 70), 4), ((33, 64, 128), 6), ((25, 90, 200), 8)])]
    singles = [run_gpu(p) for p in shots]
    for mode in (M.BATCH_STREAMS, M.BATCH_FUSED):
        props = [M.Propagator.from_problem(p) for p in shots]
        for pr, p in zip(props, shots):
            pr.set_model(torch.from_numpy(p.vel).cuda())
        b = M.Batch(props)
        b.set_mode(mode)
        tr = [torch.zeros((p.nt, len(p.rec_ijk)), device="cuda") for p in shots]
        b.forward([torch.from_numpy(p.wavelet).cuda() for p in shots], tr)
        torch.cuda.synchronize()
        for i in range(len(shots)):
            assert np.array_equal(tr[i].cpu().numpy(), singles[i][0]), (mode, i)
        b.close()


def test_free_surface_needs_five_planes():
    torch_cuda()
    with pytest.raises(M.MmodError) as ei:
        M.Propagator((4, 16, 16), (10.0, 10.0, 10.0), 1e-3, 5, free_surface=True)
    assert ei.value.status == -1
