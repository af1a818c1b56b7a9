"""mmod_forward_noalloc: the forward run for callers that may not allocate
device memory (a framework pool that accounts for every byte, a process that
reserves all device memory up front, real-time code that cannot afford an
allocation's synchronisation or failure).

It runs the same kernels as the handle API (mmod_create / mmod_set_model /
mmod_forward), so it must give the handle's bits, on consecutive calls that
share its fixed scratch block; it must match the FP64 oracle within the
forward parity gate (1e-5 after <= 100 steps); it must not change the
device's free memory; and it must refuse grids beyond its stated limit and
pointers the kernels cannot dereference with a clear error.
This file sorts last so that a run stopping at the first failure has already
run every other test.
"""
import numpy as np
import pytest

import paper_2007_06048_gb300 as M
import workloads as W
from _gpu_util import rel_l2, run_gpu, run_oracle, torch_cuda

pytestmark = pytest.mark.gpu

TOL = 1e-5   # the 100-step parity tolerance used by the other GPU tests


def _noalloc(p, torch):
    vel = torch.from_numpy(np.ascontiguousarray(p.vel)).cuda()
    wav = torch.from_numpy(np.ascontiguousarray(p.wavelet, np.float32)).cuda()
    tr = torch.full((p.nt, len(p.rec_ijk)), np.nan, device="cuda")
    fin = torch.full(p.vel.shape, np.nan, device="cuda")
    nz, ny, nx = p.vel.shape
    torch.cuda.synchronize()
    M.mmod_forward_noalloc(nx, ny, nz, p.h, p.dt, p.nt, vel, wav, tr, fin, nbl=p.nbl,
                           src_ijk=p.src_ijk, rec_ijk=p.rec_ijk, damp_R=p.refl, free_surface=p.free_surface)
    return tr.cpu().numpy(), fin.cpu().numpy()


def _case(shape, nt, nbl, fs=False, nrec=23, colocated=False):
    p = W.tiny_problem(shape=shape, nt=nt, nbl=nbl, nsrc=3, nrec=nrec, seed=sum(shape) + nrec)
    if fs:   # free surface, with a source and a receiver on its plane
        p.free_surface = True
        p.src_ijk[0] = [5, 6, 0]
        p.src_ijk[1:] = [[20, 10, 3], [40, 20, 12]]
        p.rec_ijk[0] = [7, 8, 0]
    if colocated:   # two sources at one point, one receiver on it
        p.src_ijk[2] = p.src_ijk[1]
        p.rec_ijk[1] = p.src_ijk[1]
    return p


CASES = [((30, 28, 70), 60, 4, False, 23, False), ((100, 96, 128), 100, 12, False, 23, False),
         ((30, 28, 70), 60, 4, True, 23, False), ((40, 64, 90), 50, 5, False, 1500, True)]


@pytest.mark.parametrize("shape,nt,nbl,fs,nrec,coloc", CASES)
def test_matches_handle_api_bitwise_on_two_calls(shape, nt, nbl, fs, nrec, coloc):
    torch = torch_cuda()
    p = _case(shape, nt, nbl, fs, nrec, coloc)
    tr_ref, u_ref, _ = run_gpu(p)
    assert np.abs(u_ref).max() > 0
    for _ in range(2):   # the second call reuses the block the first one left behind
        tr, u = _noalloc(p, torch)
        assert np.array_equal(u, u_ref)
        assert np.array_equal(tr, tr_ref)


@pytest.mark.parametrize("shape,nt,nbl,fs,nrec,coloc", CASES)
def test_matches_oracle(orc, shape, nt, nbl, fs, nrec, coloc):
    torch = torch_cuda()
    p = _case(shape, nt, nbl, fs, nrec, coloc)
    tr_o, _, u_o = run_oracle(orc, p)
    tr, u = _noalloc(p, torch)
    assert rel_l2(u, u_o) <= TOL
    assert rel_l2(tr, tr_o) <= TOL


def test_zero_steps_leaves_traces_and_gives_zero_state():
    torch = torch_cuda()
    p = _case((30, 28, 70), 0, 4)
    vel = torch.from_numpy(p.vel).cuda()
    tr = torch.full((1, len(p.rec_ijk)), 7.0, device="cuda")
    fin = torch.full(p.vel.shape, np.nan, device="cuda")
    nz, ny, nx = p.vel.shape
    M.mmod_forward_noalloc(nx, ny, nz, p.h, p.dt, 0, vel, None, tr, fin, nbl=p.nbl, src_ijk=p.src_ijk,
                           rec_ijk=p.rec_ijk)
    assert (tr.cpu().numpy() == 7.0).all()
    assert (fin.cpu().numpy() == 0.0).all()


def test_device_free_memory_unchanged():
    torch = torch_cuda()
    p = W.tiny_problem(shape=(40, 36, 70), nt=30, nbl=5, nsrc=2, nrec=9, seed=5)
    _noalloc(p, torch)                      # first call on the device: device code loaded
    vel = torch.from_numpy(p.vel).cuda()
    wav = torch.from_numpy(p.wavelet).cuda()
    tr = torch.zeros((p.nt, len(p.rec_ijk)), device="cuda")
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    nz, ny, nx = p.vel.shape
    for _ in range(3):
        M.mmod_forward_noalloc(nx, ny, nz, p.h, p.dt, p.nt, vel, wav, tr, None, nbl=p.nbl,
                               src_ijk=p.src_ijk, rec_ijk=p.rec_ijk)
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_rejects_grids_beyond_the_limit():
    torch = torch_cuda()
    nx = ny = nz = 160                      # 160 * 160 * 160 > 2^21 padded points
    vel = torch.full((nz, ny, nx), 2000.0, device="cuda")
    with pytest.raises(M.MmodError) as ei:
        M.mmod_forward_noalloc(nx, ny, nz, (10.0, 10.0, 10.0), 1e-3, 5, vel, None, None)
    assert ei.value.status == -1
    assert "allocation-free limits" in str(ei.value)


def test_rejects_host_memory():
    torch_cuda()
    vel = np.full((20, 20, 20), 2000.0, np.float32)   # host array: the kernels cannot read it
    with pytest.raises(M.MmodError) as ei:
        M.mmod_forward_noalloc(20, 20, 20, (10.0, 10.0, 10.0), 1e-3, 5, vel, None, None)
    assert ei.value.status == -1
    assert "memory of `device`" in str(ei.value)


def test_many_injection_buckets_within_the_limit():
    """nx = 513, ny = 1, nz = 3855 is inside the volume limit (544 x 3855 padded
    points) and has 9 x 3855 = 34695 injection buckets (x tile, plane); the
    entry point must accept it and give the handle API's bits."""
    torch = torch_cuda()
    nx, ny, nz, nt = 513, 1, 3855, 12
    p = W.Problem("buckets-513x1x3855", np.full((nz, ny, nx), 2000.0, np.float32), (10.0, 10.0, 10.0), 1e-3, nt,
                  0, np.array([[300, 0, 2000], [40, 0, 3800]], np.int32),
                  np.stack([W.ricker(25.0, 1e-3, nt), W.ricker(30.0, 1e-3, nt)]),
                  np.array([[301, 0, 2000], [40, 0, 3801], [512, 0, 3854]], np.int32))
    tr_ref, u_ref, _ = run_gpu(p)
    tr, u = _noalloc(p, torch)
    assert np.abs(tr_ref).max() > 0
    assert np.array_equal(tr, tr_ref) and np.array_equal(u, u_ref)
