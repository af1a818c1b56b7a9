"""mmod_forward_noalloc: the forward run for callers that may not allocate
device memory (a framework pool that accounts for every byte, a process that
reserves all device memory up front, real-time code that cannot afford an
allocation's synchronisation or failure).

It must give what the handle API (mmod_create / mmod_set_model / mmod_forward)
gives, within the parity tolerance of the other tests, on consecutive calls
that share its fixed scratch block; it must not change the device's free
memory; and it must refuse grids beyond its stated limit with a clear error.
This file sorts last so that a run stopping at the first failure has already
run every other test.
"""
import numpy as np
import pytest

import paper_2007_06048_gb300 as M
import workloads as W
from _gpu_util import rel_l2, run_gpu, torch_cuda

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


@pytest.mark.parametrize("shape,nt,nbl,fs", [((30, 28, 70), 60, 4, False), ((100, 96, 128), 120, 12, False),
                                             ((30, 28, 70), 60, 4, True)])
def test_matches_handle_api_on_two_calls(shape, nt, nbl, fs):
    torch = torch_cuda()
    p = W.tiny_problem(shape=shape, nt=nt, nbl=nbl, nsrc=3, nrec=23, seed=sum(shape))
    if fs:   # free surface, with a source and a receiver on its plane
        p.free_surface = True
        p.src_ijk[0] = [5, 6, 0]
        p.src_ijk[1:] = [[20, 10, 3], [40, 20, 12]]
        p.rec_ijk[0] = [7, 8, 0]
    tr_ref, u_ref, _ = run_gpu(p)
    assert np.abs(u_ref).max() > 0
    for _ in range(2):   # the second call reuses the block the first one left behind
        tr, u = _noalloc(p, torch)
        assert rel_l2(u, u_ref) <= TOL
        assert rel_l2(tr, tr_ref) <= TOL


def test_device_free_memory_unchanged():
    torch = torch_cuda()
    p = W.tiny_problem(shape=(40, 36, 70), nt=30, nbl=5, nsrc=2, nrec=9, seed=5)
    _noalloc(p, torch)                      # first call on the device: block address set-up
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
