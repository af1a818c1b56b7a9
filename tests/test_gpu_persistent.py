"""The persistent time loop (one cooperative launch, neighbour counters
between work units) against one launch per step.

Every unit performs the same per-point arithmetic in both forms, so traces
and final wavefields must agree bit for bit: on ragged grids, with sources
and receivers spread over tiles and planes, with few CTAs serving many units
each, for the adjoint run, and on the 240^3 layered workload.  The failure
path is exercised with the stall hook: waits that nothing will satisfy give
up after their bound and the call reports MMOD_ERR_TIMEOUT.
"""
import numpy as np
import pytest

import paper_2007_06048_gb300 as M
import workloads as W
from _gpu_util import torch_cuda

pytestmark = pytest.mark.gpu


def _run(p, persistent, ctas=0, variant=None, adjoint=None):
    torch = torch_cuda()
    prop = M.Propagator.from_problem(p)
    if variant is not None:
        prop.set_variant(variant)
    prop.set_option(M.OPT_PERSISTENT, persistent)
    prop.set_option(M.OPT_PERSISTENT_CTAS, ctas)
    grid = prop.persistent_grid()
    prop.set_model(torch.from_numpy(np.ascontiguousarray(p.vel)).cuda())
    if adjoint is not None:
        r = torch.from_numpy(adjoint).cuda()
        out = torch.zeros((len(p.src_ijk), p.nt), device="cuda")
        prop.adjoint(r, out)
        torch.cuda.synchronize()
        return out.cpu().numpy(), None, grid
    wav = torch.from_numpy(np.ascontiguousarray(p.wavelet, np.float32)).cuda()
    tr = torch.zeros((p.nt, len(p.rec_ijk)), device="cuda")
    fin = torch.zeros(p.vel.shape, device="cuda")
    prop.forward(wav, tr, fin)
    torch.cuda.synchronize()
    return tr.cpu().numpy(), fin.cpu().numpy(), grid


CASES = [((70, 36, 40), 4), ((131, 40, 33), 6), ((45, 20, 70), 3), ((200, 90, 25), 8), ((64, 64, 130), 5)]


@pytest.mark.parametrize("shape,nbl", CASES)
def test_persistent_equals_per_step_launches(shape, nbl):
    p = W.tiny_problem(shape=shape, nt=50, nbl=nbl, nsrc=3, nrec=40, seed=sum(shape))
    tr_s, u_s, g0 = _run(p, 0)
    assert g0 == 0
    tr_p, u_p, g1 = _run(p, 1)
    assert g1 > 0
    assert np.array_equal(u_p, u_s) and np.array_equal(tr_p, tr_s)


@pytest.mark.parametrize("ctas", [1, 7])
def test_persistent_with_many_units_per_cta(ctas):
    p = W.tiny_problem(shape=(131, 70, 150), nt=30, nbl=5, nsrc=2, nrec=60, seed=12)
    tr_s, u_s, _ = _run(p, 0)
    tr_p, u_p, g = _run(p, 1, ctas=ctas)
    assert g == ctas
    assert np.array_equal(u_p, u_s) and np.array_equal(tr_p, tr_s)


def test_persistent_second_variant():
    p = W.tiny_problem(shape=(90, 50, 70), nt=40, nbl=4, nsrc=2, nrec=30, seed=5)
    v = [i for i in range(M.mmod_tma_variant_count()) if "shallow" in M.mmod_tma_variant_name(i)
         and "2x4" in M.mmod_tma_variant_name(i)][0]
    tr_s, u_s, _ = _run(p, 0, variant=v)
    tr_p, u_p, g = _run(p, 1, variant=v)
    assert g > 0
    assert np.array_equal(u_p, u_s) and np.array_equal(tr_p, tr_s)


def test_persistent_adjoint():
    p = W.tiny_problem(shape=(60, 40, 70), nt=45, nbl=4, nsrc=3, nrec=80, seed=8)
    r = np.random.default_rng(3).standard_normal((p.nt, len(p.rec_ijk))).astype(np.float32)
    a_s, _, _ = _run(p, 0, adjoint=r)
    a_p, _, g = _run(p, 1, adjoint=r)
    assert g > 0
    assert np.array_equal(a_p, a_s)


def test_persistent_layered_240():
    p = W.layered_240(nt=100)
    tr_s, u_s, _ = _run(p, 0)
    tr_p, u_p, g = _run(p, 1)
    assert g > 0
    assert np.array_equal(u_p, u_s) and np.array_equal(tr_p, tr_s)


def test_persistent_thin_z_ranges():
    """Grids whose per-step plan cuts z into ranges thinner than the stencil
    radius: the persistent form uses ranges of at least 4 planes."""
    for shape in [(6, 16, 64), (9, 40, 40), (33, 8, 200)]:
        p = W.tiny_problem(shape=shape, nt=12, nbl=1, nsrc=1, nrec=7, seed=1)
        tr_s, u_s, _ = _run(p, 0)
        tr_p, u_p, g = _run(p, 1)
        assert g > 0
        assert np.array_equal(u_p, u_s) and np.array_equal(tr_p, tr_s), shape


def test_stalled_wait_reports_timeout_and_device_stays_usable():
    torch = torch_cuda()
    p = W.tiny_problem(shape=(64, 48, 130), nt=10, nbl=3, nsrc=1, nrec=5, seed=2)
    prop = M.Propagator.from_problem(p)
    prop.set_option(M.OPT_PERSISTENT, 1)
    assert prop.persistent_grid() > 1
    prop.set_model(torch.from_numpy(p.vel).cuda())
    wav = torch.from_numpy(p.wavelet).cuda()
    tr = torch.zeros((p.nt, len(p.rec_ijk)), device="cuda")
    prop.set_option(M.OPT_TEST_STALL, 1)
    try:
        prop.forward(wav, tr)
    except M.MmodError as e:
        assert e.status == -5
    torch.cuda.synchronize()
    with pytest.raises(M.MmodError) as ei:
        prop.forward(wav, tr)
    assert ei.value.status == -5            # MMOD_ERR_TIMEOUT, latched on the handle
    prop.close()
    # a fresh handle on the same device still runs and gives the per-step result
    tr_s, u_s, _ = _run(p, 0)
    tr_p, u_p, _ = _run(p, 1)
    assert np.array_equal(u_p, u_s) and np.array_equal(tr_p, tr_s)


def test_zlen_option_keeps_bits():
    """MMOD_OPT_ZLEN re-cuts the z ranges of the one-launch-per-step kernel
    and of the persistent units; every cut gives the same bits."""
    torch = torch_cuda()
    p = W.tiny_problem(shape=(97, 40, 70), nt=30, nbl=4, nsrc=2, nrec=25, seed=4)
    ref, u_ref, _ = _run(p, 0)
    for zlen in (1, 5, 17, 96, 500):
        for persistent in (0, 1):
            prop = M.Propagator.from_problem(p)
            prop.set_option(M.OPT_ZLEN, zlen)
            prop.set_option(M.OPT_PERSISTENT, persistent)
            prop.set_model(torch.from_numpy(p.vel).cuda())
            wav = torch.from_numpy(p.wavelet).cuda()
            tr = torch.zeros((p.nt, len(p.rec_ijk)), device="cuda")
            fin = torch.zeros(p.vel.shape, device="cuda")
            prop.forward(wav, tr, fin)
            torch.cuda.synchronize()
            assert np.array_equal(tr.cpu().numpy(), ref), (zlen, persistent)
            assert np.array_equal(fin.cpu().numpy(), u_ref), (zlen, persistent)
            prop.close()
