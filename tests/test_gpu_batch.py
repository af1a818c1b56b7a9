"""Batched shots and the autotuner on the GPU.

A batch advances shots of uneven grid sizes and damping widths together, on
overlapping streams, in one fused launch per step or in one persistent
launch for the whole run; every shot must come
out bit for bit as when it runs alone through mmod_forward (same per-point
arithmetic, only the CTA decomposition differs).  The autotuner must pick a valid variant and leave
results unchanged.
"""
import numpy as np
import pytest

import paper_2007_06048_gb300 as M
import workloads as W
from _gpu_util import run_gpu, torch_cuda

pytestmark = pytest.mark.gpu

SHAPES = [((40, 36, 70), 4), ((33, 64, 128), 6), ((70, 20, 45), 3), ((25, 90, 200), 8)]


def _shots(nt=60):
    return [W.tiny_problem(shape=s, nt=nt, nbl=L, nsrc=2, nrec=15, seed=i + 40) for i, (s, L) in enumerate(SHAPES)]


def _run_batch(shots, autotune=False, mode=M.BATCH_STREAMS):
    torch = torch_cuda()
    props = [M.Propagator.from_problem(p) for p in shots]
    for pr, p in zip(props, shots):
        pr.set_model(torch.from_numpy(p.vel).cuda())
    b = M.Batch(props)
    b.set_mode(mode)
    v = b.autotune(steps=5) if autotune else None
    wav = [torch.from_numpy(p.wavelet).cuda() for p in shots]
    tr = [torch.zeros((p.nt, len(p.rec_ijk)), device="cuda") for p in shots]
    b.forward(wav, tr)
    finals = []
    for pr, p in zip(props, shots):
        up = torch.empty(p.vel.shape, device="cuda")
        uc = torch.empty(p.vel.shape, device="cuda")
        pr.get_state(up, uc)
        finals.append(uc.cpu().numpy())
    torch.cuda.synchronize()
    assert b.loop_ms() > 0
    b.close()
    return [t.cpu().numpy() for t in tr], finals, v


@pytest.mark.parametrize("mode", [M.BATCH_STREAMS, M.BATCH_FUSED, M.BATCH_PERSISTENT])
def test_batch_matches_single_shots_bitwise(mode):
    shots = _shots()
    tr_b, u_b, _ = _run_batch(shots, mode=mode)
    for i, p in enumerate(shots):
        tr_s, u_s, _ = run_gpu(p)
        assert np.array_equal(tr_b[i], tr_s), i
        assert np.array_equal(u_b[i], u_s), i


@pytest.mark.parametrize("mode", [M.BATCH_STREAMS, M.BATCH_FUSED])
def test_batch_autotune_keeps_results(mode):
    shots = _shots(nt=30)
    tr_b, u_b, v = _run_batch(shots, autotune=True, mode=mode)
    assert 0 <= v < M.mmod_tma_variant_count()
    for i, p in enumerate(shots):
        tr_s, u_s, _ = run_gpu(p, kernel=M.KERNEL_SIMPLE)
        assert np.array_equal(tr_b[i], tr_s), i
        assert np.array_equal(u_b[i], u_s), i


def test_single_handle_autotune():
    torch = torch_cuda()
    p = W.tiny_problem(shape=(48, 64, 130), nt=40, nbl=5, nsrc=2, nrec=9, seed=77)
    prop = M.Propagator.from_problem(p)
    prop.set_model(torch.from_numpy(p.vel).cuda())
    v = prop.autotune(steps=6)
    assert 0 <= v < M.mmod_tma_variant_count()
    assert prop.plan()["variant"] == v
    wav = torch.from_numpy(p.wavelet).cuda()
    tr = torch.zeros((p.nt, len(p.rec_ijk)), device="cuda")
    fin = torch.zeros(p.vel.shape, device="cuda")
    prop.forward(wav, tr, fin)
    tr_s, u_s, _ = run_gpu(p, kernel=M.KERNEL_SIMPLE)
    assert np.array_equal(tr.cpu().numpy(), tr_s)
    assert np.array_equal(fin.cpu().numpy(), u_s)


def test_batch_rejects_mismatched_steps():
    torch_cuda()
    a = M.Propagator.from_problem(W.tiny_problem(shape=(20, 20, 40), nt=10))
    b = M.Propagator.from_problem(W.tiny_problem(shape=(20, 20, 40), nt=11))
    with pytest.raises(M.MmodError) as ei:
        M.Batch([a, b])
    assert ei.value.status == -1


def test_batch_mode_rejects_unknown():
    torch_cuda()
    a = M.Propagator.from_problem(W.tiny_problem(shape=(20, 20, 40), nt=10))
    b = M.Batch([a])
    with pytest.raises(M.MmodError):
        b.set_mode(7)
    b.close()


def test_persistent_batch_stall_reports_timeout_and_device_stays_usable():
    """The failure path of the persistent batch: a shot's test hook makes
    every unit wait for neighbour counters that nothing sets; the bounded
    waits give up, the shots report MMOD_ERR_TIMEOUT, and a new batch on the
    same device still gives every shot its single-run bits."""
    torch = torch_cuda()
    shots = _shots(nt=10)
    props = [M.Propagator.from_problem(p) for p in shots]
    for pr, p in zip(props, shots):
        pr.set_model(torch.from_numpy(p.vel).cuda())
    b = M.Batch(props)
    b.set_mode(M.BATCH_PERSISTENT)
    wav = [torch.from_numpy(p.wavelet).cuda() for p in shots]
    tr = [torch.zeros((p.nt, len(p.rec_ijk)), device="cuda") for p in shots]
    props[1].set_option(M.OPT_TEST_STALL, 1)
    try:
        b.forward(wav, tr)
    except M.MmodError as e:
        assert e.status == -5
    torch.cuda.synchronize()
    with pytest.raises(M.MmodError) as ei:
        b.forward(wav, tr)
    assert ei.value.status == -5             # latched on the shots' handles
    b.close()
    for pr in props:
        pr.close()
    tr_b, u_b, _ = _run_batch(shots, mode=M.BATCH_PERSISTENT)
    for i, p in enumerate(shots):
        tr_s, u_s, _ = run_gpu(p)
        assert np.array_equal(tr_b[i], tr_s) and np.array_equal(u_b[i], u_s), i
