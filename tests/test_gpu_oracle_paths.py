"""Every multi-shot and persistent path of the GPU library against the FP64
oracle directly, on the same inputs.

The bitwise tests elsewhere show that a batch, the persistent loop and the
single-shot forward give the same bits; they share the per-point stencil code
and the injection tables, so a mistake common to both would pass them.  Here
each path is compared with ``oracle.forward`` (Alg. 1 / Alg. 2, Eq. 5) on its
own shots, element by element, with the forward parity gates: relative L2 of
wavefield and traces <= 1e-5 after <= 100 steps, <= 1e-4 after 800 steps.

Cases: shots of uneven sizes and damping widths (ragged tiles and z ranges),
one with a free surface (reading R15) and a source and receiver on its plane,
duplicated sources, a receiver on a source point, and receivers at grid
corners; two shots of the 32-shot workload (uneven 128..320 x 128..320 x
128..256 grids, 800 steps, per-shot layered models, as the paper's nshots run
of Sec. 5.3) through all three batch modes.
"""
import numpy as np
import pytest

import paper_2007_06048_gb300 as M
import workloads as W
from _gpu_util import rel_l2, run_oracle, torch_cuda

pytestmark = pytest.mark.gpu

MODES = [M.BATCH_STREAMS, M.BATCH_FUSED, M.BATCH_PERSISTENT]
SHAPES = [((40, 36, 70), 4), ((33, 64, 128), 6), ((70, 20, 45), 3), ((25, 90, 200), 8)]


def _mixed_shots(nt=100):
    shots = []
    for i, (s, L) in enumerate(SHAPES):
        p = W.tiny_problem(shape=s, nt=nt, nbl=L, nsrc=3, nrec=19, seed=i + 140)
        nz, ny, nx = s
        if i == 0:     # free surface, a source and a receiver on its plane
            p.free_surface = True
            p.src_ijk[0] = [nx // 3, ny // 2, 0]
            p.rec_ijk[0] = [nx // 4, ny // 3, 0]
        if i == 1:     # duplicated source, a receiver on a source point
            p.src_ijk[2] = p.src_ijk[1]
            p.rec_ijk[3] = p.src_ijk[0]
        if i == 2:     # receivers at two opposite grid corners
            p.rec_ijk[0] = [0, 0, 0]
            p.rec_ijk[1] = [nx - 1, ny - 1, nz - 1]
        shots.append(p)
    return shots


def _batch(shots, mode, variant=None):
    torch = torch_cuda()
    props = [M.Propagator.from_problem(p) for p in shots]
    for pr, p in zip(props, shots):
        pr.set_model(torch.from_numpy(np.ascontiguousarray(p.vel)).cuda())
    b = M.Batch(props)
    b.set_mode(mode)
    if variant is not None:
        b.set_variant(variant)
    wav = [torch.from_numpy(np.ascontiguousarray(p.wavelet)).cuda() for p in shots]
    tr = [torch.full((p.nt, len(p.rec_ijk)), float("nan"), device="cuda") for p in shots]
    b.forward(wav, tr)
    out = []
    for pr, p, t in zip(props, shots, tr):
        up = torch.empty(p.vel.shape, device="cuda")
        uc = torch.empty(p.vel.shape, device="cuda")
        pr.get_state(up, uc)
        out.append((t.cpu().numpy(), uc.cpu().numpy()))
    torch.cuda.synchronize()
    b.close()
    for pr in props:
        pr.close()
    return out


@pytest.fixture(scope="module")
def mixed(orc):
    shots = _mixed_shots()
    refs = [run_oracle(orc, p) for p in shots]
    return shots, [(r[0], r[2]) for r in refs]


@pytest.mark.parametrize("mode", MODES)
def test_batch_matches_oracle(mixed, mode):
    shots, refs = mixed
    for i, ((tr, u), (tr_o, u_o)) in enumerate(zip(_batch(shots, mode), refs)):
        assert np.isfinite(tr).all(), i
        e_u, e_t = rel_l2(u, u_o), rel_l2(tr, tr_o)
        print(f"mode {mode} shot {i}: rel L2 u {e_u:.2e} traces {e_t:.2e}")
        assert e_u <= 1e-5 and e_t <= 1e-5, (i, e_u, e_t)


def test_persistent_batch_second_variant_matches_oracle(mixed):
    shots, refs = mixed
    for i, ((tr, u), (tr_o, u_o)) in enumerate(zip(_batch(shots, M.BATCH_PERSISTENT, variant=5), refs)):
        assert rel_l2(u, u_o) <= 1e-5 and rel_l2(tr, tr_o) <= 1e-5, i


def _single(p, options):
    torch = torch_cuda()
    prop = M.Propagator.from_problem(p)
    for k, v in options.items():
        prop.set_option(k, v)
    prop.set_model(torch.from_numpy(np.ascontiguousarray(p.vel)).cuda())
    wav = torch.from_numpy(np.ascontiguousarray(p.wavelet)).cuda()
    tr = torch.full((p.nt, len(p.rec_ijk)), float("nan"), device="cuda")
    fin = torch.zeros(p.vel.shape, device="cuda")
    grid = prop.persistent_grid()
    prop.forward(wav, tr, fin)
    torch.cuda.synchronize()
    prop.close()
    return tr.cpu().numpy(), fin.cpu().numpy(), grid


@pytest.mark.parametrize("ctas", [0, 5])
def test_persistent_loop_matches_oracle(mixed, ctas):
    shots, refs = mixed
    for i, (p, (tr_o, u_o)) in enumerate(zip(shots, refs)):
        tr, u, grid = _single(p, {M.OPT_PERSISTENT: 1, M.OPT_PERSISTENT_CTAS: ctas})
        assert grid > 0, i
        assert rel_l2(u, u_o) <= 1e-5 and rel_l2(tr, tr_o) <= 1e-5, i


def test_persistent_adjoint_matches_oracle(orc):
    torch = torch_cuda()
    p = W.tiny_problem(shape=(60, 40, 70), nt=90, nbl=4, nsrc=3, nrec=80, seed=18)
    p.rec_ijk[1] = p.rec_ijk[0]                      # duplicated receiver
    p.rec_ijk[2] = p.src_ijk[0]                      # a receiver on a source
    r = np.random.default_rng(5).standard_normal((p.nt, len(p.rec_ijk))).astype(np.float32)
    prop = M.Propagator.from_problem(p)
    prop.set_option(M.OPT_PERSISTENT, 1)
    assert prop.persistent_grid() > 0
    prop.set_model(torch.from_numpy(p.vel).cuda())
    out = torch.zeros((len(p.src_ijk), p.nt), device="cuda")
    prop.adjoint(torch.from_numpy(r).cuda(), out)
    torch.cuda.synchronize()
    a_o = orc.adjoint(p.vel, p.h, p.dt, p.nt, nbl=p.nbl, src_ijk=p.src_ijk, rec_ijk=p.rec_ijk, resid=r)
    assert rel_l2(out.cpu().numpy(), a_o) <= 1e-5


@pytest.fixture(scope="module")
def workload_shots(orc):
    """Two shots of the 32-shot workload (800 steps each) and their oracle runs."""
    shots = W.batched_shots()[:2]
    refs = [run_oracle(orc, p) for p in shots]
    return shots, [(r[0], r[2]) for r in refs]


@pytest.mark.parametrize("mode", MODES)
def test_batch_workload_shots_800_steps_match_oracle(workload_shots, mode):
    shots, refs = workload_shots
    for i, ((tr, u), (tr_o, u_o)) in enumerate(zip(_batch(shots, mode), refs)):
        e_u, e_t = rel_l2(u, u_o), rel_l2(tr, tr_o)
        print(f"{shots[i].name} mode {mode}: rel L2 u {e_u:.2e} traces {e_t:.2e}")
        assert e_u <= 1e-4 and e_t <= 1e-4, (i, e_u, e_t)
