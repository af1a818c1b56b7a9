"""Work-claiming step launches (MMOD_OPT_CLAIM) against the static plan.

With claiming on, at most one wave of CTAs serves the step's units and each
CTA claims further units from a per-launch counter; the units are the same
per-point arithmetic, so traces and final wavefields must equal the static
plan's bit for bit: for every unit size (thinner than the stencil radius, not
dividing nz, larger than nz), on ragged grids, for every variant with a
claiming form, for the adjoint and the gradient, and on consecutive runs
(the counters must be cleared by each launch for the next one).
"""
import numpy as np
import pytest

import paper_2007_06048_gb300 as M
import workloads as W
from _gpu_util import rel_l2, run_gpu, run_oracle, torch_cuda

pytestmark = pytest.mark.gpu

SHAPES = [((70, 36, 40), 4), ((131, 40, 33), 6), ((45, 20, 70), 3), ((200, 90, 25), 8)]


@pytest.mark.parametrize("shape,nbl", SHAPES)
def test_claim_equals_static_plan(shape, nbl):
    p = W.tiny_problem(shape=shape, nt=40, nbl=nbl, nsrc=3, nrec=40, seed=sum(shape) + 3)
    tr_s, u_s, _ = run_gpu(p)
    for planes in (1, 3, 5, 16, 1000):
        tr, u, prop = run_gpu(p, options={M.OPT_CLAIM: planes})
        plan = prop.plan()
        assert plan["planes_per_chunk"] == min(planes, shape[0]), plan
        assert np.array_equal(u, u_s) and np.array_equal(tr, tr_s), planes


@pytest.mark.parametrize("variant", [1, 2, 6])
def test_claim_variants_on_layered_240(variant):
    p = W.layered_240(nt=30)
    tr_s, u_s, _ = run_gpu(p, variant=variant)
    torch = torch_cuda()
    tr, u, prop = run_gpu(p, variant=variant, options={M.OPT_CLAIM: 16})
    plan = prop.plan()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    units = plan["tiles_x"] * plan["tiles_y"] * plan["z_chunks"]
    assert plan["planes_per_chunk"] == 16 and plan["grid"] == min(units, plan["ctas_per_sm"] * sms), plan
    assert np.array_equal(u, u_s) and np.array_equal(tr, tr_s)


def test_claim_repeated_runs_and_pdl_off(orc):
    """Consecutive runs on one handle reuse the counters; with and without
    programmatic dependent launch; and the result against the oracle."""
    torch = torch_cuda()
    p = W.tiny_problem(shape=(64, 48, 130), nt=60, nbl=5, nsrc=2, nrec=30, seed=21)
    tr_s, u_s, _ = run_gpu(p)
    for pdl in (1, 0):
        prop = M.Propagator.from_problem(p)
        prop.set_option(M.OPT_CLAIM, 7)
        prop.set_option(M.OPT_PDL, pdl)
        prop.set_model(torch.from_numpy(p.vel).cuda())
        wav = torch.from_numpy(p.wavelet).cuda()
        for _ in range(3):
            tr = torch.zeros((p.nt, len(p.rec_ijk)), device="cuda")
            fin = torch.zeros(p.vel.shape, device="cuda")
            prop.forward(wav, tr, fin)
            torch.cuda.synchronize()
            assert np.array_equal(fin.cpu().numpy(), u_s) and np.array_equal(tr.cpu().numpy(), tr_s)
        prop.close()
    tr_o, _, u_o = run_oracle(orc, p)
    assert rel_l2(u_s, u_o) <= 1e-5 and rel_l2(tr_s, tr_o) <= 1e-5


def test_claim_adjoint_and_gradient_keep_bits():
    torch = torch_cuda()
    p = W.tiny_problem(shape=(40, 44, 70), nt=50, nbl=4, nsrc=2, nrec=50, seed=9)
    r = np.random.default_rng(2).standard_normal((p.nt, len(p.rec_ijk))).astype(np.float32)
    out = {}
    for planes in (0, 6):
        prop = M.Propagator.from_problem(p)
        prop.set_option(M.OPT_CLAIM, planes)
        prop.set_model(torch.from_numpy(p.vel).cuda())
        a = torch.zeros((len(p.src_ijk), p.nt), device="cuda")
        prop.adjoint(torch.from_numpy(r).cuda(), a)
        g = torch.zeros(p.vel.shape, device="cuda")
        prop.gradient(torch.from_numpy(p.wavelet).cuda(), torch.from_numpy(r).cuda(), g, 5, M.CKPT_FP32)
        torch.cuda.synchronize()
        out[planes] = (a.cpu().numpy(), g.cpu().numpy())
        prop.close()
    assert np.array_equal(out[0][0], out[6][0])
    assert np.array_equal(out[0][1], out[6][1])


def test_claim_option_validation():
    torch_cuda()
    prop = M.Propagator.from_problem(W.tiny_problem(shape=(20, 20, 40), nt=5))
    with pytest.raises(M.MmodError):
        prop.set_option(M.OPT_CLAIM, -1)
    prop.set_option(M.OPT_CLAIM, 0)
    prop.close()
