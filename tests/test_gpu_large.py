"""The 1024 x 1024 x 512 shot (h = 12.5 m, L = 32, 1024^2 receivers) at its
full size.

Forward: 20 steps from a non-zero initial state (the normalised model field
itself, so every cell moves from the first step) with a white-noise source
wavelet, against the FP64 oracle over the whole final wavefield and all
1 048 576 traces (relative L2 <= 1e-5, the 100-step forward gate), and the
TMA and plain kernels bit for bit.

Gradient: 16-bit checkpoints against FP32 checkpoints at full size (40
steps, white-noise wavelet and residual): the added error stays within the
FP16 / BF16 gates that the small-grid tests hold against the FP64 oracle, and
the 500-step run fits the 180 GB device budget with FP16 checkpoints.
"""
import numpy as np
import pytest

import paper_2007_06048_gb300 as M
import workloads as W
from _gpu_util import rel_l2, run_gpu, torch_cuda

pytestmark = pytest.mark.gpu

BUDGET = 180e9


@pytest.fixture(scope="module")
def large():
    p = W.fractal_large(nt=20)
    rng = np.random.default_rng(55)
    p.wavelet = (1e3 * rng.standard_normal((1, p.nt))).astype(np.float32)
    u0 = ((p.vel - 3250.0) / 1750.0).astype(np.float32)
    return p, u0


def test_large_forward_matches_oracle(large, orc):
    p, u0 = large
    u1 = np.roll(u0, 1, axis=2)
    tr_g, u_g, _ = run_gpu(p, state=(u0, u1))
    tr_o, _, u_o = orc.forward(p.vel, p.h, p.dt, p.nt, nbl=p.nbl, src_ijk=p.src_ijk, wavelet=p.wavelet,
                               rec_ijk=p.rec_ijk, u_prev0=u0, u_cur0=u1, want_state=True)
    e_u, e_t = rel_l2(u_g, u_o), rel_l2(tr_g, tr_o)
    print(f"1024x1024x512, 20 steps: wavefield rel L2 {e_u:.2e}, traces rel L2 {e_t:.2e}")
    assert e_u <= 1e-5 and e_t <= 1e-5


def test_large_forward_kernels_bitwise(large):
    p, u0 = large
    tr_t, u_t, _ = run_gpu(p, kernel=M.KERNEL_TMA, state=(u0, None))
    tr_s, u_s, _ = run_gpu(p, kernel=M.KERNEL_SIMPLE, state=(u0, None))
    assert np.array_equal(u_t, u_s) and np.array_equal(tr_t, tr_s)


def _gradient(prop, wav, r, ckpt, dtype):
    torch = torch_cuda()
    g = torch.empty(prop.shape, device="cuda")
    prop.gradient(wav, r, g, ckpt, dtype)
    torch.cuda.synchronize()
    return g


def test_large_gradient_16bit_checkpoints(large):
    torch = torch_cuda()
    p, _ = large
    nt = 40
    prop = M.Propagator(p.vel.shape, p.h, p.dt, nt, nbl=p.nbl, src_ijk=p.src_ijk, rec_ijk=p.rec_ijk)
    prop.set_model(torch.from_numpy(p.vel).cuda())
    gen = torch.Generator(device="cuda").manual_seed(9)
    wav = 1e3 * torch.randn((1, nt), device="cuda", generator=gen)
    r = torch.randn((nt, len(p.rec_ijk)), device="cuda", generator=gen)
    g32 = _gradient(prop, wav, r, 8, M.CKPT_FP32)
    for dtype, gate in ((M.CKPT_FP16, 3e-3), (M.CKPT_BF16, 2e-2)):
        g16 = _gradient(prop, wav, r, 8, dtype)
        err = (torch.linalg.vector_norm((g16 - g32).double()) / torch.linalg.vector_norm(g32.double())).item()
        print(f"1024x1024x512, {nt} steps: checkpoint dtype {dtype} vs FP32 checkpoints, rel L2 {err:.2e}")
        assert err <= gate
        del g16
    prop.close()


def test_large_gradient_fits_budget():
    """500 steps, 25 FP16 checkpoints: the handle's volumes, the gradient's work
    space and the 1024^2 x 500 residual and staging stay under 180 GB."""
    torch_cuda()
    nz, ny, nx = 512, 1024, 1024
    prop = M.Propagator((nz, ny, nx), (12.5, 12.5, 12.5), 1e-3, 500, nbl=32, src_ijk=[[512, 512, 4]],
                        rec_ijk=W.surface_grid(nx, ny, 0))
    work = prop.gradient_memory(25, M.CKPT_FP16)
    handle = 4 * 4 * nx * ny * nz                 # u^{n-1}, u^n, c, velocity copy (FP32)
    traces = 2 * 4 * 500 * nx * ny                # residual + its reversed copy
    total = work + handle + traces
    print(f"1024x1024x512 x 500 steps, 25 FP16 checkpoints: {total / 1e9:.1f} GB")
    assert total < BUDGET
    prop.set_option(M.OPT_CKPT_SCHEME, M.SCHEME_REVOLVE)
    assert prop.gradient_memory(40, M.CKPT_FP16) + handle + traces < BUDGET
    prop.close()
