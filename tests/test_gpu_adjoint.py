"""GPU adjoint and velocity gradient against the FP64 oracle.

Tolerances (relative L2 over the whole array, FP64 norms):
  adjoint source (transpose of the forward map), <= 100 steps: 1e-5, as the
  forward parity gate (the adjoint runs the same FP32 step kernels);
  gradient, FP32 checkpoints, <= 100 steps: 1e-5, the forward gate (the
  imaging factor g^n = L u^n + s^n comes from the step kernel's own FP32
  Laplacian, so no difference of nearly equal wavefields is formed);
  16-bit checkpoints: the replayed forward starts from rounded states, so the
  gradient moves by ~ the storage precision (BF16 8 bits, FP16 11 bits of
  mantissa after per-plane scaling, BFP16 15 bits below each 32-value
  block's maximum) times the stencil's amplification of grid-scale noise:
  gates 2e-2 (BF16), 3e-3 (FP16) and 1e-3 (BFP16) on this 30 Hz case.
Dot-product test: <F w, r> = <w, F^T r> with FP32 operators and FP64 sums
(mmod_dot) to 1e-6 relative.
"""
import numpy as np
import pytest

import paper_2007_06048_gb300 as M
import workloads as W
from _gpu_util import rel_l2, run_gpu, torch_cuda

pytestmark = pytest.mark.gpu


def _problem(shape=(24, 26, 70), nt=90, nbl=4, nsrc=2, nrec=40, seed=13):
    p = W.tiny_problem(shape=shape, nt=nt, nbl=nbl, nsrc=nsrc, nrec=nrec, seed=seed)
    nz, ny, nx = shape
    p.rec_ijk[1] = p.rec_ijk[0]                      # duplicated receiver
    p.rec_ijk[2:22] = [[i, ny // 2, 1] for i in range(3, 23)]   # a dense line in one plane
    return p


def _gpu_adjoint(p, resid, kernel=M.KERNEL_AUTO):
    torch = torch_cuda()
    prop = M.Propagator.from_problem(p)
    if kernel != M.KERNEL_AUTO:
        prop.set_kernel(kernel)
    prop.set_model(torch.from_numpy(p.vel).cuda())
    r = torch.from_numpy(np.ascontiguousarray(resid, np.float32)).cuda()
    adj = torch.zeros((len(p.src_ijk), p.nt), device="cuda")
    prop.adjoint(r, adj)
    torch.cuda.synchronize()
    return adj.cpu().numpy(), prop


def test_adjoint_matches_oracle(orc):
    p = _problem()
    rng = np.random.default_rng(3)
    resid = rng.standard_normal((p.nt, len(p.rec_ijk))).astype(np.float32)
    a_gpu, _ = _gpu_adjoint(p, resid)
    a_orc = orc.adjoint(p.vel, p.h, p.dt, p.nt, nbl=p.nbl, src_ijk=p.src_ijk, rec_ijk=p.rec_ijk, resid=resid)
    assert rel_l2(a_gpu, a_orc) <= 1e-5


def test_adjoint_plain_and_tma_kernels_agree_bitwise():
    p = _problem(shape=(33, 40, 131), nt=40, nrec=60, seed=5)
    resid = np.random.default_rng(1).standard_normal((p.nt, len(p.rec_ijk))).astype(np.float32)
    a_t, _ = _gpu_adjoint(p, resid, M.KERNEL_TMA)
    a_s, _ = _gpu_adjoint(p, resid, M.KERNEL_SIMPLE)
    assert np.array_equal(a_t, a_s)


def test_dot_product_fp64_sums():
    """<F w, r> = <w, F^T r> with the FP32 GPU operators, sums in FP64 on the GPU."""
    torch = torch_cuda()
    p = _problem(shape=(40, 44, 64), nt=120, nrec=50, seed=21)
    rng = np.random.default_rng(4)
    w = torch.from_numpy(rng.standard_normal((len(p.src_ijk), p.nt)).astype(np.float32)).cuda()
    r = torch.from_numpy(rng.standard_normal((p.nt, len(p.rec_ijk))).astype(np.float32)).cuda()
    prop = M.Propagator.from_problem(p)
    prop.set_model(torch.from_numpy(p.vel).cuda())
    Fw = torch.zeros((p.nt, len(p.rec_ijk)), device="cuda")
    prop.forward(w, Fw)
    FTr = torch.zeros((len(p.src_ijk), p.nt), device="cuda")
    prop.adjoint(r, FTr)
    lhs = M.mmod_dot(Fw, r)
    rhs = M.mmod_dot(w, FTr)
    assert abs(lhs - rhs) <= 1e-6 * abs(lhs), (lhs, rhs)


def test_many_sources_with_duplicates_forward(orc):
    p = W.tiny_problem(shape=(20, 50, 70), nt=30, nbl=3, nsrc=300, nrec=7, seed=9)
    p.src_ijk[5] = p.src_ijk[4]
    p.src_ijk[6] = p.src_ijk[4]
    tr_o, _, u_o = orc.forward(p.vel, p.h, p.dt, p.nt, nbl=p.nbl, src_ijk=p.src_ijk, wavelet=p.wavelet,
                               rec_ijk=p.rec_ijk, want_state=True)
    tr_g, u_g, _ = run_gpu(p)
    assert rel_l2(u_g, u_o) <= 1e-5
    tr_s, u_s, _ = run_gpu(p, kernel=M.KERNEL_SIMPLE)
    assert np.array_equal(u_s, u_g) and np.array_equal(tr_s, tr_g)


def _gradient_case(nt=80):
    p = W.tiny_problem(shape=(26, 28, 30), nt=nt, nbl=5, nsrc=1, nrec=30, seed=31)
    p.vel = np.round(p.vel).astype(np.float32)
    p.src_ijk[0] = [15, 14, 3]
    p.rec_ijk[:] = [[3 + (r % 6) * 4, 4 + (r // 6) * 4, 1] for r in range(30)]
    p.wavelet = W.ricker(30.0, p.dt, nt)[None, :]
    return p


def _gpu_gradient(p, resid, ckpt, dtype, scheme=M.SCHEME_SEGMENTS):
    torch = torch_cuda()
    prop = M.Propagator.from_problem(p)
    prop.set_option(M.OPT_CKPT_SCHEME, scheme)
    prop.set_model(torch.from_numpy(p.vel).cuda())
    g = torch.zeros(p.vel.shape, device="cuda")
    prop.gradient(torch.from_numpy(p.wavelet).cuda(), torch.from_numpy(resid.astype(np.float32)).cuda(), g,
                  ckpt, dtype)
    torch.cuda.synchronize()
    return g.cpu().numpy()


@pytest.fixture(scope="module")
def grad_ref(orc):
    p = _gradient_case()
    vel_true = (p.vel * 1.04).astype(np.float32)
    d_obs = orc.forward(vel_true, p.h, p.dt, p.nt, nbl=p.nbl, src_ijk=p.src_ijk, wavelet=p.wavelet, rec_ijk=p.rec_ijk)
    tr = orc.forward(p.vel, p.h, p.dt, p.nt, nbl=p.nbl, src_ijk=p.src_ijk, wavelet=p.wavelet, rec_ijk=p.rec_ijk)
    resid = tr - d_obs
    g = orc.gradient(p.vel, p.h, p.dt, p.nt, nbl=p.nbl, src_ijk=p.src_ijk, wavelet=p.wavelet, rec_ijk=p.rec_ijk,
                     resid=resid)
    return p, resid, g


def test_gradient_fp32_checkpoints_matches_oracle(grad_ref):
    p, resid, g_o = grad_ref
    g = _gpu_gradient(p, resid, 8, M.CKPT_FP32)
    assert np.abs(g_o).max() > 0
    err = rel_l2(g, g_o)
    print(f"FP32 checkpoints: gradient rel L2 vs FP64 oracle {err:.3e}")
    assert err <= 1e-5


def test_gradient_fp32_is_independent_of_the_checkpoint_count(grad_ref):
    p, resid, _ = grad_ref
    ref = _gpu_gradient(p, resid, 1, M.CKPT_FP32)
    for ck in (3, 8, p.nt):
        assert np.array_equal(_gpu_gradient(p, resid, ck, M.CKPT_FP32), ref), ck


@pytest.mark.parametrize("dtype,gate", [(M.CKPT_BF16, 2e-2), (M.CKPT_FP16, 3e-3), (M.CKPT_BFP16, 1e-3)])
def test_gradient_checkpoint_precision(grad_ref, dtype, gate):
    p, resid, g_o = grad_ref
    g = _gpu_gradient(p, resid, 8, dtype)
    err = rel_l2(g, g_o)
    print(f"checkpoint dtype {dtype}: gradient rel L2 vs FP64 oracle {err:.3e}")
    assert err <= gate


def test_gradient_memory_accounting():
    torch = torch_cuda()
    p = _gradient_case(nt=100)
    prop = M.Propagator.from_problem(p)
    m32 = prop.gradient_memory(10, M.CKPT_FP32)
    m16 = prop.gradient_memory(10, M.CKPT_BF16)
    mb = prop.gradient_memory(10, M.CKPT_BFP16)
    assert 0 < m16 < mb < m32
    torch.cuda.synchronize()


def test_gradient_revolve_fp32_matches_segments_bitwise(grad_ref):
    """FP32 checkpoints replay exactly, so every schedule gives the same bits."""
    p, resid, _ = grad_ref
    ref = _gpu_gradient(p, resid, 8, M.CKPT_FP32)
    for ck in (1, 2, 5, p.nt):
        assert np.array_equal(_gpu_gradient(p, resid, ck, M.CKPT_FP32, M.SCHEME_REVOLVE), ref), ck


@pytest.mark.parametrize("dtype,gate", [(M.CKPT_BF16, 2e-2), (M.CKPT_FP16, 3e-3), (M.CKPT_BFP16, 1e-3)])
def test_gradient_revolve_16bit_checkpoints(grad_ref, dtype, gate):
    p, resid, g_o = grad_ref
    g = _gpu_gradient(p, resid, 4, dtype, M.SCHEME_REVOLVE)
    err = rel_l2(g, g_o)
    print(f"revolve, 4 slots, checkpoint dtype {dtype}: gradient rel L2 vs FP64 oracle {err:.3e}")
    assert err <= gate


def test_gradient_memory_revolve_is_smaller():
    torch_cuda()
    p = _gradient_case(nt=100)
    prop = M.Propagator.from_problem(p)
    seg = prop.gradient_memory(10, M.CKPT_FP16)
    prop.set_option(M.OPT_CKPT_SCHEME, M.SCHEME_REVOLVE)
    rev = prop.gradient_memory(10, M.CKPT_FP16)
    assert 0 < rev < seg


def test_autograd_function_matches_gradient_and_adjoint(grad_ref):
    torch = torch_cuda()
    from paper_2007_06048_gb300.autograd import forward_map
    p, resid, _ = grad_ref
    prop = M.Propagator.from_problem(p)
    vel = torch.from_numpy(p.vel).cuda().requires_grad_(True)
    wav = torch.from_numpy(p.wavelet).cuda().requires_grad_(True)
    r = torch.from_numpy(resid.astype(np.float32)).cuda()
    traces = forward_map(prop, vel, wav, ckpt_count=8)
    (traces * r).sum().backward()
    g_ref = _gpu_gradient(p, resid, 8, M.CKPT_FP32)
    a_ref, _ = _gpu_adjoint(p, resid)
    torch.cuda.synchronize()
    assert np.array_equal(vel.grad.cpu().numpy(), g_ref)
    assert np.array_equal(wav.grad.cpu().numpy(), a_ref)


@pytest.mark.parametrize("dtype,gate", [(M.CKPT_BF16, 2e-2), (M.CKPT_FP16, 3e-3), (M.CKPT_BFP16, 1e-3)])
def test_gradient_16bit_checkpoints_with_quiet_planes(dtype, gate):
    """A deep grid run for few steps: far planes hold only zeros and the
    wave's leading edge only FP32 subnormals, so a checkpoint plane's scale
    can be tiny; the 16-bit gradient must stay finite and close to FP32."""
    torch = torch_cuda()
    p = W.tiny_problem(shape=(160, 20, 20), nt=14, nbl=3, nsrc=1, nrec=12, seed=3)
    p.src_ijk[0] = [10, 10, 2]
    p.rec_ijk[:] = [[2 + r, 10, 0] for r in range(12)]
    resid = np.random.default_rng(2).standard_normal((p.nt, 12)).astype(np.float32)
    g32 = _gpu_gradient(p, resid, 7, M.CKPT_FP32)
    g16 = _gpu_gradient(p, resid, 7, dtype)
    assert np.isfinite(g16).all()
    assert rel_l2(g16, g32) <= gate
    torch.cuda.synchronize()


@pytest.mark.parametrize("scheme", [M.SCHEME_SEGMENTS, M.SCHEME_REVOLVE])
@pytest.mark.parametrize("nt", [1, 2, 3, 7])
def test_gradient_of_short_runs_matches_oracle(orc, nt, scheme):
    """Runs of a few steps, where the checkpoint layouts degenerate (one slot,
    a slot per step, every state kept): random wavelets, receivers on and next
    to the sources so that the gradient is not identically zero."""
    rng = np.random.default_rng(50 + nt)
    p = W.tiny_problem(shape=(14, 15, 16), nt=nt, nbl=2, nsrc=2, nrec=6, seed=60 + nt)
    p.wavelet = rng.standard_normal((2, nt)).astype(np.float32)
    s0, s1 = p.src_ijk
    top = np.array([16 - 1, 15 - 1, 14 - 1])
    p.rec_ijk[:] = np.clip([s0, s1, s0 + [1, 0, 0], s1 + [0, 1, 0], s0 + [0, 0, 1], s1 - [1, 0, 0]], 0, top)
    resid = rng.standard_normal((nt, 6)).astype(np.float32)
    g_o = orc.gradient(p.vel, p.h, p.dt, p.nt, nbl=p.nbl, src_ijk=p.src_ijk, wavelet=p.wavelet,
                       rec_ijk=p.rec_ijk, resid=resid)
    assert np.abs(g_o).max() > 0
    for ck, dtype, gate in ((1, M.CKPT_FP32, 1e-5), (nt, M.CKPT_FP32, 1e-5), (1, M.CKPT_BFP16, 1e-3)):
        g = _gpu_gradient(p, resid, ck, dtype, scheme)
        assert rel_l2(g, g_o) <= gate, (ck, dtype)
