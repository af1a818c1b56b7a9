"""Optimised stencil weights on the GPU (reading R16): parity with the FP64
oracle given the same weights, bit-for-bit agreement of the kernels, the
adjoint stays the transpose, a cached time loop picks up new weights, and the
stability bound follows the weights."""
import numpy as np
import pytest

import paper_2007_06048_gb300 as M
import workloads as W
from _gpu_util import rel_l2, run_oracle, torch_cuda

pytestmark = pytest.mark.gpu

KMAX = 2 * np.pi / 3


def _forward(p, c4, kernel=M.KERNEL_AUTO, variant=None, prop=None):
    torch = torch_cuda()
    own = prop is None
    if own:
        prop = M.Propagator.from_problem(p)
        if kernel != M.KERNEL_AUTO:
            prop.set_kernel(kernel)
        if variant is not None:
            prop.set_variant(variant)
        prop.set_fd_coefficients(c4)
        prop.set_model(torch.from_numpy(p.vel).cuda())
    wav = torch.from_numpy(p.wavelet).cuda()
    tr = torch.zeros((p.nt, len(p.rec_ijk)), device="cuda")
    fin = torch.zeros(p.vel.shape, device="cuda")
    prop.forward(wav, tr, fin)
    torch.cuda.synchronize()
    out = tr.cpu().numpy(), fin.cpu().numpy()
    if own:
        prop.close()
    return out


@pytest.mark.parametrize("shape,nbl", [((40, 36, 70), 4), ((33, 64, 131), 6)])
def test_optimised_weights_match_oracle(orc, shape, nbl):
    c4 = M.mmod_optimized_coefficients(KMAX)
    p = W.tiny_problem(shape=shape, nt=100, nbl=nbl, nsrc=2, nrec=20, seed=sum(shape))
    tr_g, u_g = _forward(p, c4)
    tr_o, _, u_o = run_oracle(orc, p, coef=c4)
    assert rel_l2(u_g, u_o) <= 1e-5
    _, _, u_t = run_oracle(orc, p)                # Taylor weights: a different field
    assert rel_l2(u_t, u_o) > 1e-3


def test_optimised_weights_kernels_bitwise():
    c4 = M.mmod_optimized_coefficients(KMAX)
    p = W.tiny_problem(shape=(50, 40, 90), nt=40, nbl=5, nsrc=2, nrec=20, seed=7)
    ref = _forward(p, c4, kernel=M.KERNEL_SIMPLE)
    for v in range(M.mmod_tma_variant_count()):
        got = _forward(p, c4, kernel=M.KERNEL_TMA, variant=v)
        assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1]), v


def test_new_weights_replace_the_cached_loop():
    torch = torch_cuda()
    c4 = M.mmod_optimized_coefficients(KMAX)
    p = W.tiny_problem(shape=(40, 36, 70), nt=50, nbl=4, nsrc=2, nrec=20, seed=3)
    prop = M.Propagator.from_problem(p)
    prop.set_model(torch.from_numpy(p.vel).cuda())
    taylor = _forward(p, None, prop=prop)         # captures the loop with the Taylor weights
    prop.set_fd_coefficients(c4)
    opt = _forward(p, None, prop=prop)
    prop.set_fd_coefficients(None)
    back = _forward(p, None, prop=prop)
    prop.close()
    fresh = _forward(p, c4)
    assert np.array_equal(opt[1], fresh[1]) and np.array_equal(opt[0], fresh[0])
    assert np.array_equal(back[1], taylor[1])
    assert not np.array_equal(opt[1], taylor[1])


def test_adjoint_with_optimised_weights_is_the_transpose():
    torch = torch_cuda()
    c4 = M.mmod_optimized_coefficients(KMAX)
    p = W.tiny_problem(shape=(40, 44, 64), nt=120, nsrc=2, nrec=50, seed=21)
    rng = np.random.default_rng(4)
    w = torch.from_numpy(rng.standard_normal((len(p.src_ijk), p.nt)).astype(np.float32)).cuda()
    r = torch.from_numpy(rng.standard_normal((p.nt, len(p.rec_ijk))).astype(np.float32)).cuda()
    prop = M.Propagator.from_problem(p)
    prop.set_fd_coefficients(c4)
    prop.set_model(torch.from_numpy(p.vel).cuda())
    Fw = torch.zeros((p.nt, len(p.rec_ijk)), device="cuda")
    prop.forward(w, Fw)
    FTr = torch.zeros((len(p.src_ijk), p.nt), device="cuda")
    prop.adjoint(r, FTr)
    lhs, rhs = M.mmod_dot(Fw, r), M.mmod_dot(w, FTr)
    assert abs(lhs - rhs) <= 1e-6 * abs(lhs), (lhs, rhs)


def test_stability_bound_follows_the_weights():
    torch = torch_cuda()
    c4 = M.mmod_optimized_coefficients(KMAX)
    s_opt = max(sum(2 * c4[m - 1] * (1 - np.cos(m * k)) for m in range(1, 5)) for k in np.linspace(0, np.pi, 4001))
    s_tay = 2048 / 315
    h = 10.0
    v = 3000.0
    # a dt stable for the Taylor weights, unstable for the optimised ones
    dt = 2.0 / (v * np.sqrt(3 * (s_opt + s_tay) / 2 / h ** 2))
    p = W.tiny_problem(shape=(20, 20, 20), nt=5, nbl=0, h=(h, h, h))
    vel = torch.full((20, 20, 20), v, device="cuda")
    prop = M.Propagator((20, 20, 20), (h, h, h), dt, 5, src_ijk=p.src_ijk, rec_ijk=p.rec_ijk)
    prop.set_model(vel)                           # Taylor: stable
    with pytest.raises(M.MmodError) as ei:
        prop.set_fd_coefficients(c4)              # drops the model
    assert ei.value.status == -2
    with pytest.raises(M.MmodError) as ei:
        prop.set_model(vel)
    assert ei.value.status == -2
    prop.set_fd_coefficients([1.0, 0.0, 0.0, 0.0])     # second order: symbol max 4, stable here
    prop.set_model(vel)
    with pytest.raises(M.MmodError) as ei:
        prop.set_fd_coefficients([1.0, 1.0, 0.0, 0.0])   # inconsistent
    assert ei.value.status == -1
    prop.close()
