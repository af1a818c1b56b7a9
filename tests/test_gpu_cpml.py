"""CPML layers (reading R17) on the GPU against the FP64 oracle, bit for bit
across the step kernels, absorbing on the GPU as in the oracle, and the calls
built for damping layers only refusing a CPML handle."""
import numpy as np
import pytest

import paper_2007_06048_gb300 as M
import workloads as W
from _gpu_util import rel_l2, run_gpu, run_oracle, torch_cuda

pytestmark = pytest.mark.gpu


def _cpml(p, f0=25.0, fs=False):
    p.cpml = True
    p.cpml_f0 = f0
    p.free_surface = fs
    return p


def trace_err(tr_g, tr_o, u_o):
    floor = np.abs(u_o).max() * np.sqrt(tr_o.size)
    return float(np.linalg.norm(tr_g.astype(np.float64) - tr_o) / max(np.linalg.norm(tr_o), floor))


# the layer passes work on ranges along each axis: 26-cell x layers take the
# line march (wider than a warp segment), 18 points with 8-cell layers merge
# both x ranges into one, 18-cell layers leave a 4-cell gap
# both ranges apart; 20- and 8-cell layers (with nx a multiple of 4) run the
# tiled passes, over tiles that are ragged along every line axis
CASES = [((40, 36, 70), 6, False), ((33, 64, 131), 8, False), ((9, 20, 9), 2, False), ((30, 28, 70), 5, True),
         ((64, 20, 40), 0, False), ((60, 60, 70), 26, False), ((30, 40, 18), 8, False), ((36, 40, 40), 18, True),
         ((47, 71, 100), 20, False), ((47, 71, 100), 20, True), ((40, 37, 68), 8, True)]


@pytest.mark.parametrize("shape,nbl,fs", CASES, ids=[f"{s}-L{n}-fs{int(f)}" for s, n, f in CASES])
def test_cpml_matches_oracle(orc, shape, nbl, fs):
    nz, ny, nx = shape
    p = _cpml(W.tiny_problem(shape=shape, nt=100, nbl=nbl, nsrc=3, nrec=12, seed=sum(shape) + nbl), fs=fs)
    p.src_ijk[0] = [1, 1, min(2, nz - 1)]          # inside the layers
    p.rec_ijk[0] = [nx - 1, ny - 1, nz - 1]
    tr_o, _, u_o = run_oracle(orc, p)
    tr_g, u_g, _ = run_gpu(p)
    assert rel_l2(u_g, u_o) <= 1e-5
    assert trace_err(tr_g, tr_o, u_o) <= 1e-5


def test_cpml_layered_240_1000_steps(orc):
    p = _cpml(W.layered_240(1000), f0=10.0)
    tr_o, _, u_o = run_oracle(orc, p)
    tr_g, u_g, _ = run_gpu(p)
    assert rel_l2(u_g, u_o) <= 1e-4
    assert rel_l2(tr_g, tr_o) <= 1e-4


def test_cpml_kernels_and_variants_bitwise():
    p = _cpml(W.tiny_problem(shape=(60, 50, 90), nt=40, nbl=7, nsrc=2, nrec=20, seed=3))
    tr_s, u_s, _ = run_gpu(p, kernel=M.KERNEL_SIMPLE)
    for v in range(M.mmod_tma_variant_count()):
        tr_t, u_t, _ = run_gpu(p, kernel=M.KERNEL_TMA, variant=v)
        assert np.array_equal(u_t, u_s) and np.array_equal(tr_t, tr_s), v


@pytest.mark.parametrize("fs", [False, True])
def test_cpml_interior_tiles_bitwise(orc, fs):
    """A grid with step-kernel tiles both inside and across the layers
    (70 x 80 x 200, 8-cell layers), with and without the free surface: the
    TMA step kernel equals the plain one bit for bit under CPML, and both
    match the oracle."""
    p = _cpml(W.tiny_problem(shape=(70, 80, 200), nt=60, nbl=8, nsrc=3, nrec=20, seed=12), fs=fs)
    p.src_ijk[0] = [100, 40, 3]          # in the top layer (or under the surface)
    p.src_ijk[1] = [3, 40, 35]           # in an x layer
    tr_s, u_s, _ = run_gpu(p, kernel=M.KERNEL_SIMPLE)
    tr_t, u_t, _ = run_gpu(p, kernel=M.KERNEL_TMA)
    assert np.array_equal(u_t, u_s) and np.array_equal(tr_t, tr_s)
    tr_o, _, u_o = run_oracle(orc, p)
    assert rel_l2(u_t, u_o) <= 1e-5
    assert trace_err(tr_t, tr_o, u_o) <= 1e-5


@pytest.mark.parametrize("fs", [False, True])
def test_cpml_planes_per_thread_keep_bits(fs):
    """MMOD_OPT_CPML_PLANES only regroups the layer passes' work (1 to 100
    layer lines per thread or row segments per warp): the same bits."""
    p = _cpml(W.tiny_problem(shape=(70, 45, 209), nt=30, nbl=8, nsrc=2, nrec=20, seed=14), fs=fs)
    tr_d, u_d, _ = run_gpu(p)
    for planes in (1, 3, 7, 100):
        tr_p, u_p, _ = run_gpu(p, options={M.OPT_CPML_PLANES: planes})
        assert np.array_equal(u_p, u_d) and np.array_equal(tr_p, tr_d), planes


# (45, 50, 98): nx not a multiple of 4, so x takes the marching pass while y
# and z run tiled in the same step
TILE_CASES = [((47, 71, 100), 20, False), ((47, 71, 100), 20, True), ((40, 37, 68), 8, False),
              ((41, 37, 68), 8, True), ((33, 64, 131), 8, False), ((45, 50, 98), 20, True)]


@pytest.mark.parametrize("shape,nbl,fs", TILE_CASES, ids=[f"{s}-L{n}-fs{int(f)}" for s, n, f in TILE_CASES])
def test_cpml_tiled_passes_keep_bits(shape, nbl, fs):
    """The tiled layer passes (whole units in shared memory by bulk-tensor
    copies) take the marching passes' FP32 operations: the same bits, with
    sources and receivers inside the layers."""
    nz, ny, nx = shape
    p = _cpml(W.tiny_problem(shape=shape, nt=50, nbl=nbl, nsrc=3, nrec=16, seed=nx + nbl), fs=fs)
    p.src_ijk[0] = [2, ny - 3, nz - 2]
    p.src_ijk[1] = [nx - 5, 4, nz // 2]
    p.rec_ijk[0] = [0, 0, nz - 1]
    p.rec_ijk[1] = [nx - 1, ny // 2, 1]
    tr_m, u_m, _ = run_gpu(p, options={M.OPT_CPML_TILES: 0}, pdl=0)
    assert np.abs(u_m).max() > 0
    for pdl in (0, 1):   # chained by programmatic dependent launch, or in stream order
        tr_t, u_t, _ = run_gpu(p, options={M.OPT_CPML_TILES: 1}, pdl=pdl)
        assert np.array_equal(u_t, u_m) and np.array_equal(tr_t, tr_m), pdl


def test_cpml_absorbs_on_the_gpu():
    """Against a GPU run on a grid large enough that nothing returns in the
    window: the CPML of 10 cells leaves < 2 %, the damping layer much more."""
    v, h, f = 2000.0, 10.0, 15.0
    dt = W.cfl_dt(0.35, (h, h, h), v)
    nt, L, n, big = 300, 10, 60, 150
    recs = [(18, 0, 0), (15, 15, 0), (0, 0, 17), (-16, 8, -8)]

    def run(nn, nbl, cpml):
        c = nn // 2
        p = W.Problem("absorb", np.full((nn, nn, nn), v, np.float32), (h, h, h), dt, nt, nbl,
                      np.array([[c, c, c]], np.int32), W.ricker(f, dt, nt)[None, :],
                      np.array([[c + a, c + b, c + e] for a, b, e in recs], np.int32), cpml=cpml, cpml_f0=f)
        return run_gpu(p, want_final=False)[0].astype(np.float64)

    ref = run(big, 0, False)
    err = {}
    for cpml in (True, False):
        tr = run(n, L, cpml)
        err[cpml] = max(np.linalg.norm(tr[:, r] - ref[:, r]) / np.linalg.norm(ref[:, r]) for r in range(len(recs)))
    assert err[True] < 0.02, err
    assert err[False] > 5 * err[True], err


def test_cpml_refuses_adjoint_gradient_fused_batch():
    torch = torch_cuda()
    p = _cpml(W.tiny_problem(shape=(20, 20, 40), nt=10, nbl=3))
    prop = M.Propagator.from_problem(p)
    prop.set_model(torch.from_numpy(p.vel).cuda())
    r = torch.zeros((p.nt, len(p.rec_ijk)), device="cuda")
    with pytest.raises(M.MmodError) as ei:
        prop.adjoint(r, torch.zeros((len(p.src_ijk), p.nt), device="cuda"))
    assert ei.value.status == -7
    with pytest.raises(M.MmodError) as ei:
        prop.gradient(torch.from_numpy(p.wavelet).cuda(), r, torch.zeros(p.vel.shape, device="cuda"), 2)
    assert ei.value.status == -7
    b = M.Batch([prop])
    b.set_mode(M.BATCH_FUSED)
    with pytest.raises(M.MmodError) as ei:
        b.forward([torch.from_numpy(p.wavelet).cuda()], [r])
    assert ei.value.status == -7
    b.set_mode(M.BATCH_STREAMS)            # the streams mode runs the handle's own CPML loop
    b.forward([torch.from_numpy(p.wavelet).cuda()], [r])
    torch.cuda.synchronize()
    b.close()
    prop.close()
