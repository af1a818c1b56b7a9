"""Variable-density staggered propagator on the GPU (FP32, C ABI) against the
FP64 oracle (reading R18), with the same gates as the constant-density path:
relative L2 of pressure, velocities and traces <= 1e-5 after up to 100 steps
and <= 1e-4 after 1000.  The TMA kernels and the plain kernels must agree bit
for bit."""
import numpy as np
import pytest

import paper_2007_06048_gb300 as M
import workloads as W
from _gpu_util import rel_l2, torch_cuda

pytestmark = pytest.mark.gpu


def run_vd(p, kernel=M.KERNEL_AUTO, state=None, pdl=None, zlen=None):
    torch = torch_cuda()
    prop = M.StaggeredPropagator.from_problem(p)
    if kernel != M.KERNEL_AUTO:
        prop.set_kernel(kernel)
    if pdl is not None:
        prop.set_option(M.OPT_PDL, pdl)
    if zlen is not None:
        prop.set_option(M.OPT_ZLEN, zlen)
    prop.set_model(torch.from_numpy(np.ascontiguousarray(p.vel)).cuda(),
                   torch.from_numpy(np.ascontiguousarray(p.rho)).cuda())
    nsrc, nrec = len(p.src_ijk), len(p.rec_ijk)
    wav = torch.from_numpy(np.ascontiguousarray(p.wavelet, np.float32)).cuda() if nsrc else None
    tr = torch.zeros((p.nt, nrec), device="cuda") if nrec else None
    fin = torch.zeros((4,) + p.vel.shape, device="cuda")
    if state is not None:
        prop.set_state(torch.from_numpy(np.ascontiguousarray(state, np.float32)).cuda())
    prop.forward(wav, tr, fin)
    torch.cuda.synchronize()
    return (np.zeros((p.nt, 0)) if tr is None else tr.cpu().numpy()), fin.cpu().numpy(), prop


def run_oracle_vd(orc, p, state0=None):
    return orc.forward_vd(p.vel, p.rho, p.h, p.dt, p.nt, nbl=p.nbl, refl=p.refl, cpml=p.cpml, f0=p.cpml_f0,
                          src_ijk=p.src_ijk, wavelet=p.wavelet, rec_ijk=p.rec_ijk, state0=state0,
                          want_state=True, free_surface=p.free_surface)


def check(tr_g, st_g, tr_o, st_o, tol):
    for f in range(4):
        if np.linalg.norm(st_o[f]) > 0:
            assert rel_l2(st_g[f], st_o[f]) <= tol, ("field", f, rel_l2(st_g[f], st_o[f]))
    if tr_o.size and np.linalg.norm(tr_o) > 0:
        assert rel_l2(tr_g, tr_o) <= tol, ("traces", rel_l2(tr_g, tr_o))


SHAPES = [((9, 9, 9), 0), ((13, 17, 35), 2), ((70, 33, 65), 5), ((5, 40, 3), 1), ((1, 1, 1), 0),
          ((2, 67, 129), 0), ((40, 1, 30), 0), ((37, 45, 131), 9)]


@pytest.mark.parametrize("cpml", [False, True], ids=["damping", "cpml"])
@pytest.mark.parametrize("shape,nbl", SHAPES, ids=[f"{s}-L{n}" for s, n in SHAPES])
def test_ragged_and_degenerate_shapes(orc, shape, nbl, cpml):
    nz, ny, nx = shape
    p = W.tiny_problem_vd(shape=shape, nt=60, nbl=nbl, nsrc=3, nrec=9, seed=nx * 7 + ny * 3 + nz)
    p.cpml, p.cpml_f0 = cpml, 25.0
    corners = [[0, 0, 0], [nx - 1, ny - 1, nz - 1], [nx - 1, 0, nz - 1], [0, ny - 1, 0]]
    p.src_ijk[0] = corners[1]
    p.src_ijk[1] = p.src_ijk[2]          # two sources on one point add up
    p.rec_ijk[:4] = corners
    p.rec_ijk[4] = p.rec_ijk[5]          # duplicated receiver
    p.rec_ijk[6] = p.src_ijk[0]
    tr_o, st_o = run_oracle_vd(orc, p)
    tr_g, st_g, prop = run_vd(p)
    check(tr_g, st_g, tr_o, st_o, 1e-5)
    assert np.array_equal(tr_g[:, 4], tr_g[:, 5])
    tr_s, st_s, _ = run_vd(p, kernel=M.KERNEL_SIMPLE)
    assert np.array_equal(tr_s, tr_g) and np.array_equal(st_s, st_g)
    assert prop.uses_tma


def test_layered_240_100_steps(orc):
    p = W.layered_240_vd(100)
    tr_o, st_o = run_oracle_vd(orc, p)
    tr_g, st_g, prop = run_vd(p)
    check(tr_g, st_g, tr_o, st_o, 1e-5)
    assert prop.launches >= 2 * p.nt          # velocity + pressure (sources folded in) per step


def test_layered_240_1000_steps_full_size(orc):
    """The benchmarked variable-density workload itself: 240^3, 1000 steps,
    57 600 receivers, damping layers."""
    p = W.layered_240_vd(1000)
    tr_o, st_o = run_oracle_vd(orc, p)
    tr_g, st_g, _ = run_vd(p)
    check(tr_g, st_g, tr_o, st_o, 1e-4)


def test_cpml_128_300_steps(orc):
    p = W.tiny_problem_vd(shape=(128, 120, 136), nt=300, nbl=12, nsrc=2, nrec=40, seed=4)
    p.cpml, p.cpml_f0 = True, 20.0
    tr_o, st_o = run_oracle_vd(orc, p)
    tr_g, st_g, _ = run_vd(p)
    check(tr_g, st_g, tr_o, st_o, 1e-5)


@pytest.mark.parametrize("shape,nbl,cpml", [((64, 64, 64), 8, False), ((97, 130, 200), 12, True),
                                            ((240, 240, 240), 20, False)])
def test_tma_kernels_are_bitwise_the_plain_kernels(shape, nbl, cpml):
    if shape == (240, 240, 240):
        p = W.layered_240_vd(200)
    else:
        p = W.tiny_problem_vd(shape=shape, nt=80, nbl=nbl, nsrc=2, nrec=30, seed=9)
    p.cpml, p.cpml_f0 = cpml, 15.0
    tr_t, st_t, prop = run_vd(p)
    assert prop.uses_tma
    tr_s, st_s, prop_s = run_vd(p, kernel=M.KERNEL_SIMPLE)
    assert not prop_s.uses_tma
    assert np.array_equal(tr_t, tr_s)
    assert np.array_equal(st_t, st_s)
    tr_n, st_n, _ = run_vd(p, pdl=1)           # with programmatic dependent launch
    assert np.array_equal(tr_n, tr_s) and np.array_equal(st_n, st_s)
    tr_z, st_z, _ = run_vd(p, zlen=7)          # z ranges of 7 planes
    assert np.array_equal(tr_z, tr_s) and np.array_equal(st_z, st_s)


def test_standing_wave_fp32():
    """The exact discrete standing wave (constant K, b) in FP32 on the GPU:
    p^n = P_n phi at points the zero boundary has not reached."""
    shape, h, v, rho, dt = (72, 70, 74), (10.0, 12.0, 9.0), 2200.0, 1800.0, 0.9e-3
    K, b = rho * v * v, 1.0 / rho
    k = np.array([2 * np.pi / 97.0, 2 * np.pi / 61.0, 2 * np.pi / 143.0])
    s = (0.3, 1.1, -0.4)
    a8 = [1225 / 1024, -245 / 3072, 49 / 5120, -5 / 7168]
    S = np.array([sum(2.0 / h[ax] * a8[m - 1] * np.sin((2 * m - 1) * k[ax] * h[ax] / 2) for m in range(1, 5))
                  for ax in range(3)])
    nz, ny, nx = shape
    xs = (np.arange(nx) * h[0], np.arange(ny) * h[1], np.arange(nz) * h[2])

    def field(half):
        f = [np.sin(k[a] * (xs[a] + 0.5 * h[a]) + s[a]) if a == half else np.cos(k[a] * xs[a] + s[a]) for a in range(3)]
        return f[2][:, None, None] * f[1][None, :, None] * f[0][None, None, :]

    V0 = 0.5 * dt * b * S
    st = np.stack([field(None)] + [V0[a] * field(a) for a in range(3)])
    nsteps = 4
    p = W.Problem("standing", np.full(shape, v, np.float32), h, dt, nsteps, 0, np.zeros((0, 3), np.int32),
                  np.zeros((0, nsteps), np.float32), np.zeros((0, 3), np.int32), rho=np.full(shape, rho, np.float32))
    _, out, _ = run_vd(p, state=st)
    P, V = 1.0, V0.copy()
    for _ in range(nsteps):
        V = V - dt * b * S * P
        P = P + dt * K * float(np.dot(S, V))
    m = 7 * nsteps + 1
    inner = (slice(m, -m),) * 3
    assert rel_l2(out[0][inner], (P * st[0])[inner]) < 2e-6
    for a in range(3):
        assert rel_l2(out[1 + a][inner], (V[a] / V0[a] * st[1 + a])[inner]) < 2e-6


# P = sum of coef * s^a t^b r^c, s = (i - i_c + 0.13) / 3 (t, r alike with
# other offsets): degree <= 8 per axis, where the order-8 staggered
# differences are exact (Sec. 3 system; see the oracle's pins)
_POLY = [(1.0, 8, 0, 0), (-0.7, 0, 8, 0), (0.4, 0, 0, 8), (1.3, 3, 2, 3), (-0.5, 5, 0, 4), (0.9, 2, 6, 0),
         (0.6, 7, 1, 1), (-0.8, 1, 1, 7), (0.2, 0, 0, 0)]
_A8 = (1225 / 1024, -245 / 3072, 49 / 5120, -5 / 7168)
_NP_AXIS = (2, 1, 0)   # array axis of x, y, z


def _poly_terms(shape, h, half_axis, deriv, scale=3.0):
    """sum over _POLY of d^deriv/dx_a^deriv (a = each axis in turn when
    deriv > 0, summed) at the grid points, shifted half a cell along
    half_axis; deriv 0: P itself."""
    nz, ny, nx = shape
    off = (0.13, -0.21, 0.37)
    t = [(np.arange(n) - (n - 1) / 2 + off[a] + (0.5 if a == half_axis else 0.0)) / scale
         for a, n in enumerate((nx, ny, nz))]
    Z, Y, X = np.meshgrid(t[2], t[1], t[0], indexing="ij")
    base = (X, Y, Z)
    out = np.zeros(shape)
    for coef, *pw in _POLY:
        axes = [None] if deriv == 0 else ([half_axis] if deriv == 1 else [0, 1, 2])
        for ax in axes:
            f = [base[a] ** pw[a] for a in range(3)]
            if ax is not None:
                k = pw[ax]
                if k < deriv:
                    continue
                f[ax] = (k if deriv == 1 else k * (k - 1)) * base[ax] ** (k - deriv) / (scale * h[ax]) ** deriv
            out += coef * f[0] * f[1] * f[2]
    return out


def _pair_sum(U, axis, h, shift_plus, shift_minus):
    """sum_m |a_m| (|U(i + m + shift_plus)| + |U(i - m + shift_minus)|) / h."""
    U = np.abs(U.astype(np.float64))
    ax = _NP_AXIS[axis]
    out = np.zeros(U.shape)
    for m in range(1, 5):
        out += abs(_A8[m - 1]) * (np.roll(U, -(m + shift_plus), axis=ax) + np.roll(U, m - shift_minus, axis=ax))
    return out / h[axis]


@pytest.mark.parametrize("kernel", [M.KERNEL_TMA, M.KERNEL_SIMPLE])
def test_polynomial_step_fp32(kernel):
    """The staggered polynomial pin on the GPU: from p^0 = P (degree <= 8 per
    axis), v^{-1/2} = 0 and a constant density, one step gives
    v_a^{1/2} = dt b dP/dx_a at the half points (D+ exact) and
    p^1 = P + dt^2 v^2 Laplacian(P) (D- D+ exact), per point within 8 FP32
    roundings of the pair terms (plus the products' rounding); a 1 % error
    in a_4 or order-6 weights exceed the bounds 400 to 10^5 times."""
    shape, h, dt, rho = (44, 40, 48), (9.0, 12.0, 10.0), 1.0e-3, 1800.0
    rng = np.random.default_rng(31)
    vel = rng.uniform(1500.0, 3000.0, shape).astype(np.float32)
    P = _poly_terms(shape, h, None, 0)
    P32 = P.astype(np.float32)
    st = np.zeros((4,) + shape, np.float32)
    st[0] = P32
    p = W.Problem("poly", vel, h, dt, 1, 0, np.zeros((0, 3), np.int32), np.zeros((0, 1), np.float32),
                  np.zeros((0, 3), np.int32), rho=np.full(shape, rho, np.float32))
    _, out, _ = run_vd(p, kernel=kernel, state=st)
    eps = 2.0 ** -24
    dtb = dt / rho
    inner_v = (slice(4, -5),) * 3
    vbound = []
    for a in range(3):
        exact = dtb * _poly_terms(shape, h, a, 1)
        bound = 8 * eps * dtb * _pair_sum(P32, a, h, 0, 1) + 4 * eps * np.abs(exact)
        vbound.append(bound)
        err = np.abs(out[1 + a].astype(np.float64) - exact)
        assert np.all(err[inner_v] <= bound[inner_v]), (a, float(np.max(err[inner_v] / bound[inner_v])))
    dtK = dt * rho * vel.astype(np.float64) ** 2
    update = dt * dt * vel.astype(np.float64) ** 2 * _poly_terms(shape, h, None, 2)
    bound = 2 * eps * np.abs(P) + 4 * eps * np.abs(update)
    for a in range(3):
        bound += dtK * (8 * eps * _pair_sum(out[1 + a], a, h, -1, 0) + _pair_sum(vbound[a], a, h, -1, 0))
    inner_p = (slice(8, -8),) * 3
    err = np.abs(out[0].astype(np.float64) - (P + update))
    assert np.all(err[inner_p] <= bound[inner_p]), float(np.max(err[inner_p] / bound[inner_p]))


def test_zero_steps_and_no_sources_or_receivers(orc):
    p = W.tiny_problem_vd(shape=(20, 21, 22), nt=0, nbl=2, nsrc=1, nrec=2)
    tr, st, _ = run_vd(p)
    assert tr.shape == (0, 2) and not st.any()
    q = W.tiny_problem_vd(shape=(20, 21, 22), nt=30, nbl=2, nsrc=0, nrec=0)
    rng = np.random.default_rng(3)
    st0 = rng.standard_normal((4,) + q.vel.shape).astype(np.float32)
    st0[0] *= 1e6
    _, st_g, _ = run_vd(q, state=st0)
    _, st_o = orc.forward_vd(q.vel, q.rho, q.h, q.dt, q.nt, nbl=q.nbl, state0=st0, want_state=True)
    check(np.zeros(0), st_g, np.zeros(0), st_o, 1e-5)


def test_error_paths():
    torch = torch_cuda()
    p = W.tiny_problem_vd(shape=(20, 21, 22), nt=10, nbl=2)
    base = dict(nbl=p.nbl, src_ijk=p.src_ijk, rec_ijk=p.rec_ijk)
    with pytest.raises(M.MmodError) as e:
        M.StaggeredPropagator(p.vel.shape, p.h, p.dt, p.nt, nbl=30)
    assert e.value.status == -1
    cfg = M._config(22, 21, 20, p.h, p.dt, p.nt, 2, p.src_ijk, p.rec_ijk, 6, 1e-3)
    import ctypes
    out = ctypes.c_void_p()
    assert M.load().mmod_vd_create(ctypes.byref(cfg), 0, ctypes.byref(out)) == -7     # order 6
    cfg = M._config(22, 21, 4, p.h, p.dt, p.nt, 1, np.zeros((0, 3), np.int32), np.zeros((0, 3), np.int32), 8, 1e-3,
                    free_surface=True)
    assert M.load().mmod_vd_create(ctypes.byref(cfg), 0, ctypes.byref(out)) == -1     # surface with nz < 5
    prop = M.StaggeredPropagator(p.vel.shape, p.h, p.dt, p.nt, **base)
    wav = torch.zeros((2, p.nt), device="cuda")
    tr = torch.zeros((p.nt, len(p.rec_ijk)), device="cuda")
    with pytest.raises(M.MmodError) as e:
        prop.forward(wav, tr)
    assert e.value.status == -6                                   # no model yet
    vel = torch.from_numpy(p.vel).cuda()
    rho = torch.from_numpy(p.rho).cuda()
    with pytest.raises(M.MmodError) as e:
        prop.set_model(torch.from_numpy(p.vel), rho)               # host pointer
    assert e.value.status == -1
    bad = rho.clone()
    bad[3, 4, 5] = -1.0
    with pytest.raises(M.MmodError) as e:
        prop.set_model(vel, bad)
    assert e.value.status == -1
    fast = M.StaggeredPropagator(p.vel.shape, p.h, p.dt * 4, p.nt, **base)
    with pytest.raises(M.MmodError) as e:
        fast.set_model(vel, rho)
    assert e.value.status == -2
    prop.set_model(vel, rho)
    prop.forward(wav, tr)
    torch.cuda.synchronize()
    assert prop.loop_ms() > 0


FS_SHAPES = [((13, 17, 35), 2), ((70, 33, 65), 5), ((5, 40, 3), 1), ((37, 45, 131), 9), ((6, 20, 70), 0)]


@pytest.mark.parametrize("cpml", [False, True], ids=["damping", "cpml"])
@pytest.mark.parametrize("shape,nbl", FS_SHAPES, ids=[f"{s}-L{n}" for s, n in FS_SHAPES])
def test_free_surface_ragged_shapes(orc, shape, nbl, cpml):
    """With the surface option: sources on, just under and far below the
    surface, receivers on it (they read 0) and under it; TMA = plain bits."""
    nz, ny, nx = shape
    p = W.tiny_problem_vd(shape=shape, nt=60, nbl=nbl, nsrc=3, nrec=9, seed=nx * 5 + ny * 3 + nz)
    p.cpml, p.cpml_f0, p.free_surface = cpml, 25.0, True
    p.src_ijk[0] = [nx // 2, ny // 2, 0]
    p.src_ijk[1] = [nx - 1, 0, 1]
    p.rec_ijk[0] = [0, 0, 0]
    p.rec_ijk[1] = [nx // 2, ny - 1, 1]
    tr_o, st_o = run_oracle_vd(orc, p)
    tr_g, st_g, prop = run_vd(p)
    assert prop.uses_tma
    check(tr_g, st_g, tr_o, st_o, 1e-5)
    assert not tr_g[:, 0].any() and not st_g[0][0].any()
    tr_s, st_s, _ = run_vd(p, kernel=M.KERNEL_SIMPLE)
    assert np.array_equal(tr_s, tr_g) and np.array_equal(st_s, st_g)


def test_free_surface_layered_240_1000_steps(orc):
    """The 240^3 Gardner-density workload with the surface on and the
    receivers one plane under it, over 1000 steps."""
    p = W.layered_240_vd(1000)
    p.free_surface = True
    p.rec_ijk[:, 2] = 1
    tr_o, st_o = run_oracle_vd(orc, p)
    tr_g, st_g, _ = run_vd(p)
    check(tr_g, st_g, tr_o, st_o, 1e-4)


def test_free_surface_standing_wave_fp32():
    """cos(kx x) cos(ky y) sin(kz z): exact with the images up to the surface."""
    shape, h, v, rho, dt = (60, 70, 74), (10.0, 12.0, 9.0), 2200.0, 1800.0, 0.9e-3
    K, b = rho * v * v, 1.0 / rho
    k = np.array([2 * np.pi / 97.0, 2 * np.pi / 61.0, 2 * np.pi / 143.0])
    a8 = [1225 / 1024, -245 / 3072, 49 / 5120, -5 / 7168]
    S = np.array([sum(2.0 / h[ax] * a8[m - 1] * np.sin((2 * m - 1) * k[ax] * h[ax] / 2) for m in range(1, 5))
                  for ax in range(3)])
    nz, ny, nx = shape
    x, y, z = np.arange(nx) * h[0], np.arange(ny) * h[1], np.arange(nz) * h[2]

    def prod(fz, fy, fx):
        return fz[:, None, None] * fy[None, :, None] * fx[None, None, :]

    cx, cy = np.cos(k[0] * x + 0.3), np.cos(k[1] * y + 1.1)
    f = [prod(np.sin(k[2] * z), cy, cx), prod(np.sin(k[2] * z), cy, np.sin(k[0] * (x + 0.5 * h[0]) + 0.3)),
         prod(np.sin(k[2] * z), np.sin(k[1] * (y + 0.5 * h[1]) + 1.1), cx),
         prod(np.cos(k[2] * (z + 0.5 * h[2])), cy, cx)]
    sgn = np.array([1.0, 1.0, -1.0])
    V0 = 0.5 * dt * b * S * sgn
    st = np.stack([f[0]] + [V0[a] * f[1 + a] for a in range(3)])
    nsteps = 4
    p = W.Problem("standing-fs", np.full(shape, v, np.float32), h, dt, nsteps, 0, np.zeros((0, 3), np.int32),
                  np.zeros((0, nsteps), np.float32), np.zeros((0, 3), np.int32), rho=np.full(shape, rho, np.float32),
                  free_surface=True)
    _, out, _ = run_vd(p, state=st)
    P, V = 1.0, V0.copy()
    for _ in range(nsteps):
        V = V - dt * b * S * sgn * P
        P = P + dt * K * float(np.dot(S * sgn, V))
    m = 7 * nsteps + 1
    near = (slice(0, nz - m), slice(m, -m), slice(m, -m))
    assert rel_l2(out[0][near], (P * f[0])[near]) < 2e-6
    for a in range(3):
        assert rel_l2(out[1 + a][near], (V[a] * f[1 + a])[near]) < 2e-6
