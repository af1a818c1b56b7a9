"""The byte models behind bench.py's roofline figures, on CPU.

The CPML model counts, per step, 16 B for every cell that lies in any
layer (u^n and c read, u^{n+1} read and written once) plus 16 B per layer
axis of the cell (psi_a and zeta_a read and written).  It is pinned here
against a brute-force count over the cells of small grids, with and without
a free surface (no top layer).  The gradient model is 48 B per point and
step with every state kept, and 64 B with segments.  With S FP32 segments
the first sweep writes g^n of the last one (+4 B on 1/S of the steps), and
that segment is not replayed (-20 B on 1/S).
"""
import itertools

import pytest

import bench


def brute_force_cpml(nx, ny, nz, L, free_surface):
    cells = axes = 0
    for k, j, i in itertools.product(range(nz), range(ny), range(nx)):
        in_x = i < L or i >= nx - L
        in_y = j < L or j >= ny - L
        in_z = (k < L and not free_surface) or k >= nz - L
        n = in_x + in_y + in_z
        cells += n > 0
        axes += n
    return cells, axes


@pytest.mark.parametrize("shape,L,fs", [((12, 10, 9), 3, False), ((12, 10, 9), 3, True), ((7, 30, 16), 2, False),
                                        ((20, 20, 20), 5, True)])
def test_cpml_layer_bytes_count_cells_and_axes(shape, L, fs):
    nx, ny, nz = shape
    b, cells, axes = bench.cpml_layer_bytes(nx, ny, nz, L, free_surface=fs)
    assert (cells, axes) == brute_force_cpml(nx, ny, nz, L, fs)
    assert b == 16 * cells + 16 * axes


def test_cpml_layer_bytes_on_the_bench_workload():
    # 240^3 with 20-cell layers: the cells outside the 200^3 interior, and
    # 2 x 20 x 240 x 240 cells per axis
    b, cells, axes = bench.cpml_layer_bytes(240, 240, 240, 20)
    assert cells == 240 ** 3 - 200 ** 3
    assert axes == 3 * 2 * 20 * 240 * 240
    assert b == 203_776_000


def test_gradient_bytes_per_point_and_step():
    assert bench.gradient_bytes_per_point_step(True)[0] == 48
    assert bench.gradient_bytes_per_point_step(False)[0] == 64
    assert bench.gradient_bytes_per_point_step(False, 20)[0] == pytest.approx(64 - 16 / 20)
    assert bench.gradient_bytes_per_point_step(False, 1)[0] == pytest.approx(48)   # one segment: nothing replayed


def test_roofline_arithmetic():
    r = bench.roofline_of(221_184_000, 0.0418, 6758.2, "step")
    assert r["achieved"] == pytest.approx(221_184_000 / 0.0418e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6758.2)
