// CPML layers of the constant-density propagator (mmod_cpml.cu).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include "stencil.cuh"

namespace mmod {

// CPML layers (mmod_cpml.cu): memory variables psi_a and zeta_a (padded
// volumes), per-cell coefficients b_a, g_a of each axis (g = 0 outside the
// layers), the layer width, the step kernels' weights and 1 / h_a.
struct CpmlArgs {
    int nx, ny, nz, nxp;
    long long plane;
    int fs, nbl;
    float *psi[3], *zeta[3];
    const float *b[3], *g[3];
    float inv_h[3];
    float w[3][kRadius];
    const float *c;
    int zc;      // layer lines per thread (y, z passes) or row segments per warp (x pass), about
    int tiles;   // 1: tiled passes on the axes that allow them
    int pdl;     // 1: tiled passes as programmatic dependent launches
    int *err;    // device view of the handle's error word (a bounded wait gave up)
    // x layers of the tiled pass in compact form, each [range][nzp][y][L]
    // with nzp = nz rounded up to a multiple of 4: psi_x | zeta_x | c_x
    // (null: no tiled x pass)
    float *xc;
};

// Default lines per thread of the layer passes.
constexpr int kCpmlPlanes = 1;

// Tensor maps of one axis's tiled layer pass for one buffer pair: u^n with
// the axis's 4-cell margins, and the layer boxes of u^{n+1}, psi_a, zeta_a
// and c.
struct CpmlTileMaps {
    CUtensorMap u, uout, psi, zeta, c;
};

// Tiled passes of a handle: maps per (u buffer b: u = u[b], uout = u[1 - b])
// and axis; ok[a] where axis a's pass can run tiled (two layer ranges, or
// the lower one alone under a free surface, of a compiled width; for x also
// 16-byte aligned row segments).
struct CpmlTiles {
    CpmlTileMaps maps[2][3];
    bool ok[3];
    int resident[3];   // blocks of each axis's persistent pass that fit at once
};

// Floats of the compact x-layer arrays (p.xc) the tiled x pass needs; 0
// where the x pass cannot run tiled.
long long cpml_x_compact_floats(const CpmlArgs &p);

// Builds the tile maps for the wavefield buffers u[0], u[1] and sets ok[]
// for the axes whose tiled pass can run (an axis whose maps cannot be
// encoded keeps the marching pass).  Returns true.
bool make_cpml_tiles(const CpmlArgs &p, float *const u[2], CpmlTiles *t);

// c_x of the compact x layers from c (after set_model's fill); no-op
// without p.xc.
cudaError_t launch_cpml_pack_c(const CpmlArgs &p, cudaStream_t s);

// After the undamped step (u = u^n, uout = u^{n+1}): the layer terms on the
// layer cells, one pass per axis.  tiles: the handle's tile maps (null:
// march kernels only), buffer: b with u = u[b]; *launches: the kernels
// launched.
cudaError_t launch_cpml_layers(const CpmlArgs &p, const CpmlTiles *tiles, int buffer, const float *u, float *uout,
                               cudaStream_t s, int *launches);

}  // namespace mmod
