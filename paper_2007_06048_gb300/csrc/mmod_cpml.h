// CPML layers of the constant-density propagator (mmod_cpml.cu).
#pragma once
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
    int zc;   // layer lines per thread (y, z passes) or row segments per warp (x pass), about
};

// Default lines per thread of the layer passes.
constexpr int kCpmlPlanes = 1;
// After the undamped step (u = u^n, uout = u^{n+1}): the layer terms on the
// layer cells, one pass per axis.
cudaError_t launch_cpml_layers(const CpmlArgs &p, const float *u, float *uout, cudaStream_t s);

}  // namespace mmod
