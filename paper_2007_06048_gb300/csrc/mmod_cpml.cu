// CPML layers for the second-order equation (the paper's convolutional PML,
// Sec. 3): complex-frequency-shifted stretching on each axis with two memory
// variables per axis,
//     u_tt = v^2 sum_a [ D2_a u + D1_a psi_a + zeta_a ],
//     psi_a^n  = b_a psi_a^{n-1}  + g_a D1_a u^n,
//     zeta_a^n = b_a zeta_a^{n-1} + g_a (D2_a u^n + D1_a psi_a^n),
// b = exp(-(d + alpha) dt), g = d (b - 1) / (d + alpha) per cell of the axis
// (zero outside the layers), D2_a the order-8 second difference (the step
// kernels' pair form), D1_a the order-8 centred first difference.
//
// Each step runs three kernels: psi from u^n (cells with g != 0), the usual
// step kernel without damping (u^{n+1} = 2u^n - u^{n-1} + c L u^n + sources),
// then the correction u^{n+1} += c sum_a (D1_a psi_a + zeta_a) on the layer
// cells, which also advances zeta.  u and psi are 0 outside the grid.
// Memory variables are full padded volumes; only layer cells are touched.
#include "mmod_internal.h"

namespace mmod {
namespace {

__device__ __forceinline__ float at0(const float *__restrict__ v, const CpmlArgs &p, int i, int j, int k) {
    const bool in = (unsigned)i < (unsigned)p.nx && (unsigned)j < (unsigned)p.ny && (unsigned)k < (unsigned)p.nz;
    return in ? __ldg(v + (long long)k * p.plane + (long long)j * p.nxp + i) : 0.0f;
}

// The 9 values of v along axis a centred on (i, j, k), all loads issued
// before any arithmetic (0 outside the grid).
__device__ __forceinline__ void line(const float *__restrict__ v, const CpmlArgs &p, int a, int i, int j, int k,
                                     float (&x)[2 * kRadius + 1]) {
    const int di = a == 0, dj = a == 1, dk = a == 2;
#pragma unroll
    for (int m = -kRadius; m <= kRadius; ++m) x[m + kRadius] = at0(v, p, i + m * di, j + m * dj, k + m * dk);
}

// order-8 first difference from a line of 9 values, divided by h_a
__device__ __forceinline__ float d1_line(const float (&x)[2 * kRadius + 1], float inv_h) {
    constexpr float w[4] = {4.0f / 5.0f, -1.0f / 5.0f, 4.0f / 105.0f, -1.0f / 280.0f};
    float s = 0.0f;
#pragma unroll
    for (int m = 1; m <= kRadius; ++m) s = __fmaf_rn(w[m - 1], __fsub_rn(x[kRadius + m], x[kRadius - m]), s);
    return __fmul_rn(s, inv_h);
}

__global__ void cpml_psi_kernel(const CpmlArgs p, const float *__restrict__ u) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z * blockDim.z + threadIdx.z;
    if (i >= p.nx || j >= p.ny || k >= p.nz) return;
    const int idx[3] = {i, j, k};
    const long long o = (long long)k * p.plane + (long long)j * p.nxp + i;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float g = __ldg(p.g[a] + idx[a]);
        if (g == 0.0f) continue;
        float x[2 * kRadius + 1];
        line(u, p, a, i, j, k, x);
        const float old = p.psi[a][o];
        p.psi[a][o] = __fmaf_rn(__ldg(p.b[a] + idx[a]), old, __fmul_rn(g, d1_line(x, p.inv_h[a])));
    }
}

__global__ void cpml_correct_kernel(const CpmlArgs p, const float *__restrict__ u, float *__restrict__ uout) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z * blockDim.z + threadIdx.z;
    if (i >= p.nx || j >= p.ny || k >= p.nz) return;
    if (p.fs && k == 0) return;   // the free-surface plane stays 0
    const int idx[3] = {i, j, k};
    const long long o = (long long)k * p.plane + (long long)j * p.nxp + i;
    float acc = 0.0f;
    bool any = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float g = __ldg(p.g[a] + idx[a]);
        if (g == 0.0f) continue;
        any = true;
        float x[2 * kRadius + 1], q[2 * kRadius + 1];
        line(u, p, a, i, j, k, x);
        line(p.psi[a], p, a, i, j, k, q);
        const float zold = p.zeta[a][o];
        const float two_p = __fadd_rn(x[kRadius], x[kRadius]);
        float d2 = pair_first(p.w[a][0], x[kRadius + 1], x[kRadius - 1], two_p);
#pragma unroll
        for (int m = 2; m <= kRadius; ++m) d2 = pair_acc(d2, p.w[a][m - 1], x[kRadius + m], x[kRadius - m], two_p);
        const float dpsi = d1_line(q, p.inv_h[a]);
        const float z = __fmaf_rn(__ldg(p.b[a] + idx[a]), zold, __fmul_rn(g, __fadd_rn(d2, dpsi)));
        p.zeta[a][o] = z;
        acc = __fadd_rn(acc, __fadd_rn(dpsi, z));
    }
    if (any) uout[o] = __fmaf_rn(__ldg(p.c + o), acc, uout[o]);
}

// Blocks of 32 x-consecutive points over 4 rows (other shapes up to 32 x 2 x 8
// measured the same).
constexpr dim3 kBlock(32, 4, 1);

dim3 grid_of(const CpmlArgs &p, dim3 block) {
    return dim3((p.nx + block.x - 1) / block.x, (p.ny + block.y - 1) / block.y, (p.nz + block.z - 1) / block.z);
}

}  // namespace

cudaError_t launch_cpml_psi(const CpmlArgs &p, const float *u, cudaStream_t s) {
    if (p.nx <= 0 || p.ny <= 0 || p.nz <= 0) return cudaSuccess;
    cpml_psi_kernel<<<grid_of(p, kBlock), kBlock, 0, s>>>(p, u);
    return cudaGetLastError();
}

cudaError_t launch_cpml_correct(const CpmlArgs &p, const float *u, float *uout, cudaStream_t s) {
    if (p.nx <= 0 || p.ny <= 0 || p.nz <= 0) return cudaSuccess;
    cpml_correct_kernel<<<grid_of(p, kBlock), kBlock, 0, s>>>(p, u, uout);
    return cudaGetLastError();
}

}  // namespace mmod
