// Plain step kernel: one thread per grid point, neighbours read straight from
// global memory (L1/L2 cached), u = 0 outside the grid by explicit bounds
// tests, then a separate injection kernel adds the sources.  It performs
// exactly the FP32 operations of the TMA kernel in the same order
// (stencil.cuh, inject_point), so the two agree bit for bit; it is the
// validation kernel (MMOD_KERNEL_SIMPLE), not the fast path.
#include "mmod_internal.h"

namespace mmod {
namespace {

// u = 0 outside the grid, except above a free surface: the odd image
// u(i, j, -m) = -u(i, j, m).
__device__ __forceinline__ float ld0(const float *__restrict__ u, const StepArgs &a, int i, int j,
                                     int k) {
    const bool image = a.fs && k < 0;
    if (image) k = -k;
    const bool in = (unsigned)i < (unsigned)a.nx && (unsigned)j < (unsigned)a.ny &&
                    (unsigned)k < (unsigned)a.nz;
    const float v = in ? __ldg(u + (long long)k * a.plane + (long long)j * a.nxp + i) : 0.0f;
    return image ? -v : v;
}

__global__ void __launch_bounds__(128) step_simple_kernel(const StepArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= a.nx || j >= a.ny) return;
    const long long o = (long long)k * a.plane + (long long)j * a.nxp + i;
    const float p = __ldg(a.ucur + o);
    const float two_p = __fadd_rn(p, p);
    float lx = pair_first(a.w.x[0], ld0(a.ucur, a, i + 1, j, k), ld0(a.ucur, a, i - 1, j, k), two_p);
    float ly = pair_first(a.w.y[0], ld0(a.ucur, a, i, j + 1, k), ld0(a.ucur, a, i, j - 1, k), two_p);
    float lz = pair_first(a.w.z[0], ld0(a.ucur, a, i, j, k + 1), ld0(a.ucur, a, i, j, k - 1), two_p);
#pragma unroll
    for (int m = 2; m <= kRadius; ++m) {
        lx = pair_acc(lx, a.w.x[m - 1], ld0(a.ucur, a, i + m, j, k), ld0(a.ucur, a, i - m, j, k), two_p);
        ly = pair_acc(ly, a.w.y[m - 1], ld0(a.ucur, a, i, j + m, k), ld0(a.ucur, a, i, j - m, k), two_p);
        lz = pair_acc(lz, a.w.z[m - 1], ld0(a.ucur, a, i, j, k + m), ld0(a.ucur, a, i, j, k - m), two_p);
    }
    const float lap = lap_sum(lx, ly, lz);
    const float e = __fadd_rn(__fadd_rn(__ldg(a.ex + i), __ldg(a.ey + j)), __ldg(a.ez + k));
    const float out = __fmul_rn(num_damped(two_p, a.uprev[o], __ldg(a.c + o), lap, e), damp_factor(e));
    a.uout[o] = (a.fs && k == 0) ? 0.0f : out;   // p = 0 on a free surface
    if (a.gout) a.gout[o] = (a.fs && k == 0) ? 0.0f : lap;   // g^n = L u^n (sources: inject_kernel)
}

// Sources, after the step: one thread per injection point (stencil order).
__global__ void inject_kernel(const StepArgs a) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < a.inj.npts; p += gridDim.x * blockDim.x) {
        inject_point(a, p);
        if (a.gout) inject_g_points(a, a.n, p, p + 1, 0, 1);
    }
}

__global__ void gather_kernel(const float *__restrict__ u, const long long *__restrict__ off, int nrec,
                              float *__restrict__ dst) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nrec; r += gridDim.x * blockDim.x)
        dst[r] = u[off[r]];
}

}  // namespace

cudaError_t launch_step_simple(const StepArgs &a, cudaStream_t s) {
    if (a.nx <= 0 || a.ny <= 0 || a.nz <= 0) return cudaSuccess;
    dim3 block(32, 4);
    dim3 grid((a.nx + 31) / 32, (a.ny + 3) / 4, a.nz);
    step_simple_kernel<<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_inject(const StepArgs &a, cudaStream_t s) {
    if (a.inj.npts <= 0) return cudaSuccess;
    int blocks = (a.inj.npts + 127) / 128;
    if (blocks > 1024) blocks = 1024;
    inject_kernel<<<blocks, 128, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_gather(const float *u, const long long *rec_off, int nrec, float *dst,
                          cudaStream_t s) {
    if (nrec <= 0) return cudaSuccess;
    int blocks = (nrec + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    gather_kernel<<<blocks, 256, 0, s>>>(u, rec_off, nrec, dst);
    return cudaGetLastError();
}

}  // namespace mmod
