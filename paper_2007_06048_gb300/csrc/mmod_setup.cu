// Set-up kernels (run once per model or per call, outside the time loop):
// model scan (maximum velocity, invalid-value count), c = dt^2 v^2 into the
// padded layout, source scales, and dense <-> padded copies.
#include <algorithm>

#include "mmod_internal.h"

namespace mmod {
namespace {

__global__ void model_scan_kernel(const float *__restrict__ vel, long long n, unsigned int *vmax_bits,
                                  unsigned long long *bad) {
    unsigned int local_max = 0;
    unsigned long long local_bad = 0;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
         q += (long long)gridDim.x * blockDim.x) {
        const float v = vel[q];
        if (!(v > 0.0f) || !isfinite(v)) {
            ++local_bad;
        } else {
            // positive finite floats order like their bit patterns
            const unsigned int b = __float_as_uint(v);
            local_max = b > local_max ? b : local_max;
        }
    }
    for (int off = 16; off > 0; off >>= 1) {
        const unsigned int o = __shfl_xor_sync(0xffffffffu, local_max, off);
        local_max = o > local_max ? o : local_max;
        local_bad += __shfl_xor_sync(0xffffffffu, local_bad, off);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(vmax_bits, local_max);
        if (local_bad) atomicAdd(bad, local_bad);
    }
}

// c = dt^2 v^2 formed in FP64 and rounded once to FP32; padding columns = 0.
__global__ void model_fill_kernel(const float *__restrict__ vel, int nx, int ny, int nz, int nxp,
                                  double dt, float *__restrict__ c) {
    const long long total = (long long)nxp * ny * nz;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(q % nxp);
        const long long row = q / nxp;          // k * ny + j
        float out = 0.0f;
        if (i < nx) {
            const double v = (double)vel[row * nx + i];
            out = (float)(dt * dt * v * v);
        }
        c[q] = out;
    }
}

__global__ void source_scale_kernel(const float *__restrict__ vel, int nx, int ny, int nsrc,
                                    const int *si, const int *sj, const int *sk, double dt, double cell,
                                    float *scale) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nsrc) return;
    const double v = (double)vel[((long long)sk[t] * ny + sj[t]) * nx + si[t]];
    scale[t] = (float)(dt * dt * v * v / cell);
}

__global__ void pack_kernel(const float *__restrict__ dense, int nx, int ny, int nz, int nxp,
                            float *__restrict__ padded) {
    const long long total = (long long)nxp * ny * nz;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(q % nxp);
        const long long row = q / nxp;
        padded[q] = (i < nx && dense) ? dense[row * nx + i] : 0.0f;
    }
}

__global__ void unpack_kernel(const float *__restrict__ padded, int nx, int ny, int nz, int nxp,
                              float *__restrict__ dense) {
    const long long total = (long long)nx * ny * nz;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(q % nx);
        const long long row = q / nx;
        dense[q] = padded[row * nxp + i];
    }
}

inline int grid_for(long long n, int block) {
    long long b = (n + block - 1) / block;
    if (b > 152 * 32) b = 152 * 32;
    return b < 1 ? 1 : (int)b;
}

}  // namespace

cudaError_t launch_model_scan(const float *vel, long long n, unsigned int *vmax_bits,
                              unsigned long long *bad, cudaStream_t s) {
    model_scan_kernel<<<grid_for(n, 256), 256, 0, s>>>(vel, n, vmax_bits, bad);
    return cudaGetLastError();
}

cudaError_t launch_model_fill(const float *vel, int nx, int ny, int nz, int nxp, double dt,
                              float *c, cudaStream_t s) {
    model_fill_kernel<<<grid_for((long long)nxp * ny * nz, 256), 256, 0, s>>>(vel, nx, ny, nz, nxp,
                                                                               dt, c);
    return cudaGetLastError();
}

cudaError_t launch_source_scale(const float *vel, int nx, int ny, int nsrc, const int *src_i,
                                const int *src_j, const int *src_k, double dt, double cell,
                                float *scale, cudaStream_t s) {
    if (nsrc <= 0) return cudaSuccess;
    source_scale_kernel<<<(nsrc + 127) / 128, 128, 0, s>>>(vel, nx, ny, nsrc, src_i, src_j, src_k,
                                                            dt, cell, scale);
    return cudaGetLastError();
}

cudaError_t launch_pack(const float *dense, int nx, int ny, int nz, int nxp, float *padded,
                        cudaStream_t s) {
    pack_kernel<<<grid_for((long long)nxp * ny * nz, 256), 256, 0, s>>>(dense, nx, ny, nz, nxp,
                                                                         padded);
    return cudaGetLastError();
}

cudaError_t launch_unpack(const float *padded, int nx, int ny, int nz, int nxp, float *dense,
                          cudaStream_t s) {
    unpack_kernel<<<grid_for((long long)nx * ny * nz, 256), 256, 0, s>>>(padded, nx, ny, nz, nxp,
                                                                          dense);
    return cudaGetLastError();
}

}  // namespace mmod

namespace mmod {
namespace {

// Largest difference, in units in the last place, between the kernels'
// damping reciprocal and CUDA's correctly rounded __frcp_rn over n values of
// d spread evenly over [1, 8).
__global__ void recip_check_kernel(int n, unsigned int *max_ulp) {
    unsigned int worst = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float d = 1.0f + 7.0f * ((float)i / (float)n);
        const int a = __float_as_int(recip_nr(d)), b = __float_as_int(__frcp_rn(d));
        const unsigned int ulp = (unsigned int)(a > b ? a - b : b - a);
        worst = ulp > worst ? ulp : worst;
    }
    atomicMax(max_ulp, worst);
}

}  // namespace
}  // namespace mmod

extern "C" __attribute__((visibility("default"))) int mmod_check_recip(int n, unsigned int *max_ulp_out) {
    if (n <= 0 || !max_ulp_out) return MMOD_ERR_ARG;
    unsigned int *d = nullptr;
    if (cudaMalloc(&d, sizeof(unsigned int)) != cudaSuccess) return MMOD_ERR_OOM;
    cudaMemset(d, 0, sizeof(unsigned int));
    mmod::recip_check_kernel<<<152, 256>>>(n, d);
    cudaError_t e = cudaMemcpy(max_ulp_out, d, sizeof(unsigned int), cudaMemcpyDeviceToHost);
    cudaFree(d);
    return e == cudaSuccess ? MMOD_OK : MMOD_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// Adjoint and gradient helpers.
// ---------------------------------------------------------------------------
namespace mmod {
namespace {

// adj[s][n] = g[nt-1-n][s] * scale.
__global__ void unreverse_transpose_kernel(const float *__restrict__ g, int nt, int ncol, double scale,
                                           float *__restrict__ adj) {
    const long long total = (long long)nt * ncol;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const int col = (int)(q / nt), n = (int)(q % nt);
        adj[q] = (float)((double)g[(long long)(nt - 1 - n) * ncol + col] * scale);
    }
}

// Zero-lag imaging condition: with mu = psi / c the adjoint state,
//   dJ/dc = sum_n mu^{n+1} g^n,  g^n = L u^n + s^n (written by the replay's
// step kernel), so the kernel accumulates A = sum_n psi^{n+1} g^n (FP32
// fused multiply-adds, in step order) and the factor 1 / c is applied once at
// the end (dJ/dv = 2 dt^2 v A / c = 2 A / v).
// Four consecutive x of one row per thread (16-byte loads; rows are padded to
// 32 floats, so a group never straddles rows); columns past nx are loaded
// (in bounds of the padded row) but not stored.  NS = 1: forward step n
// (psi[0] = psi^{n+1}, g[0] = g^n); NS = 2: steps n and n - 1 in that order
// (psi[1] = psi^n, g[1] = g^{n-1}), the same operations as two single-step
// passes with A read and written once.
struct ImagingArgs {
    const float4 *psi[2];
    const float4 *g[2];
    int nx, ny, nz, nxp;
    float4 *acc;
};

template <int NS>
__global__ void imaging_kernel(const ImagingArgs a) {
    const int per_row = a.nxp >> 2;
    const long long total = (long long)per_row * a.ny * a.nz;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const int row = total <= 0xffffffffLL ? (int)((unsigned)q / (unsigned)per_row) : (int)(q / per_row);
        const int i0 = (int)(q - (long long)row * per_row) * 4;
        if (i0 >= a.nx) continue;
        float4 ps[NS], gg[NS];
#pragma unroll
        for (int t = 0; t < NS; ++t) {
            ps[t] = a.psi[t][q];
            gg[t] = a.g[t][q];
        }
        float4 acc = a.acc[q];
#pragma unroll
        for (int t = 0; t < NS; ++t) {
            acc.x = __fmaf_rn(ps[t].x, gg[t].x, acc.x);
            acc.y = __fmaf_rn(ps[t].y, gg[t].y, acc.y);
            acc.z = __fmaf_rn(ps[t].z, gg[t].z, acc.z);
            acc.w = __fmaf_rn(ps[t].w, gg[t].w, acc.w);
        }
        if (i0 + 3 < a.nx) {
            a.acc[q] = acc;
        } else {   // the row's last group: keep the padding untouched
            float *ap = reinterpret_cast<float *>(a.acc + q);
            ap[0] = acc.x;
            if (i0 + 1 < a.nx) ap[1] = acc.y;
            if (i0 + 2 < a.nx) ap[2] = acc.z;
        }
    }
}

// grad_v = 2 A / v (A = sum_n psi^{n+1} g^n, c = dt^2 v^2), dense output,
// FP32 (correctly rounded division).
__global__ void grad_to_velocity_kernel(const float *__restrict__ acc, const float *__restrict__ vel, int nx,
                                        int ny, int nz, int nxp, float *__restrict__ gv) {
    const long long total = (long long)nx * ny * nz;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(q % nx);
        const long long o = (q / nx) * nxp + i;
        gv[q] = __fdiv_rn(__fmul_rn(2.0f, acc[o]), vel[q]);
    }
}

// FP64 sum of a[i] * b[i] (block partials, then one atomic per block).
__global__ void dot_kernel(const float *__restrict__ a, const float *__restrict__ b, long long n, double *out) {
    double acc = 0.0;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
        acc += (double)a[q] * (double)b[q];
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    __shared__ double part[32];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.0;
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        if (threadIdx.x == 0) atomicAdd(out, acc);
    }
}

inline int grid2(long long n) {
    long long b = (n + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    return b < 1 ? 1 : (int)b;
}

}  // namespace

cudaError_t launch_unreverse_transpose(const float *g, int nt, int ncol, double scale, float *out,
                                       cudaStream_t s) {
    if ((long long)nt * ncol == 0) return cudaSuccess;
    unreverse_transpose_kernel<<<grid2((long long)nt * ncol), 256, 0, s>>>(g, nt, ncol, scale, out);
    return cudaGetLastError();
}

cudaError_t launch_imaging(int nsteps, const float *const *psi, const float *const *g, int nx, int ny, int nz,
                           int nxp, float *acc, cudaStream_t s) {
    if (nsteps < 1 || nsteps > 2) return cudaErrorInvalidValue;
    ImagingArgs a{};
    for (int t = 0; t < nsteps; ++t) {
        a.psi[t] = reinterpret_cast<const float4 *>(psi[t]);
        a.g[t] = reinterpret_cast<const float4 *>(g[t]);
    }
    a.nx = nx; a.ny = ny; a.nz = nz; a.nxp = nxp;
    a.acc = reinterpret_cast<float4 *>(acc);
    const long long groups = (long long)(nxp / 4) * ny * nz;
    const int grid = (int)std::min<long long>((groups + 255) / 256, 152LL * 8);
    if (nsteps == 1)
        imaging_kernel<1><<<grid, 256, 0, s>>>(a);
    else
        imaging_kernel<2><<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_grad_to_velocity(const float *acc, const float *vel, int nx, int ny, int nz, int nxp,
                                    float *grad_v, cudaStream_t s) {
    grad_to_velocity_kernel<<<grid2((long long)nx * ny * nz), 256, 0, s>>>(acc, vel, nx, ny, nz, nxp, grad_v);
    return cudaGetLastError();
}

cudaError_t launch_dot(const float *a, const float *b, long long n, double *out, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    dot_kernel<<<grid2(n), 256, 0, s>>>(a, b, n, out);
    return cudaGetLastError();
}

}  // namespace mmod
