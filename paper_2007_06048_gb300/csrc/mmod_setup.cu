// Set-up kernels (run once per model or per call, outside the time loop):
// model scan (maximum velocity, invalid-value count), c = dt^2 v^2 into the
// padded layout, source scales, and dense <-> padded copies.
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
