// Internal declarations of the propagator library: the handle, the argument
// block of the step kernels and the launchers.  Not part of the public ABI.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "mmod.h"
#include "stencil.cuh"

namespace mmod {

// Everything a step kernel needs; passed by value (kernel parameter space).
struct StepArgs {
    int nx, ny, nz;            // grid
    int nxp;                   // padded row length (floats), multiple of 32
    long long plane;           // nxp * ny
    int nbl;                   // damping width: inner region is [nbl, n - 1 - nbl]
    int nt;                    // steps of the run (wavelet row length)
    int n;                     // this step: computes u^{n+1}
    Weights w;                 // c_m / h_a^2
    const float *ucur;         // u^n       (padded layout)
    float *uprev;              // u^{n-1} in, u^{n+1} out
    const float *c;            // dt^2 v^2  (padded layout)
    const float *ex, *ey, *ez; // dt * eta per axis
    // point sources, sorted by depth k: sources of plane k are
    // [src_kstart[k], src_kstart[k+1])
    const int *src_kstart;
    const int *src_i, *src_j, *src_row;   // position and wavelet row
    const float *src_scale;               // c(x_s) / (hx hy hz)
    const float *wavelet;                 // [nsrc][nt]
    // receivers: the kernel of step n copies u^n (its ucur) into traces[n-1]
    int nrec;
    const long long *rec_off;             // padded offsets
    float *traces;                        // [nt][nrec]
    int *err;                             // device view of the mapped error word
    int pdl;                              // 1: launched as a programmatic dependent of the previous step
};

// Host helpers shared by the entry points (mmod_api.cu).
void damping_profile(int n, int nbl, double h, double vmax, double R, double dt, float *out);
void set_thread_error(const char *msg);   // fixed buffer read by mmod_last_error(NULL)

// Order-8 Taylor weights of the second derivative (Sec. 3):
// c_1..c_4 = 8/5, -1/5, 8/315, -1/560.
constexpr double kTaylor8[4] = {8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0, -1.0 / 560.0};
// Largest magnitude of the order-8 stencil's symbol (at k h = pi):
// 4 (c_1 + c_3) = 2048 / 315; leapfrog is stable iff dt^2 v^2 sum_a K_a <= 4.
constexpr double kSymbolMax8 = 2048.0 / 315.0;

// Launchers (mmod_step_simple.cu, mmod_step_tma.cu, mmod_setup.cu).
cudaError_t launch_step_simple(const StepArgs &a, cudaStream_t s);
cudaError_t launch_gather(const float *u, const long long *rec_off, int nrec, float *dst,
                          cudaStream_t s);

struct TmaPlan;   // tile shape / grid decomposition of the TMA kernel
cudaError_t launch_step_tma(const StepArgs &a, const CUtensorMap *cur_map,
                            const CUtensorMap *prev_map, const CUtensorMap *c_map,
                            const TmaPlan &plan, cudaStream_t s);

cudaError_t launch_model_scan(const float *vel, long long n, unsigned int *vmax_bits,
                              unsigned long long *bad, cudaStream_t s);
cudaError_t launch_model_fill(const float *vel, int nx, int ny, int nz, int nxp, double dt,
                              float *c, cudaStream_t s);
cudaError_t launch_source_scale(const float *vel, int nx, int ny, int nsrc, const int *src_i,
                                const int *src_j, const int *src_k, double dt, double cell,
                                float *scale, cudaStream_t s);
cudaError_t launch_pack(const float *dense, int nx, int ny, int nz, int nxp, float *padded,
                        cudaStream_t s);
cudaError_t launch_unpack(const float *padded, int nx, int ny, int nz, int nxp, float *dense,
                          cudaStream_t s);

}  // namespace mmod
