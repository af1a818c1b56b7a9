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

// Point sources grouped by grid point and bucketed per (x-y tile, plane) of
// the TMA kernel (64 x 16 tiles): the points of plane k in tile (tx, ty) are
// [tile_start[b], tile_start[b+1]), b = (ty * tiles_x + tx) * nz + k, so the
// points of one tile over a z range [k0, k1) are one contiguous run.
// Point p carries the sources [pt_first[p], pt_first[p+1]) in a fixed order.
constexpr int kInjTileX = 64, kInjTileY = 16;

struct InjTable {
    const int *tile_start;      // [tiles_y * tiles_x * nz + 1]
    const int *pt_i, *pt_j, *pt_k;
    const long long *pt_off;    // padded offset of the point
    const int *pt_first;        // [npts + 1]
    const int *src_row;         // wavelet row of each source (point order)
    const float *src_scale;     // injection scale of each source
    int tiles_x, tiles_y, npts;
};

// Everything a step kernel needs; passed by value (kernel parameter space).
struct StepArgs {
    int nx, ny, nz;            // grid
    int nxp;                   // padded row length (floats), multiple of 32
    long long plane;           // nxp * ny
    int nbl;                   // damping width: inner region is [nbl, n - 1 - nbl]
    int nt;                    // steps of the run
    int n;                     // this step: computes u^{n+1}
    Weights w;                 // c_m / h_a^2
    const float *ucur;         // u^n       (padded layout)
    const float *uprev;        // u^{n-1}
    float *uout;               // u^{n+1}   (may be uprev: in-place rotation)
    const float *c;            // dt^2 v^2  (padded layout)
    const float *ex, *ey, *ez; // dt * eta per axis
    InjTable inj;              // sources of this run
    const float *wavelet;      // w(row, n) = wavelet[row * wrs + n * wcs]
    long long wrs, wcs;        // [rows][nt]: (nt, 1); the adjoint reads its residual
                               // [nt][nrec] backward in time: (1, -nrec)
    // receivers: the kernel of step n copies u^n (its ucur) into traces[n-1]
    int nrec;
    const long long *rec_off;             // padded offsets
    float *traces;                        // [nt][nrec]
    int *err;                             // device view of the mapped error word
    int fs;                               // free surface at k = 0 (odd image, p = 0 on the plane)
    int pdl;                              // 0: plain launch; 1: programmatic dependent launch;
                                          // 2: the same, and the previous kernel in the stream
                                          //    is the previous step of this run
    int *claim;                           // work-claiming launches: {next unit, CTAs done},
                                          // 0 between launches (null: the static plan)
    float *gout;                          // gradient replay: also write g^n = L u^n + s^n here
                                          // (padded layout; null: not written)
    float inv_cell;                       // 1 / (hx hy hz): s^n = w[n] / (hx hy hz) at a source
};

// Adds the sources of injection point p to u^{n+1} (already stored): the
// point's damping factor r scales each term, sources in table order.
// uout / n: the step's u^{n+1} buffer and step index.
__device__ __forceinline__ void inject_point_at(const StepArgs &a, float *uout, int n, int p) {
    const int i = __ldg(a.inj.pt_i + p), j = __ldg(a.inj.pt_j + p), k = __ldg(a.inj.pt_k + p);
    const float r = damp_factor(__fadd_rn(__fadd_rn(__ldg(a.ex + i), __ldg(a.ey + j)), __ldg(a.ez + k)));
    float *dst = uout + __ldg(a.inj.pt_off + p);
    float v = *dst;
    for (int s = __ldg(a.inj.pt_first + p); s < __ldg(a.inj.pt_first + p + 1); ++s)
        v = add_source(v, __ldg(a.inj.src_scale + s),
                       __ldg(a.wavelet + (long long)__ldg(a.inj.src_row + s) * a.wrs + (long long)n * a.wcs), r);
    *dst = v;
}

__device__ __forceinline__ void inject_point(const StepArgs &a, int p) { inject_point_at(a, a.uout, a.n, p); }

// The same for injection points [lo, hi), thread t of nthreads: each thread
// takes up to four points at a time and issues the table, profile, wavefield
// and wavelet loads of all four before it applies any, so the dependent loads
// of different points overlap (a receiver plane injected by the adjoint gives
// a CTA about a thousand points).  Per point: the same operations in the same
// order as inject_point_at.
__device__ __forceinline__ void inject_points(const StepArgs &a, float *uout, int n, int lo, int hi, int t,
                                              int nthreads) {
    constexpr int G = 4;
    for (int base = lo + t; base < hi; base += G * nthreads) {
        int p[G], s0[G], s1[G];
        long long off[G];
        float e[G], v[G], sc[G], w[G];
        bool ok[G];
#pragma unroll
        for (int q = 0; q < G; ++q) {
            p[q] = base + q * nthreads;
            ok[q] = p[q] < hi;
            if (!ok[q]) p[q] = lo;   // a valid entry, not applied
        }
#pragma unroll
        for (int q = 0; q < G; ++q) {
            const int i = __ldg(a.inj.pt_i + p[q]), j = __ldg(a.inj.pt_j + p[q]), k = __ldg(a.inj.pt_k + p[q]);
            e[q] = __fadd_rn(__fadd_rn(__ldg(a.ex + i), __ldg(a.ey + j)), __ldg(a.ez + k));
            off[q] = __ldg(a.inj.pt_off + p[q]);
            s0[q] = __ldg(a.inj.pt_first + p[q]);
            s1[q] = __ldg(a.inj.pt_first + p[q] + 1);
        }
#pragma unroll
        for (int q = 0; q < G; ++q) {
            v[q] = uout[off[q]];
            sc[q] = __ldg(a.inj.src_scale + s0[q]);
            w[q] = __ldg(a.wavelet + (long long)__ldg(a.inj.src_row + s0[q]) * a.wrs + (long long)n * a.wcs);
        }
#pragma unroll
        for (int q = 0; q < G; ++q) {
            if (!ok[q]) continue;
            const float r = damp_factor(e[q]);
            float x = add_source(v[q], sc[q], w[q], r);   // every point has at least one source
            for (int s = s0[q] + 1; s < s1[q]; ++s)
                x = add_source(x, __ldg(a.inj.src_scale + s),
                               __ldg(a.wavelet + (long long)__ldg(a.inj.src_row + s) * a.wrs + (long long)n * a.wcs),
                               r);
            uout[off[q]] = x;
        }
    }
}

// The source term of g^n = L u^n + s^n at injection points [lo, hi) of the
// step's g^n (already holding L u^n): + w[n] / (hx hy hz) per source, in table
// order; thread t of nthreads.
__device__ __forceinline__ void inject_g_points(const StepArgs &a, int n, int lo, int hi, int t, int nthreads) {
    for (int p = lo + t; p < hi; p += nthreads) {
        float *dst = a.gout + __ldg(a.inj.pt_off + p);
        float v = *dst;
        for (int s = __ldg(a.inj.pt_first + p); s < __ldg(a.inj.pt_first + p + 1); ++s)
            v = __fmaf_rn(__ldg(a.wavelet + (long long)__ldg(a.inj.src_row + s) * a.wrs + (long long)n * a.wcs),
                          a.inv_cell, v);
        *dst = v;
    }
}

// Host helpers shared by the entry points (mmod_api.cu).
void damping_profile(int n, int nbl, double h, double vmax, double R, double dt, float *out);
// With a free surface the z axis has no layer under the surface plane.
void clear_surface_layer(int nz, int nbl, float *ez);
void cpml_profile(int n, int L, double h, double vmax, double R, double f0, double dt, bool top_free, float *b,
                  float *g);
void set_thread_error(const char *msg);   // fixed buffer read by mmod_last_error(NULL)

// Order-8 Taylor weights of the second derivative (Sec. 3):
// c_1..c_4 = 8/5, -1/5, 8/315, -1/560.
constexpr double kTaylor8[4] = {8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0, -1.0 / 560.0};
// Largest magnitude of the order-8 stencil's symbol (at k h = pi):
// 4 (c_1 + c_3) = 2048 / 315; leapfrog is stable iff dt^2 v^2 sum_a K_a <= 4.
constexpr double kSymbolMax8 = 2048.0 / 315.0;

// Launchers (mmod_step_simple.cu, mmod_step_tma.cu, mmod_setup.cu).
cudaError_t launch_step_simple(const StepArgs &a, cudaStream_t s);
cudaError_t launch_inject(const StepArgs &a, cudaStream_t s);   // all points, after a plain step
cudaError_t launch_gather(const float *u, const long long *rec_off, int nrec, float *dst,
                          cudaStream_t s);

struct TmaPlan;   // tile shape / grid decomposition of the TMA kernel

// Tensor map of a padded FP32 volume [nz][ny][nxp] with logical extent
// nx x ny x nz and a bx x by x 1 box (zero fill outside the extent).  False
// when the driver's encoder is unavailable or rejects the map.
bool encode_box(CUtensorMap *map, const float *base, int nx, int ny, int nz, int nxp, int bx, int by);

// x-y tiles and z ranges of one grid (one shot) for the TMA kernel.
struct Geom {
    int tiles_x, tiles_y, zchunks, zlen;
};

// One shot of a batch as the batch kernel reads it from global memory: its
// tensor maps (both wavefield buffers as u^n and u^{n-1} operands, and c),
// its step arguments (n, buffer roles and traces are set per step by the
// kernel), buffers, traces and decomposition.
struct ShotDesc {
    CUtensorMap cur[2], prev[2], cmap;
    StepArgs args;
    float *u[2];
    float *traces;   // [nt][nrec] or null
    Geom geom;
    int nblocks;     // CTAs of this shot per step
    // receivers bucketed per (64 x 16 tile, plane), for the persistent batch
    const int *rec_start, *rec_idx;
    const long long *rec_boff;
};

// Persistent batch run: steps n0 .. n1-1 of every shot in one cooperative
// launch; unit u serves shot unit_shot[u] as its block unit_local[u]; the
// shot's units signal counters[counter_base[shot] + block].
struct BatchPersistArgs {
    int n0, n1, units;
    const int *unit_shot, *unit_local, *counter_base;
    int *counters;
    unsigned long long *queue;   // next (step, unit) item of the work list, zeroed before the launch
};
cudaError_t launch_step_tma_batch_persistent(int variant, const ShotDesc *shots, const BatchPersistArgs &pa, int grid,
                                             cudaStream_t s);
// CTAs of the persistent batch kernel of variant v that fit at once (0: none).
int batch_persistent_grid(int variant, int units);
cudaError_t launch_step_tma(const StepArgs &a, const CUtensorMap *cur_map,
                            const CUtensorMap *prev_map, const CUtensorMap *c_map,
                            const TmaPlan &plan, cudaStream_t s);

// Persistent run: one cooperative launch advances steps n0 .. n1-1.  CTAs
// claim (step, work unit) items in step-major order from a queue; an item
// starts once its unit and the unit's 26 neighbours have completed step n-1
// (counters[v] >= n: they wrote the u^n it reads and finished reading the
// u^{n-1} it overwrites), so no launch boundary separates the steps.  The
// receivers of a unit (bucketed like the injection table: entries
// [rec_start[b], rec_start[b+1]), b = tile * nz + k) are recorded by the
// unit right after its sources.
struct TmaMaps {
    CUtensorMap cur[2], prev[2], c;   // u^n / u^{n-1} operand maps of both buffers, c
};
struct PersistArgs {
    int n0, n1, units;
    int *counters;                    // per unit: steps completed, zeroed before the run
    unsigned long long *queue;        // next (step, unit) item of the work list, zeroed before the run
    const int *rec_start, *rec_idx;   // receivers bucketed per (tile, plane); original index
    const long long *rec_off;         // padded offset of each bucketed receiver
    float *traces;                    // [nt][nrec] or null
    int nrec;
    float *u[2];
};
// Work units of the persistent kernel: the plan's tiles and z ranges of at
// least kRadius planes.  Grid: CTAs that fit at once, capped by max_ctas > 0;
// 0 when the variant has no persistent instantiation.
Geom persistent_geom(const TmaPlan &plan, int nz);
int persistent_grid(const TmaPlan &plan, int nz, int max_ctas);
cudaError_t launch_step_tma_persistent(const StepArgs &a, const TmaMaps &maps, const TmaPlan &plan,
                                       const PersistArgs &pa, int grid, cudaStream_t s);

// All shots of a batch, one step (variant = compiled TMA variant index).
cudaError_t launch_step_tma_batch(int variant, const ShotDesc *shots, const int *cta_shot, const int *cta_local,
                                  int nctas, int n, bool pdl, cudaStream_t s);
bool tma_variant_shape(int v, int *block, int *smem);
// 14 ints: threads, dynamic shared bytes, then {registers, local bytes,
// static shared bytes, resident CTAs per SM} of the step, batch and
// persistent kernels (-1 where a kernel is not compiled).
bool tma_variant_info(int v, int *out);

cudaError_t launch_model_scan(const float *vel, long long n, unsigned int *vmax_bits,
                              unsigned long long *bad, cudaStream_t s);
cudaError_t launch_model_fill(const float *vel, int nx, int ny, int nz, int nxp, double dt,
                              float *c, cudaStream_t s);
cudaError_t launch_source_scale(const float *vel, int nx, int ny, int nsrc, const int *src_i,
                                const int *src_j, const int *src_k, double dt, double cell,
                                float *scale, cudaStream_t s);
// Adjoint output: the gathers g [nt][nsrc] of the backward run ->
// adj [nsrc][nt], adj[s][n] = g[nt-1-n][s] * scale.
cudaError_t launch_unreverse_transpose(const float *g, int nt, int ncol, double scale, float *out,
                                       cudaStream_t s);
// Gradient helpers (mmod_setup.cu).
// Imaging condition of nsteps (1 or 2) forward steps n, n-1: psi[t] =
// psi^{n+1-t}, g[t] = g^{n-t} = L u^{n-t} + s^{n-t}; acc += psi[t] g[t] in
// the order of the steps.
cudaError_t launch_imaging(int nsteps, const float *const *psi, const float *const *g, int nx, int ny, int nz,
                           int nxp, float *acc, cudaStream_t s);
// grad_v = 2 acc / v (dJ/dv from acc = sum_n psi^{n+1} g^n), dense output.
cudaError_t launch_grad_to_velocity(const float *acc, const float *vel, int nx, int ny, int nz, int nxp,
                                    float *grad_v, cudaStream_t s);
cudaError_t launch_dot(const float *a, const float *b, long long n, double *out, cudaStream_t s);
cudaError_t launch_pack(const float *dense, int nx, int ny, int nz, int nxp, float *padded,
                        cudaStream_t s);
cudaError_t launch_unpack(const float *padded, int nx, int ny, int nz, int nxp, float *dense,
                          cudaStream_t s);

}  // namespace mmod
