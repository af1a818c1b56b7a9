// CPML layers for the second-order equation (the paper's convolutional PML,
// Sec. 3): complex-frequency-shifted stretching on each axis with two memory
// variables per axis,
//     u_tt = v^2 sum_a [ D2_a u + D1_a psi_a + zeta_a ],
//     psi_a^n  = b_a psi_a^{n-1}  + g_a D1_a u^n,
//     zeta_a^n = b_a zeta_a^{n-1} + g_a (D2_a u^n + D1_a psi_a^n),
// b = exp(-(d + alpha) dt), g = d (b - 1) / (d + alpha) per cell of the axis
// (zero outside the layers), D2_a the order-8 second difference (the step
// kernels' pair form), D1_a the order-8 centred first difference.  The terms
// D1_a psi_a + zeta_a exist only where axis a's profile is on (g_a != 0);
// psi_a is zero elsewhere.
//
// Each step runs the usual step kernel without damping (u^{n+1} = 2u^n -
// u^{n-1} + c L u^n + sources), then one pass per axis over that axis's
// layer cells: psi_a^n, zeta_a^n and u^{n+1} += c (D1_a psi_a^n + zeta_a^n).
// A pass works on lines along its axis and on the layer ranges of a line
// ([0, L) and [n - L, n), or the whole line where the two ranges' stencils
// meet), so every psi_a value it needs is computed by the same thread or warp
// in the same pass and no gathers are needed:
//   x: one warp per row segment (lane = cell, 24 cells and a 4-cell margin
//      each side), neighbours by warp shuffles;
//   y, z (and x for ranges wider than 24): one thread per line range,
//      consecutive threads on consecutive x (coalesced), marching along the
//      axis with a 13-value window of u^n and a 9-value window of psi^n, the
//      correction trailing psi by the stencil radius.
// Per cell, psi and zeta take the same FP32 operations as before; u^{n+1}
// gains one fused multiply-add per axis whose profile is on.  u and psi are
// 0 outside the grid; with a free surface the top layer is absent and the
// plane k = 0 is left alone (u, psi and zeta stay 0).
#include "mmod_cpml.h"
#include "mmod_internal.h"

namespace mmod {
namespace {

constexpr int kLine = 2 * kRadius + 1;   // -4..4 along the axis
constexpr int kWarpCells = 32 - 2 * kRadius;   // cells per warp row segment

__device__ __forceinline__ float d1_w(int m) {   // first-difference weights: 4/5, -1/5, 4/105, -1/280
    return m == 1 ? 4.0f / 5.0f : (m == 2 ? -1.0f / 5.0f : (m == 3 ? 4.0f / 105.0f : -1.0f / 280.0f));
}

// D1 of the 9 values x[0..8] (centre x[4]), unit spacing times inv_h.
__device__ __forceinline__ float d1_of(const float *x, float inv_h) {
    float s = 0.0f;
#pragma unroll
    for (int m = 1; m <= kRadius; ++m) s = __fmaf_rn(d1_w(m), __fsub_rn(x[kRadius + m], x[kRadius - m]), s);
    return __fmul_rn(s, inv_h);
}

// D2 of the 9 values x[0..8] in the step kernels' pair form.
__device__ __forceinline__ float d2_of(const float *x, const float (&w)[kRadius]) {
    const float two_p = __fadd_rn(x[kRadius], x[kRadius]);
    float d2 = pair_first(w[0], x[kRadius + 1], x[kRadius - 1], two_p);
#pragma unroll
    for (int m = 2; m <= kRadius; ++m) d2 = pair_acc(d2, w[m - 1], x[kRadius + m], x[kRadius - m], two_p);
    return d2;
}

// Layer ranges of one axis of n points with layer width L (low_absent: no
// low layer, the z axis under a free surface).  The ranges are merged into
// one when the stencil of one reaches the other.
struct Ranges {
    int n, lo[2], hi[2];
};

Ranges axis_ranges(int n, int L, bool low_absent) {
    Ranges r{};
    if (L <= 0) return r;
    if (!low_absent && n - L < L + kRadius) {
        r.lo[0] = 0;
        r.hi[0] = n;
        r.n = 1;
        return r;
    }
    if (!low_absent) {
        r.lo[r.n] = 0;
        r.hi[r.n] = L;
        ++r.n;
    }
    r.lo[r.n] = n - L;
    r.hi[r.n] = n;
    ++r.n;
    return r;
}

// One layer range [lo, hi) of the line at offset o0 (axis stride st, n points
// along the axis) for axis A: psi_a, zeta_a and the u^{n+1} correction.  The
// march takes kGroup positions at a time (7: a 20-cell layer's 28 positions
// in four groups) and issues all their loads (u ahead of
// psi, psi, zeta, u^{n+1}, c and the profiles) before any arithmetic, so a
// thread keeps 5 kGroup loads in flight instead of waiting on one per
// position.
// kLen > 0: the range is known to hold kLen cells, so the march is unrolled in
// full and the windows are fixed registers (no shifting moves).
template <int A, int kGroup, int kLen = 0>
__device__ __forceinline__ void march_range(const CpmlArgs &p, long long o0, long long st, int n, int lo, int hi,
                                            const float *__restrict__ u, float *__restrict__ uout) {
    if (kLen > 0) hi = lo + kLen;
    const float *B = p.b[A], *G = p.g[A];
    float *psi = p.psi[A], *zeta = p.zeta[A];
    const float ih = p.inv_h[A];
    float uw[2 * kRadius + kLine - kRadius];   // u at q-8 .. q+4 (13 values)
    float pw[kLine];                           // psi at q-8 .. q
#pragma unroll
    for (int m = 0; m < 13; ++m) {
        const int q = lo - 13 + m;
        uw[m] = (q >= 0 && q < n) ? __ldg(u + o0 + q * st) : 0.0f;
    }
#pragma unroll
    for (int m = 0; m < kLine; ++m) pw[m] = 0.0f;
    constexpr int kGroups = kLen > 0 ? (kLen + 2 * kRadius + kGroup - 1) / kGroup : 1;
#pragma unroll
    for (int gi = 0; kLen > 0 ? gi < kGroups : lo - kRadius + gi * kGroup < hi + kRadius; ++gi) {
        const int q0 = lo - kRadius + gi * kGroup;
        // loads of positions q = q0 .. q0+3: u(q + 4); psi(q) and the profile at
        // q when q lies in the range; zeta, u^{n+1}, c and the profile at the
        // trailing position q - 4
        float un[kGroup], po[kGroup], bq[kGroup], gq[kGroup], zo[kGroup], uo[kGroup], co[kGroup], bp[kGroup],
            gp[kGroup];
#pragma unroll
        for (int j = 0; j < kGroup; ++j) {
            const int q = q0 + j, qa = q + kRadius, pc = q - kRadius;
            un[j] = (qa >= 0 && qa < n) ? __ldg(u + o0 + (long long)qa * st) : 0.0f;
            const bool iq = q >= lo && q < hi, ip = pc >= lo && pc < hi;
            po[j] = iq ? psi[o0 + (long long)q * st] : 0.0f;
            bq[j] = iq ? __ldg(B + q) : 0.0f;
            gq[j] = iq ? __ldg(G + q) : 0.0f;
            zo[j] = ip ? zeta[o0 + (long long)pc * st] : 0.0f;
            uo[j] = ip ? uout[o0 + (long long)pc * st] : 0.0f;
            co[j] = ip ? __ldg(p.c + o0 + (long long)pc * st) : 0.0f;
            bp[j] = ip ? __ldg(B + pc) : 0.0f;
            gp[j] = ip ? __ldg(G + pc) : 0.0f;
        }
#pragma unroll
        for (int j = 0; j < kGroup; ++j) {
            const int q = q0 + j, pc = q - kRadius;
#pragma unroll
            for (int m = 0; m < 12; ++m) uw[m] = uw[m + 1];
            uw[12] = un[j];
#pragma unroll
            for (int m = 0; m < kLine - 1; ++m) pw[m] = pw[m + 1];
            float ps = 0.0f;   // psi outside the range is 0 (outside the grid or g = 0)
            if (gq[j] != 0.0f) {
                ps = __fmaf_rn(bq[j], po[j], __fmul_rn(gq[j], d1_of(uw + kRadius, ih)));
                psi[o0 + (long long)q * st] = ps;
            }
            pw[kLine - 1] = ps;
            if (gp[j] != 0.0f) {   // the correction trails psi by the radius
                const long long o = o0 + (long long)pc * st;
                const float d2 = d2_of(uw, p.w[A]);
                const float dpsi = d1_of(pw, ih);
                const float z = __fmaf_rn(bp[j], zo[j], __fmul_rn(gp[j], __fadd_rn(d2, dpsi)));
                zeta[o] = z;
                uout[o] = __fmaf_rn(co[j], __fadd_rn(dpsi, z), uo[j]);
            }
        }
    }
}

// Layer width whose march is compiled fully unrolled (the workloads' 20 cells).
constexpr int kCommonLayer = 20;

// y and z passes (and the x pass for ranges wider than a warp row segment):
// work item t is line t % lines of range t / lines (consecutive t on
// consecutive x for y and z); grid-stride over the items, so each thread
// takes about `per` of them and neighbouring threads stay on neighbouring
// lines.
template <int A, int kGroup = 7>
__global__ void __launch_bounds__(128) cpml_line_kernel(const CpmlArgs p, const Ranges rg, const float *__restrict__ u,
                                                        float *__restrict__ uout) {
    const int n = A == 0 ? p.nx : (A == 1 ? p.ny : p.nz);
    // the other two coordinates: (x, z) for y lines, (x, y) for z lines, (y, z) for x lines
    const int n1 = A == 0 ? p.ny : p.nx, n2 = A == 2 ? p.ny : p.nz;
    const long long lines = (long long)n1 * n2;
    const long long st = A == 0 ? 1 : (A == 1 ? p.nxp : p.plane);
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < lines * rg.n; t += stride) {
        const int r = (int)(t / lines);
        const long long l = t - (long long)r * lines;
        const int c1 = (int)(l % n1), c2 = (int)(l / n1);
        long long o0;
        if (A == 0) {
            if (p.fs && c2 == 0) continue;   // the free-surface plane stays 0
            o0 = (long long)c2 * p.plane + (long long)c1 * p.nxp;
        } else if (A == 1) {
            if (p.fs && c2 == 0) continue;
            o0 = (long long)c2 * p.plane + c1;
        } else {
            o0 = (long long)c2 * p.nxp + c1;
        }
        if (rg.hi[r] - rg.lo[r] == kCommonLayer)
            march_range<A, kGroup, kCommonLayer>(p, o0, st, n, rg.lo[r], rg.hi[r], u, uout);
        else
            march_range<A, kGroup>(p, o0, st, n, rg.lo[r], rg.hi[r], u, uout);
    }
}

// x pass: one warp per row segment of one layer range (at most 24 cells,
// lanes 4..27 hold them, lanes 0..3 and 28..31 the margins); a warp takes
// kRows consecutive segments at a time and issues all their loads before the
// shuffles and arithmetic; grid-stride over the groups.
constexpr int kRows = 4;

__global__ void __launch_bounds__(128) cpml_x_warp_kernel(const CpmlArgs p, const Ranges rg, const float *__restrict__ u,
                                                          float *__restrict__ uout) {
    const int lane = threadIdx.x & 31;
    const long long rows = (long long)p.ny * p.nz, total = rows * rg.n;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const float ih = p.inv_h[0];
    for (long long t0 = (((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * kRows; t0 < total;
         t0 += nwarps * kRows) {
        float uu[kRows], po[kRows], zo[kRows], uo[kRows], co[kRows], bb[kRows], gg[kRows];
        long long off[kRows];
#pragma unroll
        for (int rr = 0; rr < kRows; ++rr) {
            const long long t = t0 + rr;
            const int r = t < total ? (int)(t / rows) : 0;
            const long long l = t - (long long)r * rows;
            const int j = (int)(l % p.ny), k = (int)(l / p.ny);
            // rows past the end and the free-surface plane take no part (uniform over the warp)
            const bool live = t < total && !(p.fs && k == 0);
            const int i = rg.lo[r] - kRadius + lane;
            const bool in_grid = live && i >= 0 && i < p.nx;
            const bool mine = live && i >= rg.lo[r] && i < rg.hi[r];
            off[rr] = (long long)k * p.plane + (long long)j * p.nxp + i;
            uu[rr] = in_grid ? __ldg(u + off[rr]) : 0.0f;
            gg[rr] = mine ? __ldg(p.g[0] + i) : 0.0f;
            bb[rr] = mine ? __ldg(p.b[0] + i) : 0.0f;
            po[rr] = mine ? p.psi[0][off[rr]] : 0.0f;
            zo[rr] = mine ? p.zeta[0][off[rr]] : 0.0f;
            uo[rr] = mine ? uout[off[rr]] : 0.0f;
            co[rr] = mine ? __ldg(p.c + off[rr]) : 0.0f;
        }
#pragma unroll
        for (int rr = 0; rr < kRows; ++rr) {
            float x[kLine];
#pragma unroll
            for (int m = 1; m <= kRadius; ++m) {
                x[kRadius + m] = __shfl_down_sync(0xffffffffu, uu[rr], m);
                x[kRadius - m] = __shfl_up_sync(0xffffffffu, uu[rr], m);
            }
            x[kRadius] = uu[rr];
            const float g = gg[rr];
            float ps = 0.0f;
            if (g != 0.0f) {
                ps = __fmaf_rn(bb[rr], po[rr], __fmul_rn(g, d1_of(x, ih)));
                p.psi[0][off[rr]] = ps;
            }
            float q[kLine];
#pragma unroll
            for (int m = 1; m <= kRadius; ++m) {
                q[kRadius + m] = __shfl_down_sync(0xffffffffu, ps, m);
                q[kRadius - m] = __shfl_up_sync(0xffffffffu, ps, m);
            }
            q[kRadius] = ps;
            if (g != 0.0f) {
                const float d2 = d2_of(x, p.w[0]);
                const float dpsi = d1_of(q, ih);
                const float z = __fmaf_rn(bb[rr], zo[rr], __fmul_rn(g, __fadd_rn(d2, dpsi)));
                p.zeta[0][off[rr]] = z;
                uout[off[rr]] = __fmaf_rn(co[rr], __fadd_rn(dpsi, z), uo[rr]);
            }
        }
    }
}

int blocks_for(long long threads) {
    const long long b = (threads + 127) / 128;
    return (int)(b < 1 ? 1 : b);
}

}  // namespace

cudaError_t launch_cpml_layers(const CpmlArgs &p, const float *u, float *uout, cudaStream_t s) {
    if (p.nbl <= 0) return cudaSuccess;
    const int per = p.zc > 0 ? p.zc : kCpmlPlanes;
    const Ranges rx = axis_ranges(p.nx, p.nbl, false), ry = axis_ranges(p.ny, p.nbl, false),
                 rz = axis_ranges(p.nz, p.nbl, p.fs != 0);
    bool x_warp = true;
    for (int r = 0; r < rx.n; ++r) x_warp = x_warp && rx.hi[r] - rx.lo[r] <= kWarpCells;
    const long long xl = (long long)p.ny * p.nz * rx.n, yl = (long long)p.nx * p.nz * ry.n,
                    zl = (long long)p.nx * p.ny * rz.n;
    if (rx.n > 0) {
        if (x_warp)
            cpml_x_warp_kernel<<<blocks_for(((xl + (long long)per * kRows - 1) / ((long long)per * kRows)) * 32), 128,
                                 0, s>>>(p, rx, u, uout);
        else
            cpml_line_kernel<0><<<blocks_for((xl + per - 1) / per), 128, 0, s>>>(p, rx, u, uout);
        if (cudaError_t e = cudaGetLastError()) return e;
    }
    if (ry.n > 0) {
        cpml_line_kernel<1><<<blocks_for((yl + per - 1) / per), 128, 0, s>>>(p, ry, u, uout);
        if (cudaError_t e = cudaGetLastError()) return e;
    }
    if (rz.n > 0) {
        cpml_line_kernel<2><<<blocks_for((zl + per - 1) / per), 128, 0, s>>>(p, rz, u, uout);
        if (cudaError_t e = cudaGetLastError()) return e;
    }
    return cudaSuccess;
}

}  // namespace mmod
