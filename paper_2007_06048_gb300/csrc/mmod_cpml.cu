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
// in the same pass and no gathers are needed.  Two forms, with the same FP32
// operations per cell (the same bits):
//   tiled (the default where the axis allows it, see below): units of 64
//      lines of a range loaded whole into shared memory by bulk-tensor
//      copies, one thread per line, results stored back by bulk-tensor
//      stores; the x layers' psi, zeta and c in compact arrays;
//   marching: x — one warp per row segment (lane = cell, 24 cells and a
//      4-cell margin each side), neighbours by warp shuffles; y, z (and x
//      for ranges wider than 24) — one thread per line range, consecutive
//      threads on consecutive x (coalesced), marching along the axis with a
//      13-value window of u^n and a 9-value window of psi^n, the correction
//      trailing psi by the stencil radius.
// u^{n+1} gains one fused multiply-add per axis whose profile is on.  u and
// psi are 0 outside the grid; with a free surface the top layer is absent
// and the plane k = 0 is left alone (u, psi and zeta stay 0).
#include "mmod_cpml.h"
#include "mmod_internal.h"
#include "tma_ptx.cuh"

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


// ---------------------------------------------------------------------------
// Tiled passes.  A unit is 2 W lines of one layer range (z: W x 2 lines over
// (x, y); y: W x 2 over (x, z); x: W x 2 rows over (y, z)) and a block loads
// the whole unit with five bulk-tensor copies on one mbarrier: u^n over the
// range and its 4-cell margins (zeros outside the grid), psi_a, zeta_a,
// u^{n+1} and c over the range.  Each thread then marches its line from
// shared memory (the same FP32 operations as march_range), updates psi,
// zeta and u^{n+1} in place, and the three boxes go back by bulk-tensor
// stores.  All of a unit's bytes are in flight at once, which the per-thread
// marches over global memory cannot reach.
// ---------------------------------------------------------------------------

constexpr int kTileW = 32;                 // line-box width W
constexpr int kTileLines = 2 * kTileW;     // lines per unit

// Orders this thread's shared-memory writes before later bulk copies.
__device__ __forceinline__ void fence_tile_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Tiled bulk-tensor store of a shared-memory box; elements outside the
// tensor are not written.
__device__ __forceinline__ void tma_store_3d(const CUtensorMap *map, int x, int y, int z, const float *src) {
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y), "r"(z), "r"(smem_u32(src))
                 : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }

// Until every committed bulk store of this thread has completed.
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Until every committed bulk store of this thread has read its source.
__device__ __forceinline__ void bulk_wait_read_all() {
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

template <int kLen>
struct TileGeom {
    static constexpr int kU = kLen + 2 * kRadius;        // u positions of a line
    static constexpr int kUF = kU * kTileLines;          // floats of the u box
    static constexpr int kOF = kLen * kTileLines;        // floats of each layer box
    static constexpr int kBytes = (kUF + 4 * kOF) * 4;   // bytes of the five boxes
};

// Box shape of axis A's pass: lines (x extent, y extent, z extent) with the
// axis extent set to `len`.
__host__ __device__ constexpr int box_x(int A, int len) { return A == 0 ? len : kTileW; }
__host__ __device__ constexpr int box_y(int A, int len) { return A == 0 ? kTileW : (A == 1 ? len : 2); }
__host__ __device__ constexpr int box_z(int A, int len) { return A == 2 ? len : 2; }

// Line t's element at position j of a box with `len` positions per line.
template <int A, int len>
__device__ __forceinline__ int tile_index(int t, int j) {
    if (A == 0) return t * len + j;                               // [z][y][x]: row t, x = j
    if (A == 1) return ((t / kTileW) * len + j) * kTileW + t % kTileW;   // [z][y][x]: z = t / W, y = j
    return j * kTileLines + t;                                    // [z][y][x]: z = j
}

// Positions [start, start + N) of line t of a box with `len` positions per
// line into v (0 outside [0, len)); rows of the x pass in 16- or 8-byte
// vectors where the positions allow (a row is 16-byte aligned).
template <int A, int len, int N, int start>
__device__ __forceinline__ void tile_get(const float *s, int t, float (&v)[N]) {
    constexpr int lo = start < 0 ? 0 : start, hi = start + N > len ? len : start + N;
#pragma unroll
    for (int j = 0; j < N; ++j) v[j] = 0.0f;
    if constexpr (A == 0 && lo % 4 == 0 && (hi - lo) % 4 == 0) {
        const float4 *q = reinterpret_cast<const float4 *>(s + t * len + lo);
#pragma unroll
        for (int k = 0; k < (hi - lo) / 4; ++k) {
            const float4 f = q[k];
            v[lo - start + 4 * k] = f.x; v[lo - start + 4 * k + 1] = f.y;
            v[lo - start + 4 * k + 2] = f.z; v[lo - start + 4 * k + 3] = f.w;
        }
    } else if constexpr (A == 0 && lo % 2 == 0 && (hi - lo) % 2 == 0) {
        const float2 *q = reinterpret_cast<const float2 *>(s + t * len + lo);
#pragma unroll
        for (int k = 0; k < (hi - lo) / 2; ++k) {
            const float2 f = q[k];
            v[lo - start + 2 * k] = f.x; v[lo - start + 2 * k + 1] = f.y;
        }
    } else {
#pragma unroll
        for (int j = lo; j < hi; ++j) v[j - start] = s[tile_index<A, len>(t, j)];
    }
}

// v into positions [start, start + N) of line t (all inside [0, len)).
template <int A, int len, int N, int start>
__device__ __forceinline__ void tile_put(float *s, int t, const float (&v)[N]) {
    static_assert(start >= 0 && start + N <= len, "a store stays inside the line");
    if constexpr (A == 0 && start % 4 == 0 && N % 4 == 0) {
        float4 *q = reinterpret_cast<float4 *>(s + t * len + start);
#pragma unroll
        for (int k = 0; k < N / 4; ++k) q[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
    } else if constexpr (A == 0 && start % 2 == 0 && N % 2 == 0) {
        float2 *q = reinterpret_cast<float2 *>(s + t * len + start);
#pragma unroll
        for (int k = 0; k < N / 2; ++k) q[k] = make_float2(v[2 * k], v[2 * k + 1]);
    } else {
#pragma unroll
        for (int j = 0; j < N; ++j) s[tile_index<A, len>(t, start + j)] = v[j];
    }
}

// Global coordinate of line t along the slowest line axis (z for the x and y
// passes), for the free-surface plane.
template <int A>
__device__ __forceinline__ int tile_line_z(int i2, int t) {
    return i2 * 2 + t / kTileW;
}

// One thread per line: psi_a, zeta_a and u^{n+1} of line t, in place, with
// the same FP32 operations as march_range.  The range's profiles are loaded
// once per warp (lane i holds cell i) and broadcast by shuffles; where g = 0
// the results are selected away (psi taken as 0, the stored values kept).
// Called by whole warps; lines that are not live write nothing back.
template <int A, int kLen>
__device__ __forceinline__ void tile_unit(const CpmlArgs &p, float *base, int t, int lo, bool live) {
    static_assert(kLen <= 32, "one profile value per lane");
    using G = TileGeom<kLen>;
    float *su = base, *sp = su + G::kUF, *sz = sp + G::kOF, *so = sz + G::kOF, *sc = so + G::kOF;
    const int lane = t & 31;
    const float gl = lane < kLen ? __ldg(p.g[A] + lo + lane) : 0.0f;
    const float bl = lane < kLen ? __ldg(p.b[A] + lo + lane) : 0.0f;
    const float ih = p.inv_h[A];
    float uu[G::kU], ps[kLen], v[kLen];
    tile_get<A, G::kU, G::kU, 0>(su, t, uu);
    tile_get<A, kLen, kLen, 0>(sp, t, v);
    // psi^n at each cell of the range
#pragma unroll
    for (int i = 0; i < kLen; ++i) {
        const float g = __shfl_sync(0xffffffffu, gl, i), b = __shfl_sync(0xffffffffu, bl, i);
        const float nv = __fmaf_rn(b, v[i], __fmul_rn(g, d1_of(uu + i, ih)));
        ps[i] = g != 0.0f ? nv : 0.0f;
        v[i] = g != 0.0f ? nv : v[i];
    }
    if (live) tile_put<A, kLen, kLen, 0>(sp, t, v);
    // zeta^n and the u^{n+1} term, psi taken as 0 outside the range
    float zo[kLen], uo[kLen], co[kLen];
    tile_get<A, kLen, kLen, 0>(sz, t, zo);
    tile_get<A, kLen, kLen, 0>(so, t, uo);
    tile_get<A, kLen, kLen, 0>(sc, t, co);
#pragma unroll
    for (int i = 0; i < kLen; ++i) {
        const float g = __shfl_sync(0xffffffffu, gl, i), b = __shfl_sync(0xffffffffu, bl, i);
        float pw[kLine];
#pragma unroll
        for (int k = 0; k < kLine; ++k) {
            const int j = i - kRadius + k;
            pw[k] = (j >= 0 && j < kLen) ? ps[j] : 0.0f;
        }
        const float d2 = d2_of(uu + i, p.w[A]);
        const float dpsi = d1_of(pw, ih);
        const float zn = __fmaf_rn(b, zo[i], __fmul_rn(g, __fadd_rn(d2, dpsi)));
        const float un = __fmaf_rn(co[i], __fadd_rn(dpsi, zn), uo[i]);
        zo[i] = g != 0.0f ? zn : zo[i];
        uo[i] = g != 0.0f ? un : uo[i];
    }
    if (live) {
        tile_put<A, kLen, kLen, 0>(sz, t, zo);
        tile_put<A, kLen, kLen, 0>(so, t, uo);
    }
}

// Unit -> layer-box origin (x, y, z), the range's first cell lo and the
// slowest line-axis tile i2; r the range.
template <int A>
__device__ __forceinline__ void tile_origin(const Ranges &rg, int n1, int n2, int unit, int &x, int &y, int &z,
                                            int &lo, int &i2, int &r) {
    const int per_range = n1 * n2, rem = unit - (unit / per_range) * per_range;
    r = unit / per_range;
    const int i1 = rem % n1;
    i2 = rem / n1;
    lo = rg.lo[r];
    x = A == 0 ? lo : i1 * kTileW;
    y = A == 0 ? i1 * kTileW : (A == 1 ? lo : i2 * 2);
    z = A == 2 ? lo : i2 * 2;
}

// Planes per range of the compact x-layer arrays: nz rounded up to the x
// pass's 2-plane boxes, so that no box reaches into the next range.
__host__ __device__ constexpr int compact_planes(int nz) { return (nz + 1) / 2 * 2; }

// Origin of the psi, zeta and c boxes: the volumes' layer box, or for the x
// pass the compact arrays' box (x = 0, z = r * nzp + z).
template <int A>
__device__ __forceinline__ void tile_aux_origin(int nz, int r, int x, int y, int z, int &ax, int &ay, int &az) {
    ax = A == 0 ? 0 : x;
    ay = y;
    az = A == 0 ? r * compact_planes(nz) + z : z;
}

// Persistent over the units (unit = block + k * grid), kTileStages
// shared-memory stages: the loads of the next units are in flight while unit
// k is computed;
// a stage is refilled once the bulk stores of its previous unit have read
// it.
constexpr int kTileThreads = kTileLines;   // one thread per line
// Shared-memory stages per block.  Measured on 240^3 (us per CPML step):
// 32-cell boxes with 1 / 2 / 3 / 4 stages 95.0 / 85.5 / 89.2 / 91.0, 16-cell
// boxes with 2 / 3 / 4 stages 86.4 / 87.8 / 90.0.
constexpr int kTileStages = 2;

template <int A, int kLen>
__global__ void __launch_bounds__(kTileThreads, 2)
    cpml_tile_kernel(const __grid_constant__ CpmlTileMaps m, const CpmlArgs p, const Ranges rg, int n1, int n2,
                     int units) {
    using G = TileGeom<kLen>;
    constexpr int kStage = G::kBytes / 4;   // floats per stage
    extern __shared__ __align__(128) float tile_smem[];
    __shared__ __align__(8) uint64_t full[kTileStages];
    __shared__ int abort_flag;
    const int t = threadIdx.x;
    // thread 0: a unit's copies into stage st; `stable` the four that no
    // earlier pass of the step writes (u^n, psi_a, zeta_a, c), `after` u^{n+1}
    auto issue = [&](int unit, int st, bool stable, bool after) {
        int x, y, z, lo, i2, r, ax, ay, az;
        tile_origin<A>(rg, n1, n2, unit, x, y, z, lo, i2, r);
        tile_aux_origin<A>(p.nz, r, x, y, z, ax, ay, az);
        float *su = tile_smem + st * kStage, *sp = su + G::kUF, *sz = sp + G::kOF, *so = sz + G::kOF,
              *sc = so + G::kOF;
        if (stable) {
            mbar_expect_tx(&full[st], G::kBytes);
            tma_load_3d(su, &m.u, A == 0 ? x - kRadius : x, A == 1 ? y - kRadius : y, A == 2 ? z - kRadius : z,
                        &full[st]);
            tma_load_3d(sp, &m.psi, ax, ay, az, &full[st]);
            tma_load_3d(sz, &m.zeta, ax, ay, az, &full[st]);
            tma_load_3d(sc, &m.c, ax, ay, az, &full[st]);
        }
        if (after) tma_load_3d(so, &m.uout, x, y, z, &full[st]);
    };
    if (t == 0) {
        abort_flag = 0;
        for (int s = 0; s < kTileStages; ++s) mbar_init(&full[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_tile_shared();
    }
    __syncthreads();
    // the first units' copies of data the previous kernels of the step do not
    // write go out before the programmatic-launch wait, u^{n+1} after it
    if (t == 0)
        for (int s = 0; s < kTileStages; ++s)
            if ((int)(blockIdx.x + s * gridDim.x) < units) issue(blockIdx.x + s * gridDim.x, s, true, false);
    if (p.pdl) {
        asm volatile("griddepcontrol.wait;" ::: "memory");
        asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    }
    if (t == 0)
        for (int s = 0; s < kTileStages; ++s)
            if ((int)(blockIdx.x + s * gridDim.x) < units) issue(blockIdx.x + s * gridDim.x, s, false, true);
    int k = 0;
    for (int unit = blockIdx.x; unit < units; unit += gridDim.x, ++k) {
        const int st = k % kTileStages;
        float *base = tile_smem + st * kStage;
        const bool ready = mbar_wait(&full[st], (k / kTileStages) & 1, &abort_flag, p.err);
        int x, y, z, lo, i2, r;
        tile_origin<A>(rg, n1, n2, unit, x, y, z, lo, i2, r);
        // every lane computes (the profiles are shuffled across the warp); the
        // free-surface plane keeps its values
        const bool live = ready && !(A != 2 && p.fs && tile_line_z<A>(i2, t) == 0);
        tile_unit<A, kLen>(p, base, t, lo, live);
        fence_tile_shared();   // this thread's shared-memory writes before the bulk stores
        __syncthreads();
        if (abort_flag) {      // uniform: read after the barrier
            if (t == 0)        // no copy may still be landing when the block exits
                for (int j = 0; j < kTileStages; ++j)
                    if (unit + j * (int)gridDim.x < units)
                        mbar_drain(&full[(k + j) % kTileStages], ((k + j) / kTileStages) & 1);
            break;
        }
        if (t == 0) {
            float *sp = base + G::kUF, *sz = sp + G::kOF, *so = sz + G::kOF;
            int ax, ay, az;
            tile_aux_origin<A>(p.nz, r, x, y, z, ax, ay, az);
            tma_store_3d(&m.psi, ax, ay, az, sp);
            tma_store_3d(&m.zeta, ax, ay, az, sz);
            tma_store_3d(&m.uout, x, y, z, so);
            bulk_commit();
            const int next = unit + kTileStages * (int)gridDim.x;
            if (next < units) {
                bulk_wait_read_all();   // the stage's stores have read it
                issue(next, st, true, true);
            }
        }
    }
    if (t == 0) bulk_wait_all();
}

// Compiled layer widths of the tiled passes.
constexpr int kTileWidths[] = {8, 20};

template <int A, int kLen>
cudaError_t tile_attr() {
    return cudaFuncSetAttribute(cpml_tile_kernel<A, kLen>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                kTileStages * TileGeom<kLen>::kBytes);
}

// Resident blocks of the persistent tiled pass on the current device.
template <int A, int kLen>
int tile_blocks() {
    int dev = 0, sms = 0, occ = 0;
    if (cudaGetDevice(&dev) || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, cpml_tile_kernel<A, kLen>, kTileThreads,
                                                      kTileStages * TileGeom<kLen>::kBytes)) {
        cudaGetLastError();
        return 0;
    }
    return sms * occ;
}

template <int A>
void tile_grid(const CpmlArgs &p, int *n1, int *n2) {
    if (A == 0) {
        *n1 = (p.ny + kTileW - 1) / kTileW;
        *n2 = (p.nz + 1) / 2;
    } else {
        *n1 = (p.nx + kTileW - 1) / kTileW;
        *n2 = ((A == 1 ? p.nz : p.ny) + 1) / 2;
    }
}

template <int A, int kLen>
cudaError_t launch_tile(const CpmlTileMaps &m, const CpmlArgs &p, const Ranges &rg, int resident, cudaStream_t s) {
    int n1, n2;
    tile_grid<A>(p, &n1, &n2);
    // as many units per block everywhere: ceil(units / resident) rounds, and
    // only as many blocks as those rounds need
    const int units = rg.n * n1 * n2;
    const int rounds = resident > 0 ? (units + resident - 1) / resident : 1;
    const int grid = (units + rounds - 1) / rounds;
    cudaLaunchConfig_t lc{};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    lc.gridDim = dim3(grid);
    lc.blockDim = dim3(kTileThreads);
    lc.dynamicSmemBytes = kTileStages * TileGeom<kLen>::kBytes;
    lc.stream = s;
    lc.attrs = at;
    lc.numAttrs = p.pdl ? 1 : 0;
    return cudaLaunchKernelEx(&lc, cpml_tile_kernel<A, kLen>, m, p, rg, n1, n2, units);
}

template <int A>
cudaError_t launch_tile_axis(const CpmlTiles &tl, int buffer, const CpmlArgs &p, const Ranges &rg, cudaStream_t s) {
    return p.nbl == 8 ? launch_tile<A, 8>(tl.maps[buffer][A], p, rg, tl.resident[A], s)
                      : launch_tile<A, 20>(tl.maps[buffer][A], p, rg, tl.resident[A], s);
}

// c_x[r][z][y][i] = c(lo_r + i, y, z) over the x layer ranges (z < nz of
// each range's nzp planes).
__global__ void cpml_pack_c_kernel(const CpmlArgs p, const Ranges rg, float *__restrict__ cx) {
    const int L = p.nbl, nzp = compact_planes(p.nz);
    const long long per = (long long)p.nz * p.ny * L, n = per * rg.n;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(e / per);
        long long q = e - (long long)r * per;
        const int i = (int)(q % L);
        q /= L;
        const int y = (int)(q % p.ny), z = (int)(q / p.ny);
        cx[(((long long)r * nzp + z) * p.ny + y) * L + i] =
            p.c[(long long)z * p.plane + (long long)y * p.nxp + rg.lo[r] + i];
    }
}

int blocks_for(long long threads) {
    const long long b = (threads + 127) / 128;
    return (int)(b < 1 ? 1 : b);
}

}  // namespace

namespace {

using EncodeFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                              const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn tile_encoder() {
    static EncodeFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeFn>(f);
        else
            cudaGetLastError();
    }
    return fn;
}

// A 3-D FP32 array of dims (nx, ny, nz), row and plane pitches in floats,
// with a box of (bx, by, bz).
bool encode_array(CUtensorMap *map, const float *base, long long nx, long long ny, long long nz, long long row,
                  long long plane, int bx, int by, int bz) {
    const EncodeFn fn = tile_encoder();
    if (!fn) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
    const cuuint64_t strides[2] = {(cuuint64_t)row * 4, (cuuint64_t)plane * 4};
    const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz};
    const cuuint32_t estr[3] = {1, 1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// A padded volume (x pitch nxp, plane pitch `plane`) with a box of (bx, by, bz).
bool encode_tile(CUtensorMap *map, const float *base, const CpmlArgs &p, int bx, int by, int bz) {
    return encode_array(map, base, p.nx, p.ny, p.nz, p.nxp, p.plane, bx, by, bz);
}

// The x pass can run tiled: a compiled width, two layer ranges of L cells,
// 16-byte aligned row segments (lo = 0 or nx - L, and lo - 4).
bool x_tileable(const CpmlArgs &p, Ranges *rx) {
    const int L = p.nbl;
    bool width = false;
    for (int w : kTileWidths) width = width || w == L;
    *rx = axis_ranges(p.nx, L, false);
    bool ok = width && rx->n > 0 && L % 4 == 0 && p.nx % 4 == 0;
    for (int r = 0; r < rx->n; ++r) ok = ok && rx->hi[r] - rx->lo[r] == L;
    return ok;
}

template <int A>
bool encode_axis(const CpmlArgs &p, const float *u, const float *uout, CpmlTileMaps *m) {
    const int L = p.nbl, lu = L + 2 * kRadius;
    if (!encode_tile(&m->u, u, p, box_x(A, lu), box_y(A, lu), box_z(A, lu)) ||
        !encode_tile(&m->uout, uout, p, box_x(A, L), box_y(A, L), box_z(A, L)))
        return false;
    if (A == 0) {   // compact [range][z][y][L] arrays: rows of L, planes of ny rows
        Ranges rx;
        x_tileable(p, &rx);
        const long long zr = (long long)rx.n * compact_planes(p.nz), cnt = zr * p.ny * L;
        return encode_array(&m->psi, p.xc, L, p.ny, zr, L, (long long)L * p.ny, L, kTileW, 2) &&
               encode_array(&m->zeta, p.xc + cnt, L, p.ny, zr, L, (long long)L * p.ny, L, kTileW, 2) &&
               encode_array(&m->c, p.xc + 2 * cnt, L, p.ny, zr, L, (long long)L * p.ny, L, kTileW, 2);
    }
    return encode_tile(&m->psi, p.psi[A], p, box_x(A, L), box_y(A, L), box_z(A, L)) &&
           encode_tile(&m->zeta, p.zeta[A], p, box_x(A, L), box_y(A, L), box_z(A, L)) &&
           encode_tile(&m->c, p.c, p, box_x(A, L), box_y(A, L), box_z(A, L));
}

}  // namespace

long long cpml_x_compact_floats(const CpmlArgs &p) {
    Ranges rx;
    if (!x_tileable(p, &rx)) return 0;
    return 3LL * rx.n * compact_planes(p.nz) * p.ny * p.nbl;
}

cudaError_t launch_cpml_pack_c(const CpmlArgs &p, cudaStream_t s) {
    Ranges rx;
    if (!p.xc || !x_tileable(p, &rx)) return cudaSuccess;
    const long long cnt = (long long)rx.n * compact_planes(p.nz) * p.ny * p.nbl;
    const long long blocks = ((long long)rx.n * p.nz * p.ny * p.nbl + 255) / 256;
    cpml_pack_c_kernel<<<(int)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(p, rx, p.xc + 2 * cnt);
    return cudaGetLastError();
}

bool make_cpml_tiles(const CpmlArgs &p, float *const u[2], CpmlTiles *t) {
    for (int a = 0; a < 3; ++a) t->ok[a] = false;
    const int L = p.nbl;
    bool width = false;
    for (int w : kTileWidths) width = width || w == L;
    if (!width) return true;
    const Ranges rr[3] = {axis_ranges(p.nx, L, false), axis_ranges(p.ny, L, false), axis_ranges(p.nz, L, p.fs != 0)};
    bool ok[3];
    for (int a = 0; a < 3; ++a) {
        ok[a] = rr[a].n > 0;
        for (int r = 0; r < rr[a].n; ++r) ok[a] = ok[a] && rr[a].hi[r] - rr[a].lo[r] == L;
    }
    // x: row segments start on 16-byte boundaries, and the compact arrays exist
    Ranges rx;
    ok[0] = ok[0] && x_tileable(p, &rx) && p.xc != nullptr;
    // an axis whose maps cannot be encoded keeps the marching pass
    for (int b = 0; b < 2; ++b) {
        ok[0] = ok[0] && encode_axis<0>(p, u[b], u[1 - b], &t->maps[b][0]);
        ok[1] = ok[1] && encode_axis<1>(p, u[b], u[1 - b], &t->maps[b][1]);
        ok[2] = ok[2] && encode_axis<2>(p, u[b], u[1 - b], &t->maps[b][2]);
    }
    if (tile_attr<0, 8>() || tile_attr<1, 8>() || tile_attr<2, 8>() || tile_attr<0, 20>() || tile_attr<1, 20>() ||
        tile_attr<2, 20>()) {
        cudaGetLastError();
        return true;   // no tiled pass: the marching passes serve every axis
    }
    const bool w8 = L == 8;
    t->resident[0] = w8 ? tile_blocks<0, 8>() : tile_blocks<0, 20>();
    t->resident[1] = w8 ? tile_blocks<1, 8>() : tile_blocks<1, 20>();
    t->resident[2] = w8 ? tile_blocks<2, 8>() : tile_blocks<2, 20>();
    for (int a = 0; a < 3; ++a) ok[a] = ok[a] && t->resident[a] > 0;
    for (int a = 0; a < 3; ++a) t->ok[a] = ok[a];
    return true;
}

cudaError_t launch_cpml_layers(const CpmlArgs &p, const CpmlTiles *tiles, int buffer, const float *u, float *uout,
                               cudaStream_t s, int *launches) {
    *launches = 0;
    if (p.nbl <= 0) return cudaSuccess;
    const int per = p.zc > 0 ? p.zc : kCpmlPlanes;
    const Ranges rx = axis_ranges(p.nx, p.nbl, false), ry = axis_ranges(p.ny, p.nbl, false),
                 rz = axis_ranges(p.nz, p.nbl, p.fs != 0);
    const bool use = tiles && p.tiles && (buffer == 0 || buffer == 1);
    bool x_warp = true;
    for (int r = 0; r < rx.n; ++r) x_warp = x_warp && rx.hi[r] - rx.lo[r] <= kWarpCells;
    const long long xl = (long long)p.ny * p.nz * rx.n, yl = (long long)p.nx * p.nz * ry.n,
                    zl = (long long)p.nx * p.ny * rz.n;
    if (rx.n > 0) {
        if (use && tiles->ok[0])
            launch_tile_axis<0>(*tiles, buffer, p, rx, s);
        else if (x_warp)
            cpml_x_warp_kernel<<<blocks_for(((xl + (long long)per * kRows - 1) / ((long long)per * kRows)) * 32), 128,
                                 0, s>>>(p, rx, u, uout);
        else
            cpml_line_kernel<0><<<blocks_for((xl + per - 1) / per), 128, 0, s>>>(p, rx, u, uout);
        if (cudaError_t e = cudaGetLastError()) return e;
        ++*launches;
    }
    if (ry.n > 0) {
        if (use && tiles->ok[1])
            launch_tile_axis<1>(*tiles, buffer, p, ry, s);
        else
            cpml_line_kernel<1><<<blocks_for((yl + per - 1) / per), 128, 0, s>>>(p, ry, u, uout);
        if (cudaError_t e = cudaGetLastError()) return e;
        ++*launches;
    }
    if (rz.n > 0) {
        if (use && tiles->ok[2])
            launch_tile_axis<2>(*tiles, buffer, p, rz, s);
        else
            cpml_line_kernel<2><<<blocks_for((zl + per - 1) / per), 128, 0, s>>>(p, rz, u, uout);
        if (cudaError_t e = cudaGetLastError()) return e;
        ++*launches;
    }
    return cudaSuccess;
}

}  // namespace mmod
