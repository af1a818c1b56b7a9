// Variable-density acoustic propagator on a staggered (Yee) grid: the paper's
// first-order system (Sec. 3, "acoustic_iso"),
//     (1 / (rho v^2)) p_t - div vel = f,     rho vel_t - grad p = 0,
// i.e. p_t = K (div vel + f), vel_t = b grad p with K = rho v^2, b = 1 / rho.
// p, K and b live at the grid points; the velocity component along axis a
// lives half a cell further along a.  Leapfrog in time, velocities at half
// steps.  Per time step n:
//   velocity kernel  vel_a += dt bh_a D+_a p^n          (in place)
//   pressure kernel  p     += dt K (sum_a D-_a vel_a)   (in place)
//   injection        p(x_s) += dt K w[n] / (hx hy hz (1 + eps))
// with the order-8 staggered differences
//   D+_a p (i + 1/2) = sum_m a_m (p(i + m) - p(i - m + 1)) / h_a,
//   D-_a q (i)       = sum_m a_m (q(i + m - 1) - q(i - m)) / h_a,
// a_m = 1225/1024, -245/3072, 49/5120, -5/7168, zero outside the grid;
// buoyancy at a half point the mean of b at its two grid points (b itself
// past the last point).  Layers: damping (both fields relax at the summed
// profile, centred: x <- [(1 - eps) x + dt (...)] / (1 + eps), eps = dt eta / 2
// at each field's own position) or CPML (one memory variable per derivative
// in its axis's layers, recursive convolution m = B m + G D).  Receivers
// record p^{n+1} after the injection of step n.  Free surface (option): p = 0
// on the plane k = 0; above it p is the odd image p(-m) = -p(m) and v_z (at
// the half points) the even image v_z(-m) = v_z(m - 1); no top layer.
//
// Kernels.  Both step kernels give a CTA a 64 x 16 x-y tile and a range of
// planes; one elected thread streams planes into shared-memory rings with
// cp.async.bulk.tensor (mbarrier per slot, transaction bytes, bounded waits),
// the tensor maps' zero fill being the "zero outside the grid" reading:
//   velocity kernel: p planes with a 4-cell x-y halo (72 x 24) and the own
//     velocity planes (3 x 64 x 16) and buoyancy planes with a +1 x-y halo
//     (68 x 17); z neighbours of p from a register queue of 8 planes;
//   pressure kernel: vx planes with an x halo (72 x 16), vy planes with a y
//     halo (64 x 24), own p and dt K planes, and vz own planes feeding a
//     register queue of 8 planes for the z difference.
// Each thread computes 2 (x) x 2 (y) points.  The plain kernels (one thread
// per point, bounds-checked global loads) perform the same per-point FP32
// operations in the same order: the two paths agree bit for bit.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "mmod_handle.h"
#include "tma_ptx.cuh"

#define MMOD_API extern "C" __attribute__((visibility("default")))

namespace mmod {

// Order-8 staggered first-derivative weights (unit spacing) and the largest
// magnitude of their symbol, sum_m |a_m| (at k h = pi the symbol of D+ is
// 2 sum_m a_m sin((2m - 1) pi / 2) / h = 2 sum_m |a_m| / h).
constexpr double kStag8[kRadius] = {1225.0 / 1024.0, -245.0 / 3072.0, 49.0 / 5120.0, -5.0 / 7168.0};
constexpr double kStagSymbol8 = 1225.0 / 1024.0 + 245.0 / 3072.0 + 49.0 / 5120.0 + 5.0 / 7168.0;

struct VdArgs {
    int nx, ny, nz, nxp;
    long long plane;
    int nbl;
    int cpml;
    int fs;                    // free surface at k = 0
    float w[3][kRadius];       // a_m / h_a
    float *p;                  // pressure (padded)
    float *v[3];               // velocities (padded)
    const float *kd;           // dt rho v^2
    const float *bd;           // dt / rho
    // damping: eps = dt eta / 2 at the grid points (g) and half points (h) of each axis
    const float *eg[3], *eh[3];
    // CPML: memory volumes and coefficients B, G at grid / half points per axis
    float *psi[3], *phi[3];
    const float *Bg[3], *Gg[3], *Bh[3], *Gh[3];
    int *err;
    // programmatic dependent launch: each kernel may start before its
    // predecessor ends; it reads the predecessor's output after
    // griddepcontrol.wait and lets its own dependents start only after that
    int pdl;
    // sources added by the pressure kernel of the TMA path (ngrp = 0: by the
    // separate injection kernel): groups of sources on one grid point
    int ngrp, nt, n;
    const int *grp_ijk;        // [ngrp][3]
    const long long *grp_off;
    const int *grp_first, *src_id;
    const float *src_scale, *wavelet;
    // receivers of the previous step, gathered by the velocity kernel
    int nrec;
    const long long *rec_off;
    float *traces;             // row to fill, or null
};

namespace {

constexpr int TX = 64, TY = 16, RY = 2, NWARP = TY / RY, NT = NWARP * 32;
constexpr int PHX = TX + 2 * kRadius, PHY = TY + 2 * kRadius;   // 72 x 24: p with its halo
constexpr int BX = TX + 4, BY = TY + 1;                         // 68 x 17: b with +1 halo (16-byte rows)
constexpr int OWN = TX * TY;

// ---------------------------------------------------------------------------
// Per-point arithmetic shared by the TMA and plain kernels.
// ---------------------------------------------------------------------------

// sum_m w_m (hi_m - lo_m), m = 1..4, in that order (first term a product).
__device__ __forceinline__ float stag_diff(const float (&w)[kRadius], float h1, float l1, float h2, float l2,
                                           float h3, float l3, float h4, float l4) {
    float d = __fmul_rn(w[0], __fsub_rn(h1, l1));
    d = __fmaf_rn(w[1], __fsub_rn(h2, l2), d);
    d = __fmaf_rn(w[2], __fsub_rn(h3, l3), d);
    return __fmaf_rn(w[3], __fsub_rn(h4, l4), d);
}

// Mean of dt * b over a half point's two grid points (own value past the edge).
__device__ __forceinline__ float half_b(float b0, float b1, bool inside) {
    return inside ? __fmul_rn(0.5f, __fadd_rn(b0, b1)) : b0;
}

// x <- [(1 - eps) x + c d] / (1 + eps), the reciprocal by recip_nr (within
// one ulp of the correctly rounded one); with eps = 0 exactly x + c d.
__device__ __forceinline__ float relax(float x, float c, float d, float eps) {
    const float t = __fmaf_rn(c, d, __fmul_rn(__fsub_rn(1.0f, eps), x));
    return __fmul_rn(t, recip_nr(__fadd_rn(1.0f, eps)));
}

__device__ __forceinline__ float undamped(float x, float c, float d) { return __fmaf_rn(c, d, x); }

// CPML: memory m <- B m + G d (stored), returns d + m.
__device__ __forceinline__ float cpml_mem(float *m, float B, float G, float d) {
    const float nm = __fmaf_rn(B, *m, __fmul_rn(G, d));
    *m = nm;
    return __fadd_rn(d, nm);
}

__device__ __forceinline__ int zero_clip(int v, int n) { return v < 0 ? 0 : (v >= n ? n - 1 : v); }

// Programmatic dependent launch (no-ops without it): wait for the previous
// kernel of the stream; allow the next one to start.  The step kernels
// release their dependents after their plane loop, so that the next kernel's
// CTAs take SM slots only as this kernel's CTAs finish.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait_then_release() {
    pdl_wait();
    pdl_release();
}

// ---------------------------------------------------------------------------
// Plain kernels: one thread per point.
// ---------------------------------------------------------------------------

__device__ __forceinline__ float at_or0(const float *f, const VdArgs &a, int i, int j, int k) {
    const bool in = (unsigned)i < (unsigned)a.nx && (unsigned)j < (unsigned)a.ny && (unsigned)k < (unsigned)a.nz;
    return in ? f[(long long)k * a.plane + (long long)j * a.nxp + i] : 0.0f;
}

// p above a free surface: the odd image; v_z: the even image shifted by the
// half cell, v_z(-m) = v_z(m - 1).
__device__ __forceinline__ float p_at(const VdArgs &a, int i, int j, int k) {
    if (a.fs && k < 0) return -at_or0(a.p, a, i, j, -k);
    return at_or0(a.p, a, i, j, k);
}

__device__ __forceinline__ float vz_at(const VdArgs &a, int i, int j, int k) {
    if (a.fs && k < 0) return at_or0(a.v[2], a, i, j, -k - 1);
    return at_or0(a.v[2], a, i, j, k);
}

__global__ void vd_velocity_simple(VdArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (blockIdx.x == 0 && blockIdx.y == 0 && a.traces) {
        for (int r = threadIdx.y * blockDim.x + threadIdx.x + k * blockDim.x * blockDim.y; r < a.nrec;
             r += blockDim.x * blockDim.y * gridDim.z)
            a.traces[r] = a.p[a.rec_off[r]];
    }
    if (i >= a.nx || j >= a.ny) return;
    const long long o = (long long)k * a.plane + (long long)j * a.nxp + i;
    const int idx[3] = {i, j, k};
    const int n3[3] = {a.nx, a.ny, a.nz};
    const float b0 = a.bd[o];
    for (int ax = 0; ax < 3; ++ax) {
        const int di = ax == 0, dj = ax == 1, dk = ax == 2;
        float h[kRadius], l[kRadius];
        for (int m = 1; m <= kRadius; ++m) {
            h[m - 1] = p_at(a, i + m * di, j + m * dj, k + m * dk);
            l[m - 1] = p_at(a, i - (m - 1) * di, j - (m - 1) * dj, k - (m - 1) * dk);
        }
        float d = stag_diff(a.w[ax], h[0], l[0], h[1], l[1], h[2], l[2], h[3], l[3]);
        const bool nxt = idx[ax] + 1 < n3[ax];
        const float b1 = nxt ? at_or0(a.bd, a, i + di, j + dj, k + dk) : 0.0f;
        const float bh = half_b(b0, b1, nxt);
        float *v = a.v[ax] + o;
        if (a.cpml) {
            const float G = a.Gh[ax][idx[ax]];
            if (G != 0.0f) d = cpml_mem(a.psi[ax] + o, a.Bh[ax][idx[ax]], G, d);
            *v = undamped(*v, bh, d);
        } else {
            float eps = 0.0f;
            // e_x + e_y + e_z, each at the component's own position
            eps = __fadd_rn(__fadd_rn(ax == 0 ? a.eh[0][i] : a.eg[0][i], ax == 1 ? a.eh[1][j] : a.eg[1][j]),
                            ax == 2 ? a.eh[2][k] : a.eg[2][k]);
            *v = relax(*v, bh, d, eps);
        }
    }
}

__global__ void vd_pressure_simple(VdArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= a.nx || j >= a.ny) return;
    const long long o = (long long)k * a.plane + (long long)j * a.nxp + i;
    const int idx[3] = {i, j, k};
    float dv[3];
    for (int ax = 0; ax < 3; ++ax) {
        const int di = ax == 0, dj = ax == 1, dk = ax == 2;
        float h[kRadius], l[kRadius];
        for (int m = 1; m <= kRadius; ++m) {
            if (ax == 2) {
                h[m - 1] = vz_at(a, i, j, k + (m - 1));
                l[m - 1] = vz_at(a, i, j, k - m);
            } else {
                h[m - 1] = at_or0(a.v[ax], a, i + (m - 1) * di, j + (m - 1) * dj, k);
                l[m - 1] = at_or0(a.v[ax], a, i - m * di, j - m * dj, k);
            }
        }
        dv[ax] = stag_diff(a.w[ax], h[0], l[0], h[1], l[1], h[2], l[2], h[3], l[3]);
        if (a.cpml) {
            const float G = a.Gg[ax][idx[ax]];
            if (G != 0.0f) dv[ax] = cpml_mem(a.phi[ax] + o, a.Bg[ax][idx[ax]], G, dv[ax]);
        }
    }
    const float div = __fadd_rn(__fadd_rn(dv[0], dv[1]), dv[2]);
    if (a.fs && k == 0) {
        a.p[o] = 0.0f;   // p = 0 on the free surface
    } else if (a.cpml) {
        a.p[o] = undamped(a.p[o], a.kd[o], div);
    } else {
        const float eps = __fadd_rn(__fadd_rn(a.eg[0][i], a.eg[1][j]), a.eg[2][k]);
        a.p[o] = relax(a.p[o], a.kd[o], div, eps);
    }
}

// ---------------------------------------------------------------------------
// TMA kernels.
// ---------------------------------------------------------------------------

constexpr int VNSP = 8;    // p halo slots (8-plane window from the queue's leading plane to the centre + prefetch)
constexpr int VNSO = 3;    // own velocity slots
constexpr int VNSB = 4;    // buoyancy slots (planes k and k + 1 resident)
// slots start on 128-byte boundaries (the b box, 68 x 17 floats, is padded)
constexpr int V_SLOT_P = PHX * PHY, V_SLOT_O = 3 * OWN, V_BOX_B = BX * BY, V_SLOT_B = (V_BOX_B + 31) / 32 * 32;
static_assert(V_SLOT_P % 32 == 0 && V_SLOT_O % 32 == 0, "128-byte slots");
constexpr int V_SMEM = (VNSP * V_SLOT_P + VNSO * V_SLOT_O + VNSB * V_SLOT_B) * 4 + (VNSP + VNSO + VNSB) * 8 + 16;

constexpr int PNSC = 3;    // centre slots: vx (72 x 16), vy (64 x 24), p, dt K (64 x 16)
constexpr int PNSZ = 8;    // vz own slots feeding the queue
constexpr int P_VX = PHX * TY, P_VY = TX * PHY;
constexpr int P_SLOT_C = P_VX + P_VY + 2 * OWN;
constexpr int P_SMEM = (PNSC * P_SLOT_C + PNSZ * OWN) * 4 + (PNSC + PNSZ) * 8 + 16;

static_assert(V_SMEM <= 113 * 1024 && P_SMEM <= 113 * 1024, "two CTAs per SM");

struct VdMaps {
    CUtensorMap p_halo;          // p, 72 x 24 box
    CUtensorMap own[3];          // vx, vy, vz, 64 x 16 box
    CUtensorMap b_box;           // dt / rho, 68 x 17 box
    CUtensorMap vx_halo;         // vx, 72 x 16 box
    CUtensorMap vy_halo;         // vy, 64 x 24 box
    CUtensorMap p_own, k_own;    // p, dt K, 64 x 16 box
};

struct VdGeom {
    int tiles_x, tiles_y, zchunks, zlen;
};

__device__ __forceinline__ void tile_of(const VdGeom &g, int bid, int nz, int &x0, int &y0, int &z0, int &T) {
    const int tx = bid % g.tiles_x;
    const int ty = (bid / g.tiles_x) % g.tiles_y;
    const int ch = bid / (g.tiles_x * g.tiles_y);
    x0 = tx * TX;
    y0 = ty * TY;
    z0 = ch * g.zlen;
    T = min(nz - z0, g.zlen);
}

// Every thread stops at the next block barrier once a wait gave up; the
// elected thread then waits (bounded) for the copies it issued.  Sequences
// 0 .. hi-1 went to slot seq % nslots, so slot s saw (hi - s + nslots - 1) / nslots
// phases and its last one has parity (that count - 1) & 1.
__device__ __forceinline__ void drain(uint64_t *bars, int hi, int nslots) {
    for (int s = 0; s < nslots && s < hi; ++s) mbar_drain(&bars[s], (unsigned)(((hi - s + nslots - 1) / nslots - 1) & 1));
}

// Packed FP32x2 forms of the per-point helpers: per component exactly the
// scalar operations above (a - b is a + (-b), negation being exact).
__device__ __forceinline__ float2 bc2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }

__device__ __forceinline__ float2 stag_diff2(const float (&w)[kRadius], float2 h1, float2 l1, float2 h2, float2 l2,
                                             float2 h3, float2 l3, float2 h4, float2 l4) {
    float2 d = __fmul2_rn(bc2(w[0]), sub2(h1, l1));
    d = __ffma2_rn(bc2(w[1]), sub2(h2, l2), d);
    d = __ffma2_rn(bc2(w[2]), sub2(h3, l3), d);
    return __ffma2_rn(bc2(w[3]), sub2(h4, l4), d);
}

__device__ __forceinline__ float2 half_b2(float2 b0, float2 b1, bool in0, bool in1) {
    const float2 m = __fmul2_rn(bc2(0.5f), __fadd2_rn(b0, b1));
    return make_float2(in0 ? m.x : b0.x, in1 ? m.y : b0.y);
}

__device__ __forceinline__ float2 relax2(float2 x, float2 c, float2 d, float2 eps) {
    const float2 t = __ffma2_rn(c, d, __fmul2_rn(sub2(bc2(1.0f), eps), x));
    const float2 one_e = __fadd2_rn(bc2(1.0f), eps);
    return __fmul2_rn(t, make_float2(recip_nr(one_e.x), recip_nr(one_e.y)));
}

__device__ __forceinline__ float2 undamped2(float2 x, float2 c, float2 d) { return __ffma2_rn(c, d, x); }

// CPML of two x-adjacent points (skipped where G = 0 or outside the grid).
__device__ __forceinline__ float2 cpml_pair(float *mem, const float *B, const float *G, int i0, int i1, int n,
                                            bool in0, bool in1, float2 d) {
    if (in0) {
        const float g0 = G[min(i0, n - 1)];
        if (g0 != 0.0f) d.x = cpml_mem(mem, B[min(i0, n - 1)], g0, d.x);
    }
    if (in1) {
        const float g1 = G[min(i1, n - 1)];
        if (g1 != 0.0f) d.y = cpml_mem(mem + 1, B[min(i1, n - 1)], g1, d.y);
    }
    return d;
}

__device__ __forceinline__ void store_pair(float *dst, float2 v, bool in0, bool in1) {
    if (in1)
        *reinterpret_cast<float2 *>(dst) = v;
    else if (in0)
        dst[0] = v.x;
}

// ---------------------------------------------------------------------------
// Velocity kernel.  Rings (sequence -> plane): p halo tiles, seq s -> z0-3+s
// (the queue window of plane k is p(k-3 .. k+4), the centre tile is seq t+3);
// own velocity tiles and buoyancy tiles, seq s -> z0+s (planes k and k+1 of
// b are resident during step t).  The plane loop is unrolled kVU times: at
// step J of a group queue slot J + i holds p(k - 3 + i) (kVQ = 7 + kVU slots),
// and after each group the queue shifts down by kVU.  With kVU = 8 the
// slots are used modulo 8 instead and nothing shifts (more code per loop).
// ---------------------------------------------------------------------------
constexpr int kVU = 4;
constexpr int kVQ = kVU == 8 ? 8 : 2 * kRadius - 1 + kVU;
__host__ __device__ constexpr int vq(int J, int i) { return kVU == 8 ? (J + i) % 8 : J + i; }

struct VCtx {
    float *ring_p, *ring_o, *ring_b;
    uint64_t *bar_p, *bar_o, *bar_b;
    int *abort_flag;
    int x0, y0, z0, T, lane, warp, xl, x;
    float2 egx, ehx;       // eps at this thread's two columns (grid, half points)
    float egy[RY], ehy[RY];
    bool lay_xy[RY];       // tile columns or this row pair touch an x or y layer (half points included)
    bool in0, in1;         // columns x, x+1 inside the grid
};

__device__ __forceinline__ void v_read_q(const VCtx &c, int seq, float2 (&dst)[RY]) {
    const float *base = c.ring_p + (seq % VNSP) * V_SLOT_P + (kRadius + RY * c.warp) * PHX + kRadius + c.xl;
#pragma unroll
    for (int r = 0; r < RY; ++r) dst[r] = *reinterpret_cast<const float2 *>(base + r * PHX);
}

template <int J, bool C>
__device__ __forceinline__ bool v_plane(const VdArgs &a, const VCtx &c, int t, float2 (&q)[kVQ][RY]) {
    const int k = c.z0 + t;
    if (!(mbar_wait(&c.bar_p[(t + 7) % VNSP], ((t + 7) / VNSP) & 1, c.abort_flag, a.err) &&
          mbar_wait(&c.bar_o[t % VNSO], (t / VNSO) & 1, c.abort_flag, a.err) &&
          mbar_wait(&c.bar_b[t % VNSB], (t / VNSB) & 1, c.abort_flag, a.err) &&
          mbar_wait(&c.bar_b[(t + 1) % VNSB], ((t + 1) / VNSB) & 1, c.abort_flag, a.err)))
        return false;
    v_read_q(c, t + 7, q[vq(J, 7)]);
    const float *ctr = c.ring_p + ((t + 3) % VNSP) * V_SLOT_P;
    const float *own = c.ring_o + (t % VNSO) * V_SLOT_O;
    const float *bk = c.ring_b + (t % VNSB) * V_SLOT_B;
    const float *bk1 = c.ring_b + ((t + 1) % VNSB) * V_SLOT_B;
    const bool zl = !C && (k < a.nbl || k >= a.nz - 1 - a.nbl);
    const float egz = C ? 0.0f : a.eg[2][k], ehz = C ? 0.0f : a.eh[2][k];
    const bool zin = k + 1 < a.nz;
    // y neighbours: rows 2w+1 .. 2w+9 of the centre tile, columns xl+4, xl+5
    float2 yc[RY + 2 * kRadius - 1];
#pragma unroll
    for (int i = 0; i < RY + 2 * kRadius - 1; ++i)
        yc[i] = *reinterpret_cast<const float2 *>(ctr + (RY * c.warp + 1 + i) * PHX + kRadius + c.xl);
#pragma unroll
    for (int r = 0; r < RY; ++r) {
        const int yl = RY * c.warp + r, y = c.y0 + yl;
        // x neighbours: columns xl .. xl+9 of row yl+4 as pairs xa[j] = (col 2j, col 2j+1)
        float2 xa[5];
        const float *row = ctr + (yl + kRadius) * PHX + c.xl;
#pragma unroll
        for (int j = 0; j < 5; ++j) xa[j] = *reinterpret_cast<const float2 *>(row + 2 * j);
        // D+_x: point c uses cols (5+c, 4+c), (6+c, 3+c), (7+c, 2+c), (8+c, 1+c)
        const float2 dx = stag_diff2(a.w[0], make_float2(xa[2].y, xa[3].x), xa[2], xa[3], make_float2(xa[1].y, xa[2].x),
                                     make_float2(xa[3].y, xa[4].x), xa[1], xa[4], make_float2(xa[0].y, xa[1].x));
        // D+_y: rows yl+4+m and yl+5-m -> yc[r+3+m], yc[r+4-m]
        const float2 dy = stag_diff2(a.w[1], yc[r + 4], yc[r + 3], yc[r + 5], yc[r + 2], yc[r + 6], yc[r + 1],
                                     yc[r + 7], yc[r + 0]);
        // D+_z: planes k+m and k-m+1 -> queue entries 3+m and 4-m
        const float2 dz = stag_diff2(a.w[2], q[vq(J, 4)][r], q[vq(J, 3)][r], q[vq(J, 5)][r], q[vq(J, 2)][r],
                                     q[vq(J, 6)][r], q[vq(J, 1)][r], q[vq(J, 7)][r], q[vq(J, 0)][r]);
        // dt b at the half points
        const float *brow = bk + yl * BX + c.xl;
        const float2 b01 = *reinterpret_cast<const float2 *>(brow);
        const float b2 = brow[2];
        const float2 bn = *reinterpret_cast<const float2 *>(brow + BX);
        const float2 bz = *reinterpret_cast<const float2 *>(bk1 + yl * BX + c.xl);
        const bool yin = y + 1 < a.ny;
        const float2 bhx = half_b2(b01, make_float2(b01.y, b2), c.x + 1 < a.nx, c.x + 2 < a.nx);
        const float2 bhy = half_b2(b01, bn, yin, yin);
        const float2 bhz = half_b2(b01, bz, zin, zin);
        const float *orow = own + yl * TX + c.xl;
        const float2 vx = *reinterpret_cast<const float2 *>(orow);
        const float2 vy = *reinterpret_cast<const float2 *>(orow + OWN);
        const float2 vz = *reinterpret_cast<const float2 *>(orow + 2 * OWN);
        const bool in0 = c.in0 && y < a.ny, in1 = c.in1 && y < a.ny;
        const long long o = (long long)k * a.plane + (long long)y * a.nxp + c.x;
        float2 nx_, ny_, nz_;
        if (!C && (c.lay_xy[r] || zl)) {
            // eps = (e_x + e_y) + e_z at each component's own position
            const float2 ex = __fadd2_rn(__fadd2_rn(c.ehx, bc2(c.egy[r])), bc2(egz));
            const float2 ey = __fadd2_rn(__fadd2_rn(c.egx, bc2(c.ehy[r])), bc2(egz));
            const float2 ez = __fadd2_rn(__fadd2_rn(c.egx, bc2(c.egy[r])), bc2(ehz));
            nx_ = relax2(vx, bhx, dx, ex);
            ny_ = relax2(vy, bhy, dy, ey);
            nz_ = relax2(vz, bhz, dz, ez);
        } else if (C) {
            const float2 ddx = cpml_pair(a.psi[0] + o, a.Bh[0], a.Gh[0], c.x, c.x + 1, a.nx, in0, in1, dx);
            const float2 ddy = cpml_pair(a.psi[1] + o, a.Bh[1], a.Gh[1], y, y, a.ny, in0, in1, dy);
            const float2 ddz = cpml_pair(a.psi[2] + o, a.Bh[2], a.Gh[2], k, k, a.nz, in0, in1, dz);
            nx_ = undamped2(vx, bhx, ddx);
            ny_ = undamped2(vy, bhy, ddy);
            nz_ = undamped2(vz, bhz, ddz);
        } else {
            nx_ = undamped2(vx, bhx, dx);
            ny_ = undamped2(vy, bhy, dy);
            nz_ = undamped2(vz, bhz, dz);
        }
        store_pair(a.v[0] + o, nx_, in0, in1);
        store_pair(a.v[1] + o, ny_, in0, in1);
        store_pair(a.v[2] + o, nz_, in0, in1);
    }
    return true;
}

template <bool C>
__global__ void __launch_bounds__(NT, 2)
    vd_velocity_tma(const __grid_constant__ VdArgs a, const __grid_constant__ VdMaps maps, VdGeom g) {
    extern __shared__ __align__(128) unsigned char smem[];
    VCtx c;
    c.ring_p = reinterpret_cast<float *>(smem);
    c.ring_o = c.ring_p + VNSP * V_SLOT_P;
    c.ring_b = c.ring_o + VNSO * V_SLOT_O;
    c.bar_p = reinterpret_cast<uint64_t *>(c.ring_b + VNSB * V_SLOT_B);
    c.bar_o = c.bar_p + VNSP;
    c.bar_b = c.bar_o + VNSO;
    c.abort_flag = reinterpret_cast<int *>(c.bar_b + VNSB);
    const int tid = threadIdx.x;
    c.lane = tid & 31;
    c.warp = tid >> 5;
    tile_of(g, blockIdx.x, a.nz, c.x0, c.y0, c.z0, c.T);
    const int x0 = c.x0, y0 = c.y0, z0 = c.z0, T = c.T;
    const int nseq_p = T + 2 * kRadius - 1;   // p planes z0-3 .. z0+T+3
    const int nseq_b = T + 1;                 // b planes z0 .. z0+T
    int hi_p = 0, hi_o = 0, hi_b = 0;         // sequences issued per ring (elected thread only)

    auto issue_p = [&](int seq) {
        const int s = seq % VNSP;
        int z = z0 - (kRadius - 1) + seq;
        if (a.fs && z < 0) z = -z;   // plane -m holds the odd image of plane m (negated in the queue)
        mbar_expect_tx(&c.bar_p[s], V_SLOT_P * 4);
        tma_load_3d(c.ring_p + s * V_SLOT_P, &maps.p_halo, x0 - kRadius, y0 - kRadius, z, &c.bar_p[s]);
        hi_p = seq + 1;
    };
    auto issue_o = [&](int seq) {
        const int s = seq % VNSO;
        mbar_expect_tx(&c.bar_o[s], V_SLOT_O * 4);
#pragma unroll
        for (int f = 0; f < 3; ++f)
            tma_load_3d(c.ring_o + s * V_SLOT_O + f * OWN, &maps.own[f], x0, y0, z0 + seq, &c.bar_o[s]);
        hi_o = seq + 1;
    };
    auto issue_b = [&](int seq) {
        const int s = seq % VNSB;
        mbar_expect_tx(&c.bar_b[s], V_BOX_B * 4);
        tma_load_3d(c.ring_b + s * V_SLOT_B, &maps.b_box, x0, y0, z0 + seq, &c.bar_b[s]);
        hi_b = seq + 1;
    };

    if (tid == 0) {
        for (int s = 0; s < VNSP; ++s) mbar_init(&c.bar_p[s], 1);
        for (int s = 0; s < VNSO; ++s) mbar_init(&c.bar_o[s], 1);
        for (int s = 0; s < VNSB; ++s) mbar_init(&c.bar_b[s], 1);
        *c.abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        // own velocities (last written two launches back) and buoyancy first
        if (T > 0) {
            for (int q = 0; q < VNSO && q < T; ++q) issue_o(q);
            for (int q = 0; q < VNSB && q < nseq_b; ++q) issue_b(q);
        }
    }
    pdl_wait();   // p^n of the pressure kernel and the source add
    if (tid == 0 && T > 0)
        for (int q = 0; q < VNSP && q < nseq_p; ++q) issue_p(q);
    // receivers of the previous step: p^n, read-only in this kernel
    if (a.traces)
        for (int r = blockIdx.x * NT + tid; r < a.nrec; r += gridDim.x * NT) a.traces[r] = a.p[a.rec_off[r]];
    __syncthreads();
    if (T <= 0) return;

    c.xl = 2 * c.lane;
    c.x = x0 + c.xl;
    c.in0 = c.x < a.nx;
    c.in1 = c.x + 1 < a.nx;
    c.egx = C ? bc2(0.0f) : make_float2(a.eg[0][zero_clip(c.x, a.nx)], a.eg[0][zero_clip(c.x + 1, a.nx)]);
    c.ehx = C ? bc2(0.0f) : make_float2(a.eh[0][zero_clip(c.x, a.nx)], a.eh[0][zero_clip(c.x + 1, a.nx)]);
    // the half point after the last inner index (n - 1 - nbl) already lies in the layer
    const bool lay_x = x0 < a.nbl || x0 + TX - 1 >= a.nx - 1 - a.nbl;
#pragma unroll
    for (int r = 0; r < RY; ++r) {
        const int y = y0 + RY * c.warp + r, yi = zero_clip(y, a.ny);
        c.egy[r] = C ? 0.0f : a.eg[1][yi];
        c.ehy[r] = C ? 0.0f : a.eh[1][yi];
        c.lay_xy[r] = lay_x || y < a.nbl || y >= a.ny - 1 - a.nbl;
    }

    float2 q[kVQ][RY];
    bool ok = true;
    for (int s = 0; s < 2 * kRadius - 1 && ok; ++s) {
        ok = mbar_wait(&c.bar_p[s % VNSP], (s / VNSP) & 1, c.abort_flag, a.err);
        if (ok) {
#pragma unroll
            for (int i = 0; i < 2 * kRadius - 1; ++i)
                if (i == s) v_read_q(c, s, q[i]);
        }
    }
    if (a.fs && ok) {   // queue planes above k = 0 (z0-3+i < 0) hold the images: negate
#pragma unroll
        for (int i = 0; i < kRadius - 1; ++i)
            if (z0 - (kRadius - 1) + i < 0) {
#pragma unroll
                for (int r = 0; r < RY; ++r) q[i][r] = make_float2(-q[i][r].x, -q[i][r].y);
            }
    }
    __syncthreads();
    // the slots of planes z0-3 .. z0-1 (never a centre) are refilled now
    if (!*c.abort_flag && tid == 0)
        for (int s = 0; s < kRadius - 1; ++s)
            if (s + VNSP < nseq_p) issue_p(s + VNSP);

    // end of step t: the centre tile (seq t+3), the own tile and b plane k are free
#define VD_VSTEP(J)                                                                   \
    if (t + (J) < T) {                                                                \
        v_plane<(J), C>(a, c, t + (J), q);                                               \
        __syncthreads();                                                              \
        if (*c.abort_flag) break;                                                     \
        if (tid == 0) {                                                               \
            if (t + (J) + 3 + VNSP < nseq_p) issue_p(t + (J) + 3 + VNSP);             \
            if (t + (J) + VNSO < T) issue_o(t + (J) + VNSO);                          \
            if (t + (J) + VNSB < nseq_b) issue_b(t + (J) + VNSB);                     \
        }                                                                             \
    }
    if (!*c.abort_flag) {
#pragma unroll 1
        for (int t = 0; t < T; t += kVU) {
            VD_VSTEP(0) VD_VSTEP(1) VD_VSTEP(2) VD_VSTEP(3)
            if constexpr (kVU == 8) {
                VD_VSTEP(4) VD_VSTEP(5) VD_VSTEP(6) VD_VSTEP(7)
            } else {
#pragma unroll
                for (int i = 0; i < 2 * kRadius - 1; ++i) {
#pragma unroll
                    for (int r = 0; r < RY; ++r) q[i][r] = q[i + kVU][r];
                }
            }
        }
    }
#undef VD_VSTEP
    pdl_release();
    if (*c.abort_flag && tid == 0) {
        drain(c.bar_p, hi_p, VNSP);
        drain(c.bar_o, hi_o, VNSO);
        drain(c.bar_b, hi_b, VNSB);
    }
}

// ---------------------------------------------------------------------------
// Pressure kernel.  Rings: centre tiles (vx with its x halo, vy with its y
// halo, p, dt K), seq s -> z0+s; vz own tiles, seq s -> z0-4+s, read into the
// queue.  The plane loop is unrolled kPU times: at step J of a group queue
// slot J + i holds vz(k - 4 + i), and the queue shifts down by kPU after each
// group (kPU = 8: slots modulo 8, no shifts).  The pressure kernel's code is
// small enough at 8 (240^3: 101.8 against 101.4 Gpoint-updates/s at 4).
// ---------------------------------------------------------------------------
constexpr int kPU = 8;
constexpr int kPQ = kPU == 8 ? 8 : 2 * kRadius - 1 + kPU;
__host__ __device__ constexpr int pq(int J, int i) { return kPU == 8 ? (J + i) % 8 : J + i; }
struct PCtx {
    float *ring_c, *ring_z;
    uint64_t *bar_c, *bar_z;
    int *abort_flag;
    int x0, y0, z0, T, lane, warp, xl, x;
    float2 egx;
    float egy[RY];
    bool lay_xy[RY];
    bool in0, in1;
};

__device__ __forceinline__ void p_read_q(const PCtx &c, int seq, float2 (&dst)[RY]) {
    const float *base = c.ring_z + (seq % PNSZ) * OWN + RY * c.warp * TX + c.xl;
#pragma unroll
    for (int r = 0; r < RY; ++r) dst[r] = *reinterpret_cast<const float2 *>(base + r * TX);
}

template <int J, bool C>
__device__ __forceinline__ bool p_plane(const VdArgs &a, const PCtx &c, int t, float2 (&q)[kPQ][RY]) {
    const int k = c.z0 + t;
    if (!(mbar_wait(&c.bar_z[(t + 7) % PNSZ], ((t + 7) / PNSZ) & 1, c.abort_flag, a.err) &&
          mbar_wait(&c.bar_c[t % PNSC], (t / PNSC) & 1, c.abort_flag, a.err)))
        return false;
    p_read_q(c, t + 7, q[pq(J, 7)]);
    const float *base = c.ring_c + (t % PNSC) * P_SLOT_C;
    const float *tvx = base, *tvy = base + P_VX, *tp = base + P_VX + P_VY, *tk = tp + OWN;
    const bool zl = !C && (k < a.nbl || k > a.nz - 1 - a.nbl);
    const float egz = C ? 0.0f : a.eg[2][k];
    // vy rows 2w .. 2w+8 at columns xl, xl+1
    float2 yc[RY + 2 * kRadius - 1];
#pragma unroll
    for (int i = 0; i < RY + 2 * kRadius - 1; ++i)
        yc[i] = *reinterpret_cast<const float2 *>(tvy + (RY * c.warp + i) * TX + c.xl);
#pragma unroll
    for (int r = 0; r < RY; ++r) {
        const int yl = RY * c.warp + r, y = c.y0 + yl;
        float2 xa[5];
        const float *row = tvx + yl * PHX + c.xl;
#pragma unroll
        for (int j = 0; j < 5; ++j) xa[j] = *reinterpret_cast<const float2 *>(row + 2 * j);
        // D-_x: point c uses cols (4+c, 3+c), (5+c, 2+c), (6+c, 1+c), (7+c, 0+c)
        float2 dx = stag_diff2(a.w[0], xa[2], make_float2(xa[1].y, xa[2].x), make_float2(xa[2].y, xa[3].x), xa[1],
                               xa[3], make_float2(xa[0].y, xa[1].x), make_float2(xa[3].y, xa[4].x), xa[0]);
        // D-_y: rows yl+3+m and yl+4-m -> yc[r+3+m], yc[r+4-m]
        float2 dy = stag_diff2(a.w[1], yc[r + 4], yc[r + 3], yc[r + 5], yc[r + 2], yc[r + 6], yc[r + 1], yc[r + 7],
                               yc[r + 0]);
        // D-_z: planes k+m-1 and k-m -> queue entries 3+m and 4-m
        float2 dz = stag_diff2(a.w[2], q[pq(J, 4)][r], q[pq(J, 3)][r], q[pq(J, 5)][r], q[pq(J, 2)][r],
                               q[pq(J, 6)][r], q[pq(J, 1)][r], q[pq(J, 7)][r], q[pq(J, 0)][r]);
        const bool in0 = c.in0 && y < a.ny, in1 = c.in1 && y < a.ny;
        const long long o = (long long)k * a.plane + (long long)y * a.nxp + c.x;
        if (C) {
            dx = cpml_pair(a.phi[0] + o, a.Bg[0], a.Gg[0], c.x, c.x + 1, a.nx, in0, in1, dx);
            dy = cpml_pair(a.phi[1] + o, a.Bg[1], a.Gg[1], y, y, a.ny, in0, in1, dy);
            dz = cpml_pair(a.phi[2] + o, a.Bg[2], a.Gg[2], k, k, a.nz, in0, in1, dz);
        }
        const float2 div = __fadd2_rn(__fadd2_rn(dx, dy), dz);
        const float2 po = *reinterpret_cast<const float2 *>(tp + yl * TX + c.xl);
        const float2 ko = *reinterpret_cast<const float2 *>(tk + yl * TX + c.xl);
        float2 pn;
        if (a.fs && k == 0)
            pn = make_float2(0.0f, 0.0f);   // p = 0 on the free surface
        else if (!C && (c.lay_xy[r] || zl))
            pn = relax2(po, ko, div, __fadd2_rn(__fadd2_rn(c.egx, bc2(c.egy[r])), bc2(egz)));
        else
            pn = undamped2(po, ko, div);
        store_pair(a.p + o, pn, in0, in1);
    }
    return true;
}

template <bool C>
__global__ void __launch_bounds__(NT, 2)
    vd_pressure_tma(const __grid_constant__ VdArgs a, const __grid_constant__ VdMaps maps, VdGeom g) {
    extern __shared__ __align__(128) unsigned char smem[];
    PCtx c;
    c.ring_c = reinterpret_cast<float *>(smem);
    c.ring_z = c.ring_c + PNSC * P_SLOT_C;
    c.bar_c = reinterpret_cast<uint64_t *>(c.ring_z + PNSZ * OWN);
    c.bar_z = c.bar_c + PNSC;
    c.abort_flag = reinterpret_cast<int *>(c.bar_z + PNSZ);
    const int tid = threadIdx.x;
    c.lane = tid & 31;
    c.warp = tid >> 5;
    tile_of(g, blockIdx.x, a.nz, c.x0, c.y0, c.z0, c.T);
    const int x0 = c.x0, y0 = c.y0, z0 = c.z0, T = c.T;
    const int nseq_z = T + 2 * kRadius - 1;   // vz planes z0-4 .. z0+T+2
    int hi_c = 0, hi_z = 0;                   // sequences issued per ring (elected thread only)

    // a centre slot: p and dt K (own part), then vx, vy (velocity part); one
    // barrier counts the bytes of all four boxes
    auto issue_c_own = [&](int seq) {
        const int s = seq % PNSC;
        float *base = c.ring_c + s * P_SLOT_C;
        mbar_expect_tx(&c.bar_c[s], P_SLOT_C * 4);
        tma_load_3d(base + P_VX + P_VY, &maps.p_own, x0, y0, z0 + seq, &c.bar_c[s]);
        tma_load_3d(base + P_VX + P_VY + OWN, &maps.k_own, x0, y0, z0 + seq, &c.bar_c[s]);
        hi_c = seq + 1;
    };
    auto issue_c_vel = [&](int seq) {
        const int s = seq % PNSC;
        float *base = c.ring_c + s * P_SLOT_C;
        tma_load_3d(base, &maps.vx_halo, x0 - kRadius, y0, z0 + seq, &c.bar_c[s]);
        tma_load_3d(base + P_VX, &maps.vy_halo, x0, y0 - kRadius, z0 + seq, &c.bar_c[s]);
    };
    auto issue_c = [&](int seq) {
        issue_c_own(seq);
        issue_c_vel(seq);
    };
    auto issue_z = [&](int seq) {
        const int s = seq % PNSZ;
        int z = z0 - kRadius + seq;
        if (a.fs && z < 0) z = -z - 1;   // v_z(-m) = v_z(m - 1): the even image across the surface
        mbar_expect_tx(&c.bar_z[s], OWN * 4);
        tma_load_3d(c.ring_z + s * OWN, &maps.own[2], x0, y0, z, &c.bar_z[s]);
        hi_z = seq + 1;
    };

    if (tid == 0) {
        for (int s = 0; s < PNSC; ++s) mbar_init(&c.bar_c[s], 1);
        for (int s = 0; s < PNSZ; ++s) mbar_init(&c.bar_z[s], 1);
        *c.abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        // p and dt K first (p was last written two launches back)
        if (T > 0)
            for (int q = 0; q < PNSC && q < T; ++q) issue_c_own(q);
    }
    pdl_wait();   // the velocities of the velocity kernel
    if (tid == 0 && T > 0) {
        for (int q = 0; q < PNSC && q < T; ++q) issue_c_vel(q);
        for (int q = 0; q < PNSZ && q < nseq_z; ++q) issue_z(q);
    }
    __syncthreads();
    if (T <= 0) return;

    c.xl = 2 * c.lane;
    c.x = x0 + c.xl;
    c.in0 = c.x < a.nx;
    c.in1 = c.x + 1 < a.nx;
    c.egx = C ? bc2(0.0f) : make_float2(a.eg[0][zero_clip(c.x, a.nx)], a.eg[0][zero_clip(c.x + 1, a.nx)]);
    const bool lay_x = x0 < a.nbl || x0 + TX - 1 > a.nx - 1 - a.nbl;
#pragma unroll
    for (int r = 0; r < RY; ++r) {
        const int y = y0 + RY * c.warp + r;
        c.egy[r] = C ? 0.0f : a.eg[1][zero_clip(y, a.ny)];
        c.lay_xy[r] = lay_x || y < a.nbl || y > a.ny - 1 - a.nbl;
    }

    float2 q[kPQ][RY];
    bool ok = true;
    for (int s = 0; s < 2 * kRadius - 1 && ok; ++s) {
        ok = mbar_wait(&c.bar_z[s % PNSZ], (s / PNSZ) & 1, c.abort_flag, a.err);
        if (ok) {
#pragma unroll
            for (int i = 0; i < 2 * kRadius - 1; ++i)
                if (i == s) p_read_q(c, s, q[i]);
        }
    }
    __syncthreads();
    if (!*c.abort_flag && tid == 0)
        for (int s = 0; s < 2 * kRadius - 1; ++s)
            if (s + PNSZ < nseq_z) issue_z(s + PNSZ);

    // end of step t: the vz tile read into the queue (seq t+7) and the centre slot are free
#define VD_PSTEP(J)                                                                   \
    if (t + (J) < T) {                                                                \
        p_plane<(J), C>(a, c, t + (J), q);                                               \
        __syncthreads();                                                              \
        if (*c.abort_flag) break;                                                     \
        if (tid == 0) {                                                               \
            if (t + (J) + 7 + PNSZ < nseq_z) issue_z(t + (J) + 7 + PNSZ);             \
            if (t + (J) + PNSC < T) issue_c(t + (J) + PNSC);                          \
        }                                                                             \
    }
    if (!*c.abort_flag) {
#pragma unroll 1
        for (int t = 0; t < T; t += kPU) {
            VD_PSTEP(0) VD_PSTEP(1) VD_PSTEP(2) VD_PSTEP(3)
            if constexpr (kPU == 8) {
                VD_PSTEP(4) VD_PSTEP(5) VD_PSTEP(6) VD_PSTEP(7)
            } else {
#pragma unroll
                for (int i = 0; i < 2 * kRadius - 1; ++i) {
#pragma unroll
                    for (int r = 0; r < RY; ++r) q[i][r] = q[i + kPU][r];
                }
            }
        }
    }
#undef VD_PSTEP
    // Sources of this CTA's tile and planes, once its whole z range is stored
    // (the block barrier makes the stores visible); one thread per group,
    // sources in their order: the separate injection kernel's operations.
    if (a.ngrp > 0) {
        __syncthreads();
        if (!*c.abort_flag)
            for (int gi = tid; gi < a.ngrp; gi += NT) {
                const int *q = a.grp_ijk + 3 * gi;
                if (q[0] < x0 || q[0] >= x0 + TX || q[1] < y0 || q[1] >= y0 + TY || q[2] < z0 || q[2] >= z0 + T)
                    continue;
                float *dst = a.p + a.grp_off[gi];
                float v = *dst;
                for (int m = a.grp_first[gi]; m < a.grp_first[gi + 1]; ++m) {
                    const int sid = a.src_id[m];
                    v = __fmaf_rn(a.src_scale[sid], a.wavelet[(long long)sid * a.nt + a.n], v);
                }
                *dst = v;
            }
    }
    pdl_release();
    if (*c.abort_flag && tid == 0) {
        drain(c.bar_c, hi_c, PNSC);
        drain(c.bar_z, hi_z, PNSZ);
    }
}

// Sources grouped by grid point (groups in first-occurrence order, sources
// of a group in their original order): p(x_g) += scale_s w_s[n], in FP32.
__global__ void vd_inject(float *p, int ngrp, const long long *grp_off, const int *grp_first, const int *src_id,
                          const float *scale, const float *wavelet, int nt, int n) {
    pdl_wait_then_release();   // p^{n+1} of the pressure kernel
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ngrp) return;
    float *dst = p + grp_off[g];
    float v = *dst;
    for (int q = grp_first[g]; q < grp_first[g + 1]; ++q) {
        const int s = src_id[q];
        v = __fmaf_rn(scale[s], wavelet[(long long)s * nt + n], v);
    }
    *dst = v;
}

// dense vel, rho -> padded dt rho v^2, dt / rho (FP64 products, rounded once);
// counts non-positive or non-finite inputs; max of v and of
// rho v^2 / min(rho over the 7-point star) (stability), as float bits.
__global__ void vd_model(const float *vel, const float *rho, int nx, int ny, int nz, int nxp, double dt, float *kd,
                         float *bd, unsigned int *maxbits, unsigned long long *bad) {
    const long long n = (long long)nx * ny * nz;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(q % nx);
        const int j = (int)((q / nx) % ny);
        const int k = (int)(q / ((long long)nx * ny));
        const float v = vel[q], r = rho[q];
        if (!(v > 0.0f) || !(r > 0.0f) || !isfinite(v) || !isfinite(r)) {
            atomicAdd(bad, 1ull);
            continue;
        }
        const long long o = (long long)k * ny * nxp + (long long)j * nxp + i;
        kd[o] = (float)(dt * (double)r * (double)v * (double)v);
        bd[o] = (float)(dt / (double)r);
        float rmin = r;
        if (i > 0) rmin = fminf(rmin, rho[q - 1]);
        if (i + 1 < nx) rmin = fminf(rmin, rho[q + 1]);
        if (j > 0) rmin = fminf(rmin, rho[q - nx]);
        if (j + 1 < ny) rmin = fminf(rmin, rho[q + nx]);
        if (k > 0) rmin = fminf(rmin, rho[q - (long long)nx * ny]);
        if (k + 1 < nz) rmin = fminf(rmin, rho[q + (long long)nx * ny]);
        const float veff2 = (float)((double)r * (double)v * (double)v / (double)rmin);
        atomicMax(maxbits, __float_as_uint(v));
        atomicMax(maxbits + 1, __float_as_uint(veff2));
    }
}

// scale_s = dt rho v^2 / (hx hy hz (1 + eps_s)) at each source point (FP64).
__global__ void vd_source_scale(const float *vel, const float *rho, int nx, int ny, int nsrc, const int *ijk,
                                const double *eps, double dt, double cell, float *scale) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsrc) return;
    const long long q = ((long long)ijk[3 * s + 2] * ny + ijk[3 * s + 1]) * nx + ijk[3 * s];
    const double v = vel[q], r = rho[q];
    scale[s] = (float)(dt * r * v * v / (cell * (1.0 + eps[s])));
}

int grid_for(long long n, int block) { return (int)std::min<long long>((n + block - 1) / block, 152LL * 32); }

// Source groups the pressure kernel adds itself (each CTA scans the list).
constexpr int kFoldSources = 1024;

}  // namespace
}  // namespace mmod

using namespace mmod;

struct mmod_vd {
    mmod_config cfg{};
    std::vector<int> src, rec;
    int device = 0, nxp = 0;
    long long plane = 0, vol = 0, npts = 0;
    float *mem = nullptr;             // p, vx, vy, vz, dt K, dt b [, psi x3, phi x3] (padded volumes)
    float *p = nullptr, *v[3] = {nullptr, nullptr, nullptr}, *kd = nullptr, *bd = nullptr;
    float *psi[3] = {nullptr, nullptr, nullptr}, *phi[3] = {nullptr, nullptr, nullptr};
    float *prof = nullptr;            // eps g/h per axis, then CPML B g/h, G g/h per axis
    const float *eg[3] = {}, *eh[3] = {}, *Bg[3] = {}, *Gg[3] = {}, *Bh[3] = {}, *Gh[3] = {};
    float w[3][kRadius] = {};
    // sources grouped by point, receivers
    long long *grp_off = nullptr;
    int *grp_ijk = nullptr;           // [ngrp][3] grid point of each source group
    int *grp_first = nullptr, *src_id = nullptr, *src_ijk_d = nullptr;
    double *src_eps = nullptr;
    float *src_scale = nullptr;
    int ngrp = 0;
    long long *rec_off = nullptr;
    unsigned int *maxbits = nullptr;
    unsigned long long *bad = nullptr;
    float *st_dense = nullptr;        // [nz][ny][nx] staging for state in / out
    int *err_host = nullptr, *err_dev = nullptr;
    cudaStream_t cap = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaGraphExec_t exec = nullptr;
    const void *gkey[2] = {nullptr, nullptr};
    int gkernel = -1;
    long long glaunches = 0, last_launches = 0;
    bool tma_ok = false;
    VdMaps maps{};
    VdGeom geom{};
    int kernel = MMOD_KERNEL_AUTO;
    int pdl = 0;                      // programmatic dependent launch of the TMA step kernels (measured
                                      // equal on 240^3 with the release after the plane loop)
    int zlen = 0;                     // planes per z range (0: the plan's choice)
    VdGeom geom_plan{};               // the plan's decomposition
    bool model_set = false, ran = false, state_pending = false;
    double vmax = 0.0, veff = 0.0;
    cudaError_t latched = cudaSuccess;
    std::string err;
};

namespace {

mmod_status vd_fail(mmod_vd *h, mmod_status st, const std::string &m) {
    h->err = m;
    return st;
}

mmod_status vd_cuda(mmod_vd *h, cudaError_t e, const char *what) {
    h->latched = e;
    h->err = std::string(what) + ": " + cudaGetErrorString(e);
    return MMOD_ERR_CUDA;
}

#define VD_CK(h, call)                                       \
    do {                                                     \
        cudaError_t _e = (call);                             \
        if (_e != cudaSuccess) return vd_cuda((h), _e, #call); \
    } while (0)

mmod_status vd_latched(mmod_vd *h) {
    if (h->err_host && *(volatile int *)h->err_host) {
        h->err = "a device-side wait gave up (timeout)";
        return MMOD_ERR_TIMEOUT;
    }
    if (h->latched != cudaSuccess) {
        h->err = std::string("earlier CUDA failure: ") + cudaGetErrorName(h->latched);
        return MMOD_ERR_CUDA;
    }
    return MMOD_OK;
}

// Depth of the continuous position x into the layers of an axis (capped at
// L); top_free drops the layer at index 0 (free surface).
double layer_depth(double x, int n, int L, bool top_free) {
    double d = 0.0;
    if (!top_free && L - x > d) d = L - x;
    if (x - (n - 1 - L) > d) d = x - (n - 1 - L);
    return d > L ? (double)L : d;
}

// Profiles of one axis at grid (half = 0) or half points: eps = dt eta / 2,
// and the CPML pair B, G (reading shared with the oracle).
void axis_profiles(int n, int L, double h, double vmax, double R, double f0, double dt, int half, bool top_free,
                   double *eps, float *B, float *G) {
    const double d0 = L > 0 ? 3.0 * vmax * std::log(1.0 / R) / (2.0 * L * h) : 0.0;
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < n; ++i) {
        const double x = L > 0 ? layer_depth(i + 0.5 * half, n, L, top_free) : 0.0;
        const double s = L > 0 ? x / L : 0.0;
        const double d = d0 * s * s;
        eps[i] = 0.5 * dt * d;
        if (x == 0.0) {
            B[i] = 1.0f;
            G[i] = 0.0f;
            continue;
        }
        const double alpha = pi * f0 * (1.0 - s);
        const double b = std::exp(-(d + alpha) * dt);
        B[i] = (float)b;
        G[i] = (float)(d * (b - 1.0) / (d + alpha));
    }
}

VdArgs vd_args(mmod_vd *h) {
    VdArgs a{};
    const mmod_config &c = h->cfg;
    a.nx = c.nx; a.ny = c.ny; a.nz = c.nz; a.nxp = h->nxp; a.plane = h->plane;
    a.nbl = c.nbl;
    a.cpml = c.boundary == MMOD_BOUNDARY_CPML;
    a.fs = c.free_surface ? 1 : 0;
    std::memcpy(a.w, h->w, sizeof(a.w));
    a.p = h->p;
    for (int ax = 0; ax < 3; ++ax) {
        a.v[ax] = h->v[ax];
        a.eg[ax] = h->eg[ax]; a.eh[ax] = h->eh[ax];
        a.psi[ax] = h->psi[ax]; a.phi[ax] = h->phi[ax];
        a.Bg[ax] = h->Bg[ax]; a.Gg[ax] = h->Gg[ax]; a.Bh[ax] = h->Bh[ax]; a.Gh[ax] = h->Gh[ax];
    }
    a.kd = h->kd;
    a.bd = h->bd;
    a.err = h->err_dev;
    a.nrec = c.nrec;
    a.rec_off = h->rec_off;
    return a;
}

bool vd_use_tma(const mmod_vd *h) { return h->tma_ok && h->kernel != MMOD_KERNEL_SIMPLE; }

// One time step: velocity, pressure, injection.  traces_prev: row n-1 for
// the receivers of p^n (null: none).
cudaError_t enqueue_vd_step(mmod_vd *h, int n, const float *wav, float *traces_prev, cudaStream_t s, long long *cnt) {
    VdArgs a = vd_args(h);
    a.traces = traces_prev;
    // the pressure kernel adds the sources when the TMA path runs and the
    // source list is short (each CTA scans it); else the injection kernel
    const bool fold = vd_use_tma(h) && h->ngrp > 0 && h->ngrp <= kFoldSources;
    if (fold) {
        a.ngrp = h->ngrp;
        a.nt = h->cfg.nt;
        a.n = n;
        a.grp_ijk = h->grp_ijk;
        a.grp_off = h->grp_off;
        a.grp_first = h->grp_first;
        a.src_id = h->src_id;
        a.src_scale = h->src_scale;
        a.wavelet = wav;
    }
    cudaError_t e;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t lc = {};
    lc.stream = s;
    lc.attrs = attr;
    lc.numAttrs = h->pdl ? 1 : 0;
    a.pdl = h->pdl;
    if (vd_use_tma(h)) {
        lc.gridDim = dim3(h->geom.tiles_x * h->geom.tiles_y * h->geom.zchunks);
        lc.blockDim = dim3(NT);
        lc.dynamicSmemBytes = V_SMEM;
        if ((e = cudaLaunchKernelEx(&lc, a.cpml ? vd_velocity_tma<true> : vd_velocity_tma<false>, a, h->maps,
                                    h->geom)) != cudaSuccess)
            return e;
        a.traces = nullptr;
        lc.dynamicSmemBytes = P_SMEM;
        if ((e = cudaLaunchKernelEx(&lc, a.cpml ? vd_pressure_tma<true> : vd_pressure_tma<false>, a, h->maps,
                                    h->geom)) != cudaSuccess)
            return e;
    } else {
        const dim3 blk(32, 8, 1), grd((h->cfg.nx + 31) / 32, (h->cfg.ny + 7) / 8, h->cfg.nz);
        vd_velocity_simple<<<grd, blk, 0, s>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        vd_pressure_simple<<<grd, blk, 0, s>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    *cnt += 2;
    if (h->ngrp > 0 && !fold) {
        lc.gridDim = dim3((h->ngrp + 127) / 128);
        lc.blockDim = dim3(128);
        lc.dynamicSmemBytes = 0;
        lc.numAttrs = (h->pdl && vd_use_tma(h)) ? 1 : 0;
        if ((e = cudaLaunchKernelEx(&lc, vd_inject, h->p, h->ngrp, (const long long *)h->grp_off,
                                    (const int *)h->grp_first, (const int *)h->src_id, (const float *)h->src_scale,
                                    wav, h->cfg.nt, n)) != cudaSuccess)
            return e;
        ++*cnt;
    }
    return cudaSuccess;
}

mmod_status vd_loop(mmod_vd *h, const float *wav, float *tr, cudaStream_t s, long long *launches) {
    const mmod_config &c = h->cfg;
    const int kern = (vd_use_tma(h) ? 1 : 0) + 2 * h->pdl + 4 * h->zlen;
    const void *key[2] = {wav, tr};
    if (!h->exec || std::memcmp(h->gkey, key, sizeof(key)) != 0 || h->gkernel != kern) {
        if (h->exec) cudaGraphExecDestroy(h->exec);
        h->exec = nullptr;
        cudaGraph_t graph = nullptr;
        VD_CK(h, cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
        long long n_l = 0;
        cudaError_t e = cudaEventRecordWithFlags(h->ev0, h->cap, cudaEventRecordExternal);
        for (int n = 0; n < c.nt && e == cudaSuccess; ++n)
            e = enqueue_vd_step(h, n, wav, (tr && n > 0) ? tr + (long long)(n - 1) * c.nrec : nullptr, h->cap, &n_l);
        if (e == cudaSuccess && tr && c.nt > 0) {
            e = launch_gather(h->p, h->rec_off, c.nrec, tr + (long long)(c.nt - 1) * c.nrec, h->cap);
            ++n_l;
        }
        if (e == cudaSuccess) e = cudaEventRecordWithFlags(h->ev1, h->cap, cudaEventRecordExternal);
        cudaError_t e_end = cudaStreamEndCapture(h->cap, &graph);
        if (e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return vd_cuda(h, e, "capturing the time loop");
        }
        if (e_end != cudaSuccess) return vd_cuda(h, e_end, "cudaStreamEndCapture");
        cudaError_t e_inst = cudaGraphInstantiate(&h->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e_inst != cudaSuccess) {
            h->exec = nullptr;
            return vd_cuda(h, e_inst, "cudaGraphInstantiate");
        }
        std::memcpy(h->gkey, key, sizeof(key));
        h->gkernel = kern;
        h->glaunches = n_l;
    }
    VD_CK(h, cudaGraphLaunch(h->exec, s));
    *launches += h->glaunches;
    return MMOD_OK;
}

// Tile decomposition: x-y tiles of 64 x 16, z ranges chosen to minimise
// waves x (planes per range + 7) over two resident CTAs per SM.
VdGeom plan_geom(int nx, int ny, int nz, int sms) {
    VdGeom g{};
    g.tiles_x = (nx + TX - 1) / TX;
    g.tiles_y = (ny + TY - 1) / TY;
    const long long tiles = (long long)g.tiles_x * g.tiles_y, slots = 2LL * std::max(sms, 1);
    long long best = -1;
    for (int zc = 1; zc <= nz; ++zc) {
        const int zlen = (nz + zc - 1) / zc;
        const int zcount = (nz + zlen - 1) / zlen;
        const long long waves = (tiles * zcount + slots - 1) / slots;
        const long long cost = waves * (zlen + 2 * kRadius - 1);
        if (best < 0 || cost < best) {
            best = cost;
            g.zchunks = zcount;
            g.zlen = zlen;
        }
    }
    return g;
}

void vd_free(mmod_vd *h) {
    if (h->exec) cudaGraphExecDestroy(h->exec);
    void *ptrs[] = {h->mem, h->prof, h->grp_off, h->grp_ijk, h->grp_first, h->src_id, h->src_ijk_d, h->src_eps, h->src_scale,
                    h->rec_off, h->maxbits, h->bad, h->st_dense};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (h->err_host) cudaFreeHost(h->err_host);
    if (h->cap) cudaStreamDestroy(h->cap);
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
}

std::string vd_validate(const mmod_config *c, mmod_status *st) {
    *st = MMOD_ERR_ARG;
    if (!c) return "null config";
    if (c->nx < 1 || c->ny < 1 || c->nz < 1) return "grid sizes must be >= 1";
    if ((long long)c->nx * c->ny * c->nz > (1LL << 34)) return "grid too large";
    if (!(c->hx > 0) || !(c->hy > 0) || !(c->hz > 0) || !(c->dt > 0)) return "spacing and dt must be > 0";
    if (c->nt < 0 || c->nbl < 0) return "nt and nbl must be >= 0";
    if (2 * c->nbl > c->nx || 2 * c->nbl > c->ny || 2 * c->nbl > c->nz) return "layers wider than half the grid";
    if (c->nbl > 0 && !(c->damp_R > 0 && c->damp_R < 1)) return "damp_R must be in (0, 1)";
    if (c->nsrc < 0 || c->nrec < 0 || (c->nsrc > 0 && !c->src_ijk) || (c->nrec > 0 && !c->rec_ijk))
        return "bad source / receiver lists";
    for (int s = 0; s < c->nsrc + c->nrec; ++s) {
        const int *q = s < c->nsrc ? c->src_ijk + 3 * s : c->rec_ijk + 3 * (s - c->nsrc);
        if (q[0] < 0 || q[0] >= c->nx || q[1] < 0 || q[1] >= c->ny || q[2] < 0 || q[2] >= c->nz)
            return "source or receiver outside the grid";
    }
    if (c->boundary != MMOD_BOUNDARY_DAMPING && c->boundary != MMOD_BOUNDARY_CPML) return "unknown boundary";
    if (c->boundary == MMOD_BOUNDARY_CPML && !(c->cpml_f0 >= 0.0 && std::isfinite(c->cpml_f0)))
        return "cpml_f0 must be finite and >= 0";
    *st = MMOD_ERR_UNSUPPORTED;
    if (c->order != 8) return "the staggered propagator supports order 8 only";
    *st = MMOD_ERR_ARG;
    if (c->free_surface && c->nz <= kRadius) return "a free surface needs nz >= 5";
    *st = MMOD_OK;
    return "";
}

}  // namespace

MMOD_API mmod_status mmod_vd_create(const mmod_config *cfg, int device, mmod_vd **out) {
    if (!out) return MMOD_ERR_ARG;
    *out = nullptr;
    mmod_status st;
    const std::string msg = vd_validate(cfg, &st);
    if (st != MMOD_OK) {
        set_thread_error(msg.c_str());
        return st;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        set_thread_error("no such CUDA device");
        return MMOD_ERR_ARG;
    }
    DeviceGuard guard(device);
    mmod_vd *h = new (std::nothrow) mmod_vd();
    if (!h) return MMOD_ERR_OOM;
    h->cfg = *cfg;
    h->device = device;
    h->src.assign(cfg->src_ijk, cfg->src_ijk + 3 * cfg->nsrc);
    h->rec.assign(cfg->rec_ijk, cfg->rec_ijk + 3 * cfg->nrec);
    h->cfg.src_ijk = h->src.data();
    h->cfg.rec_ijk = h->rec.data();
    const mmod_config &c = h->cfg;
    h->nxp = (c.nx + 31) / 32 * 32;
    h->plane = (long long)h->nxp * c.ny;
    h->vol = h->plane * c.nz;
    h->npts = (long long)c.nx * c.ny * c.nz;
    const double hh[3] = {c.hx, c.hy, c.hz};
    for (int ax = 0; ax < 3; ++ax)
        for (int m = 0; m < kRadius; ++m) h->w[ax][m] = (float)(kStag8[m] / hh[ax]);
    const bool cpml = c.boundary == MMOD_BOUNDARY_CPML;
    const int nvol = cpml ? 12 : 6;
    auto bail = [&](mmod_status s, const char *m, cudaError_t e) {
        std::string full = m;
        if (e != cudaSuccess) full += std::string(": ") + cudaGetErrorString(e);
        set_thread_error(full.c_str());
        cudaGetLastError();
        vd_free(h);
        delete h;
        return s;
    };
#define VD_CREATE(call, what)                                                                            \
    do {                                                                                                 \
        cudaError_t _e = (call);                                                                         \
        if (_e != cudaSuccess)                                                                           \
            return bail(_e == cudaErrorMemoryAllocation ? MMOD_ERR_OOM : MMOD_ERR_CUDA, what, _e);       \
    } while (0)
    VD_CREATE(cudaMalloc(&h->mem, sizeof(float) * (size_t)h->vol * nvol), "wavefield volumes");
    VD_CREATE(cudaMemset(h->mem, 0, sizeof(float) * (size_t)h->vol * nvol), "clearing the volumes");
    h->p = h->mem;
    for (int ax = 0; ax < 3; ++ax) h->v[ax] = h->mem + (size_t)(1 + ax) * h->vol;
    h->kd = h->mem + 4 * (size_t)h->vol;
    h->bd = h->mem + 5 * (size_t)h->vol;
    if (cpml)
        for (int ax = 0; ax < 3; ++ax) {
            h->psi[ax] = h->mem + (size_t)(6 + ax) * h->vol;
            h->phi[ax] = h->mem + (size_t)(9 + ax) * h->vol;
        }
    const int n3[3] = {c.nx, c.ny, c.nz};
    const size_t nsum = (size_t)c.nx + c.ny + c.nz;
    VD_CREATE(cudaMalloc(&h->prof, sizeof(float) * 6 * nsum), "profiles");
    VD_CREATE(cudaMemset(h->prof, 0, sizeof(float) * 6 * nsum), "profiles");
    size_t off = 0;
    for (int ax = 0; ax < 3; ++ax) {
        h->eg[ax] = h->prof + off;
        h->eh[ax] = h->prof + nsum + off;
        h->Bg[ax] = h->prof + 2 * nsum + off;
        h->Gg[ax] = h->prof + 3 * nsum + off;
        h->Bh[ax] = h->prof + 4 * nsum + off;
        h->Gh[ax] = h->prof + 5 * nsum + off;
        off += n3[ax];
    }
    // sources grouped by point (first-occurrence order), receivers
    if (c.nsrc > 0) {
        std::vector<long long> goff;
        std::vector<int> gfirst, sid;
        std::vector<std::vector<int>> members;
        for (int s = 0; s < c.nsrc; ++s) {
            const int *q = &h->src[3 * s];
            const long long o = (long long)q[2] * h->plane + (long long)q[1] * h->nxp + q[0];
            size_t g = 0;
            while (g < goff.size() && goff[g] != o) ++g;
            if (g == goff.size()) {
                goff.push_back(o);
                members.emplace_back();
            }
            members[g].push_back(s);
        }
        gfirst.push_back(0);
        for (auto &m : members) {
            sid.insert(sid.end(), m.begin(), m.end());
            gfirst.push_back((int)sid.size());
        }
        h->ngrp = (int)goff.size();
        std::vector<int> gijk;
        for (auto &m : members) gijk.insert(gijk.end(), &h->src[3 * m[0]], &h->src[3 * m[0]] + 3);
        VD_CREATE(cudaMalloc(&h->grp_ijk, sizeof(int) * gijk.size()), "source table");
        VD_CREATE(cudaMemcpy(h->grp_ijk, gijk.data(), sizeof(int) * gijk.size(), cudaMemcpyHostToDevice),
                  "source table");
        VD_CREATE(cudaMalloc(&h->grp_off, sizeof(long long) * goff.size()), "source table");
        VD_CREATE(cudaMalloc(&h->grp_first, sizeof(int) * gfirst.size()), "source table");
        VD_CREATE(cudaMalloc(&h->src_id, sizeof(int) * sid.size()), "source table");
        VD_CREATE(cudaMalloc(&h->src_ijk_d, sizeof(int) * 3 * c.nsrc), "source table");
        VD_CREATE(cudaMalloc(&h->src_eps, sizeof(double) * c.nsrc), "source table");
        VD_CREATE(cudaMalloc(&h->src_scale, sizeof(float) * c.nsrc), "source table");
        VD_CREATE(cudaMemcpy(h->grp_off, goff.data(), sizeof(long long) * goff.size(), cudaMemcpyHostToDevice), "source table");
        VD_CREATE(cudaMemcpy(h->grp_first, gfirst.data(), sizeof(int) * gfirst.size(), cudaMemcpyHostToDevice), "source table");
        VD_CREATE(cudaMemcpy(h->src_id, sid.data(), sizeof(int) * sid.size(), cudaMemcpyHostToDevice), "source table");
        VD_CREATE(cudaMemcpy(h->src_ijk_d, h->src.data(), sizeof(int) * 3 * c.nsrc, cudaMemcpyHostToDevice), "source table");
    }
    if (c.nrec > 0) {
        std::vector<long long> ro(c.nrec);
        for (int r = 0; r < c.nrec; ++r)
            ro[r] = (long long)h->rec[3 * r + 2] * h->plane + (long long)h->rec[3 * r + 1] * h->nxp + h->rec[3 * r];
        VD_CREATE(cudaMalloc(&h->rec_off, sizeof(long long) * c.nrec), "receiver table");
        VD_CREATE(cudaMemcpy(h->rec_off, ro.data(), sizeof(long long) * c.nrec, cudaMemcpyHostToDevice), "receiver table");
    }
    VD_CREATE(cudaMalloc(&h->maxbits, sizeof(unsigned int) * 2), "scan words");
    VD_CREATE(cudaMalloc(&h->bad, sizeof(unsigned long long)), "scan words");
    VD_CREATE(cudaHostAlloc(&h->err_host, sizeof(int), cudaHostAllocMapped), "error word");
    *h->err_host = 0;
    VD_CREATE(cudaHostGetDevicePointer(&h->err_dev, h->err_host, 0), "error word");
    VD_CREATE(cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking), "capture stream");
    VD_CREATE(cudaEventCreate(&h->ev0), "events");
    VD_CREATE(cudaEventCreate(&h->ev1), "events");
    // TMA plan: tensor maps of every operand, two CTAs per SM
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    h->geom = plan_geom(c.nx, c.ny, c.nz, sms);
    h->geom_plan = h->geom;
    bool ok = true;
    for (const void *f : {(const void *)vd_velocity_tma<false>, (const void *)vd_velocity_tma<true>})
        ok = ok && cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, V_SMEM) == cudaSuccess;
    for (const void *f : {(const void *)vd_pressure_tma<false>, (const void *)vd_pressure_tma<true>})
        ok = ok && cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, P_SMEM) == cudaSuccess;
    ok = ok && encode_box(&h->maps.p_halo, h->p, c.nx, c.ny, c.nz, h->nxp, PHX, PHY);
    for (int ax = 0; ax < 3; ++ax) ok = ok && encode_box(&h->maps.own[ax], h->v[ax], c.nx, c.ny, c.nz, h->nxp, TX, TY);
    ok = ok && encode_box(&h->maps.b_box, h->bd, c.nx, c.ny, c.nz, h->nxp, BX, BY);
    ok = ok && encode_box(&h->maps.vx_halo, h->v[0], c.nx, c.ny, c.nz, h->nxp, PHX, TY);
    ok = ok && encode_box(&h->maps.vy_halo, h->v[1], c.nx, c.ny, c.nz, h->nxp, TX, PHY);
    ok = ok && encode_box(&h->maps.p_own, h->p, c.nx, c.ny, c.nz, h->nxp, TX, TY);
    ok = ok && encode_box(&h->maps.k_own, h->kd, c.nx, c.ny, c.nz, h->nxp, TX, TY);
    cudaGetLastError();
    h->tma_ok = ok;
#undef VD_CREATE
    *out = h;
    return MMOD_OK;
}

MMOD_API mmod_status mmod_vd_destroy(mmod_vd *h) {
    if (!h) return MMOD_OK;
    {
        DeviceGuard guard(h->device);
        cudaDeviceSynchronize();
        vd_free(h);
    }
    delete h;
    return MMOD_OK;
}

MMOD_API mmod_status mmod_vd_set_model(mmod_vd *h, const float *vel, const float *rho, mmod_stream stream) {
    if (!h) return MMOD_ERR_ARG;
    if (!vel || !rho) return vd_fail(h, MMOD_ERR_ARG, "null model");
    if (!is_device_ptr(vel) || !is_device_ptr(rho)) return vd_fail(h, MMOD_ERR_ARG, "vel and rho must be device pointers");
    if (mmod_status st = vd_latched(h)) return st;
    DeviceGuard guard(h->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const mmod_config &c = h->cfg;
    h->model_set = false;
    VD_CK(h, cudaMemsetAsync(h->maxbits, 0, sizeof(unsigned int) * 2, s));
    VD_CK(h, cudaMemsetAsync(h->bad, 0, sizeof(unsigned long long), s));
    vd_model<<<grid_for(h->npts, 256), 256, 0, s>>>(vel, rho, c.nx, c.ny, c.nz, h->nxp, c.dt, h->kd, h->bd,
                                                    h->maxbits, h->bad);
    VD_CK(h, cudaGetLastError());
    unsigned int bits[2];
    unsigned long long bad = 0;
    VD_CK(h, cudaMemcpyAsync(bits, h->maxbits, sizeof(bits), cudaMemcpyDeviceToHost, s));
    VD_CK(h, cudaMemcpyAsync(&bad, h->bad, sizeof(bad), cudaMemcpyDeviceToHost, s));
    VD_CK(h, cudaStreamSynchronize(s));
    if (bad) return vd_fail(h, MMOD_ERR_ARG, "velocities and densities must be finite and > 0");
    float vmaxf, veff2;
    std::memcpy(&vmaxf, &bits[0], 4);
    std::memcpy(&veff2, &bits[1], 4);
    h->vmax = vmaxf;
    h->veff = std::sqrt((double)veff2);
    // staggered leapfrog: dt veff sqrt(sum_a (2 S / h_a)^2) <= 2, S = sum |a_m|
    const double bound = c.dt * h->veff * kStagSymbol8 *
                         std::sqrt(1.0 / (c.hx * c.hx) + 1.0 / (c.hy * c.hy) + 1.0 / (c.hz * c.hz));
    if (bound > 1.0)
        return vd_fail(h, MMOD_ERR_UNSTABLE, "dt too large for the model (staggered CFL bound)");
    // profiles (host, FP64 -> FP32) and source scales
    const int n3[3] = {c.nx, c.ny, c.nz};
    const double hh[3] = {c.hx, c.hy, c.hz};
    const size_t nsum = (size_t)c.nx + c.ny + c.nz;
    std::vector<float> prof(6 * nsum, 0.0f);
    std::vector<double> epsg[3];
    size_t off = 0;
    for (int ax = 0; ax < 3; ++ax) {
        std::vector<double> eg(n3[ax]), eh(n3[ax]);
        const bool top_free = ax == 2 && c.free_surface;
        axis_profiles(n3[ax], c.nbl, hh[ax], h->vmax, c.damp_R, c.cpml_f0, c.dt, 0, top_free, eg.data(),
                      &prof[2 * nsum + off], &prof[3 * nsum + off]);
        axis_profiles(n3[ax], c.nbl, hh[ax], h->vmax, c.damp_R, c.cpml_f0, c.dt, 1, top_free, eh.data(),
                      &prof[4 * nsum + off], &prof[5 * nsum + off]);
        for (int i = 0; i < n3[ax]; ++i) {
            prof[off + i] = (float)eg[i];
            prof[nsum + off + i] = (float)eh[i];
        }
        epsg[ax] = eg;
        off += n3[ax];
    }
    VD_CK(h, cudaMemcpyAsync(h->prof, prof.data(), sizeof(float) * prof.size(), cudaMemcpyHostToDevice, s));
    if (c.nsrc > 0) {
        std::vector<double> se(c.nsrc, 0.0);
        if (c.boundary != MMOD_BOUNDARY_CPML)
            for (int q = 0; q < c.nsrc; ++q)
                se[q] = epsg[0][h->src[3 * q]] + epsg[1][h->src[3 * q + 1]] + epsg[2][h->src[3 * q + 2]];
        VD_CK(h, cudaMemcpyAsync(h->src_eps, se.data(), sizeof(double) * c.nsrc, cudaMemcpyHostToDevice, s));
        vd_source_scale<<<(c.nsrc + 127) / 128, 128, 0, s>>>(vel, rho, c.nx, c.ny, c.nsrc, h->src_ijk_d, h->src_eps,
                                                             c.dt, c.hx * c.hy * c.hz, h->src_scale);
        VD_CK(h, cudaGetLastError());
        if (c.free_surface)   // sources on the surface plane do nothing
            for (int q = 0; q < c.nsrc; ++q)
                if (h->src[3 * q + 2] == 0) VD_CK(h, cudaMemsetAsync(h->src_scale + q, 0, sizeof(float), s));
    }
    VD_CK(h, cudaStreamSynchronize(s));
    h->model_set = true;
    return MMOD_OK;
}

MMOD_API mmod_status mmod_vd_set_state(mmod_vd *h, const float *state, mmod_stream stream) {
    if (!h) return MMOD_ERR_ARG;
    if (state && !is_device_ptr(state)) return vd_fail(h, MMOD_ERR_ARG, "state must be a device pointer");
    if (mmod_status st = vd_latched(h)) return st;
    DeviceGuard guard(h->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const mmod_config &c = h->cfg;
    float *dst[4] = {h->p, h->v[0], h->v[1], h->v[2]};
    for (int f = 0; f < 4; ++f) {
        if (state) {
            VD_CK(h, launch_pack(state + (size_t)f * h->npts, c.nx, c.ny, c.nz, h->nxp, dst[f], s));
        } else {
            VD_CK(h, cudaMemsetAsync(dst[f], 0, sizeof(float) * (size_t)h->vol, s));
        }
    }
    if (c.free_surface) VD_CK(h, cudaMemsetAsync(h->p, 0, sizeof(float) * (size_t)h->plane, s));   // p = 0 on k = 0
    h->state_pending = true;
    return MMOD_OK;
}

MMOD_API mmod_status mmod_vd_forward(mmod_vd *h, const float *wavelet, float *traces, float *final_state,
                                     mmod_stream stream) {
    if (!h) return MMOD_ERR_ARG;
    if (mmod_status st = vd_latched(h)) return st;
    if (!h->model_set) return vd_fail(h, MMOD_ERR_STATE, "no model: call mmod_vd_set_model first");
    const mmod_config &c = h->cfg;
    if (c.nsrc > 0 && c.nt > 0 && !wavelet) return vd_fail(h, MMOD_ERR_ARG, "null wavelet");
    if (c.nrec > 0 && c.nt > 0 && !traces) return vd_fail(h, MMOD_ERR_ARG, "null traces");
    if ((wavelet && !is_device_ptr(wavelet)) || (traces && !is_device_ptr(traces)) ||
        (final_state && !is_device_ptr(final_state)))
        return vd_fail(h, MMOD_ERR_ARG, "wavelet, traces and final_state must be device pointers");
    DeviceGuard guard(h->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    long long launches = 0;
    if (!h->state_pending) {
        VD_CK(h, cudaMemsetAsync(h->mem, 0, sizeof(float) * 4 * (size_t)h->vol, s));
    }
    h->state_pending = false;
    if (c.boundary == MMOD_BOUNDARY_CPML)
        VD_CK(h, cudaMemsetAsync(h->psi[0], 0, sizeof(float) * 6 * (size_t)h->vol, s));
    if (c.nt > 0) {
        if (mmod_status st = vd_loop(h, wavelet, c.nrec > 0 ? traces : nullptr, s, &launches)) return st;
        h->ran = true;
    }
    if (final_state) {
        const float *src[4] = {h->p, h->v[0], h->v[1], h->v[2]};
        for (int f = 0; f < 4; ++f) {
            VD_CK(h, launch_unpack(src[f], c.nx, c.ny, c.nz, h->nxp, final_state + (size_t)f * h->npts, s));
            ++launches;
        }
    }
    h->last_launches = launches;
    return vd_latched(h);
}

MMOD_API mmod_status mmod_vd_set_kernel(mmod_vd *h, int kernel) {
    if (!h) return MMOD_ERR_ARG;
    if (kernel != MMOD_KERNEL_AUTO && kernel != MMOD_KERNEL_SIMPLE && kernel != MMOD_KERNEL_TMA)
        return vd_fail(h, MMOD_ERR_ARG, "unknown kernel");
    if (kernel == MMOD_KERNEL_TMA && !h->tma_ok) return vd_fail(h, MMOD_ERR_UNSUPPORTED, "no TMA plan for this grid");
    h->kernel = kernel;
    return MMOD_OK;
}

MMOD_API int mmod_vd_uses_tma(const mmod_vd *h) { return h ? (vd_use_tma(h) ? 1 : 0) : -1; }

MMOD_API mmod_status mmod_vd_set_option(mmod_vd *h, int option, int value) {
    if (!h) return MMOD_ERR_ARG;
    if (option == MMOD_OPT_PDL && (value == 0 || value == 1)) {
        h->pdl = value;
        return MMOD_OK;
    }
    if (option == MMOD_OPT_ZLEN && value >= 0) {
        h->zlen = value;
        h->geom = h->geom_plan;
        if (value > 0) {
            h->geom.zlen = std::min(value, h->cfg.nz);
            h->geom.zchunks = (h->cfg.nz + h->geom.zlen - 1) / h->geom.zlen;
        }
        return MMOD_OK;
    }
    return vd_fail(h, MMOD_ERR_ARG, "unknown option or value");
}

MMOD_API float mmod_vd_last_loop_ms(mmod_vd *h) {
    if (!h || !h->ran) return -1.0f;
    DeviceGuard guard(h->device);
    float ms = -1.0f;
    if (cudaEventSynchronize(h->ev1) != cudaSuccess || cudaEventElapsedTime(&ms, h->ev0, h->ev1) != cudaSuccess) {
        cudaGetLastError();
        return -1.0f;
    }
    return ms;
}

MMOD_API long long mmod_vd_last_launch_count(const mmod_vd *h) { return h ? h->last_launches : -1; }

MMOD_API const char *mmod_vd_last_error(const mmod_vd *h) { return h ? h->err.c_str() : mmod_last_error(nullptr); }

MMOD_API mmod_status mmod_vd_get_plan(const mmod_vd *h, int *out6) {
    if (!h || !out6) return MMOD_ERR_ARG;
    out6[0] = h->geom.tiles_x;
    out6[1] = h->geom.tiles_y;
    out6[2] = h->geom.zchunks;
    out6[3] = h->geom.zlen;
    out6[4] = h->geom.tiles_x * h->geom.tiles_y * h->geom.zchunks;
    out6[5] = NT;
    return h->tma_ok ? MMOD_OK : MMOD_ERR_UNSUPPORTED;
}
