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
// Each step runs the usual step kernel without damping (u^{n+1} = 2u^n -
// u^{n-1} + c L u^n + sources) and then one layer kernel over the six layer
// slabs only, which adds c sum_a (D1_a psi_a^n + zeta_a^n) to u^{n+1}.  The
// layer kernel needs psi_a^n at the eight neighbours along a; it recomputes
// them from a 17-point line of u^n and psi_a^{n-1} (every thread performs the
// same operations for a given cell, so the recomputed values equal the one
// the cell's own thread stores), which removes a separate psi pass.  psi is
// ping-ponged: step n reads psi[n & 1] and writes psi[(n + 1) & 1].  u and psi
// are 0 outside the grid; with a free surface the top layer is absent and the
// plane k = 0 is left alone (u, psi and zeta stay 0 there).
#include "mmod_cpml.h"
#include "mmod_internal.h"

namespace mmod {
namespace {

constexpr int kLine = 4 * kRadius + 1;   // u^n from -8 to +8 along the axis

// First-difference weights (unit spacing): 4/5, -1/5, 4/105, -1/280.
__device__ __forceinline__ float d1_at(const float *x, int c, float inv_h) {
    constexpr float w[4] = {4.0f / 5.0f, -1.0f / 5.0f, 4.0f / 105.0f, -1.0f / 280.0f};
    float s = 0.0f;
#pragma unroll
    for (int m = 1; m <= kRadius; ++m) s = __fmaf_rn(w[m - 1], __fsub_rn(x[c + m], x[c - m]), s);
    return __fmul_rn(s, inv_h);
}

struct Box {
    int x0, y0, z0, ex, ey, ez, tx, ty;
    int first;   // first block of this box
};
struct Boxes {
    Box b[6];
    int n;
    long long blocks;
};

constexpr int kBX = 32, kBY = 4;

// The layer terms of axis A at cell (idx, o): psi^n at the nine cells along A
// recomputed from u^n (-8..8) and psi^{n-1} (-4..4), the own psi^n stored,
// zeta advanced; returns D1 psi^n + zeta^n.  Lines that stay inside the grid
// take unchecked loads.
template <int A>
__device__ __forceinline__ float axis_term(const CpmlArgs &p, const float *__restrict__ u, const float *psi_old,
                                           float *psi_new, float *zeta, int q0, int n, long long o, long long st,
                                           float g0) {
    float x[kLine], po[2 * kRadius + 1], bb[2 * kRadius + 1], gg[2 * kRadius + 1];
    const float *bA = p.b[A], *gA = p.g[A];
    if (q0 >= 2 * kRadius && q0 + 2 * kRadius < n) {
        const float *up = u + o - 2 * kRadius * st;
#pragma unroll
        for (int m = 0; m < kLine; ++m) x[m] = __ldg(up + m * st);
        const float *pp = psi_old + o - kRadius * st;
#pragma unroll
        for (int m = 0; m <= 2 * kRadius; ++m) {
            po[m] = pp[m * st];
            bb[m] = __ldg(bA + q0 - kRadius + m);
            gg[m] = __ldg(gA + q0 - kRadius + m);
        }
    } else {
#pragma unroll
        for (int m = 0; m < kLine; ++m) {
            const int q = q0 - 2 * kRadius + m;
            x[m] = ((unsigned)q < (unsigned)n) ? __ldg(u + o + (m - 2 * kRadius) * st) : 0.0f;
        }
#pragma unroll
        for (int m = 0; m <= 2 * kRadius; ++m) {
            const int q = q0 - kRadius + m;
            const bool in = (unsigned)q < (unsigned)n;
            po[m] = in ? psi_old[o + (m - kRadius) * st] : 0.0f;
            bb[m] = in ? __ldg(bA + q) : 1.0f;
            gg[m] = in ? __ldg(gA + q) : 0.0f;
        }
    }
    // psi_a^n at the nine cells: b psi^{n-1} + g D1 u^n (0 outside the grid)
    float pn[2 * kRadius + 1];
#pragma unroll
    for (int m = 0; m <= 2 * kRadius; ++m) {
        const int q = q0 - kRadius + m;
        const float d1 = d1_at(x, m + kRadius, p.inv_h[A]);
        pn[m] = ((unsigned)q < (unsigned)n) ? __fmaf_rn(bb[m], po[m], __fmul_rn(gg[m], d1)) : 0.0f;
    }
    psi_new[o] = pn[kRadius];
    const float c2 = x[2 * kRadius];
    const float two_p = __fadd_rn(c2, c2);
    float d2 = pair_first(p.w[A][0], x[2 * kRadius + 1], x[2 * kRadius - 1], two_p);
#pragma unroll
    for (int m = 2; m <= kRadius; ++m) d2 = pair_acc(d2, p.w[A][m - 1], x[2 * kRadius + m], x[2 * kRadius - m], two_p);
    const float dpsi = d1_at(pn, kRadius, p.inv_h[A]);
    const float z = __fmaf_rn(bb[kRadius], zeta[o], __fmul_rn(g0, __fadd_rn(d2, dpsi)));
    zeta[o] = z;
    return __fadd_rn(dpsi, z);
}

__global__ void __launch_bounds__(kBX *kBY)
    cpml_layer_kernel(const CpmlArgs p, const Boxes boxes, const float *__restrict__ u, float *__restrict__ uout,
                      const float *psi_old0, const float *psi_old1, const float *psi_old2, float *psi_new0,
                      float *psi_new1, float *psi_new2) {
    const int blk = blockIdx.x;
    int bi = 0;
    while (bi + 1 < boxes.n && blk >= boxes.b[bi + 1].first) ++bi;
    const Box &B = boxes.b[bi];
    int local = blk - B.first;
    const int tx = local % B.tx;
    local /= B.tx;
    const int ty = local % B.ty;
    const int tz = local / B.ty;
    const int li = tx * kBX + threadIdx.x, lj = ty * kBY + threadIdx.y;
    if (li >= B.ex || lj >= B.ey) return;
    const int i = B.x0 + li, j = B.y0 + lj, k = B.z0 + tz;
    if (p.fs && k == 0) return;   // the free-surface plane stays 0
    const long long o = (long long)k * p.plane + (long long)j * p.nxp + i;
    float acc = 0.0f;
    bool any = false;
    const float gx = __ldg(p.g[0] + i), gy = __ldg(p.g[1] + j), gz = __ldg(p.g[2] + k);
    if (gx != 0.0f) {
        acc = __fadd_rn(acc, axis_term<0>(p, u, psi_old0, psi_new0, p.zeta[0], i, p.nx, o, 1, gx));
        any = true;
    }
    if (gy != 0.0f) {
        acc = __fadd_rn(acc, axis_term<1>(p, u, psi_old1, psi_new1, p.zeta[1], j, p.ny, o, p.nxp, gy));
        any = true;
    }
    if (gz != 0.0f) {
        acc = __fadd_rn(acc, axis_term<2>(p, u, psi_old2, psi_new2, p.zeta[2], k, p.nz, o, p.plane, gz));
        any = true;
    }
    if (any) uout[o] = __fmaf_rn(__ldg(p.c + o), acc, uout[o]);
}

void add_box(Boxes &bx, int x0, int y0, int z0, int ex, int ey, int ez) {
    if (ex <= 0 || ey <= 0 || ez <= 0) return;
    Box &b = bx.b[bx.n++];
    b.x0 = x0; b.y0 = y0; b.z0 = z0; b.ex = ex; b.ey = ey; b.ez = ez;
    b.tx = (ex + kBX - 1) / kBX;
    b.ty = (ey + kBY - 1) / kBY;
    b.first = (int)bx.blocks;
    bx.blocks += (long long)b.tx * b.ty * ez;
}

// The layer cells as six disjoint slabs: z layers (whole planes), y layers
// between them, x layers between those.  With a free surface the top z layer
// is absent and the y and x slabs reach the surface.
Boxes layer_boxes(const CpmlArgs &p) {
    Boxes bx{};
    const int L = p.nbl;
    if (L <= 0) return bx;
    const int zlo = p.fs ? 0 : L, zhi = p.nz - L;
    if (!p.fs) add_box(bx, 0, 0, 0, p.nx, p.ny, L);
    add_box(bx, 0, 0, p.nz - L, p.nx, p.ny, L);
    add_box(bx, 0, 0, zlo, p.nx, L, zhi - zlo);
    add_box(bx, 0, p.ny - L, zlo, p.nx, L, zhi - zlo);
    add_box(bx, 0, L, zlo, L, p.ny - 2 * L, zhi - zlo);
    add_box(bx, p.nx - L, L, zlo, L, p.ny - 2 * L, zhi - zlo);
    return bx;
}

}  // namespace

cudaError_t launch_cpml_layers(const CpmlArgs &p, int n, const float *u, float *uout, cudaStream_t s) {
    const Boxes bx = layer_boxes(p);
    if (bx.blocks == 0) return cudaSuccess;
    if (bx.blocks >= (1LL << 31)) return cudaErrorInvalidConfiguration;
    float *const *po = p.psi[n & 1];
    float *const *pn = p.psi[(n + 1) & 1];
    cpml_layer_kernel<<<(unsigned)bx.blocks, dim3(kBX, kBY, 1), 0, s>>>(p, bx, u, uout, po[0], po[1], po[2], pn[0],
                                                                          pn[1], pn[2]);
    return cudaGetLastError();
}

}  // namespace mmod
