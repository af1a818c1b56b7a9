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
// u^{n-1} + c L u^n + sources), then two passes over the six layer slabs
// only: the psi pass (psi_a^n from u^n, in place) and the correction pass
// (zeta_a^n, and u^{n+1} += c sum_a (D1_a psi_a^n + zeta_a^n)).  One thread
// per layer column over a z range of at most CpmlArgs::zc planes (a block
// takes 128 consecutive columns of one slab); each cell loads its 9-point lines
// before the arithmetic, without bounds tests where the line stays inside
// the grid.  u and psi are 0 outside the grid; with a free surface the top
// layer is absent and the plane k = 0 is left alone (u, psi and zeta stay 0).
#include "mmod_cpml.h"
#include "mmod_internal.h"

namespace mmod {
namespace {

constexpr int kLine = 2 * kRadius + 1;   // -4..4 along the axis

// First-difference weights (unit spacing): 4/5, -1/5, 4/105, -1/280.
__device__ __forceinline__ float d1_of(const float (&x)[kLine], float inv_h) {
    constexpr float w[4] = {4.0f / 5.0f, -1.0f / 5.0f, 4.0f / 105.0f, -1.0f / 280.0f};
    float s = 0.0f;
#pragma unroll
    for (int m = 1; m <= kRadius; ++m) s = __fmaf_rn(w[m - 1], __fsub_rn(x[kRadius + m], x[kRadius - m]), s);
    return __fmul_rn(s, inv_h);
}

// The 9 values of f along an axis (stride st) centred on offset o, index q0
// of n along the axis; 0 outside the grid.
__device__ __forceinline__ void line9(const float *__restrict__ f, long long o, long long st, int q0, int n,
                                      float (&x)[kLine]) {
    if (q0 >= kRadius && q0 + kRadius < n) {
        const float *fp = f + o - kRadius * st;
#pragma unroll
        for (int m = 0; m < kLine; ++m, fp += st) x[m] = __ldg(fp);
    } else {
#pragma unroll
        for (int m = 0; m < kLine; ++m) {
            const int q = q0 - kRadius + m;
            x[m] = ((unsigned)q < (unsigned)n) ? __ldg(f + o + (m - kRadius) * st) : 0.0f;
        }
    }
}

struct Box {
    int x0, y0, z0, ex, ey, ez;
    int ncb;      // blocks over the ex * ey columns of the box
    int zc, tz;   // planes per z range, z ranges
    int first;    // first block of this box
};
struct Boxes {
    Box b[6];
    int n;
    long long blocks;
};

constexpr int kBT = 128;   // a block: 128 consecutive columns of one box (row-major in x, y)

// Column of this thread in the layer slabs and its planes [k0, k1); false
// when outside its box.  Consecutive threads take consecutive columns of the
// box's rows, so a 20-wide x slab fills whole warps (1.6 rows per warp).
__device__ __forceinline__ bool layer_column(const CpmlArgs &p, const Boxes &boxes, int &i, int &j, int &k0,
                                             int &k1) {
    const int blk = blockIdx.x;
    int bi = 0;
    while (bi + 1 < boxes.n && blk >= boxes.b[bi + 1].first) ++bi;
    const Box &B = boxes.b[bi];
    const int local = blk - B.first;
    const int cb = local % B.ncb;
    const int tz = local / B.ncb;
    const int col = cb * kBT + threadIdx.x;
    if (col >= B.ex * B.ey) return false;
    const int lj = col / B.ex;
    i = B.x0 + (col - lj * B.ex);
    j = B.y0 + lj;
    k0 = B.z0 + tz * B.zc;
    k1 = min(k0 + B.zc, B.z0 + B.ez);
    if (p.fs && k0 == 0) k0 = 1;   // the free-surface plane stays 0
    return true;
}

template <int A>
__device__ __forceinline__ void psi_axis(const CpmlArgs &p, const float *__restrict__ u, long long o, long long st,
                                         int q0, int n, float g) {
    float x[kLine];
    line9(u, o, st, q0, n, x);
    float *ps = p.psi[A] + o;
    *ps = __fmaf_rn(__ldg(p.b[A] + q0), *ps, __fmul_rn(g, d1_of(x, p.inv_h[A])));
}

// 16 blocks per SM: 32 registers, full occupancy for the latency-bound line
// gathers (the correction pass would spill at that cap and keeps 40)
__global__ void __launch_bounds__(kBT, 16)
    cpml_psi_kernel(const CpmlArgs p, const Boxes boxes, const float *__restrict__ u) {
    int i, j, k0, k1;
    if (!layer_column(p, boxes, i, j, k0, k1)) return;
    const float gx = __ldg(p.g[0] + i), gy = __ldg(p.g[1] + j);
    long long o = (long long)k0 * p.plane + (long long)j * p.nxp + i;
    for (int k = k0; k < k1; ++k, o += p.plane) {
        const float gz = __ldg(p.g[2] + k);
        if (gx != 0.0f) psi_axis<0>(p, u, o, 1, i, p.nx, gx);
        if (gy != 0.0f) psi_axis<1>(p, u, o, p.nxp, j, p.ny, gy);
        if (gz != 0.0f) psi_axis<2>(p, u, o, p.plane, k, p.nz, gz);
    }
}

// zeta_a^n and the axis's term D1_a psi_a^n + zeta_a^n.
template <int A>
__device__ __forceinline__ float correct_axis(const CpmlArgs &p, const float *__restrict__ u, long long o,
                                              long long st, int q0, int n, float g) {
    float x[kLine], q[kLine];
    line9(u, o, st, q0, n, x);
    line9(p.psi[A], o, st, q0, n, q);
    const float two_p = __fadd_rn(x[kRadius], x[kRadius]);
    float d2 = pair_first(p.w[A][0], x[kRadius + 1], x[kRadius - 1], two_p);
#pragma unroll
    for (int m = 2; m <= kRadius; ++m) d2 = pair_acc(d2, p.w[A][m - 1], x[kRadius + m], x[kRadius - m], two_p);
    const float dpsi = d1_of(q, p.inv_h[A]);
    float *ze = p.zeta[A] + o;
    const float z = __fmaf_rn(__ldg(p.b[A] + q0), *ze, __fmul_rn(g, __fadd_rn(d2, dpsi)));
    *ze = z;
    return __fadd_rn(dpsi, z);
}

__global__ void __launch_bounds__(kBT)
    cpml_correct_kernel(const CpmlArgs p, const Boxes boxes, const float *__restrict__ u, float *__restrict__ uout) {
    int i, j, k0, k1;
    if (!layer_column(p, boxes, i, j, k0, k1)) return;
    const float gx = __ldg(p.g[0] + i), gy = __ldg(p.g[1] + j);
    long long o = (long long)k0 * p.plane + (long long)j * p.nxp + i;
    for (int k = k0; k < k1; ++k, o += p.plane) {
        const float gz = __ldg(p.g[2] + k);
        float acc = 0.0f;
        bool any = false;
        if (gx != 0.0f) {
            acc = __fadd_rn(acc, correct_axis<0>(p, u, o, 1, i, p.nx, gx));
            any = true;
        }
        if (gy != 0.0f) {
            acc = __fadd_rn(acc, correct_axis<1>(p, u, o, p.nxp, j, p.ny, gy));
            any = true;
        }
        if (gz != 0.0f) {
            acc = __fadd_rn(acc, correct_axis<2>(p, u, o, p.plane, k, p.nz, gz));
            any = true;
        }
        if (any) uout[o] = __fmaf_rn(__ldg(p.c + o), acc, uout[o]);
    }
}

void add_box(Boxes &bx, int x0, int y0, int z0, int ex, int ey, int ez, int zc_max) {
    if (ex <= 0 || ey <= 0 || ez <= 0) return;
    Box &b = bx.b[bx.n++];
    b.x0 = x0; b.y0 = y0; b.z0 = z0; b.ex = ex; b.ey = ey; b.ez = ez;
    b.ncb = (int)(((long long)ex * ey + kBT - 1) / kBT);
    b.tz = (ez + zc_max - 1) / zc_max;    // equal ranges of at most zc_max planes
    b.zc = (ez + b.tz - 1) / b.tz;
    b.tz = (ez + b.zc - 1) / b.zc;
    b.first = (int)bx.blocks;
    bx.blocks += (long long)b.ncb * b.tz;
}

// The layer cells as six disjoint slabs: z layers (whole planes), y layers
// between them, x layers between those.  With a free surface the top z layer
// is absent and the y and x slabs reach the surface.
Boxes layer_boxes(const CpmlArgs &p) {
    Boxes bx{};
    const int L = p.nbl;
    if (L <= 0) return bx;
    const int zlo = p.fs ? 0 : L, zhi = p.nz - L, zc = p.zc > 0 ? p.zc : kCpmlPlanes;
    if (!p.fs) add_box(bx, 0, 0, 0, p.nx, p.ny, L, zc);
    add_box(bx, 0, 0, p.nz - L, p.nx, p.ny, L, zc);
    add_box(bx, 0, 0, zlo, p.nx, L, zhi - zlo, zc);
    add_box(bx, 0, p.ny - L, zlo, p.nx, L, zhi - zlo, zc);
    add_box(bx, 0, L, zlo, L, p.ny - 2 * L, zhi - zlo, zc);
    add_box(bx, p.nx - L, L, zlo, L, p.ny - 2 * L, zhi - zlo, zc);
    return bx;
}

}  // namespace

cudaError_t launch_cpml_layers(const CpmlArgs &p, const float *u, float *uout, cudaStream_t s) {
    const Boxes bx = layer_boxes(p);
    if (bx.blocks == 0) return cudaSuccess;
    if (bx.blocks >= (1LL << 31)) return cudaErrorInvalidConfiguration;
    cpml_psi_kernel<<<(unsigned)bx.blocks, kBT, 0, s>>>(p, bx, u);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    cpml_correct_kernel<<<(unsigned)bx.blocks, kBT, 0, s>>>(p, bx, u, uout);
    return cudaGetLastError();
}

}  // namespace mmod
