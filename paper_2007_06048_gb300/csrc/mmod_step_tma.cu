// TMA-pipelined step kernel for sm_103a: one launch computes u^{n+1} on the
// whole grid (inner region, damping layers, source add) and gathers the
// receivers of the previous step.
//
// Decomposition.  A CTA owns a 64 x TY tile in (x, y) and a range of planes in
// z, and marches down z.  Each thread owns 2 (x) x 4 (y) points.
//
// Data movement.  One elected thread issues cp.async.bulk.tensor loads:
//   * u^n planes with a 4-cell x-y halo, (64+8) x (TY+8) floats, into an
//     NSU-slot ring.  The tensor map's zero fill outside the grid is exactly
//     the u = 0 reading, so no thread tests bounds on loads.
//   * u^{n-1} and c planes, 64 x TY floats each, into an NSC-slot ring.
// Each slot has an mbarrier (transaction count = box bytes).  A slot is
// refilled after the __syncthreads that ends the step that last reads it, so
// up to four planes per ring are in flight while the CTA computes.
//
// Stencil.  x and y neighbours come from the centre plane in shared memory
// (8-byte loads, conflict-free: a warp reads 64 consecutive floats per row);
// z neighbours come from a register queue of 9 planes per point, rotated by
// unrolling the z loop 9 times (no register moves).  The arithmetic per point
// is stencil.cuh's, in the same order as the plain kernel: bit-identical.
//
// Waits are bounded (100 ms of wall-clock time each): a wait that gives up sets
// the mapped error word, the CTA stops at the next block barrier, drains its
// outstanding copies (bounded) and returns; the host reports MMOD_ERR_TIMEOUT.
#include <cstdint>

#include "mmod_internal.h"
#include "tma_plan.h"

namespace mmod {
namespace {

constexpr int TX = 64;                 // tile width: 32 lanes x 2 points
constexpr int RX = 2;                  // points per thread along x
constexpr int RY = 4;                  // points per thread along y
constexpr int HX = TX + 2 * kRadius;   // 72: halo tile width
constexpr int NSU = 8;                 // u^n slots: 5 resident planes + prefetch
constexpr int NSC = 4;                 // u^{n-1}, c slots
constexpr int QN = 2 * kRadius + 1;    // z register queue depth
constexpr unsigned long long kWaitNs = 100000000ull;   // a wait gives up after 100 ms

template <int TY>
struct Shape {
    static constexpr int NWARP = TY / RY;
    static constexpr int NT = NWARP * 32;
    static constexpr int HY = TY + 2 * kRadius;
    static constexpr int CUR = HX * HY;             // floats per u^n slot
    static constexpr int PC = TX * TY;              // floats per u^{n-1} or c slot
    static constexpr int SMEM = (NSU * CUR + NSC * 2 * PC) * 4 + (NSU + NSC) * 8 + 16;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for a phase for at most kWaitNs of wall-clock time (try_wait suspends
// the thread in hardware between polls).  The slow path gives up at once if
// another CTA already reported a failure.  On give-up it records the failure
// and returns false.
__device__ __noinline__ bool mbar_wait_slow(uint64_t *bar, uint32_t parity, int *abort_flag, int *err) {
    const unsigned long long t0 = global_ns();
    while (!(err && *(volatile int *)err) && global_ns() - t0 < kWaitNs)
        if (mbar_try_wait(bar, parity)) return true;
    *abort_flag = 1;
    if (err) atomicExch(err, 1);
    return false;
}

__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int *abort_flag, int *err) {
    if (mbar_try_wait(bar, parity)) return true;
    return mbar_wait_slow(bar, parity, abort_flag, err);
}

// Bounded drain wait used after a give-up: no error reporting.
__device__ __noinline__ void mbar_drain(uint64_t *bar, uint32_t parity) {
    const unsigned long long t0 = global_ns();
    while (global_ns() - t0 < kWaitNs)
        if (mbar_try_wait(bar, parity)) return;
}

__device__ __forceinline__ void tma_load_3d(float *dst, const CUtensorMap *map, int x, int y, int z,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

struct Geom {
    int tiles_x, tiles_y, zchunks, zlen;
};

template <int TY>
struct Ctx {
    using S = Shape<TY>;
    float *cur;          // NSU u^n slots
    float *up;           // NSC u^{n-1} slots
    float *cc;           // NSC c slots
    uint64_t *full_u;    // NSU barriers
    uint64_t *full_c;    // NSC barriers
    int *abort_flag;
    int x0, y0, z0, T;
    int lane, warp;
};

template <int TY>
__device__ __forceinline__ void issue_u(const Ctx<TY> &c, const CUtensorMap *map, int seq) {
    const int s = seq % NSU;
    mbar_expect_tx(&c.full_u[s], Shape<TY>::CUR * 4);
    tma_load_3d(c.cur + s * Shape<TY>::CUR, map, c.x0 - kRadius, c.y0 - kRadius, c.z0 - kRadius + seq,
                &c.full_u[s]);
}

template <int TY>
__device__ __forceinline__ void issue_c(const Ctx<TY> &c, const CUtensorMap *pmap, const CUtensorMap *cmap,
                                        int t) {
    const int s = t % NSC;
    mbar_expect_tx(&c.full_c[s], 2 * Shape<TY>::PC * 4);
    tma_load_3d(c.up + s * Shape<TY>::PC, pmap, c.x0, c.y0, c.z0 + t, &c.full_c[s]);
    tma_load_3d(c.cc + s * Shape<TY>::PC, cmap, c.x0, c.y0, c.z0 + t, &c.full_c[s]);
}

// Own points of plane seq (rows 4+4w+r, columns 4+2*lane) into queue slot Q.
template <int TY, int Q>
__device__ __forceinline__ void read_own(const Ctx<TY> &c, int seq, float2 (&q)[QN][RY]) {
    const float *base = c.cur + (seq % NSU) * Shape<TY>::CUR + (kRadius + RY * c.warp) * HX + kRadius + 2 * c.lane;
#pragma unroll
    for (int r = 0; r < RY; ++r) q[Q][r] = *reinterpret_cast<const float2 *>(base + r * HX);
}

__device__ __forceinline__ float2 neg2(float2 v) { return make_float2(-v.x, -v.y); }
__device__ __forceinline__ float2 bcast(float v) { return make_float2(v, v); }

// Packed pair_acc: per component exactly stencil.cuh's pair_acc.
__device__ __forceinline__ float2 pair_acc2(float2 acc, float2 w, float2 a, float2 b, float2 neg_two_p) {
    return __ffma2_rn(w, __fadd2_rn(__fadd2_rn(a, b), neg_two_p), acc);
}

// Sources of plane k that fall on this thread's points (rare: one plane per
// source).  Each thread re-reads the value it has just stored, so program
// order makes it visible; the term is scaled by the point's damping factor.
__device__ __noinline__ void add_plane_sources(const StepArgs &a, int k, int s_lo, int s_hi, int x, int y0,
                                               float2 exr, const float (&eyr)[RY], float ez) {
    for (int s = s_lo; s < s_hi; ++s) {
        const int si = __ldg(a.src_i + s), sj = __ldg(a.src_j + s);
        const int r = sj - y0;
        if ((si != x && si != x + 1) || r < 0 || r >= RY) continue;
        const float ex = si == x ? exr.x : exr.y;
        float ey = eyr[0];
#pragma unroll
        for (int i = 1; i < RY; ++i)
            if (r == i) ey = eyr[i];
        const float e = __fadd_rn(__fadd_rn(ex, ey), ez);
        float *dst = a.uprev + (long long)k * a.plane + (long long)sj * a.nxp + si;
        const float wv = __ldg(a.wavelet + (long long)__ldg(a.src_row + s) * a.nt + a.n);
        *dst = add_source(*dst, __ldg(a.src_scale + s), wv, damp_factor(e));
    }
}

struct Wts {
    float2 x2, x4, y[kRadius], z[kRadius];   // broadcast pairs of w_am
    float x1, x3;
};

// One z step computing plane z0 + t.  R is the queue rotation (0 when the
// queue is shifted after every step instead).
template <int TY, int R>
__device__ __forceinline__ void step(const StepArgs &a, const Ctx<TY> &c, int t, float2 (&q)[QN][RY],
                                     const Wts &w, float2 exr, const float (&eyr)[RY], bool xy_damped) {
    using S = Shape<TY>;
    const int k = c.z0 + t;
    // 1. the leading plane k+4 (sequence t+8) enters the queue
    {
        const int seq = t + 2 * kRadius;
        if (!mbar_wait(&c.full_u[seq % NSU], (seq / NSU) & 1, c.abort_flag, a.err)) return;
        read_own<TY, (2 * kRadius + R) % QN>(c, seq, q);
    }
    if (!mbar_wait(&c.full_c[t % NSC], (t / NSC) & 1, c.abort_flag, a.err)) return;

    // 2. y neighbour columns: rows 4w .. 4w+11 of the centre plane (sequence t+4)
    const float *ctr = c.cur + ((t + kRadius) % NSU) * S::CUR;
    float2 yc[RY + 2 * kRadius];
#pragma unroll
    for (int rr = 0; rr < RY + 2 * kRadius; ++rr)
        yc[rr] = *reinterpret_cast<const float2 *>(ctr + (RY * c.warp + rr) * HX + kRadius + 2 * c.lane);
    const float *upp = c.up + (t % NSC) * S::PC + (RY * c.warp) * TX + 2 * c.lane;
    const float *ccp = c.cc + (t % NSC) * S::PC + (RY * c.warp) * TX + 2 * c.lane;
    const bool damped = xy_damped || k < a.nbl || k > a.nz - 1 - a.nbl;
    const float ez = __ldg(a.ez + k);   // e is exactly 0 on planes without damping
    const int x = c.x0 + 2 * c.lane;
#pragma unroll
    for (int r = 0; r < RY; ++r) {
        // x neighbours: columns 2*lane .. 2*lane+9 of row 4+4w+r, as 5 aligned pairs
        float2 xa[(RX + 2 * kRadius) / 2];
        const float *row = ctr + (kRadius + RY * c.warp + r) * HX + 2 * c.lane;
#pragma unroll
        for (int j = 0; j < (RX + 2 * kRadius) / 2; ++j) xa[j] = *reinterpret_cast<const float2 *>(row + 2 * j);
        const float2 p = q[(kRadius + R) % QN][r];
        const float2 two_p = __fadd2_rn(p, p);
        const float2 ntp = neg2(two_p);
        float2 lap = make_float2(0.0f, 0.0f);
        // x, m = 1 (odd offsets do not form aligned pairs: scalar)
        lap.x = pair_acc(lap.x, w.x1, xa[2].y, xa[1].y, two_p.x);
        lap.y = pair_acc(lap.y, w.x1, xa[3].x, xa[2].x, two_p.y);
        lap = pair_acc2(lap, w.x2, xa[3], xa[1], ntp);
        lap.x = pair_acc(lap.x, w.x3, xa[3].y, xa[0].y, two_p.x);
        lap.y = pair_acc(lap.y, w.x3, xa[4].x, xa[1].x, two_p.y);
        lap = pair_acc2(lap, w.x4, xa[4], xa[0], ntp);
#pragma unroll
        for (int m = 1; m <= kRadius; ++m) lap = pair_acc2(lap, w.y[m - 1], yc[kRadius + r + m], yc[kRadius + r - m], ntp);
#pragma unroll
        for (int m = 1; m <= kRadius; ++m)
            lap = pair_acc2(lap, w.z[m - 1], q[(kRadius + m + R) % QN][r], q[(kRadius - m + R) % QN][r], ntp);
        const float2 pp = *reinterpret_cast<const float2 *>(upp + r * TX);
        const float2 cc = *reinterpret_cast<const float2 *>(ccp + r * TX);
        // e = (e_x + e_y) + e_z; zero on planes without damping
        const float2 e = __fadd2_rn(__fadd2_rn(exr, bcast(eyr[r])), bcast(ez));
        float2 num = __ffma2_rn(cc, lap, __ffma2_rn(e, pp, __fadd2_rn(two_p, neg2(pp))));
        if (damped) num = __fmul2_rn(num, make_float2(damp_factor(e.x), damp_factor(e.y)));
        // 3. store u^{n+1} over u^{n-1}
        const int y = c.y0 + RY * c.warp + r;
        if (y < a.ny && x < a.nx) {
            float *dst = a.uprev + (long long)k * a.plane + (long long)y * a.nxp + x;
            if (x + 1 < a.nx)
                *reinterpret_cast<float2 *>(dst) = num;
            else
                dst[0] = num.x;
        }
    }
    const int s_lo = __ldg(a.src_kstart + k), s_hi = __ldg(a.src_kstart + k + 1);
    if (s_lo < s_hi) add_plane_sources(a, k, s_lo, s_hi, x, c.y0 + RY * c.warp, exr, eyr, ez);
}

template <int TY, bool ROT>
__global__ void __launch_bounds__(Shape<TY>::NT, 2)
    step_tma_kernel(const StepArgs a, const __grid_constant__ CUtensorMap cur_map,
                    const __grid_constant__ CUtensorMap prev_map, const __grid_constant__ CUtensorMap c_map,
                    const Geom g) {
    using S = Shape<TY>;
    extern __shared__ __align__(128) unsigned char smem[];
    Ctx<TY> c;
    c.cur = reinterpret_cast<float *>(smem);
    c.up = c.cur + NSU * S::CUR;
    c.cc = c.up + NSC * S::PC;
    c.full_u = reinterpret_cast<uint64_t *>(c.cc + NSC * S::PC);
    c.full_c = c.full_u + NSU;
    c.abort_flag = reinterpret_cast<int *>(c.full_c + NSC);
    const int tid = threadIdx.x;
    c.lane = tid & 31;
    c.warp = tid >> 5;
    int b = blockIdx.x;
    const int tx = b % g.tiles_x;
    b /= g.tiles_x;
    const int ty = b % g.tiles_y;
    const int chunk = b / g.tiles_y;
    c.x0 = tx * TX;
    c.y0 = ty * TY;
    c.z0 = chunk * g.zlen;
    c.T = min(a.nz - c.z0, g.zlen);
    const int T = c.T;
    const int nseq = T + 2 * kRadius;   // u^n planes z0-4 .. z0+T+3

    if (tid == 0) {
        for (int s = 0; s < NSU; ++s) mbar_init(&c.full_u[s], 1);
        for (int s = 0; s < NSC; ++s) mbar_init(&c.full_c[s], 1);
        *c.abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0 && T > 0) {
        for (int seq = 0; seq < NSU && seq < nseq; ++seq) issue_u(c, &cur_map, seq);
        for (int t = 0; t < NSC && t < T; ++t) issue_c(c, &prev_map, &c_map, t);
    }
    // receivers of the previous step (u^n, read-only during this launch)
    if (a.traces) {
        for (int r = blockIdx.x * S::NT + tid; r < a.nrec; r += gridDim.x * S::NT)
            a.traces[r] = a.ucur[__ldg(a.rec_off + r)];
    }
    if (T <= 0) return;

    Wts w;
    w.x1 = a.w.x[0];
    w.x2 = bcast(a.w.x[1]);
    w.x3 = a.w.x[2];
    w.x4 = bcast(a.w.x[3]);
#pragma unroll
    for (int m = 0; m < kRadius; ++m) {
        w.y[m] = bcast(a.w.y[m]);
        w.z[m] = bcast(a.w.z[m]);
    }
    float2 exr;
    {
        const int x = c.x0 + 2 * c.lane;
        exr.x = x < a.nx ? __ldg(a.ex + x) : 0.0f;
        exr.y = x + 1 < a.nx ? __ldg(a.ex + x + 1) : 0.0f;
    }
    float eyr[RY];
#pragma unroll
    for (int r = 0; r < RY; ++r) {
        const int y = c.y0 + RY * c.warp + r;
        eyr[r] = y < a.ny ? __ldg(a.ey + y) : 0.0f;
    }
    const bool xy_damped = c.x0 < a.nbl || c.x0 + TX - 1 > a.nx - 1 - a.nbl || c.y0 < a.nbl ||
                           c.y0 + TY - 1 > a.ny - 1 - a.nbl;

    float2 q[QN][RY];
    // Issue order of u^n sequences is 0, 1, 2, ... with no gaps: the prologue
    // issues 0..NSU-1, the fill below 4 more, then one per finished step.
    int u_hi = min(NSU, nseq);
    int c_hi = min(NSC, T);
    // planes z0-4 .. z0+3 (sequences 0..7) fill queue slots 0..7
    bool filled = true;
#pragma unroll 1
    for (int seq = 0; seq < 2 * kRadius; ++seq)
        filled = filled && mbar_wait(&c.full_u[seq % NSU], (seq / NSU) & 1, c.abort_flag, a.err);
    if (filled) {
        read_own<TY, 0>(c, 0, q); read_own<TY, 1>(c, 1, q); read_own<TY, 2>(c, 2, q); read_own<TY, 3>(c, 3, q);
        read_own<TY, 4>(c, 4, q); read_own<TY, 5>(c, 5, q); read_own<TY, 6>(c, 6, q); read_own<TY, 7>(c, 7, q);
    }
    __syncthreads();
    // sequences 0..3 are only needed in registers: their slots take NSU..NSU+3
    if (!*c.abort_flag) {
        if (tid == 0)
            for (int seq = u_hi; seq < NSU + kRadius && seq < nseq; ++seq) issue_u(c, &cur_map, seq);
        u_hi = min(NSU + kRadius, nseq);
        // end of step t: every thread is done with u^n sequence t+4 (the centre)
        // and with u^{n-1}/c slot t, so both slots are refilled
#define MMOD_RELEASE(t)                                                                    \
    __syncthreads();                                                                       \
    if (*c.abort_flag) break;                                                              \
    if (tid == 0) {                                                                        \
        if ((t) + kRadius + NSU < nseq) issue_u(c, &cur_map, (t) + kRadius + NSU);         \
        if ((t) + NSC < T) issue_c(c, &prev_map, &c_map, (t) + NSC);                       \
    }                                                                                      \
    u_hi = min((t) + kRadius + NSU + 1, nseq);                                             \
    c_hi = min((t) + NSC + 1, T);
        if constexpr (ROT) {
            // queue rotated by unrolling 9 steps: no register moves, larger code
#define MMOD_STEP(R)                                                   \
    if (t + (R) < T) {                                                 \
        step<TY, (R)>(a, c, t + (R), q, w, exr, eyr, xy_damped);       \
        MMOD_RELEASE(t + (R))                                          \
    }
#pragma unroll 1
            for (int t = 0; t < T; t += QN) {
                MMOD_STEP(0) MMOD_STEP(1) MMOD_STEP(2) MMOD_STEP(3) MMOD_STEP(4)
                MMOD_STEP(5) MMOD_STEP(6) MMOD_STEP(7) MMOD_STEP(8)
            }
#undef MMOD_STEP
        } else {
            // queue shifted by one plane after every step: compact code
#pragma unroll 1
            for (int t = 0; t < T; ++t) {
                step<TY, 0>(a, c, t, q, w, exr, eyr, xy_damped);
#pragma unroll
                for (int i = 0; i < QN - 1; ++i)
#pragma unroll
                    for (int r = 0; r < RY; ++r) q[i][r] = q[i + 1][r];
                MMOD_RELEASE(t)
            }
        }
#undef MMOD_RELEASE
    }
    // After a give-up, wait (bounded) for the copies this CTA still has in
    // flight (the latest sequence of every slot) before its shared memory is
    // released.
    if (*c.abort_flag && tid == 0) {
        for (int seq = max(0, u_hi - NSU); seq < u_hi; ++seq) mbar_drain(&c.full_u[seq % NSU], (seq / NSU) & 1);
        for (int t = max(0, c_hi - NSC); t < c_hi; ++t) mbar_drain(&c.full_c[t % NSC], (t / NSC) & 1);
    }
}

using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder() {
    static EncodeTiled fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

bool encode(CUtensorMap *map, const float *base, const mmod_config &cfg, int nxp, int bx, int by) {
    EncodeTiled fn = encoder();
    if (!fn) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)cfg.nx, (cuuint64_t)cfg.ny, (cuuint64_t)cfg.nz};
    const cuuint64_t strides[2] = {(cuuint64_t)nxp * 4, (cuuint64_t)nxp * cfg.ny * 4};
    const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

constexpr int kTY = 16;

}  // namespace

bool make_tma_plan(const mmod_config &cfg, int nxp, float *const u[2], const float *c, CUtensorMap cur_map[2],
                   CUtensorMap prev_map[2], CUtensorMap *c_map, TmaPlan *plan) {
    using S = Shape<kTY>;
    for (int b = 0; b < 2; ++b) {
        if (!encode(&cur_map[b], u[b], cfg, nxp, HX, S::HY)) return false;
        if (!encode(&prev_map[b], u[b], cfg, nxp, TX, kTY)) return false;
    }
    if (!encode(c_map, c, cfg, nxp, TX, kTY)) return false;
    auto kern = step_tma_kernel<kTY, false>;
    for (auto k : {step_tma_kernel<kTY, false>, step_tma_kernel<kTY, true>}) {
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
    }
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, S::NT, S::SMEM) != cudaSuccess || occ < 1) {
        cudaGetLastError();
        return false;
    }
    const int tiles_x = (cfg.nx + TX - 1) / TX, tiles_y = (cfg.ny + kTY - 1) / kTY;
    const long long tiles = (long long)tiles_x * tiles_y;
    const long long slots = (long long)sms * occ;
    // pick the z split that minimises (waves) x (planes per CTA + halo cost)
    int best_c = 1;
    double best = 1e300;
    for (int zc = 1; zc <= cfg.nz; ++zc) {
        const int zlen = (cfg.nz + zc - 1) / zc;
        const int used = (cfg.nz + zlen - 1) / zlen;
        if (used != zc) continue;
        const long long ctas = tiles * zc;
        if (ctas > (1LL << 31) - 1) break;
        const double waves = (double)((ctas + slots - 1) / slots);
        const double cost = waves * (zlen + 2.0);
        if (cost < best - 1e-9) {
            best = cost;
            best_c = zc;
        }
    }
    plan->tiles_x = tiles_x;
    plan->tiles_y = tiles_y;
    plan->zchunks = best_c;
    plan->zlen = (cfg.nz + best_c - 1) / best_c;
    plan->grid = (int)(tiles * best_c);
    plan->smem = S::SMEM;
    plan->rotate = false;
    return true;
}

cudaError_t launch_step_tma(const StepArgs &a, const CUtensorMap *cur_map, const CUtensorMap *prev_map,
                            const CUtensorMap *c_map, const TmaPlan &plan, bool rotate, cudaStream_t s) {
    using S = Shape<kTY>;
    const Geom g{plan.tiles_x, plan.tiles_y, plan.zchunks, plan.zlen};
    if (plan.rotate || rotate)
        step_tma_kernel<kTY, true><<<plan.grid, S::NT, plan.smem, s>>>(a, *cur_map, *prev_map, *c_map, g);
    else
        step_tma_kernel<kTY, false><<<plan.grid, S::NT, plan.smem, s>>>(a, *cur_map, *prev_map, *c_map, g);
    return cudaGetLastError();
}

}  // namespace mmod
