// TMA-pipelined step kernel for sm_103a: one launch computes u^{n+1} on the
// whole grid (inner region, damping layers, source add) and gathers the
// receivers of the previous step.
//
// Decomposition.  A CTA owns a 64 x TY tile in (x, y) and a range of planes in
// z, and marches down z.  Each thread owns 2 (x) x RY (y) points: lane l holds
// columns x0+2l, x0+2l+1, warp w rows y0+RY*w .. y0+RY*w+RY-1.
//
// Data movement.  One elected thread issues cp.async.bulk.tensor loads:
//   * u^n planes with a 4-cell x-y halo, (64+8) x (TY+8) floats, into an
//     S::NSU-slot ring.  The tensor map's zero fill outside the grid is exactly
//     the u = 0 reading, so no thread tests bounds on loads.
//   * u^{n-1} and c planes, 64 x TY floats each, into an S::NSC-slot ring.
// Each slot has an mbarrier (transaction count = box bytes).  A slot is
// refilled after the block barrier that ends the last step reading it, so
// several planes per ring are in flight while the CTA computes.
//
// Stencil.  x and y neighbours come from the centre plane in shared memory
// (8-byte loads, conflict-free: a warp reads 64 consecutive floats per row);
// z neighbours come from a register queue of 9 planes per point, either
// shifted by one plane after every step (compact code) or rotated by
// unrolling nine steps (no moves).  The two points of a thread share every
// operation, so the arithmetic runs as packed FP32x2 (__ffma2_rn, __fadd2_rn:
// per component the same rounding as the scalar intrinsics), except the x
// offsets 1 and 3 whose operands do not form aligned register pairs.  The
// per-point arithmetic and its order are stencil.cuh's: the result is bit for
// bit the plain kernel's.
//
// Waits are bounded (100 ms of wall-clock time each): a wait that gives up sets
// the mapped error word, the CTA stops at the next block barrier, drains its
// outstanding copies (bounded) and returns; the host reports MMOD_ERR_TIMEOUT.
#include <algorithm>
#include <cstdint>

#include "mmod_internal.h"
#include "tma_plan.h"
#include "tma_ptx.cuh"

namespace mmod {
namespace {

constexpr int TX = 64;                 // tile width: 32 lanes x 2 points
constexpr int HX = TX + 2 * kRadius;   // 72: halo tile width

template <int TY_, int RY_, int U_, int NSU_ = 8, int NSC_ = 4, int MINB_ = 1>
struct Shape {
    static constexpr int MINB = MINB_;              // resident CTAs per SM the registers are capped for
    // the batch and persistent kernels always keep two CTAs per SM resident
    static constexpr int MINB2 = MINB_ > 2 ? MINB_ : 2;
    static constexpr int TY = TY_;
    static constexpr int RY = RY_;
    static constexpr int U = U_;                    // z steps per unrolled block
    static constexpr int NSU = NSU_;                // u^n slots: 5 resident planes + prefetch
    static constexpr int NSC = NSC_;                // u^{n-1}, c slots
    static constexpr int QD = 2 * kRadius + U;      // register queue depth
    static constexpr int NWARP = TY / RY;
    static constexpr int NT = NWARP * 32;
    static constexpr int HY = TY + 2 * kRadius;
    static constexpr int CUR = HX * HY;             // floats per u^n slot
    static constexpr int PC = TX * TY;              // floats per u^{n-1} or c slot
    static constexpr int SMEM = (NSU * CUR + NSC * 2 * PC) * 4 + (NSU + NSC) * 8 + 16;
    static_assert(TY % RY == 0, "rows per thread must divide the tile height");
    static_assert(NSU >= 6 && NSU <= 8 && NSC >= 2, "ring depth outside the fill / release schedule");
};

struct Ctx {
    float *cur;          // S::NSU u^n slots
    float *up;           // S::NSC u^{n-1} slots
    float *cc;           // S::NSC c slots
    uint64_t *full_u;    // S::NSU barriers: data landed
    uint64_t *full_c;    // S::NSC barriers
    int *abort_flag;
    int x0, y0, z0, T;
    int lane, warp;
    bool mirror;         // free surface and z0 < 4: the halo planes above k = 0 are odd images
};

template <class S>
__device__ __forceinline__ void issue_u(const Ctx &c, const CUtensorMap *map, int seq) {
    const int s = seq % S::NSU;
    int z = c.z0 - kRadius + seq;
    if (c.mirror && z < 0) z = -z;   // plane -m is the image of plane m (negated when read)
    mbar_expect_tx(&c.full_u[s], S::CUR * 4);
    tma_load_3d(c.cur + s * S::CUR, map, c.x0 - kRadius, c.y0 - kRadius, z, &c.full_u[s]);
}

template <class S>
__device__ __forceinline__ void issue_c(const Ctx &c, const CUtensorMap *pmap, const CUtensorMap *cmap, int t) {
    const int s = t % S::NSC;
    mbar_expect_tx(&c.full_c[s], 2 * S::PC * 4);
    tma_load_3d(c.up + s * S::PC, pmap, c.x0, c.y0, c.z0 + t, &c.full_c[s]);
    tma_load_3d(c.cc + s * S::PC, cmap, c.x0, c.y0, c.z0 + t, &c.full_c[s]);
}

// Own points of plane seq (rows 4+RY*w+r, columns 4+2*lane) into queue slot Q.
template <class S, int Q>
__device__ __forceinline__ void read_own(const Ctx &c, int seq, float2 (&q)[S::QD][S::RY]) {
    const float *base = c.cur + (seq % S::NSU) * S::CUR + (kRadius + S::RY * c.warp) * HX + kRadius + 2 * c.lane;
#pragma unroll
    for (int r = 0; r < S::RY; ++r) q[Q][r] = *reinterpret_cast<const float2 *>(base + r * HX);
}

__device__ __forceinline__ float2 neg2(float2 v) { return make_float2(-v.x, -v.y); }
__device__ __forceinline__ float2 bcast(float v) { return make_float2(v, v); }

// Packed pair terms: per component exactly stencil.cuh's pair_first / pair_acc.
__device__ __forceinline__ float2 pair_first2(float2 w, float2 a, float2 b, float2 neg_two_p) {
    return __fmul2_rn(w, __fadd2_rn(__fadd2_rn(a, b), neg_two_p));
}

__device__ __forceinline__ float2 pair_acc2(float2 acc, float2 w, float2 a, float2 b, float2 neg_two_p) {
    return __ffma2_rn(w, __fadd2_rn(__fadd2_rn(a, b), neg_two_p), acc);
}

struct Wts {
    float2 x2, x4, y[kRadius], z[kRadius];   // broadcast pairs of w_am
    float x1, x3;
};

// Per-plane values every thread needs, loaded one step ahead.
struct PlaneInfo {
    float ez;        // dt * eta_z(k)
};

__device__ __forceinline__ PlaneInfo plane_info(const StepArgs &a, int k) {
    PlaneInfo p;
    p.ez = __ldg(a.ez + min(k, a.nz - 1));
    return p;
}

// One z step computing plane z0 + t.  The queue window of this step is
// q[J .. J+8] (planes k-4 .. k+4); the leading plane k+4 lands in q[J+8].
template <class S, int J, bool G>
__device__ __forceinline__ void step(const StepArgs &a, const Ctx &c, int t, float2 (&q)[S::QD][S::RY],
                                     const Wts &w, float2 exr, const float (&eyr)[S::RY], bool xy_damped,
                                     const PlaneInfo &pi, float *const (&out_row)[S::RY],
                                     float *const (&g_row)[S::RY]) {
    constexpr int RY = S::RY;
    const int k = c.z0 + t;
    // 1. the leading plane k+4 (sequence t+8) enters the queue
    {
        const int seq = t + 2 * kRadius;
        if (!mbar_wait(&c.full_u[seq % S::NSU], (seq / S::NSU) & 1, c.abort_flag, a.err)) return;
        read_own<S, J + 2 * kRadius>(c, seq, q);
    }
    if (!mbar_wait(&c.full_c[t % S::NSC], (t / S::NSC) & 1, c.abort_flag, a.err)) return;

    // 2. y neighbour columns: rows RY*w .. RY*w+RY+7 of the centre plane (sequence t+4)
    const float *ctr = c.cur + ((t + kRadius) % S::NSU) * S::CUR + (RY * c.warp) * HX + 2 * c.lane;
    float2 yc[RY + 2 * kRadius];
#pragma unroll
    for (int rr = 0; rr < RY + 2 * kRadius; ++rr) yc[rr] = *reinterpret_cast<const float2 *>(ctr + rr * HX + kRadius);
    const float *upp = c.up + (t % S::NSC) * S::PC + (RY * c.warp) * TX + 2 * c.lane;
    const float *ccp = c.cc + (t % S::NSC) * S::PC + (RY * c.warp) * TX + 2 * c.lane;
    const bool damped = xy_damped || k < a.nbl || k > a.nz - 1 - a.nbl;
    const long long koff = (long long)k * a.plane;   // out_row already points into uout
#pragma unroll
    for (int r = 0; r < RY; ++r) {
        // x neighbours: columns 2*lane .. 2*lane+9 of row 4+RY*w+r, as 5 aligned pairs
        float2 xa[1 + kRadius];
        const float *row = ctr + (kRadius + r) * HX;
#pragma unroll
        for (int j = 0; j <= kRadius; ++j) xa[j] = *reinterpret_cast<const float2 *>(row + 2 * j);
        const float2 p = q[J + kRadius][r];
        const float2 two_p = __fadd2_rn(p, p);
        const float2 ntp = neg2(two_p);
        // x: offsets 1 and 3 do not form aligned pairs, so they run scalar
        float2 lx;
        lx.x = pair_first(w.x1, xa[2].y, xa[1].y, two_p.x);
        lx.y = pair_first(w.x1, xa[3].x, xa[2].x, two_p.y);
        lx = pair_acc2(lx, w.x2, xa[3], xa[1], ntp);
        lx.x = pair_acc(lx.x, w.x3, xa[3].y, xa[0].y, two_p.x);
        lx.y = pair_acc(lx.y, w.x3, xa[4].x, xa[1].x, two_p.y);
        lx = pair_acc2(lx, w.x4, xa[4], xa[0], ntp);
        float2 ly = pair_first2(w.y[0], yc[kRadius + r + 1], yc[kRadius + r - 1], ntp);
        float2 lz = pair_first2(w.z[0], q[J + kRadius + 1][r], q[J + kRadius - 1][r], ntp);
#pragma unroll
        for (int m = 2; m <= kRadius; ++m) {
            ly = pair_acc2(ly, w.y[m - 1], yc[kRadius + r + m], yc[kRadius + r - m], ntp);
            lz = pair_acc2(lz, w.z[m - 1], q[J + kRadius + m][r], q[J + kRadius - m][r], ntp);
        }
        const float2 lap = __fadd2_rn(__fadd2_rn(lx, ly), lz);
        const float2 pp = *reinterpret_cast<const float2 *>(upp + r * TX);
        const float2 cc = *reinterpret_cast<const float2 *>(ccp + r * TX);
        // e = (e_x + e_y) + e_z; exactly 0 on planes without damping
        const float2 e = __fadd2_rn(__fadd2_rn(exr, bcast(eyr[r])), bcast(pi.ez));
        float2 num = __ffma2_rn(cc, lap, __ffma2_rn(e, pp, __fadd2_rn(two_p, neg2(pp))));
        if (damped) num = __fmul2_rn(num, make_float2(damp_factor(e.x), damp_factor(e.y)));
        if (a.fs && k == 0) num = make_float2(0.0f, 0.0f);   // p = 0 on a free surface
        // 3. store u^{n+1} over u^{n-1} (out_row is null for rows and columns
        // outside the grid; its x+1 twin is stored only inside the grid)
        if (out_row[r]) {
            float *dst = out_row[r] + koff;
            if (c.x0 + 2 * c.lane + 1 < a.nx)
                *reinterpret_cast<float2 *>(dst) = num;
            else
                dst[0] = num.x;
        }
        if constexpr (G) {   // g^n = L u^n (sources added after the z range), 0 on a free surface
            if (g_row[r]) {
                const float2 gv = (a.fs && k == 0) ? make_float2(0.0f, 0.0f) : lap;
                float *dst = g_row[r] + koff;
                if (c.x0 + 2 * c.lane + 1 < a.nx)
                    *reinterpret_cast<float2 *>(dst) = gv;
                else
                    dst[0] = gv.x;
            }
        }
    }
}

// Per-step values of a launch, kept apart from StepArgs so the persistent
// kernel can take StepArgs from its (constant) parameters: the step, the
// u^{n+1} buffer, and for one-launch-per-step runs the previous step's
// receivers (traces[n-1] = u^n, gathered from ucur; null: none).
struct StepVar {
    int n;
    float *uout;
    const float *ucur;
    float *traces;
};

// What a CTA waits for before it reads u^n and overwrites u^{n-1}.
//
// One launch per step: the previous step's grid, through programmatic
// dependent launch (pdl 1 or 2) or the launch order (pdl 0).  With pdl == 2
// the previous kernel is the previous step, which only reads u^{n-1}, so the
// c and u^{n-1} planes are requested before the wait.
struct PdlDep {
    int pdl;
    static constexpr bool kProxyFence = false;
    __device__ bool early() const { return pdl == 2; }
    __device__ bool reinit() const { return false; }
    __device__ void wait(int, int *, int *) const {
        if (pdl) {
            asm volatile("griddepcontrol.wait;" ::: "memory");
            asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
        }
    }
};

// Persistent run: the 26 neighbouring units (x-y tiles and z ranges, with
// diagonals: the u^n halo box touches all of them) and the unit itself must
// have completed step n-1 (the unit's own u^n and u^{n-1} may have been
// written by another CTA).  One thread polls each counter (acquire, bounded
// by kWaitNs; a give-up sets the abort flag and the error word).  Nothing is
// requested before the wait.  Barriers of an earlier unit are invalidated and
// set up again.
struct NeighborDep {
    const int *counters;
    int unit, n;
    Geom g;
    bool first;
    static constexpr bool kProxyFence = true;
    __device__ bool early() const { return false; }
    __device__ bool reinit() const { return !first; }
    __device__ void wait(int tid, int *abort_flag, int *err) const;
};

__device__ __noinline__ void NeighborDep::wait(int tid, int *abort_flag, int *err) const {
    if (tid >= 27) return;   // 27 units: the unit (13) and its neighbours
    int b = unit;
    const int tx = b % g.tiles_x;
    b /= g.tiles_x;
    const int ty = b % g.tiles_y;
    const int ch = b / g.tiles_y;
    const int vx = tx + tid % 3 - 1, vy = ty + (tid / 3) % 3 - 1, vz = ch + tid / 9 - 1;
    if (vx < 0 || vx >= g.tiles_x || vy < 0 || vy >= g.tiles_y || vz < 0 || vz >= g.zchunks) return;
    const int *cnt = counters + (vz * g.tiles_y + vy) * g.tiles_x + vx;
    if (ld_acquire_gpu(cnt) >= n) return;
    const unsigned long long t0 = global_ns();
    while (ld_acquire_gpu(cnt) < n) {
        if (*(volatile int *)err || global_ns() - t0 >= kWaitNs) {
            *(volatile int *)abort_flag = 1;
            atomicExch(err, 1);
            return;
        }
        __nanosleep(64);
    }
}

// The work of one CTA: block `bid` of the `nbid` blocks of one grid (one
// shot).  The single-shot kernel passes its parameters; the batch kernel a
// shot's arguments staged in shared memory and that shot's tensor maps in
// global memory.
template <class S, class Dep, bool G = false>
__device__ __forceinline__ void step_tma_body(const StepArgs &a, const StepVar &v, const CUtensorMap *cur_map,
                                              const CUtensorMap *prev_map, const CUtensorMap *c_map, const Geom &g,
                                              int bid, int nbid, const Dep &dep) {
    constexpr int RY = S::RY;
    constexpr int U = S::U;
    extern __shared__ __align__(128) unsigned char smem[];
    Ctx c;
    c.cur = reinterpret_cast<float *>(smem);
    c.up = c.cur + S::NSU * S::CUR;
    c.cc = c.up + S::NSC * S::PC;
    c.full_u = reinterpret_cast<uint64_t *>(c.cc + S::NSC * S::PC);
    c.full_c = c.full_u + S::NSU;
    c.abort_flag = reinterpret_cast<int *>(c.full_c + S::NSC);
    const int tid = threadIdx.x;
    c.lane = tid & 31;
    c.warp = tid >> 5;
    int b = bid;
    const int tx = b % g.tiles_x;
    b /= g.tiles_x;
    const int ty = b % g.tiles_y;
    const int chunk = b / g.tiles_y;
    c.x0 = tx * TX;
    c.y0 = ty * S::TY;
    c.z0 = chunk * g.zlen;
    c.T = min(a.nz - c.z0, g.zlen);
    c.mirror = a.fs && c.z0 < kRadius;
    const int T = c.T;
    const int nseq = T + 2 * kRadius;   // u^n planes z0-4 .. z0+T+3

    if (tid == 0) {
        if (dep.reinit()) {   // the previous unit consumed every copy it issued
            for (int s = 0; s < S::NSU; ++s) mbar_inval(&c.full_u[s]);
            for (int s = 0; s < S::NSC; ++s) mbar_inval(&c.full_c[s]);
        }
        for (int s = 0; s < S::NSU; ++s) mbar_init(&c.full_u[s], 1);
        for (int s = 0; s < S::NSC; ++s) mbar_init(&c.full_c[s], 1);
        *c.abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if constexpr (Dep::kProxyFence) __syncthreads();   // the flag is 0 before any waiter may set it
    // c and u^{n-1} first where the dependency allows it (see PdlDep and
    // NeighborDep), then wait, then u^n.
    const bool early = dep.early();
    if (early && tid == 0 && T > 0) {
        if constexpr (Dep::kProxyFence) fence_proxy_async_global();
        for (int t = 0; t < S::NSC && t < T; ++t) issue_c<S>(c, prev_map, c_map, t);
    }
    dep.wait(tid, c.abort_flag, a.err);
    __syncthreads();
    const bool dep_ok = !*c.abort_flag;
    if (tid == 0 && T > 0 && dep_ok) {
        if constexpr (Dep::kProxyFence) fence_proxy_async_global();
        for (int seq = 0; seq < S::NSU && seq < nseq; ++seq) issue_u<S>(c, cur_map, seq);
        if (!early)
            for (int t = 0; t < S::NSC && t < T; ++t) issue_c<S>(c, prev_map, c_map, t);
    }
    // receivers of the previous step (u^n, read-only during this launch)
    if (v.traces) {
        for (int r = bid * S::NT + tid; r < a.nrec; r += nbid * S::NT)
            v.traces[r] = v.ucur[__ldg(a.rec_off + r)];
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
    const int x = c.x0 + 2 * c.lane;
    float2 exr;
    exr.x = x < a.nx ? __ldg(a.ex + x) : 0.0f;
    exr.y = x + 1 < a.nx ? __ldg(a.ex + x + 1) : 0.0f;
    float eyr[RY];
    float *out_row[RY];   // u^{n+1} row pointers at plane 0; null outside the grid
    float *g_row[RY];     // the same rows of g^n (G only)
#pragma unroll
    for (int r = 0; r < RY; ++r) {
        const int y = c.y0 + RY * c.warp + r;
        eyr[r] = y < a.ny ? __ldg(a.ey + y) : 0.0f;
        out_row[r] = (y < a.ny && x < a.nx) ? v.uout + (long long)y * a.nxp + x : nullptr;
        g_row[r] = (G && y < a.ny && x < a.nx) ? a.gout + (long long)y * a.nxp + x : nullptr;
    }
    const bool xy_damped = c.x0 < a.nbl || c.x0 + TX - 1 > a.nx - 1 - a.nbl || c.y0 < a.nbl ||
                           c.y0 + S::TY - 1 > a.ny - 1 - a.nbl;

    float2 q[S::QD][RY];
    // Issue order of u^n sequences is 0, 1, 2, ... with no gaps: the prologue
    // issues 0..S::NSU-1, the fill below 4 more, then one per finished step.
    int u_hi = dep_ok ? min(S::NSU, nseq) : 0;
    int c_hi = (dep_ok || early) ? min(S::NSC, T) : 0;
    // planes z0-4 .. z0+3 (sequences 0..7) fill queue slots 0..7.  Phase A
    // reads what the prologue issued (sequences 0..min(NSU,8)-1); the slots
    // of sequences 0..3 (never a centre) then take NSU..NSU+3; phase B reads
    // sequences NSU..7 when the ring is shallower than 8.
    constexpr int NA = S::NSU < 2 * kRadius ? S::NSU : 2 * kRadius;
    bool filled = true;
#pragma unroll 1
    for (int seq = 0; seq < NA; ++seq)
        filled = filled && mbar_wait(&c.full_u[seq % S::NSU], (seq / S::NSU) & 1, c.abort_flag, a.err);
    if (filled) {
        read_own<S, 0>(c, 0, q); read_own<S, 1>(c, 1, q); read_own<S, 2>(c, 2, q); read_own<S, 3>(c, 3, q);
        read_own<S, 4>(c, 4, q); read_own<S, 5>(c, 5, q);
        if constexpr (NA > 6) read_own<S, 6>(c, 6, q);
        if constexpr (NA > 7) read_own<S, 7>(c, 7, q);
    }
    __syncthreads();
    if (!*c.abort_flag) {
        if (tid == 0)
            for (int seq = u_hi; seq < S::NSU + kRadius && seq < nseq; ++seq) issue_u<S>(c, cur_map, seq);
        u_hi = min(S::NSU + kRadius, nseq);
        if constexpr (NA < 2 * kRadius) {
#pragma unroll 1
            for (int seq = NA; seq < 2 * kRadius; ++seq)
                filled = filled && mbar_wait(&c.full_u[seq % S::NSU], (seq / S::NSU) & 1, c.abort_flag, a.err);
            if (filled) {
                if constexpr (NA <= 6) read_own<S, 6>(c, 6, q);
                read_own<S, 7>(c, 7, q);
            }
        }
        if (c.mirror && filled) {   // queue planes above k = 0 (z0-4+i < 0) hold the images: negate
#pragma unroll
            for (int i = 0; i < kRadius; ++i)
                if (i < kRadius - c.z0) {
#pragma unroll
                    for (int r = 0; r < RY; ++r) q[i][r] = neg2(q[i][r]);
                }
        }
        PlaneInfo pi = plane_info(a, c.z0);
        // Steps run in blocks of U; step J of a block uses queue window
        // q[J .. J+8], and the block ends by moving its last 8 planes down.
        // End of step t: every thread is done with u^n sequence t+4 (the
        // centre) and with u^{n-1}/c slot t, so both slots are refilled.
#define MMOD_STEP(J)                                                                        \
    if (t + (J) < T) {                                                                      \
        const PlaneInfo pi_next = plane_info(a, c.z0 + t + (J) + 1);                        \
        step<S, (J), G>(a, c, t + (J), q, w, exr, eyr, xy_damped, pi, out_row, g_row);     \
        pi = pi_next;                                                                       \
        __syncthreads();                                                                    \
        if (*c.abort_flag) break;                                                           \
        if (tid == 0) {                                                                     \
            if (t + (J) + kRadius + S::NSU < nseq) issue_u<S>(c, cur_map, t + (J) + kRadius + S::NSU); \
            if (t + (J) + S::NSC < T) issue_c<S>(c, prev_map, c_map, t + (J) + S::NSC);        \
        }                                                                                   \
        u_hi = min(t + (J) + kRadius + S::NSU + 1, nseq);                                      \
        c_hi = min(t + (J) + S::NSC + 1, T);                                                   \
    }
#pragma unroll 1
        for (int t = 0; t < T; t += U) {
            MMOD_STEP(0)
            if constexpr (U > 1) { MMOD_STEP(1) }
            if constexpr (U > 2) { MMOD_STEP(2) }
            if constexpr (U > 3) { MMOD_STEP(3) }
#pragma unroll
            for (int i = 0; i < 2 * kRadius; ++i)
#pragma unroll
                for (int r = 0; r < RY; ++r) q[i][r] = q[i + U][r];
        }
#undef MMOD_STEP
    }
    // Sources of this CTA's tile and planes: nothing in this launch reads the
    // u^{n+1} it writes, so they are added once the whole z range is stored
    // (the block barrier makes every thread's stores visible).  The points of
    // one tile over planes [z0, z0 + T) are one run of the table; one thread
    // per injection point.
    __syncthreads();
    if (!*c.abort_flag && a.inj.npts > 0) {
        const long long b = ((long long)(c.y0 / kInjTileY) * a.inj.tiles_x + c.x0 / kInjTileX) * a.nz + c.z0;
        const int lo = __ldg(a.inj.tile_start + b), hi = __ldg(a.inj.tile_start + b + T);
        inject_points(a, v.uout, v.n, lo, hi, tid, S::NT);
        if constexpr (G) inject_g_points(a, v.n, lo, hi, tid, S::NT);
    }
    // After a give-up, wait (bounded) for the copies this CTA still has in
    // flight (the latest sequence of every slot) before its shared memory is
    // released.
    if (*c.abort_flag && tid == 0) {
        for (int seq = max(0, u_hi - S::NSU); seq < u_hi; ++seq) mbar_drain(&c.full_u[seq % S::NSU], (seq / S::NSU) & 1);
        for (int t = max(0, c_hi - S::NSC); t < c_hi; ++t) mbar_drain(&c.full_c[t % S::NSC], (t / S::NSC) & 1);
    }
}

// G: also write g^n = L u^n + s^n into a.gout (the gradient's imaging factor).
template <class S, bool G = false>
__global__ void __launch_bounds__(S::NT, S::MINB)
    step_tma_kernel(const StepArgs a, const __grid_constant__ CUtensorMap cur_map,
                    const __grid_constant__ CUtensorMap prev_map, const __grid_constant__ CUtensorMap c_map,
                    const Geom g) {
    step_tma_body<S, PdlDep, G>(a, StepVar{a.n, a.uout, a.ucur, a.traces}, &cur_map, &prev_map, &c_map, g,
                                blockIdx.x, gridDim.x, PdlDep{a.pdl});
}

// Work-claiming step (StepArgs::claim set): at most one wave of CTAs covers
// the grid's units (64 x TY tile x g.zlen planes).  CTA b serves unit b, then
// claims the next unserved unit from the launch's counter (claim[0]) until
// none is left, so a CTA that finishes early takes more work and every SM
// keeps its CTAs busy until the last units; the units are independent within
// a step (each reads u^n, its own u^{n-1} and c, and writes its own u^{n+1}),
// so the order does not matter and the bits are those of the static plan.
// Only a CTA's first unit waits for the previous step (PDL); later units
// request their planes at once.  The last CTA to stop claiming (claim[1]
// counts them) clears both counters for the next launch, which reads them
// only after its own griddepcontrol.wait or stream order.
struct ClaimDep {
    int pdl;
    bool first;
    static constexpr bool kProxyFence = false;
    __device__ bool early() const { return first ? pdl == 2 : true; }
    __device__ bool reinit() const { return !first; }
    __device__ void wait(int, int *, int *) const {
        if (first && pdl) {
            asm volatile("griddepcontrol.wait;" ::: "memory");
            asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
        }
    }
};

template <class S, bool G = false>
__global__ void __launch_bounds__(S::NT, S::MINB2)
    step_tma_claim_kernel(const StepArgs a, const __grid_constant__ CUtensorMap cur_map,
                          const __grid_constant__ CUtensorMap prev_map, const __grid_constant__ CUtensorMap c_map,
                          const Geom g, int units) {
    extern __shared__ __align__(128) unsigned char smem[];
    // the body's abort flag and, next to it, the claimed unit
    int *abort_flag = reinterpret_cast<int *>(smem + (S::NSU * S::CUR + S::NSC * 2 * S::PC) * 4 +
                                              (S::NSU + S::NSC) * 8);
    int *next = abort_flag + 1;
    bool first = true;
    for (int unit = blockIdx.x; unit < units;) {
        step_tma_body<S, ClaimDep, G>(a, StepVar{a.n, a.uout, a.ucur, a.traces}, &cur_map, &prev_map, &c_map, g,
                                      unit, units, ClaimDep{a.pdl, first});
        first = false;
        __syncthreads();
        if (*abort_flag) break;   // the body drained its copies
        if (threadIdx.x == 0) *next = (int)gridDim.x + atomicAdd(a.claim, 1);
        __syncthreads();
        unit = *next;
    }
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(a.claim + 1, 1) == (int)gridDim.x - 1) {   // every CTA has stopped claiming
            atomicExch(a.claim, 0);
            atomicExch(a.claim + 1, 0);
        }
    }
}

// Batch: every shot of the batch advances one step in one launch.  CTA b
// serves shot cta_shot[b] as its block cta_local[b]; the shot's arguments
// are copied to shared memory, its buffer roles follow the step parity.
// The shot's StepArgs live in dynamic shared memory just past the body's
// rings and barriers, so the kernel declares no static shared memory and the
// rings keep the dynamic window's 128-byte alignment.
template <class S>
__host__ __device__ constexpr int batch_args_offset() {
    return (S::SMEM + 15) / 16 * 16;
}
template <class S>
__host__ __device__ constexpr int batch_smem() {
    return batch_args_offset<S>() + (int)sizeof(StepArgs);
}

template <class S>
__global__ void __launch_bounds__(S::NT, S::MINB2)
    step_tma_batch_kernel(const ShotDesc *__restrict__ shots, const int *__restrict__ cta_shot,
                          const int *__restrict__ cta_local, int n) {
    extern __shared__ __align__(128) unsigned char smem[];
    StepArgs &sa = *reinterpret_cast<StepArgs *>(smem + batch_args_offset<S>());
    const int shot = __ldg(cta_shot + blockIdx.x);
    const ShotDesc *d = shots + shot;
    {
        const int *src = reinterpret_cast<const int *>(&d->args);
        int *dst = reinterpret_cast<int *>(&sa);
        for (int i = threadIdx.x; i < (int)(sizeof(StepArgs) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        sa.n = n;
        sa.ucur = d->u[(n + 1) & 1];
        sa.uprev = d->u[n & 1];
        sa.uout = d->u[n & 1];
        sa.traces = (n >= 1 && d->traces && sa.nrec > 0) ? d->traces + (long long)(n - 1) * sa.nrec : nullptr;
    }
    __syncthreads();
    step_tma_body<S>(sa, StepVar{sa.n, sa.uout, sa.ucur, sa.traces}, &d->cur[(n + 1) & 1], &d->prev[n & 1],
                     &d->cmap, d->geom, __ldg(cta_local + blockIdx.x), d->nblocks, PdlDep{sa.pdl});
}

// Persistent run (PersistArgs): steps n0 .. n1-1 in one cooperative launch,
// as a work list.  Item i is step n0 + i / units of unit i % units (step
// major); CTAs claim items from pa.queue in that order, one at a time, so
// every item before a claimed one is held by a resident CTA and the waits of
// NeighborDep always end.  StepArgs stay in the kernel's constant parameters
// (a.pdl is ignored); the step and the buffer roles go in a StepVar; each
// unit signals its counter once its u^{n+1} (sources and receivers included)
// is complete.
__device__ __forceinline__ unsigned long long *claimed_item(unsigned char *smem_reserved) {
    return reinterpret_cast<unsigned long long *>(smem_reserved + 8);   // next to the abort flag
}

template <class S>
__global__ void __launch_bounds__(S::NT, S::MINB2)
    step_tma_persistent_kernel(const StepArgs a, const __grid_constant__ TmaMaps maps, const Geom g,
                               const PersistArgs pa) {
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char *reserved = smem + (S::NSU * S::CUR + S::NSC * 2 * S::PC) * 4 + (S::NSU + S::NSC) * 8;
    const int *abort_flag = reinterpret_cast<const int *>(reserved);
    unsigned long long *claimed = claimed_item(reserved);
    const unsigned long long total = (unsigned long long)(pa.n1 - pa.n0) * pa.units;
    bool first = true;
    for (;;) {
        __syncthreads();   // every thread has read the previous claim
        if (threadIdx.x == 0) *claimed = atomicAdd(pa.queue, 1ULL);
        __syncthreads();
        const unsigned long long item = *claimed;
        if (item >= total) break;
        const int n = pa.n0 + (int)(item / pa.units), unit = (int)(item % pa.units);
        float *uout = pa.u[n & 1];
        step_tma_body<S>(a, StepVar{n, uout, nullptr, nullptr}, &maps.cur[(n + 1) & 1], &maps.prev[n & 1], &maps.c,
                         g, unit, pa.units, NeighborDep{pa.counters, unit, n, g, first});
        first = false;
        __syncthreads();
        if (*abort_flag) return;   // the body drained its copies; waiters give up on the error word
        // receivers of this unit: u^{n+1} after its sources
        if (pa.traces && pa.nrec > 0) {
            int b = unit;
            const int tx = b % g.tiles_x;
            b /= g.tiles_x;
            const int ty = b % g.tiles_y;
            const int z0 = (b / g.tiles_y) * g.zlen;
            const int T = min(a.nz - z0, g.zlen);
            const long long q = ((long long)ty * g.tiles_x + tx) * a.nz + z0;
            const int lo = __ldg(pa.rec_start + q), hi = __ldg(pa.rec_start + q + T);
            float *row = pa.traces + (long long)n * pa.nrec;
            for (int p = lo + threadIdx.x; p < hi; p += blockDim.x)
                row[__ldg(pa.rec_idx + p)] = uout[__ldg(pa.rec_off + p)];
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            fence_proxy_async_global();
            __threadfence();
            st_release_gpu(pa.counters + unit, n + 1);
        }
    }
}

// Persistent batch run: every shot's time loop in one cooperative launch,
// as a work list over all shots' units (the batch decomposition: unit u is
// shot unit_shot[u], block unit_local[u]).  Item i is step n0 + i / units of
// unit i % units; CTAs claim items in that order from pa.queue, one at a
// time, wait until the unit and its 26 neighbours of the same shot have
// completed step n-1 (bounded polls), run the step, record the unit's
// receivers and signal its counter.  The shot's arguments are staged in
// shared memory per item, as in the one-launch-per-step batch kernel.
template <class S>
__global__ void __launch_bounds__(S::NT, S::MINB2)
    step_tma_batch_persistent_kernel(const ShotDesc *__restrict__ shots, const BatchPersistArgs pa) {
    extern __shared__ __align__(128) unsigned char smem[];
    StepArgs &sa = *reinterpret_cast<StepArgs *>(smem + batch_args_offset<S>());
    unsigned char *reserved = smem + (S::NSU * S::CUR + S::NSC * 2 * S::PC) * 4 + (S::NSU + S::NSC) * 8;
    const int *abort_flag = reinterpret_cast<const int *>(reserved);
    unsigned long long *claimed = claimed_item(reserved);
    const unsigned long long total = (unsigned long long)(pa.n1 - pa.n0) * pa.units;
    bool first = true;
    for (;;) {
        __syncthreads();   // the previous item is done with the staged arguments and the claim
        if (threadIdx.x == 0) *claimed = atomicAdd(pa.queue, 1ULL);
        __syncthreads();
        const unsigned long long item = *claimed;
        if (item >= total) break;
        const int n = pa.n0 + (int)(item / pa.units), unit = (int)(item % pa.units);
        const int shot = __ldg(pa.unit_shot + unit), local = __ldg(pa.unit_local + unit);
        const ShotDesc *d = shots + shot;
        {
            const int *src = reinterpret_cast<const int *>(&d->args);
            int *dst = reinterpret_cast<int *>(&sa);
            for (int i = threadIdx.x; i < (int)(sizeof(StepArgs) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
        }
        __syncthreads();
        float *uout = d->u[n & 1];
        int *counters = pa.counters + __ldg(pa.counter_base + shot);
        step_tma_body<S>(sa, StepVar{n, uout, nullptr, nullptr}, &d->cur[(n + 1) & 1], &d->prev[n & 1], &d->cmap,
                         d->geom, local, d->nblocks, NeighborDep{counters, local, n, d->geom, first});
        first = false;
        __syncthreads();
        if (*abort_flag) return;   // the body drained its copies; waiters give up on the error word
        // receivers of this unit: u^{n+1} after its sources
        if (d->traces && sa.nrec > 0) {
            int b = local;
            const int tx = b % d->geom.tiles_x;
            b /= d->geom.tiles_x;
            const int ty = b % d->geom.tiles_y;
            const int z0 = (b / d->geom.tiles_y) * d->geom.zlen;
            const int T = min(sa.nz - z0, d->geom.zlen);
            const long long q = ((long long)ty * d->geom.tiles_x + tx) * sa.nz + z0;
            const int lo = __ldg(d->rec_start + q), hi = __ldg(d->rec_start + q + T);
            float *row = d->traces + (long long)n * sa.nrec;
            for (int p = lo + threadIdx.x; p < hi; p += blockDim.x)
                row[__ldg(d->rec_idx + p)] = uout[__ldg(d->rec_boff + p)];
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            fence_proxy_async_global();
            __threadfence();
            st_release_gpu(counters + local, n + 1);
        }
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

// Compiled variants.  All use tile height 16 (the tensor maps' box).
constexpr int kTY = 16;
static_assert(kTY == kInjTileY && TX == kInjTileX, "injection buckets must match the kernel's tiles");
using V22_1 = Shape<kTY, 2, 1>;
using V22_2 = Shape<kTY, 2, 2>;
using V22_4 = Shape<kTY, 2, 4>;
using V24_1 = Shape<kTY, 4, 1>;
using V24_2 = Shape<kTY, 4, 2>;
using V24_2s = Shape<kTY, 4, 2, 6, 2>;
using V22_4s = Shape<kTY, 2, 4, 6, 2>;
using V22_4s3 = Shape<kTY, 2, 4, 6, 2, 3>;
using V22_2s3 = Shape<kTY, 2, 2, 6, 2, 3>;
static_assert(kTmaGVariant == 2, "the g^n forms are compiled for V22_4, variant 2");

struct Variant {
    const char *name;
    const void *fn;
    const void *batch_fn;
    const void *persist_fn;   // null: no persistent form compiled
    const void *claim_fn;     // null: no work-claiming form compiled
    int nt, smem, batch_smem;
};

#define MMOD_VARIANT(V, desc, P, C) \
    {desc, (const void *)step_tma_kernel<V>, (const void *)step_tma_batch_kernel<V>, P, C, V::NT, V::SMEM, \
     batch_smem<V>()}
const Variant kVariants[] = {
    MMOD_VARIANT(V22_1, "64x16 tile, 2x2 points/thread, z unroll 1", nullptr, nullptr),
    MMOD_VARIANT(V22_2, "64x16 tile, 2x2 points/thread, z unroll 2", nullptr,
                 (const void *)step_tma_claim_kernel<V22_2>),
    MMOD_VARIANT(V22_4, "64x16 tile, 2x2 points/thread, z unroll 4",
                 (const void *)step_tma_persistent_kernel<V22_4>, (const void *)step_tma_claim_kernel<V22_4>),
    MMOD_VARIANT(V24_1, "64x16 tile, 2x4 points/thread, z unroll 1", nullptr, nullptr),
    MMOD_VARIANT(V24_2, "64x16 tile, 2x4 points/thread, z unroll 2", nullptr, nullptr),
    MMOD_VARIANT(V24_2s, "64x16 tile, 2x4 points/thread, z unroll 2, shallow rings",
                 (const void *)step_tma_persistent_kernel<V24_2s>, nullptr),
    MMOD_VARIANT(V22_4s, "64x16 tile, 2x2 points/thread, z unroll 4, shallow rings", nullptr,
                 (const void *)step_tma_claim_kernel<V22_4s>),
    MMOD_VARIANT(V22_4s3, "64x16 tile, 2x2 points/thread, z unroll 4, shallow rings, 3 CTAs/SM", nullptr, nullptr),
    MMOD_VARIANT(V22_2s3, "64x16 tile, 2x2 points/thread, z unroll 2, shallow rings, 3 CTAs/SM", nullptr, nullptr),
};
#undef MMOD_VARIANT
constexpr int kNumVariants = sizeof(kVariants) / sizeof(kVariants[0]);

}  // namespace

int tma_variant_count() { return kNumVariants; }

const char *tma_variant_name(int v) { return (v >= 0 && v < kNumVariants) ? kVariants[v].name : ""; }

bool encode_box(CUtensorMap *map, const float *base, int nx, int ny, int nz, int nxp, int bx, int by) {
    mmod_config c{};
    c.nx = nx;
    c.ny = ny;
    c.nz = nz;
    return encode(map, base, c, nxp, bx, by);
}

bool encode_maps(const mmod_config &cfg, int nxp, const float *buf, CUtensorMap *cur, CUtensorMap *prev) {
    return encode(cur, buf, cfg, nxp, HX, kTY + 2 * kRadius) && encode(prev, buf, cfg, nxp, TX, kTY);
}

bool make_tma_plan(const mmod_config &cfg, int nxp, float *const u[2], const float *c, CUtensorMap cur_map[2],
                   CUtensorMap prev_map[2], CUtensorMap *c_map, TmaPlan plans[]) {
    for (int b = 0; b < 2; ++b) {
        if (!encode(&cur_map[b], u[b], cfg, nxp, HX, kTY + 2 * kRadius)) return false;
        if (!encode(&prev_map[b], u[b], cfg, nxp, TX, kTY)) return false;
    }
    if (!encode(c_map, c, cfg, nxp, TX, kTY)) return false;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int tiles_x = (cfg.nx + TX - 1) / TX, tiles_y = (cfg.ny + kTY - 1) / kTY;
    const long long tiles = (long long)tiles_x * tiles_y;
    for (int v = 0; v < kNumVariants; ++v) {
        const Variant &var = kVariants[v];
        int occ = 0;
        if (cudaFuncSetAttribute(var.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, var.smem) != cudaSuccess ||
            cudaFuncSetAttribute(var.batch_fn, cudaFuncAttributeMaxDynamicSharedMemorySize, var.batch_smem) != cudaSuccess ||
            (var.claim_fn &&
             cudaFuncSetAttribute(var.claim_fn, cudaFuncAttributeMaxDynamicSharedMemorySize, var.smem) !=
                 cudaSuccess) ||
            (var.persist_fn &&
             cudaFuncSetAttribute(var.persist_fn, cudaFuncAttributeMaxDynamicSharedMemorySize, var.smem) !=
                 cudaSuccess) ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, var.fn, var.nt, var.smem) != cudaSuccess || occ < 1) {
            cudaGetLastError();
            return false;
        }
        if (v == kTmaGVariant &&
            (cudaFuncSetAttribute((const void *)step_tma_kernel<V22_4, true>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, var.smem) != cudaSuccess ||
             cudaFuncSetAttribute((const void *)step_tma_claim_kernel<V22_4, true>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, var.smem) != cudaSuccess)) {
            cudaGetLastError();
            return false;
        }
        const long long slots = (long long)sms * occ;
        // the z split that minimises (waves) x (planes per CTA + halo cost)
        int best_c = 1;
        double best = 1e300;
        for (int zc = 1; zc <= cfg.nz; ++zc) {
            const int zlen = (cfg.nz + zc - 1) / zc;
            if ((cfg.nz + zlen - 1) / zlen != zc) continue;
            const long long ctas = tiles * zc;
            if (ctas > (1LL << 31) - 1) break;
            const double waves = (double)((ctas + slots - 1) / slots);
            const double cost = waves * (zlen + 2.0);
            if (cost < best - 1e-9) {
                best = cost;
                best_c = zc;
            }
        }
        TmaPlan &p = plans[v];
        p.variant = v;
        p.tiles_x = tiles_x;
        p.tiles_y = tiles_y;
        p.zchunks = best_c;
        p.zlen = (cfg.nz + best_c - 1) / best_c;
        p.grid = (int)(tiles * best_c);
        p.block = var.nt;
        p.smem = var.smem;
        p.occupancy = occ;
        p.slots = (int)std::min<long long>(slots, 1LL << 30);
        p.claim = 0;
    }
    return true;
}

bool claim_geom(const TmaPlan &plan, int nz, Geom *g, int *units, int *grid) {
    if (plan.claim <= 0 || plan.variant < 0 || plan.variant >= kNumVariants || !kVariants[plan.variant].claim_fn ||
        plan.slots < 1 || nz < 1)
        return false;
    const int zlen = std::min(plan.claim, nz);
    *g = Geom{plan.tiles_x, plan.tiles_y, (nz + zlen - 1) / zlen, zlen};
    const long long u = (long long)g->tiles_x * g->tiles_y * g->zchunks;
    if (u > (1LL << 30)) return false;
    *units = (int)u;
    *grid = (int)std::min<long long>(u, plan.slots);
    return true;
}

cudaError_t launch_step_tma(const StepArgs &a, const CUtensorMap *cur_map, const CUtensorMap *prev_map,
                            const CUtensorMap *c_map, const TmaPlan &plan, cudaStream_t s) {
    Geom cg;
    int units = 0, cgrid = 0;
    const bool claim = a.claim && claim_geom(plan, a.nz, &cg, &units, &cgrid);
    if (a.gout) {   // g^n as well: variant 2 only (the caller passes its plan)
        if (plan.variant != kTmaGVariant) return cudaErrorInvalidValue;
        cudaLaunchConfig_t lc = {};
        lc.gridDim = dim3(claim ? cgrid : plan.grid);
        lc.blockDim = dim3(plan.block);
        lc.dynamicSmemBytes = plan.smem;
        lc.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        lc.attrs = attr;
        lc.numAttrs = a.pdl ? 1 : 0;
        const Geom g{plan.tiles_x, plan.tiles_y, plan.zchunks, plan.zlen};
        const cudaError_t e =
            claim ? cudaLaunchKernelEx(&lc, step_tma_claim_kernel<V22_4, true>, a, *cur_map, *prev_map, *c_map, cg, units)
                  : cudaLaunchKernelEx(&lc, step_tma_kernel<V22_4, true>, a, *cur_map, *prev_map, *c_map, g);
        if (e != cudaSuccess) return e;
        return cudaGetLastError();
    }
    if (claim) {
        cudaLaunchConfig_t lc = {};
        lc.gridDim = dim3(cgrid);
        lc.blockDim = dim3(plan.block);
        lc.dynamicSmemBytes = plan.smem;
        lc.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        lc.attrs = attr;
        lc.numAttrs = a.pdl ? 1 : 0;
        cudaError_t e;
        switch (plan.variant) {
            case 1: e = cudaLaunchKernelEx(&lc, step_tma_claim_kernel<V22_2>, a, *cur_map, *prev_map, *c_map, cg, units); break;
            case 2: e = cudaLaunchKernelEx(&lc, step_tma_claim_kernel<V22_4>, a, *cur_map, *prev_map, *c_map, cg, units); break;
            case 6: e = cudaLaunchKernelEx(&lc, step_tma_claim_kernel<V22_4s>, a, *cur_map, *prev_map, *c_map, cg, units); break;
            default: return cudaErrorInvalidValue;
        }
        if (e != cudaSuccess) return e;
        return cudaGetLastError();
    }
    const Geom g{plan.tiles_x, plan.tiles_y, plan.zchunks, plan.zlen};
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(plan.grid);
    lc.blockDim = dim3(plan.block);
    lc.dynamicSmemBytes = plan.smem;
    lc.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    lc.attrs = attr;
    lc.numAttrs = a.pdl ? 1 : 0;
#define MMOD_LAUNCH(V) cudaLaunchKernelEx(&lc, step_tma_kernel<V>, a, *cur_map, *prev_map, *c_map, g)
    switch (plan.variant) {
        case 0: MMOD_LAUNCH(V22_1); break;
        case 1: MMOD_LAUNCH(V22_2); break;
        case 2: MMOD_LAUNCH(V22_4); break;
        case 3: MMOD_LAUNCH(V24_1); break;
        case 4: MMOD_LAUNCH(V24_2); break;
        case 5: MMOD_LAUNCH(V24_2s); break;
        case 6: MMOD_LAUNCH(V22_4s); break;
        case 7: MMOD_LAUNCH(V22_4s3); break;
        case 8: MMOD_LAUNCH(V22_2s3); break;
        default: return cudaErrorInvalidValue;
    }
#undef MMOD_LAUNCH
    return cudaGetLastError();
}

Geom persistent_geom(const TmaPlan &plan, int nz) {
    // z ranges at least as thick as the stencil radius: a unit's halo then
    // reaches only the adjacent range
    const int zlen = std::max(plan.zlen, kRadius);
    return Geom{plan.tiles_x, plan.tiles_y, (nz + zlen - 1) / zlen, zlen};
}

int persistent_grid(const TmaPlan &plan, int nz, int max_ctas) {
    if (plan.variant < 0 || plan.variant >= kNumVariants || nz < 1) return 0;
    const Variant &var = kVariants[plan.variant];
    if (!var.persist_fn) return 0;
    const Geom g = persistent_geom(plan, nz);
    int dev = 0, sms = 0, occ = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, var.persist_fn, var.nt, var.smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    long long grid = std::min<long long>((long long)sms * occ, (long long)g.tiles_x * g.tiles_y * g.zchunks);
    if (max_ctas > 0) grid = std::min<long long>(grid, max_ctas);
    return (int)std::max<long long>(grid, 0);
}

cudaError_t launch_step_tma_persistent(const StepArgs &a, const TmaMaps &maps, const TmaPlan &plan,
                                       const PersistArgs &pa, int grid, cudaStream_t s) {
    if (plan.variant < 0 || plan.variant >= kNumVariants || !kVariants[plan.variant].persist_fn || grid < 1)
        return cudaErrorInvalidValue;
    const Geom g = persistent_geom(plan, a.nz);
    if (pa.units != g.tiles_x * g.tiles_y * g.zchunks) return cudaErrorInvalidValue;
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(grid);
    lc.blockDim = dim3(kVariants[plan.variant].nt);
    lc.dynamicSmemBytes = kVariants[plan.variant].smem;
    lc.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;   // all CTAs resident: units wait on one another
    attr[0].val.cooperative = 1;
    lc.attrs = attr;
    lc.numAttrs = 1;
    cudaError_t e;
    switch (plan.variant) {
        case 2: e = cudaLaunchKernelEx(&lc, step_tma_persistent_kernel<V22_4>, a, maps, g, pa); break;
        case 5: e = cudaLaunchKernelEx(&lc, step_tma_persistent_kernel<V24_2s>, a, maps, g, pa); break;
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

int batch_persistent_grid(int variant, int units) {
    const void *fn = variant == 2 ? (const void *)step_tma_batch_persistent_kernel<V22_4>
                                  : (variant == 5 ? (const void *)step_tma_batch_persistent_kernel<V24_2s> : nullptr);
    if (!fn || units < 1) return 0;
    const int smem = kVariants[variant].batch_smem;
    int dev = 0, sms = 0, occ = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kVariants[variant].nt, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return (int)std::min<long long>((long long)sms * occ, units);
}

cudaError_t launch_step_tma_batch_persistent(int variant, const ShotDesc *shots, const BatchPersistArgs &pa, int grid,
                                             cudaStream_t s) {
    if ((variant != 2 && variant != 5) || grid < 1) return cudaErrorInvalidValue;
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(grid);
    lc.blockDim = dim3(kVariants[variant].nt);
    lc.dynamicSmemBytes = kVariants[variant].batch_smem;
    lc.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;   // all CTAs resident: units wait on one another
    attr[0].val.cooperative = 1;
    lc.attrs = attr;
    lc.numAttrs = 1;
    cudaError_t e = variant == 2 ? cudaLaunchKernelEx(&lc, step_tma_batch_persistent_kernel<V22_4>, shots, pa)
                                 : cudaLaunchKernelEx(&lc, step_tma_batch_persistent_kernel<V24_2s>, shots, pa);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

bool tma_variant_info(int v, int *out) {
    if (v < 0 || v >= kNumVariants) return false;
    const Variant &var = kVariants[v];
    const void *fns[3] = {var.fn, var.batch_fn, var.persist_fn};
    const int dyn[3] = {var.smem, var.batch_smem, var.smem};
    out[0] = var.nt;
    out[1] = var.smem;
    for (int k = 0; k < 3; ++k) {
        int *o = out + 2 + 4 * k;
        o[0] = o[1] = o[2] = o[3] = -1;
        if (!fns[k]) continue;
        cudaFuncAttributes fa;
        int occ = 0;
        if (cudaFuncSetAttribute(fns[k], cudaFuncAttributeMaxDynamicSharedMemorySize, dyn[k]) != cudaSuccess ||
            cudaFuncGetAttributes(&fa, fns[k]) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fns[k], var.nt, dyn[k]) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        o[0] = fa.numRegs;
        o[1] = (int)fa.localSizeBytes;
        o[2] = (int)fa.sharedSizeBytes;
        o[3] = occ;
    }
    return true;
}

bool tma_variant_shape(int v, int *block, int *smem) {
    if (v < 0 || v >= kNumVariants) return false;
    *block = kVariants[v].nt;
    *smem = kVariants[v].smem;
    return true;
}

cudaError_t launch_step_tma_batch(int variant, const ShotDesc *shots, const int *cta_shot, const int *cta_local,
                                  int nctas, int n, bool pdl, cudaStream_t s) {
    if (variant < 0 || variant >= kNumVariants) return cudaErrorInvalidValue;
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(nctas);
    lc.blockDim = dim3(kVariants[variant].nt);
    lc.dynamicSmemBytes = kVariants[variant].batch_smem;
    lc.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    lc.attrs = attr;
    lc.numAttrs = pdl ? 1 : 0;
    cudaError_t e;
#define MMOD_LAUNCH_B(V) e = cudaLaunchKernelEx(&lc, step_tma_batch_kernel<V>, shots, cta_shot, cta_local, n)
    switch (variant) {
        case 0: MMOD_LAUNCH_B(V22_1); break;
        case 1: MMOD_LAUNCH_B(V22_2); break;
        case 2: MMOD_LAUNCH_B(V22_4); break;
        case 3: MMOD_LAUNCH_B(V24_1); break;
        case 4: MMOD_LAUNCH_B(V24_2); break;
        case 5: MMOD_LAUNCH_B(V24_2s); break;
        case 6: MMOD_LAUNCH_B(V22_4s); break;
        case 7: MMOD_LAUNCH_B(V22_4s3); break;
        case 8: MMOD_LAUNCH_B(V22_2s3); break;
        default: return cudaErrorInvalidValue;
    }
#undef MMOD_LAUNCH_B
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace mmod
