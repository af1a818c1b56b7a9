// Batched shots and the variant autotuner.
//
// A batch groups handles (one per shot; grids of any size, the same number of
// steps) and runs them in one of two ways:
//   streams (default): each shot's own time loop (its cached graph of
//     one-step kernels) on one of kSubStreams internal streams, forked from
//     and joined back to the caller's stream, so the shots' waves overlap and
//     hide one another's tails;
//   fused: one kernel launch per step advances every shot: CTA b serves shot
//     cta_shot[b] as its block cta_local[b], reading the shot's arguments and
//     tensor maps from a descriptor table in device memory.  The nt launches
//     are captured once into a CUDA graph; the descriptor table is uploaded
//     per call, so new wavelet / trace buffers need no new capture.  CTAs are
//     ordered longest first so the last wave is made of short ones;
//   persistent: one cooperative launch runs every shot's whole time loop as
//     a work list: CTAs claim (step, unit) items in step-major order, a unit
//     being a shot's tile and z range; an item starts when the unit and its
//     neighbouring units of the same shot have finished the previous step
//     (per-unit counters, bounded waits).
//
// The autotuner times each compiled TMA variant (points per thread, z
// unroll, ring depths) for a few steps on the real problem and keeps the
// fastest.
#include <algorithm>
#include <cstring>
#include <numeric>
#include <vector>

#include "mmod_handle.h"

#define MMOD_API extern "C" __attribute__((visibility("default")))

using namespace mmod;

constexpr int kSubStreams = 4;

struct mmod_batch {
    std::vector<mmod_handle *> shots;
    int device = 0, nt = 0;
    int mode = MMOD_BATCH_STREAMS;
    int variant = kTmaDefaultVariant;
    bool variant_set = false;
    int pdl = 1;
    cudaStream_t sub[kSubStreams] = {};
    cudaEvent_t fork = nullptr, join[kSubStreams] = {};
    std::vector<ShotDesc> desc;       // host copy, uploaded per call
    ShotDesc *d_desc = nullptr;
    int *d_cta_shot = nullptr, *d_cta_local = nullptr;
    int nctas = 0;
    // persistent mode: units in shot order, counters per unit, counter base per shot
    int *d_unit_shot = nullptr, *d_unit_local = nullptr, *d_counter_base = nullptr, *d_counters = nullptr;
    unsigned long long *d_queue = nullptr;   // next (step, unit) item of the persistent work list
    int units = 0;
    GraphSlot graph;
    cudaEvent_t ev_t0 = nullptr, ev_t1 = nullptr;
    bool ran = false;
    std::string err;
};

namespace {

// Planes per CTA (or per persistent work unit) in a batch: whole columns of
// the shots up to 256 planes (few halo planes and unit set-ups), since a batch
// has many CTAs per wave anyway.
constexpr int kBatchZlen = 256;

__global__ void batch_gather_kernel(const ShotDesc *__restrict__ shots, int nt) {
    const ShotDesc *d = shots + blockIdx.y;
    const int nrec = d->args.nrec;
    if (!d->traces || nrec <= 0 || nt <= 0) return;
    const float *u = d->u[(nt - 1) & 1];   // u^{nt}
    float *dst = d->traces + (long long)(nt - 1) * nrec;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nrec; r += gridDim.x * blockDim.x)
        dst[r] = u[__ldg(d->args.rec_off + r)];
}

mmod_status bfail(mmod_batch *b, mmod_status st, const std::string &msg) {
    if (b) b->err = msg;
    return st;
}

mmod_status bfail_cuda(mmod_batch *b, cudaError_t e, const char *what) {
    if (b) b->err = std::string(what) + ": " + cudaGetErrorName(e);
    return e == cudaErrorMemoryAllocation ? MMOD_ERR_OOM : MMOD_ERR_CUDA;
}

#define BCK(b, call)                                          \
    do {                                                      \
        cudaError_t _e = (call);                              \
        if (_e != cudaSuccess) return bfail_cuda((b), _e, #call); \
    } while (0)

void free_batch(mmod_batch *b) {
    for (int k = 0; k < kSubStreams; ++k) {
        if (b->sub[k]) cudaStreamDestroy(b->sub[k]);
        if (b->join[k]) cudaEventDestroy(b->join[k]);
    }
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->graph.exec) cudaGraphExecDestroy(b->graph.exec);
    if (b->d_desc) cudaFree(b->d_desc);
    if (b->d_cta_shot) cudaFree(b->d_cta_shot);
    if (b->d_cta_local) cudaFree(b->d_cta_local);
    if (b->d_unit_shot) cudaFree(b->d_unit_shot);
    if (b->d_unit_local) cudaFree(b->d_unit_local);
    if (b->d_counter_base) cudaFree(b->d_counter_base);
    if (b->d_counters) cudaFree(b->d_counters);
    if (b->d_queue) cudaFree(b->d_queue);
    if (b->ev_t0) cudaEventDestroy(b->ev_t0);
    if (b->ev_t1) cudaEventDestroy(b->ev_t1);
}

// The batch's steps n0 .. n1-1 on stream s (all shots), direct launches.
mmod_status enqueue_batch_steps(mmod_batch *b, int n0, int n1, cudaStream_t s) {
    for (int n = n0; n < n1; ++n)
        BCK(b, launch_step_tma_batch(b->variant, b->d_desc, b->d_cta_shot, b->d_cta_local, b->nctas, n, b->pdl != 0, s));
    return MMOD_OK;
}

mmod_status zero_states(mmod_batch *b, cudaStream_t s) {
    for (mmod_handle *h : b->shots) {
        BCK(b, cudaMemsetAsync(h->u[0], 0, sizeof(float) * (size_t)h->vol, s));
        BCK(b, cudaMemsetAsync(h->u[1], 0, sizeof(float) * (size_t)h->vol, s));
        h->state_pending = false;
        h->ran = false;
    }
    return MMOD_OK;
}

// Time `steps` steps of the time loop from zero state (ms, events on s).
float time_steps(mmod_batch *b, int steps, cudaStream_t s, mmod_status *st) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    *st = zero_states(b, s);
    cudaEventRecord(e0, s);
    if (*st == MMOD_OK) *st = enqueue_batch_steps(b, 0, std::min(steps, b->nt), s);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = -1.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ms;
}

// Fork the internal streams from s (after everything already on s).
mmod_status fork_streams(mmod_batch *b, cudaStream_t s) {
    BCK(b, cudaEventRecord(b->fork, s));
    for (int k = 0; k < kSubStreams; ++k) BCK(b, cudaStreamWaitEvent(b->sub[k], b->fork, 0));
    return MMOD_OK;
}

// Join the internal streams back into s.
mmod_status join_streams(mmod_batch *b, cudaStream_t s) {
    for (int k = 0; k < kSubStreams; ++k) {
        BCK(b, cudaEventRecord(b->join[k], b->sub[k]));
        BCK(b, cudaStreamWaitEvent(s, b->join[k], 0));
    }
    return MMOD_OK;
}

}  // namespace

namespace mmod {

// `steps` steps of h's time loop from zero state without sources or
// receivers, direct launches on s (autotuning).
mmod_status enqueue_tune_steps(mmod_handle *h, int steps, cudaStream_t s) {
    MMOD_CK(h, cudaMemsetAsync(h->u[0], 0, sizeof(float) * (size_t)h->vol, s));
    MMOD_CK(h, cudaMemsetAsync(h->u[1], 0, sizeof(float) * (size_t)h->vol, s));
    StepArgs a = base_args(h, h->fwd, nullptr);
    a.inj.npts = 0;   // no sources while tuning
    a.nrec = 0;
    long long count = 0;
    for (int n = 0; n < std::min(steps, h->cfg.nt); ++n) {
        a.n = n;
        a.ucur = h->u[(n + 1) & 1];
        a.uprev = h->u[n & 1];
        a.uout = h->u[n & 1];
        MMOD_CK(h, enqueue_step(h, a, &h->cur_map[(n + 1) & 1], &h->prev_map[n & 1], true, nullptr, s, &count));
    }
    h->state_pending = false;
    h->ran = false;
    return MMOD_OK;
}

}  // namespace mmod

MMOD_API mmod_status mmod_batch_create(mmod_handle *const *shots, int nshots, mmod_batch **out) {
    set_thread_error("");
    if (!out) return MMOD_ERR_ARG;
    *out = nullptr;
    if (!shots || nshots < 1) {
        set_thread_error("a batch needs at least one handle");
        return MMOD_ERR_ARG;
    }
    for (int i = 0; i < nshots; ++i) {
        if (!shots[i]) {
            set_thread_error("null handle in the batch");
            return MMOD_ERR_ARG;
        }
        if (shots[i]->device != shots[0]->device || shots[i]->cfg.nt != shots[0]->cfg.nt) {
            set_thread_error("the handles of a batch need the same device and the same nt");
            return MMOD_ERR_ARG;
        }
        if (!shots[i]->tma_ok) {
            set_thread_error("a handle of the batch has no TMA plan");
            return MMOD_ERR_UNSUPPORTED;
        }
    }
    mmod_batch *b = new mmod_batch();
    b->shots.assign(shots, shots + nshots);
    b->device = shots[0]->device;
    b->nt = shots[0]->cfg.nt;
    DeviceGuard guard(b->device);
    b->desc.resize(nshots);
    std::vector<int> cta_shot, cta_local, cta_len, counter_base;
    for (int i = 0; i < nshots; ++i) {
        mmod_handle *h = shots[i];
        ShotDesc &d = b->desc[i];
        std::memset(&d, 0, sizeof(d));
        d.rec_start = h->fwd.g_start;
        d.rec_idx = h->fwd.g_idx;
        d.rec_boff = h->fwd.g_off;
        for (int k = 0; k < 2; ++k) {
            d.cur[k] = h->cur_map[k];
            d.prev[k] = h->prev_map[k];
            d.u[k] = h->u[k];
        }
        d.cmap = h->c_map;
        d.args = base_args(h, h->fwd, nullptr);
        const TmaPlan &p = h->plans[0];
        // MMOD_OPT_ZLEN of the shot, at least the stencil radius (a persistent
        // unit's halo then reaches only the adjacent z ranges)
        const int zt = h->zlen_override > 0 ? std::max(h->zlen_override, kRadius) : kBatchZlen;
        const int zchunks = (h->cfg.nz + zt - 1) / zt;
        const int zlen = (h->cfg.nz + zchunks - 1) / zchunks;
        d.geom = Geom{p.tiles_x, p.tiles_y, (h->cfg.nz + zlen - 1) / zlen, zlen};
        d.nblocks = d.geom.tiles_x * d.geom.tiles_y * d.geom.zchunks;
        counter_base.push_back((int)cta_shot.size());
        for (int lb = 0; lb < d.nblocks; ++lb) {
            const int chunk = lb / (d.geom.tiles_x * d.geom.tiles_y);
            cta_shot.push_back(i);
            cta_local.push_back(lb);
            cta_len.push_back(std::min(zlen, h->cfg.nz - chunk * zlen));
        }
    }
    // persistent mode: units in shot order (unit = counter index)
    const std::vector<int> unit_shot = cta_shot, unit_local = cta_local;
    // longest z ranges first: the last wave holds the short ones
    std::vector<int> order(cta_shot.size());
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return cta_len[a] > cta_len[c]; });
    std::vector<int> cs(order.size()), cl(order.size());
    for (size_t q = 0; q < order.size(); ++q) {
        cs[q] = cta_shot[order[q]];
        cl[q] = cta_local[order[q]];
    }
    b->nctas = (int)cs.size();
    auto bail = [&](cudaError_t e, const char *what) {
        set_thread_error((std::string(what) + ": " + cudaGetErrorName(e)).c_str());
        free_batch(b);
        delete b;
        return e == cudaErrorMemoryAllocation ? MMOD_ERR_OOM : MMOD_ERR_CUDA;
    };
#define CKB(call)                                  \
    do {                                           \
        cudaError_t _e = (call);                   \
        if (_e != cudaSuccess) return bail(_e, #call); \
    } while (0)
    CKB(cudaMalloc(&b->d_desc, sizeof(ShotDesc) * nshots));
    CKB(cudaMalloc(&b->d_cta_shot, sizeof(int) * cs.size()));
    CKB(cudaMalloc(&b->d_cta_local, sizeof(int) * cl.size()));
    CKB(cudaMemcpy(b->d_cta_shot, cs.data(), sizeof(int) * cs.size(), cudaMemcpyHostToDevice));
    CKB(cudaMemcpy(b->d_cta_local, cl.data(), sizeof(int) * cl.size(), cudaMemcpyHostToDevice));
    b->units = (int)unit_shot.size();
    CKB(cudaMalloc(&b->d_unit_shot, sizeof(int) * unit_shot.size()));
    CKB(cudaMalloc(&b->d_unit_local, sizeof(int) * unit_local.size()));
    CKB(cudaMalloc(&b->d_counter_base, sizeof(int) * counter_base.size()));
    CKB(cudaMalloc(&b->d_counters, sizeof(int) * unit_shot.size()));
    CKB(cudaMalloc(&b->d_queue, sizeof(unsigned long long)));
    CKB(cudaMemcpy(b->d_unit_shot, unit_shot.data(), sizeof(int) * unit_shot.size(), cudaMemcpyHostToDevice));
    CKB(cudaMemcpy(b->d_unit_local, unit_local.data(), sizeof(int) * unit_local.size(), cudaMemcpyHostToDevice));
    CKB(cudaMemcpy(b->d_counter_base, counter_base.data(), sizeof(int) * counter_base.size(), cudaMemcpyHostToDevice));
    CKB(cudaEventCreate(&b->ev_t0));
    CKB(cudaEventCreate(&b->ev_t1));
    CKB(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
    for (int k = 0; k < kSubStreams; ++k) {
        CKB(cudaStreamCreateWithFlags(&b->sub[k], cudaStreamNonBlocking));
        CKB(cudaEventCreateWithFlags(&b->join[k], cudaEventDisableTiming));
    }
#undef CKB
    *out = b;
    return MMOD_OK;
}

MMOD_API mmod_status mmod_batch_destroy(mmod_batch *b) {
    if (!b) return MMOD_OK;
    {
        DeviceGuard guard(b->device);
        cudaDeviceSynchronize();
        free_batch(b);
    }
    delete b;
    return MMOD_OK;
}

MMOD_API const char *mmod_batch_last_error(const mmod_batch *b) { return b ? b->err.c_str() : ""; }

MMOD_API mmod_status mmod_batch_set_variant(mmod_batch *b, int v) {
    if (!b) return MMOD_ERR_ARG;
    int block, smem;
    if (v < 0 || !tma_variant_shape(v, &block, &smem)) return bfail(b, MMOD_ERR_ARG, "unknown TMA variant");
    b->variant = v;
    b->variant_set = true;
    for (mmod_handle *h : b->shots) h->variant = v;   // streams mode runs each handle's own plan
    return MMOD_OK;
}

MMOD_API mmod_status mmod_batch_set_mode(mmod_batch *b, int mode) {
    if (!b) return MMOD_ERR_ARG;
    if (mode != MMOD_BATCH_STREAMS && mode != MMOD_BATCH_FUSED && mode != MMOD_BATCH_PERSISTENT)
        return bfail(b, MMOD_ERR_ARG, "unknown batch mode");
    b->mode = mode;
    return MMOD_OK;
}

MMOD_API mmod_status mmod_batch_forward(mmod_batch *b, const float *const *wavelets, float *const *traces,
                                        mmod_stream stream) {
    if (!b) return MMOD_ERR_ARG;
    DeviceGuard guard(b->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int ns = (int)b->shots.size();
    if (b->mode == MMOD_BATCH_STREAMS) {
        for (int i = 0; i < ns; ++i) {
            mmod_handle *h = b->shots[i];
            const float *w = wavelets ? wavelets[i] : nullptr;
            float *t = traces ? traces[i] : nullptr;
            if (h->cfg.nsrc > 0 && b->nt > 0 && (!w || !is_device_ptr(w)))
                return bfail(b, MMOD_ERR_ARG, "shot " + std::to_string(i) + ": wavelet must be a device pointer");
            if (h->cfg.nrec > 0 && b->nt > 0 && (!t || !is_device_ptr(t)))
                return bfail(b, MMOD_ERR_ARG, "shot " + std::to_string(i) + ": traces must be a device pointer");
        }
        BCK(b, cudaEventRecord(b->ev_t0, s));
        if (mmod_status st = fork_streams(b, s)) return st;
        for (int i = 0; i < ns; ++i) {
            mmod_handle *h = b->shots[i];
            if (mmod_status st = mmod_forward(h, wavelets ? wavelets[i] : nullptr, traces ? traces[i] : nullptr,
                                              nullptr, (mmod_stream)b->sub[i % kSubStreams])) {
                join_streams(b, s);
                return bfail(b, st, "shot " + std::to_string(i) + ": " + h->err);
            }
        }
        if (mmod_status st = join_streams(b, s)) return st;
        BCK(b, cudaEventRecord(b->ev_t1, s));
        b->ran = b->nt > 0;
        return MMOD_OK;
    }
    for (int i = 0; i < ns; ++i) {
        mmod_handle *h = b->shots[i];
        if (mmod_status st = check_latched(h)) return bfail(b, st, "shot " + std::to_string(i) + ": " + h->err);
        if (!h->model_set) return bfail(b, MMOD_ERR_STATE, "shot " + std::to_string(i) + " has no model");
        const float *w = wavelets ? wavelets[i] : nullptr;
        float *t = traces ? traces[i] : nullptr;
        if (h->cfg.nsrc > 0 && b->nt > 0 && (!w || !is_device_ptr(w)))
            return bfail(b, MMOD_ERR_ARG, "shot " + std::to_string(i) + ": wavelet must be a device pointer");
        if (h->cfg.nrec > 0 && b->nt > 0 && (!t || !is_device_ptr(t)))
            return bfail(b, MMOD_ERR_ARG, "shot " + std::to_string(i) + ": traces must be a device pointer");
        b->desc[i].args.wavelet = w;
        b->desc[i].args.w = h->w;                // the handle's current stencil weights
        b->desc[i].args.pdl = b->pdl ? 2 : 0;   // the captured steps follow one another
        b->desc[i].args.err = h->err_dev;
        b->desc[i].traces = t;
    }
    for (int i = 0; i < ns; ++i)
        if (is_cpml(b->shots[i]))
            return bfail(b, MMOD_ERR_UNSUPPORTED, "the fused batch kernels have no CPML; use MMOD_BATCH_STREAMS");
    int pgrid = 0;
    if (b->mode == MMOD_BATCH_PERSISTENT) {
        pgrid = batch_persistent_grid(b->variant, b->units);
        if (pgrid < 1)
            return bfail(b, MMOD_ERR_UNSUPPORTED, "the persistent batch kernel needs TMA variant 2 or 5");
    }
    BCK(b, cudaMemcpyAsync(b->d_desc, b->desc.data(), sizeof(ShotDesc) * ns, cudaMemcpyHostToDevice, s));
    if (mmod_status st = zero_states(b, s)) return st;
    if (b->mode == MMOD_BATCH_PERSISTENT) {
        // every shot's loop in one cooperative launch (no graph: one node)
        BCK(b, cudaMemsetAsync(b->d_counters, 0, sizeof(int) * (size_t)b->units, s));
        BCK(b, cudaMemsetAsync(b->d_queue, 0, sizeof(unsigned long long), s));
        BCK(b, cudaEventRecord(b->ev_t0, s));
        if (b->nt > 0) {
            BatchPersistArgs pa{};
            // MMOD_OPT_TEST_STALL on any shot: start at step 1 with the
            // counters at 0, so every unit waits for neighbours that never
            // signal and gives up (bounded); the shots then report TIMEOUT
            pa.n0 = 0;
            for (mmod_handle *h : b->shots)
                if (h->test_stall) {
                    pa.n0 = 1;
                    h->test_stall = 0;
                }
            pa.n1 = b->nt;
            pa.units = b->units;
            pa.unit_shot = b->d_unit_shot;
            pa.unit_local = b->d_unit_local;
            pa.counter_base = b->d_counter_base;
            pa.counters = b->d_counters;
            pa.queue = b->d_queue;
            BCK(b, launch_step_tma_batch_persistent(b->variant, b->d_desc, pa, pgrid, s));
        }
        BCK(b, cudaEventRecord(b->ev_t1, s));
        b->ran = b->nt > 0;
        for (mmod_handle *h : b->shots) {
            if (mmod_status st = check_latched(h)) return bfail(b, st, h->err);
            h->ran = true;
        }
        return MMOD_OK;
    }
    if (b->nt > 0) {
        GraphSlot &g = b->graph;
        if (!g.exec || g.kernel != b->variant || g.opts != b->pdl) {
            if (g.exec) cudaGraphExecDestroy(g.exec);
            g = GraphSlot();
            mmod_handle *h0 = b->shots[0];
            cudaGraph_t graph = nullptr;
            BCK(b, cudaStreamBeginCapture(h0->cap, cudaStreamCaptureModeThreadLocal));
            mmod_status st = MMOD_OK;
            if (cudaEventRecordWithFlags(b->ev_t0, h0->cap, cudaEventRecordExternal) != cudaSuccess)
                st = MMOD_ERR_CUDA;
            if (st == MMOD_OK) st = enqueue_batch_steps(b, 0, b->nt, h0->cap);
            if (st == MMOD_OK) {
                batch_gather_kernel<<<dim3(64, ns), 256, 0, h0->cap>>>(b->d_desc, b->nt);
                if (cudaGetLastError() != cudaSuccess) st = MMOD_ERR_CUDA;
            }
            if (st == MMOD_OK && cudaEventRecordWithFlags(b->ev_t1, h0->cap, cudaEventRecordExternal) != cudaSuccess)
                st = MMOD_ERR_CUDA;
            cudaError_t e_end = cudaStreamEndCapture(h0->cap, &graph);
            if (st != MMOD_OK || e_end != cudaSuccess) {
                if (graph) cudaGraphDestroy(graph);
                return bfail(b, st != MMOD_OK ? st : MMOD_ERR_CUDA, "capturing the batch loop failed");
            }
            cudaError_t e_inst = cudaGraphInstantiate(&g.exec, graph, 0);
            cudaGraphDestroy(graph);
            if (e_inst != cudaSuccess) {
                g.exec = nullptr;
                return bfail_cuda(b, e_inst, "cudaGraphInstantiate");
            }
            g.kernel = b->variant;
            g.opts = b->pdl;
            g.launches = b->nt + 1;
        }
        BCK(b, cudaGraphLaunch(g.exec, s));
    }
    b->ran = b->nt > 0;
    for (mmod_handle *h : b->shots) {
        if (mmod_status st = check_latched(h)) return bfail(b, st, h->err);
        h->ran = true;   // each handle's buffers hold its shot's final state
    }
    return MMOD_OK;
}

MMOD_API float mmod_batch_last_loop_ms(mmod_batch *b) {
    if (!b || !b->ran) return -1.0f;
    DeviceGuard guard(b->device);
    float ms = -1.0f;
    if (cudaEventSynchronize(b->ev_t1) != cudaSuccess || cudaEventElapsedTime(&ms, b->ev_t0, b->ev_t1) != cudaSuccess) {
        cudaGetLastError();
        return -1.0f;
    }
    return ms;
}

MMOD_API mmod_status mmod_batch_autotune(mmod_batch *b, int steps, mmod_stream stream, int *variant_out) {
    if (!b || steps < 1) return MMOD_ERR_ARG;
    if (b->mode == MMOD_BATCH_PERSISTENT)
        return bfail(b, MMOD_ERR_UNSUPPORTED, "the persistent batch runs TMA variant 2 or 5; tune another mode");
    DeviceGuard guard(b->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int ns = (int)b->shots.size();
    if (b->mode == MMOD_BATCH_STREAMS) {
        for (int i = 0; i < ns; ++i)
            if (!b->shots[i]->model_set) return bfail(b, MMOD_ERR_STATE, "shot " + std::to_string(i) + " has no model");
        cudaEvent_t e0, e1;
        BCK(b, cudaEventCreate(&e0));
        BCK(b, cudaEventCreate(&e1));
        int best = kTmaDefaultVariant;
        float best_ms = 1e30f;
        mmod_status st = MMOD_OK;
        for (int v = 0; v < tma_variant_count() && st == MMOD_OK; ++v) {
            for (mmod_handle *h : b->shots) h->variant = v;
            float ms = -1.0f;
            for (int rep = 0; rep < 2 && st == MMOD_OK; ++rep) {   // the first repetition warms up
                if (cudaEventRecord(e0, s) != cudaSuccess) st = MMOD_ERR_CUDA;
                if (st == MMOD_OK) st = fork_streams(b, s);
                for (int i = 0; i < ns && st == MMOD_OK; ++i)
                    st = enqueue_tune_steps(b->shots[i], steps, b->sub[i % kSubStreams]);
                if (st == MMOD_OK) st = join_streams(b, s);
                if (st == MMOD_OK && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                                      cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
                    st = MMOD_ERR_CUDA;
            }
            if (st == MMOD_OK && ms > 0 && ms < best_ms) {
                best_ms = ms;
                best = v;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        for (mmod_handle *h : b->shots) h->variant = best;
        if (st != MMOD_OK) return bfail(b, st, "autotuning the batch failed");
        b->variant = best;
        b->variant_set = true;
        if (variant_out) *variant_out = best;
        return MMOD_OK;
    }
    for (int i = 0; i < ns; ++i) {
        if (!b->shots[i]->model_set) return bfail(b, MMOD_ERR_STATE, "shot " + std::to_string(i) + " has no model");
        b->desc[i].args.wavelet = nullptr;   // no sources while tuning
        b->desc[i].args.inj.npts = 0;
        b->desc[i].traces = nullptr;
        b->desc[i].args.err = b->shots[i]->err_dev;
        b->desc[i].args.pdl = b->pdl;
    }
    BCK(b, cudaMemcpyAsync(b->d_desc, b->desc.data(), sizeof(ShotDesc) * ns, cudaMemcpyHostToDevice, s));
    const int keep = b->variant;
    int best = keep;
    float best_ms = 1e30f;
    for (int v = 0; v < tma_variant_count(); ++v) {
        b->variant = v;
        mmod_status st;
        time_steps(b, std::min(2, steps), s, &st);   // warm-up
        const float ms = time_steps(b, steps, s, &st);
        if (st != MMOD_OK) {
            b->variant = keep;
            return st;
        }
        if (ms > 0 && ms < best_ms) {
            best_ms = ms;
            best = v;
        }
    }
    for (int i = 0; i < ns; ++i) b->desc[i].args.inj.npts = b->shots[i]->fwd.inj.npts;
    b->variant = best;
    if (variant_out) *variant_out = best;
    return MMOD_OK;
}

MMOD_API mmod_status mmod_autotune(mmod_handle *h, int steps, mmod_stream stream, int *variant_out) {
    if (!h || steps < 1) return MMOD_ERR_ARG;
    if (mmod_status st = check_latched(h)) return st;
    if (!h->model_set) return fail(h, MMOD_ERR_STATE, "mmod_set_model has not succeeded");
    if (!h->tma_ok) return fail(h, MMOD_ERR_UNSUPPORTED, "TMA kernel unavailable for this grid");
    DeviceGuard guard(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    int best = kTmaDefaultVariant;
    float best_ms = 1e30f;
    cudaEvent_t e0, e1;
    MMOD_CK(h, cudaEventCreate(&e0));
    MMOD_CK(h, cudaEventCreate(&e1));
    for (int v = 0; v < tma_variant_count(); ++v) {
        h->variant = v;
        float ms = 0.0f;
        for (int rep = 0; rep < 2; ++rep) {   // the first repetition warms up
            MMOD_CK(h, cudaEventRecord(e0, s));
            if (mmod_status st = enqueue_tune_steps(h, steps, s)) return st;
            MMOD_CK(h, cudaEventRecord(e1, s));
            MMOD_CK(h, cudaEventSynchronize(e1));
            MMOD_CK(h, cudaEventElapsedTime(&ms, e0, e1));
        }
        if (ms < best_ms) {
            best_ms = ms;
            best = v;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->variant = best;
    if (variant_out) *variant_out = best;
    return check_latched(h);
}
