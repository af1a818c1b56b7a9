// C ABI of the propagator (include/mmod.h): validation, the handle, the
// source/receiver geometry, staging of host buffers, the CUDA-graph-captured
// time loop (Alg. 1) and error latching.  The adjoint and gradient entry
// points are in mmod_adjoint.cu.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "mmod_handle.h"

#define MMOD_API extern "C" __attribute__((visibility("default")))

using namespace mmod;

namespace {

// Defaults of the tuning options (see mmod_set_option).
constexpr int kDefaultPdl = 1;   // measured +1% on 240^3
constexpr int kDefaultPersistent = 0;   // slower than one launch per step on 240^3 (55 vs 45.5 us)

// Message of the calling thread's last failure outside a handle (mmod_create,
// mmod_forward_noalloc); a fixed buffer, so recording it never allocates.
thread_local char g_thread_err[256] = "";

void set_thread_error_str(const std::string &msg) { set_thread_error(msg.c_str()); }

bool in_grid(const mmod_config &c, const int *p) {
    return p[0] >= 0 && p[0] < c.nx && p[1] >= 0 && p[1] < c.ny && p[2] >= 0 && p[2] < c.nz;
}

std::string validate(const mmod_config *c, mmod_status *st) {
    *st = MMOD_ERR_ARG;
    if (!c) return "null config";
    if (c->nx < 1 || c->ny < 1 || c->nz < 1) return "grid sizes must be >= 1";
    if ((long long)c->nx * c->ny * c->nz > (1LL << 36)) return "grid too large";
    if (!(c->hx > 0 && c->hy > 0 && c->hz > 0) || !std::isfinite(c->hx) ||
        !std::isfinite(c->hy) || !std::isfinite(c->hz))
        return "grid spacings must be positive and finite";
    if (!(c->dt > 0) || !std::isfinite(c->dt)) return "dt must be positive and finite";
    if (c->nt < 0) return "nt must be >= 0";
    if (c->nbl < 0 || 2LL * c->nbl > c->nx || 2LL * c->nbl > c->ny || 2LL * c->nbl > c->nz)
        return "damping width must satisfy 0 <= 2*nbl <= n on every axis";
    if (c->nbl > 0 && !(c->damp_R > 0 && c->damp_R < 1)) return "damp_R must be in (0, 1)";
    if (c->nsrc < 0 || c->nrec < 0) return "negative source/receiver count";
    if (c->nsrc > 0 && !c->src_ijk) return "null source list";
    if (c->nrec > 0 && !c->rec_ijk) return "null receiver list";
    for (int s = 0; s < c->nsrc; ++s)
        if (!in_grid(*c, c->src_ijk + 3 * s)) return "source " + std::to_string(s) + " outside the grid";
    for (int r = 0; r < c->nrec; ++r)
        if (!in_grid(*c, c->rec_ijk + 3 * r)) return "receiver " + std::to_string(r) + " outside the grid";
    if (c->free_surface != 0 && c->free_surface != 1) return "free_surface must be 0 or 1";
    if (c->boundary != MMOD_BOUNDARY_DAMPING && c->boundary != MMOD_BOUNDARY_CPML) return "unknown boundary";
    if (c->boundary == MMOD_BOUNDARY_CPML && !(c->cpml_f0 >= 0.0 && std::isfinite(c->cpml_f0)))
        return "cpml_f0 must be finite and >= 0";
    if (c->free_surface && c->nz < kRadius + 1) return "a free surface needs nz >= 5";
    if (c->order != 8) {
        *st = MMOD_ERR_UNSUPPORTED;
        return "the GPU path implements order 8 only";
    }
    *st = MMOD_OK;
    return "";
}

void free_inj(DevInj &t) {
    for (int *p : {t.tile_start, t.pt_i, t.pt_j, t.pt_k, t.pt_first, t.src_row, t.src_i, t.src_j, t.src_k})
        if (p) cudaFree(p);
    if (t.pt_off) cudaFree(t.pt_off);
    if (t.src_scale) cudaFree(t.src_scale);
    t = DevInj();
}

void free_graph(GraphSlot &g) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g = GraphSlot();
}

void free_all(mmod_handle *h) {
    free_graph(h->g_fwd);
    free_graph(h->g_adj);
    free_grad_work(h);
    for (float *p : {h->u[0], h->u[1], h->c, h->eta, h->vel_copy, h->st_vol, h->st_wav, h->st_tr, h->st_adjw,
                     h->st_adjg, h->st_adjo})
        if (p) cudaFree(p);
    free_inj(h->fwd.inj);
    free_inj(h->adj.inj);
    for (Geometry *g : {&h->fwd, &h->adj}) {
        if (g->gather_off) cudaFree(g->gather_off);
        if (g->g_start) cudaFree(g->g_start);
        if (g->g_idx) cudaFree(g->g_idx);
        if (g->g_off) cudaFree(g->g_off);
    }
    if (h->counters) cudaFree(h->counters);
    if (h->claim_ctr) cudaFree(h->claim_ctr);
    if (h->queue) cudaFree(h->queue);
    if (h->cpml_mem) cudaFree(h->cpml_mem);
    if (h->cpml_bg) cudaFree(h->cpml_bg);
    if (h->cpml_xc) cudaFree(h->cpml_xc);
    if (h->vmax_bits) cudaFree(h->vmax_bits);
    if (h->bad) cudaFree(h->bad);
    if (h->ev_t0) cudaEventDestroy(h->ev_t0);
    if (h->ev_t1) cudaEventDestroy(h->ev_t1);
    for (cudaEvent_t e : h->ev_rows)
        if (e) cudaEventDestroy(e);
    if (h->ev_copied) cudaEventDestroy(h->ev_copied);
    if (h->st_copy) cudaStreamDestroy(h->st_copy);
    if (h->cap) cudaStreamDestroy(h->cap);
    if (h->err_host) cudaFreeHost(h->err_host);
}

template <class T>
cudaError_t upload(T **dst, const std::vector<T> &v) {
    const size_t n = std::max<size_t>(v.size(), 1);
    cudaError_t e = cudaMalloc(dst, sizeof(T) * n);
    if (e != cudaSuccess) return e;
    if (v.empty()) return cudaMemset(*dst, 0, sizeof(T));
    return cudaMemcpy(*dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice);
}

// Injection table of the positions pos[n][3]: sources grouped by grid point
// (stable order), points sorted by (tile, plane, j, i) and bucketed per
// (64 x 16 tile, plane).  src_row = index of the position in pos.
cudaError_t build_inj(const mmod_config &c, long long plane, int nxp, const int *pos, int n, DevInj *t) {
    t->tiles_x = (c.nx + kInjTileX - 1) / kInjTileX;
    t->tiles_y = (c.ny + kInjTileY - 1) / kInjTileY;
    const long long tiles = (long long)t->tiles_x * t->tiles_y;
    auto bucket = [&](int s) {
        const int *p = pos + 3 * s;
        return ((long long)(p[1] / kInjTileY) * t->tiles_x + p[0] / kInjTileX) * c.nz + p[2];
    };
    // with a free surface, positions on the plane k = 0 inject nothing
    std::vector<int> order;
    for (int q = 0; q < n; ++q)
        if (!(c.free_surface && pos[3 * q + 2] == 0)) order.push_back(q);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        const long long ba = bucket(a), bb = bucket(b);
        if (ba != bb) return ba < bb;
        const int *pa = pos + 3 * a, *pb = pos + 3 * b;
        if (pa[1] != pb[1]) return pa[1] < pb[1];
        return pa[0] < pb[0];
    });
    const int m = (int)order.size();
    std::vector<int> pt_i, pt_j, pt_k, pt_first, src_row(m), si(m), sj(m), sk(m);
    std::vector<long long> pt_off;
    std::vector<int> tile_start((size_t)(c.nz * tiles + 1), 0);
    for (int q = 0; q < m; ++q) {
        const int s = order[q];
        const int *p = pos + 3 * s;
        src_row[q] = s;
        si[q] = p[0];
        sj[q] = p[1];
        sk[q] = p[2];
        const bool same = q > 0 && std::memcmp(pos + 3 * order[q - 1], p, 3 * sizeof(int)) == 0;
        if (!same) {
            pt_i.push_back(p[0]);
            pt_j.push_back(p[1]);
            pt_k.push_back(p[2]);
            pt_off.push_back((long long)p[2] * plane + (long long)p[1] * nxp + p[0]);
            pt_first.push_back(q);
            tile_start[(size_t)bucket(s) + 1]++;
        }
    }
    pt_first.push_back(m);
    for (size_t b = 1; b < tile_start.size(); ++b) tile_start[b] += tile_start[b - 1];
    t->npts = (int)pt_i.size();
    t->nsrc = m;
    cudaError_t e;
    if ((e = upload(&t->tile_start, tile_start)) || (e = upload(&t->pt_i, pt_i)) || (e = upload(&t->pt_j, pt_j)) ||
        (e = upload(&t->pt_k, pt_k)) || (e = upload(&t->pt_off, pt_off)) || (e = upload(&t->pt_first, pt_first)) ||
        (e = upload(&t->src_row, src_row)) || (e = upload(&t->src_i, si)) || (e = upload(&t->src_j, sj)) ||
        (e = upload(&t->src_k, sk)))
        return e;
    e = cudaMalloc(&t->src_scale, sizeof(float) * std::max(m, 1));
    if (e != cudaSuccess) return e;
    return cudaMemset(t->src_scale, 0, sizeof(float) * std::max(m, 1));
}

// Gather positions pos[n][3] bucketed per (64 x 16 tile, plane), tile-major
// as the injection table: entries [start[b], start[b+1]) of bucket
// b = tile * nz + k hold the original index and the padded offset.
cudaError_t build_gather_buckets(const mmod_config &c, long long plane, int nxp, const int *pos, int n,
                                 Geometry *g) {
    const int tiles_x = (c.nx + kInjTileX - 1) / kInjTileX, tiles_y = (c.ny + kInjTileY - 1) / kInjTileY;
    auto bucket = [&](int r) {
        const int *p = pos + 3 * r;
        return ((long long)(p[1] / kInjTileY) * tiles_x + p[0] / kInjTileX) * c.nz + p[2];
    };
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return bucket(a) < bucket(b); });
    std::vector<int> start((size_t)tiles_x * tiles_y * c.nz + 1, 0), idx(n);
    std::vector<long long> off(n);
    for (int q = 0; q < n; ++q) {
        const int r = order[q];
        const int *p = pos + 3 * r;
        idx[q] = r;
        off[q] = (long long)p[2] * plane + (long long)p[1] * nxp + p[0];
        start[(size_t)bucket(r) + 1]++;
    }
    for (size_t b = 1; b < start.size(); ++b) start[b] += start[b - 1];
    cudaError_t e;
    if ((e = upload(&g->g_start, start)) || (e = upload(&g->g_idx, idx)) || (e = upload(&g->g_off, off))) return e;
    return cudaSuccess;
}

cudaError_t build_gather(long long plane, int nxp, const int *pos, int n, long long **off) {
    std::vector<long long> o(n);
    for (int r = 0; r < n; ++r) o[r] = (long long)pos[3 * r + 2] * plane + (long long)pos[3 * r + 1] * nxp + pos[3 * r];
    return upload(off, o);
}

}  // namespace

namespace mmod {

void set_thread_error(const char *msg) {
    std::snprintf(g_thread_err, sizeof(g_thread_err), "%s", msg ? msg : "");
}

// Damping profile of one axis (the ABI's reading of the layers), FP64 -> FP32
// after multiplying by dt.
void damping_profile(int n, int nbl, double h, double vmax, double R, double dt, float *out) {
    if (nbl == 0) {
        std::fill(out, out + n, 0.0f);
        return;
    }
    const double eta_max = 1.5 * vmax * std::log(1.0 / R) / (nbl * h);
    for (int i = 0; i < n; ++i) {
        const int d = std::max({nbl - i, i - (n - 1 - nbl), 0});
        const double s = (double)d / nbl;
        out[i] = (float)(dt * eta_max * s * s);
    }
}

// CPML coefficients of one axis: b = exp(-(d + alpha) dt), g = d (b - 1) /
// (d + alpha) with d = d0 (x/L)^2, alpha = pi f0 (1 - x/L), x the depth into
// the layer (L at the outer cell, 0 from cell L inward); b = 1, g = 0
// elsewhere.  top_free drops the layer at index 0 (free surface).
void cpml_profile(int n, int L, double h, double vmax, double R, double f0, double dt, bool top_free, float *b,
                  float *g) {
    const double d0 = L > 0 ? 3.0 * vmax * std::log(1.0 / R) / (2.0 * L * h) : 0.0;
    for (int i = 0; i < n; ++i) {
        const int x = std::max({top_free ? 0 : L - i, i - (n - 1 - L), 0});
        if (L == 0 || x == 0) {
            b[i] = 1.0f;
            g[i] = 0.0f;
            continue;
        }
        const double sx = (double)x / L, d = d0 * sx * sx, alpha = M_PI * f0 * (1.0 - sx);
        const double bb = std::exp(-(d + alpha) * dt);
        b[i] = (float)bb;
        g[i] = (float)(d * (bb - 1.0) / (d + alpha));
    }
}

CpmlArgs cpml_args(const mmod_handle *h) {
    const auto &c = h->cfg;
    CpmlArgs p{};
    p.nx = c.nx; p.ny = c.ny; p.nz = c.nz; p.nxp = h->nxp; p.plane = h->plane; p.fs = c.free_surface;
    p.nbl = c.nbl;
    const size_t n3 = (size_t)(c.nx + c.ny + c.nz);
    const int off[3] = {0, c.nx, c.nx + c.ny};
    for (int a = 0; a < 3; ++a) {
        p.psi[a] = h->cpml_mem + (size_t)a * h->vol;
        p.zeta[a] = h->cpml_mem + (size_t)(3 + a) * h->vol;
        p.b[a] = h->cpml_bg + off[a];
        p.g[a] = h->cpml_bg + n3 + off[a];
    }
    p.inv_h[0] = (float)(1.0 / c.hx); p.inv_h[1] = (float)(1.0 / c.hy); p.inv_h[2] = (float)(1.0 / c.hz);
    for (int m = 0; m < kRadius; ++m) {
        p.w[0][m] = h->w.x[m]; p.w[1][m] = h->w.y[m]; p.w[2][m] = h->w.z[m];
    }
    p.c = h->c;
    p.zc = h->cpml_planes > 0 ? h->cpml_planes : kCpmlPlanes;
    p.tiles = h->cpml_tiles_on;
    p.err = h->err_dev;
    p.xc = h->cpml_xc;
    return p;
}

void clear_surface_layer(int nz, int nbl, float *ez) {
    for (int k = 0; k < nbl && k < nz - 1 - nbl; ++k) ez[k] = 0.0f;
}

mmod_status fail(mmod_handle *h, mmod_status st, const std::string &msg) {
    if (h) h->err = msg;
    return st;
}

mmod_status fail_cuda(mmod_handle *h, cudaError_t e, const char *what) {
    if (h) {
        if (h->latched == cudaSuccess) h->latched = e;
        h->err = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    }
    return e == cudaErrorMemoryAllocation ? MMOD_ERR_OOM : MMOD_ERR_CUDA;
}

mmod_status check_latched(mmod_handle *h) {
    if (h->err_host && *(volatile int *)h->err_host) {
        h->err = "a step kernel gave up waiting for its copies (device-side timeout)";
        return MMOD_ERR_TIMEOUT;
    }
    if (h->latched != cudaSuccess) {
        h->err = std::string("earlier CUDA failure: ") + cudaGetErrorName(h->latched);
        return MMOD_ERR_CUDA;
    }
    return MMOD_OK;
}

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

bool use_tma(const mmod_handle *h) { return h->tma_ok && h->kernel != MMOD_KERNEL_SIMPLE; }

void drop_graphs(mmod_handle *h) {
    free_graph(h->g_fwd);
    free_graph(h->g_adj);
}

// CTAs of the persistent kernel for the next run (0: one launch per step).
int persistent_grid_of(const mmod_handle *h) {
    if (!use_tma(h) || !h->persistent || !h->counters || is_cpml(h)) return 0;
    const TmaPlan &plan = active_plan(h);
    const Geom g = persistent_geom(plan, h->cfg.nz);
    if ((long long)g.tiles_x * g.tiles_y * g.zchunks > h->ncounters) return 0;
    return persistent_grid(plan, h->cfg.nz, h->persistent_ctas);
}

// The plan of variant v with the handle's z-range and work-claiming options.
static const TmaPlan &plan_with_options(const mmod_handle *h, int v, TmaPlan &q) {
    const TmaPlan &p = h->plans[v];
    if (h->zlen_override <= 0 && h->claim_planes <= 0) return p;
    q = p;
    if (h->zlen_override > 0) {   // MMOD_OPT_ZLEN: the same tiles, z ranges of the requested thickness
        q.zlen = std::min(h->zlen_override, h->cfg.nz);
        q.zchunks = (h->cfg.nz + q.zlen - 1) / q.zlen;
        q.grid = q.tiles_x * q.tiles_y * q.zchunks;
    }
    q.claim = h->claim_planes;   // MMOD_OPT_CLAIM: units of this many planes, claimed by one wave of CTAs
    return q;
}

const TmaPlan &active_plan(const mmod_handle *h) {
    return plan_with_options(h, h->variant >= 0 ? h->variant : kTmaDefaultVariant, h->plan_tmp);
}

// Steps that also write g^n run the variant compiled with that output (the
// same bits as every other variant).
static const TmaPlan &g_plan(const mmod_handle *h) { return plan_with_options(h, kTmaGVariant, h->plan_tmp_g); }

// Step arguments shared by every step of a run (n, buffers and gathers are
// filled per step).
StepArgs base_args(mmod_handle *h, const Geometry &geo, const float *wavelet) {
    StepArgs a{};
    a.nx = h->cfg.nx; a.ny = h->cfg.ny; a.nz = h->cfg.nz;
    a.nxp = h->nxp; a.plane = h->plane; a.nbl = h->cfg.nbl; a.nt = h->cfg.nt;
    a.w = h->w;
    a.c = h->c;
    a.ex = h->eta; a.ey = h->eta + h->cfg.nx; a.ez = h->eta + h->cfg.nx + h->cfg.ny;
    a.inj = geo.inj.view();
    a.wavelet = wavelet;
    a.wrs = h->cfg.nt;
    a.wcs = 1;
    if (&geo == &h->adj && wavelet) {
        // the adjoint's injection points are the receivers and its wavelet
        // the residual [nt][nrec] in time order: step n reads row nt-1-n
        a.wavelet = wavelet + (long long)(h->cfg.nt - 1) * h->cfg.nrec;
        a.wrs = 1;
        a.wcs = -(long long)h->cfg.nrec;
    }
    a.nrec = geo.ngather; a.rec_off = geo.gather_off;
    a.traces = nullptr;
    a.err = h->err_dev;
    a.fs = h->cfg.free_surface;
    a.pdl = h->pdl;
    a.claim = h->claim_ctr;
    return a;
}

// Enqueue one step of a run on stream s.  Plain path: step kernel, then the
// injection kernel, then (if plain_gather_dst) the receivers of u^{n+1}.
// TMA path: one kernel (injection inside; receivers of u^n go to a.traces).
cudaError_t enqueue_step(mmod_handle *h, const StepArgs &a, const CUtensorMap *cur, const CUtensorMap *prev,
                         bool tma, float *plain_gather_dst, cudaStream_t s, long long *count) {
    cudaError_t e;
    if (tma) {
        e = launch_step_tma(a, cur, prev, &h->c_map, a.gout ? g_plan(h) : active_plan(h), s);
        ++*count;
        return e;
    }
    StepArgs b = a;
    b.traces = nullptr;
    if ((e = launch_step_simple(b, s)) != cudaSuccess) return e;
    ++*count;
    if (a.inj.npts > 0) {
        if ((e = launch_inject(b, s)) != cudaSuccess) return e;
        ++*count;
    }
    if (plain_gather_dst && a.nrec > 0) {
        if ((e = launch_gather(a.uout, a.rec_off, a.nrec, plain_gather_dst, s)) != cudaSuccess) return e;
        ++*count;
    }
    return cudaSuccess;
}

// The time loop of a run from the state in u[0] (u^{-1}) and u[1] (u^0): nt
// steps with the geometry geo, traces [nt][ngather] (nullable), bracketed by
// the loop events.  Returns the number of kernels launched in *count.
static mmod_status enqueue_loop(mmod_handle *h, const Geometry &geo, const float *wav, float *tr, cudaStream_t s,
                                long long *count) {
    const int nt = h->cfg.nt, ng = geo.ngather;
    const bool tma = use_tma(h);
    *count = 0;
    MMOD_CK(h, cudaEventRecordWithFlags(h->ev_t0, s, cudaEventRecordExternal));
    // trace rows [0, done) are final: record the chunk events that wait for them
    const bool marks = tr && ng > 0 && &geo == &h->fwd;
    int next_mark = 0;
    auto mark = [&](long long done) -> cudaError_t {
        for (; marks && next_mark < mmod_handle::kTraceChunks && h->rows_at[next_mark] <= done; ++next_mark)
            if (cudaError_t e = cudaEventRecordWithFlags(h->ev_rows[next_mark], s, cudaEventRecordExternal))
                return e;
        return cudaSuccess;
    };
    MMOD_CK(h, mark(0));
    StepArgs a = base_args(h, geo, wav);
    if (is_cpml(h)) {
        // CPML: the undamped step (sources included), the layer terms of
        // u^{n+1}, then (plain kernel) the receivers of u^{n+1}
        // with PDL each kernel requests the data its predecessors do not
        // write before its wait: the step kernel c and u^{n-1} (the layer
        // passes only read u^n), a tiled pass u^n, psi_a, zeta_a and c
        CpmlArgs cp = cpml_args(h);
        cp.pdl = h->pdl;
        a.pdl = h->pdl ? 2 : 0;
        for (int n = 0; n < nt; ++n) {
            a.n = n;
            a.ucur = h->u[(n + 1) & 1];
            a.uprev = h->u[n & 1];
            a.uout = h->u[n & 1];
            a.traces = (n >= 1 && tr && ng > 0) ? tr + (long long)(n - 1) * ng : nullptr;
            MMOD_CK(h, enqueue_step(h, a, &h->cur_map[(n + 1) & 1], &h->prev_map[n & 1], tma, nullptr, s, count));
            int passes = 0;
            MMOD_CK(h, launch_cpml_layers(cp, &h->cpml_tiles, (n + 1) & 1, a.ucur, a.uout, s, &passes));
            *count += passes;
            if (!tma && tr && ng > 0) {
                MMOD_CK(h, launch_gather(a.uout, geo.gather_off, ng, tr + (long long)n * ng, s));
                ++*count;
            }
            MMOD_CK(h, mark(tma ? n : n + 1));
        }
        if (tma && nt > 0 && ng > 0 && tr) {
            MMOD_CK(h, launch_gather(h->u[(nt - 1) & 1], geo.gather_off, ng, tr + (long long)(nt - 1) * ng, s));
            ++*count;
        }
        MMOD_CK(h, mark(nt));
        MMOD_CK(h, cudaEventRecordWithFlags(h->ev_t1, s, cudaEventRecordExternal));
        return MMOD_OK;
    }
    // inside the loop every step kernel follows the previous step (the
    // first follows no kernel of the captured graph)
    if (a.pdl) a.pdl = 2;
    for (int n = 0; n < nt; ++n) {
        a.n = n;
        a.ucur = h->u[(n + 1) & 1];
        a.uprev = h->u[n & 1];
        a.uout = h->u[n & 1];
        a.traces = (n >= 1 && tr && ng > 0) ? tr + (long long)(n - 1) * ng : nullptr;
        MMOD_CK(h, enqueue_step(h, a, &h->cur_map[(n + 1) & 1], &h->prev_map[n & 1], tma,
                                (tr && ng > 0) ? tr + (long long)n * ng : nullptr, s, count));
        MMOD_CK(h, mark(tma ? n : n + 1));   // the TMA kernel of step n gathers row n - 1
    }
    if (tma && nt > 0 && ng > 0 && tr) {
        // u^{nt} sits in u[(nt - 1) & 1]; the last step kernel had no successor
        MMOD_CK(h, launch_gather(h->u[(nt - 1) & 1], geo.gather_off, ng, tr + (long long)(nt - 1) * ng, s));
        ++*count;
    }
    MMOD_CK(h, mark(nt));
    MMOD_CK(h, cudaEventRecordWithFlags(h->ev_t1, s, cudaEventRecordExternal));
    return MMOD_OK;
}

// Launch the cached graph of a loop, capturing it first when its inputs
// changed.
mmod_status run_loop_graph(mmod_handle *h, GraphSlot &g, const Geometry &geo, const float *wav, float *tr,
                           cudaStream_t s, long long *launches) {
    const int pgrid = persistent_grid_of(h);
    if (pgrid > 0 && h->cfg.nt > 0) {
        // one cooperative launch for the whole loop: no graph needed
        const TmaPlan &plan = active_plan(h);
        const Geom pg = persistent_geom(plan, h->cfg.nz);
        const int units = pg.tiles_x * pg.tiles_y * pg.zchunks;
        MMOD_CK(h, cudaMemsetAsync(h->counters, 0, sizeof(int) * (size_t)units, s));
        MMOD_CK(h, cudaMemsetAsync(h->queue, 0, sizeof(unsigned long long), s));
        MMOD_CK(h, cudaEventRecord(h->ev_t0, s));
        StepArgs a = base_args(h, geo, wav);
        a.pdl = 0;
        PersistArgs pa{};
        // MMOD_OPT_TEST_STALL: start at step 1 with the counters at 0, so
        // every unit waits for neighbours that never signal and gives up
        pa.n0 = h->test_stall ? 1 : 0;
        h->test_stall = 0;
        pa.n1 = h->cfg.nt;
        pa.units = units;
        pa.counters = h->counters;
        pa.queue = h->queue;
        pa.rec_start = geo.g_start;
        pa.rec_idx = geo.g_idx;
        pa.rec_off = geo.g_off;
        pa.traces = geo.ngather > 0 ? tr : nullptr;
        pa.nrec = geo.ngather;
        pa.u[0] = h->u[0];
        pa.u[1] = h->u[1];
        TmaMaps maps;
        for (int b = 0; b < 2; ++b) {
            maps.cur[b] = h->cur_map[b];
            maps.prev[b] = h->prev_map[b];
        }
        maps.c = h->c_map;
        MMOD_CK(h, launch_step_tma_persistent(a, maps, plan, pa, pgrid, s));
        MMOD_CK(h, cudaEventRecord(h->ev_t1, s));
        *launches += 1;
        return MMOD_OK;
    }
    const int kern = use_tma(h) ? 100 + active_plan(h).variant : MMOD_KERNEL_SIMPLE;
    const long long opts = h->pdl + 2LL * h->zlen_override + (1LL << 20) * h->claim_planes +
                           (1LL << 40) * h->cpml_planes;
    const void *key[4] = {wav, tr, &geo, nullptr};
    if (!g.exec || std::memcmp(g.key, key, sizeof(key)) != 0 || g.kernel != kern || g.opts != opts) {
        free_graph(g);
        cudaGraph_t graph = nullptr;
        MMOD_CK(h, cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
        long long n_l = 0;
        mmod_status st = enqueue_loop(h, geo, wav, tr, h->cap, &n_l);
        cudaError_t e_end = cudaStreamEndCapture(h->cap, &graph);
        if (st != MMOD_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        if (e_end != cudaSuccess) return fail_cuda(h, e_end, "cudaStreamEndCapture");
        cudaError_t e_inst = cudaGraphInstantiate(&g.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e_inst != cudaSuccess) {
            g.exec = nullptr;
            return fail_cuda(h, e_inst, "cudaGraphInstantiate");
        }
        std::memcpy(g.key, key, sizeof(key));
        g.kernel = kern;
        g.opts = opts;
        g.launches = n_l;
    }
    MMOD_CK(h, cudaGraphLaunch(g.exec, s));
    *launches += g.launches;
    return MMOD_OK;
}

}  // namespace mmod

MMOD_API double mmod_cfl_dt(double cfl, double hmin, double vmax) {
    if (!(cfl > 0) || !(hmin > 0) || !(vmax > 0)) return -1.0;
    return cfl * hmin / vmax;
}

MMOD_API const char *mmod_version(void) { return "mmod-gb300 0.2 sm_103a"; }

MMOD_API const char *mmod_last_error(const mmod_handle *h) { return h ? h->err.c_str() : g_thread_err; }

MMOD_API long long mmod_last_launch_count(const mmod_handle *h) { return h ? h->last_launches : -1; }

MMOD_API mmod_status mmod_create(const mmod_config *cfg, int device, mmod_handle **out) {
    set_thread_error("");
    if (!out) {
        set_thread_error("null output pointer");
        return MMOD_ERR_ARG;
    }
    *out = nullptr;
    mmod_status st;
    const std::string why = validate(cfg, &st);
    if (st != MMOD_OK) {
        set_thread_error_str(why);
        return st;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        set_thread_error_str("CUDA device " + std::to_string(device) + " not available");
        return MMOD_ERR_CUDA;
    }
    DeviceGuard guard(device);
    mmod_handle *h = new (std::nothrow) mmod_handle();
    if (!h) return MMOD_ERR_OOM;
    h->cfg = *cfg;
    h->device = device;
    h->pdl = kDefaultPdl;
    h->persistent = kDefaultPersistent;
    h->src.assign(cfg->src_ijk, cfg->src_ijk + 3 * (size_t)cfg->nsrc);
    h->rec.assign(cfg->rec_ijk, cfg->rec_ijk + 3 * (size_t)cfg->nrec);
    h->cfg.src_ijk = h->src.data();
    h->cfg.rec_ijk = h->rec.data();
    const int nx = cfg->nx, ny = cfg->ny, nz = cfg->nz;
    h->nxp = (nx + 31) / 32 * 32;
    h->plane = (long long)h->nxp * ny;
    h->vol = h->plane * nz;
    h->npts = (long long)nx * ny * nz;
    set_weights(h, kTaylor8);

    auto bail = [&](cudaError_t e, const char *what) {
        set_thread_error_str(std::string(what) + ": " + cudaGetErrorString(e));
        free_all(h);
        delete h;
        return e == cudaErrorMemoryAllocation ? MMOD_ERR_OOM : MMOD_ERR_CUDA;
    };
#define CKC(call)                                  \
    do {                                           \
        cudaError_t _e = (call);                   \
        if (_e != cudaSuccess) return bail(_e, #call); \
    } while (0)

    const size_t vbytes = sizeof(float) * (size_t)h->vol;
    CKC(cudaMalloc(&h->u[0], vbytes));
    CKC(cudaMalloc(&h->u[1], vbytes));
    CKC(cudaMalloc(&h->c, vbytes));
    CKC(cudaMalloc(&h->eta, sizeof(float) * (size_t)(nx + ny + nz)));
    CKC(cudaMemset(h->u[0], 0, vbytes));
    CKC(cudaMemset(h->u[1], 0, vbytes));
    CKC(cudaMemset(h->c, 0, vbytes));
    CKC(cudaMemset(h->eta, 0, sizeof(float) * (size_t)(nx + ny + nz)));
    if (is_cpml(h)) {
        CKC(cudaMalloc(&h->cpml_mem, 6 * vbytes));
        CKC(cudaMemset(h->cpml_mem, 0, 6 * vbytes));
        CKC(cudaMalloc(&h->cpml_bg, sizeof(float) * 2 * (size_t)(nx + ny + nz)));
        CKC(cudaMemset(h->cpml_bg, 0, sizeof(float) * 2 * (size_t)(nx + ny + nz)));
        h->cpml_xc_floats = cpml_x_compact_floats(cpml_args(h));
        if (h->cpml_xc_floats > 0) {
            CKC(cudaMalloc(&h->cpml_xc, sizeof(float) * (size_t)h->cpml_xc_floats));
            CKC(cudaMemset(h->cpml_xc, 0, sizeof(float) * (size_t)h->cpml_xc_floats));
        }
    }
    CKC(cudaMalloc(&h->vmax_bits, sizeof(unsigned int)));
    CKC(cudaMalloc(&h->bad, sizeof(unsigned long long)));
    // forward: sources injected, receivers gathered; adjoint: the reverse
    CKC(build_inj(h->cfg, h->plane, h->nxp, h->src.data(), cfg->nsrc, &h->fwd.inj));
    CKC(build_gather(h->plane, h->nxp, h->rec.data(), cfg->nrec, &h->fwd.gather_off));
    h->fwd.ngather = cfg->nrec;
    h->fwd.cell = cfg->hx * cfg->hy * cfg->hz;
    CKC(build_inj(h->cfg, h->plane, h->nxp, h->rec.data(), cfg->nrec, &h->adj.inj));
    CKC(build_gather(h->plane, h->nxp, h->src.data(), cfg->nsrc, &h->adj.gather_off));
    h->adj.ngather = cfg->nsrc;
    h->adj.cell = 1.0;
    CKC(build_gather_buckets(h->cfg, h->plane, h->nxp, h->rec.data(), cfg->nrec, &h->fwd));
    CKC(build_gather_buckets(h->cfg, h->plane, h->nxp, h->src.data(), cfg->nsrc, &h->adj));
    CKC(cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking));
    CKC(cudaEventCreate(&h->ev_t0));
    CKC(cudaEventCreate(&h->ev_t1));
    CKC(cudaStreamCreateWithFlags(&h->st_copy, cudaStreamNonBlocking));
    CKC(cudaEventCreateWithFlags(&h->ev_copied, cudaEventDisableTiming));
    for (int i = 0; i < mmod_handle::kTraceChunks; ++i) {
        CKC(cudaEventCreateWithFlags(&h->ev_rows[i], cudaEventDisableTiming));
        h->rows_at[i] = (long long)cfg->nt * (i + 1) / mmod_handle::kTraceChunks;
    }
    CKC(cudaHostAlloc(&h->err_host, sizeof(int), cudaHostAllocMapped));
    *h->err_host = 0;
    CKC(cudaHostGetDevicePointer(&h->err_dev, h->err_host, 0));
    if (is_cpml(h)) make_cpml_tiles(cpml_args(h), h->u, &h->cpml_tiles);   // axes it cannot tile keep the march
    h->tma_ok = make_tma_plan(h->cfg, h->nxp, h->u, h->c, h->cur_map, h->prev_map, &h->c_map, h->plans);
    if (h->tma_ok) {   // counters of the persistent kernel, sized for the plan with the most units
        for (int v = 0; v < tma_variant_count(); ++v)
            h->ncounters = std::max<long long>(h->ncounters, (long long)h->plans[v].tiles_x * h->plans[v].tiles_y *
                                                                 h->plans[v].zchunks);
        CKC(cudaMalloc(&h->counters, sizeof(int) * (size_t)h->ncounters));
        CKC(cudaMalloc(&h->queue, sizeof(unsigned long long)));
        CKC(cudaMalloc(&h->claim_ctr, 2 * sizeof(int)));
        CKC(cudaMemset(h->claim_ctr, 0, 2 * sizeof(int)));
    }
#undef CKC
    *out = h;
    return MMOD_OK;
}

MMOD_API mmod_status mmod_destroy(mmod_handle *h) {
    if (!h) return MMOD_OK;
    {
        DeviceGuard guard(h->device);
        cudaDeviceSynchronize();
        free_all(h);
    }
    delete h;
    return MMOD_OK;
}

MMOD_API mmod_status mmod_set_kernel(mmod_handle *h, int kernel) {
    if (!h) return MMOD_ERR_ARG;
    if (kernel != MMOD_KERNEL_AUTO && kernel != MMOD_KERNEL_SIMPLE && kernel != MMOD_KERNEL_TMA)
        return fail(h, MMOD_ERR_ARG, "unknown kernel id");
    if (kernel == MMOD_KERNEL_TMA && !h->tma_ok)
        return fail(h, MMOD_ERR_UNSUPPORTED, "TMA kernel unavailable for this grid");
    h->kernel = kernel;
    return MMOD_OK;
}

MMOD_API int mmod_tma_variant_count(void) { return tma_variant_count(); }

MMOD_API const char *mmod_tma_variant_name(int v) { return tma_variant_name(v); }

MMOD_API mmod_status mmod_set_tma_variant(mmod_handle *h, int v) {
    if (!h) return MMOD_ERR_ARG;
    if (v < -1 || v >= tma_variant_count()) return fail(h, MMOD_ERR_ARG, "unknown TMA variant");
    if (v >= 0 && !h->tma_ok) return fail(h, MMOD_ERR_UNSUPPORTED, "TMA kernel unavailable for this grid");
    h->variant = v;
    return MMOD_OK;
}

MMOD_API mmod_status mmod_set_option(mmod_handle *h, int option, int value) {
    if (!h) return MMOD_ERR_ARG;
    if (option == MMOD_OPT_ZLEN) {
        if (value < 0) return fail(h, MMOD_ERR_ARG, "MMOD_OPT_ZLEN must be >= 0");
        h->zlen_override = value;
        return MMOD_OK;
    }
    if (option == MMOD_OPT_CPML_PLANES) {
        if (value < 0 || value > 4096) return fail(h, MMOD_ERR_ARG, "MMOD_OPT_CPML_PLANES must be in [0, 4096]");
        h->cpml_planes = value;
        return MMOD_OK;
    }
    if (option == MMOD_OPT_CPML_TILES) {
        if (value != 0 && value != 1) return fail(h, MMOD_ERR_ARG, "MMOD_OPT_CPML_TILES must be 0 or 1");
        h->cpml_tiles_on = value;
        return MMOD_OK;
    }
    if (option == MMOD_OPT_CLAIM) {
        if (value < 0 || value > 1 << 20) return fail(h, MMOD_ERR_ARG, "MMOD_OPT_CLAIM must be in [0, 2^20]");
        h->claim_planes = value;
        return MMOD_OK;
    }
    if (option == MMOD_OPT_PERSISTENT_CTAS) {
        if (value < 0) return fail(h, MMOD_ERR_ARG, "MMOD_OPT_PERSISTENT_CTAS must be >= 0");
        h->persistent_ctas = value;
        return MMOD_OK;
    }
    if (value != 0 && value != 1) return fail(h, MMOD_ERR_ARG, "option values are 0 or 1");
    switch (option) {
        case MMOD_OPT_PDL: h->pdl = value; return MMOD_OK;
        case MMOD_OPT_CKPT_SCHEME: h->ckpt_scheme = value; return MMOD_OK;
        case MMOD_OPT_PERSISTENT: h->persistent = value; return MMOD_OK;
        case MMOD_OPT_TEST_STALL: h->test_stall = value; return MMOD_OK;
        default: return fail(h, MMOD_ERR_ARG, "unknown option");
    }
}

MMOD_API mmod_status mmod_tma_variant_info(int v, int *out14) {
    if (!out14) return MMOD_ERR_ARG;
    return tma_variant_info(v, out14) ? MMOD_OK : MMOD_ERR_ARG;
}

MMOD_API int mmod_persistent_grid(const mmod_handle *h) {
    if (!h) return -1;
    DeviceGuard guard(h->device);
    return persistent_grid_of(h);
}

MMOD_API mmod_status mmod_get_plan(const mmod_handle *h, int *out8) {
    if (!h || !out8) return MMOD_ERR_ARG;
    if (!h->tma_ok) return MMOD_ERR_UNSUPPORTED;
    const TmaPlan &p = active_plan(h);
    int v[8] = {p.variant, p.tiles_x, p.tiles_y, p.zchunks, p.zlen, p.grid, p.block, p.occupancy};
    Geom cg;
    int units = 0, cgrid = 0;
    if (claim_geom(p, h->cfg.nz, &cg, &units, &cgrid)) {   // a work-claiming launch: its units and grid
        v[3] = cg.zchunks;
        v[4] = cg.zlen;
        v[5] = cgrid;
    }
    for (int i = 0; i < 8; ++i) out8[i] = v[i];
    return MMOD_OK;
}

MMOD_API mmod_status mmod_set_model(mmod_handle *h, const float *vel, mmod_stream stream) {
    if (!h) return MMOD_ERR_ARG;
    if (!vel) return fail(h, MMOD_ERR_ARG, "null velocity");
    if (mmod_status st = check_latched(h)) return st;
    DeviceGuard guard(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    const auto &c = h->cfg;
    const float *dvel = vel;
    if (!is_device_ptr(vel)) {
        if (!h->st_vol) MMOD_CK(h, cudaMalloc(&h->st_vol, sizeof(float) * (size_t)h->npts));
        MMOD_CK(h, cudaMemcpyAsync(h->st_vol, vel, sizeof(float) * (size_t)h->npts, cudaMemcpyHostToDevice, s));
        dvel = h->st_vol;
    }
    MMOD_CK(h, cudaMemsetAsync(h->vmax_bits, 0, sizeof(unsigned int), s));
    MMOD_CK(h, cudaMemsetAsync(h->bad, 0, sizeof(unsigned long long), s));
    MMOD_CK(h, launch_model_scan(dvel, h->npts, h->vmax_bits, h->bad, s));
    unsigned int vbits = 0;
    unsigned long long nbad = 0;
    MMOD_CK(h, cudaMemcpyAsync(&vbits, h->vmax_bits, sizeof(vbits), cudaMemcpyDeviceToHost, s));
    MMOD_CK(h, cudaMemcpyAsync(&nbad, h->bad, sizeof(nbad), cudaMemcpyDeviceToHost, s));
    MMOD_CK(h, cudaStreamSynchronize(s));
    if (nbad) return fail(h, MMOD_ERR_ARG, std::to_string(nbad) + " velocities are not positive and finite");
    float vmaxf;
    std::memcpy(&vmaxf, &vbits, sizeof(vmaxf));
    const double vmax = vmaxf;
    const double ksum = h->symbol_max * (1.0 / (c.hx * c.hx) + 1.0 / (c.hy * c.hy) + 1.0 / (c.hz * c.hz));
    if (c.dt * vmax * std::sqrt(ksum) > 2.0) {
        h->model_set = false;
        return fail(h, MMOD_ERR_UNSTABLE, "dt too large: dt*vmax*sqrt(sum S_max/h^2) = " +
                                              std::to_string(c.dt * vmax * std::sqrt(ksum)) + " > 2");
    }
    MMOD_CK(h, launch_model_fill(dvel, c.nx, c.ny, c.nz, h->nxp, c.dt, h->c, s));
    if (is_cpml(h)) MMOD_CK(h, launch_cpml_pack_c(cpml_args(h), s));
    for (Geometry *g : {&h->fwd, &h->adj})
        MMOD_CK(h, launch_source_scale(dvel, c.nx, c.ny, g->inj.nsrc, g->inj.src_i, g->inj.src_j, g->inj.src_k,
                                       c.dt, g->cell, g->inj.src_scale, s));
    if (!h->vel_copy) MMOD_CK(h, cudaMalloc(&h->vel_copy, sizeof(float) * (size_t)h->npts));
    MMOD_CK(h, cudaMemcpyAsync(h->vel_copy, dvel, sizeof(float) * (size_t)h->npts, cudaMemcpyDeviceToDevice, s));
    std::vector<float> eta(c.nx + c.ny + c.nz);
    damping_profile(c.nx, c.nbl, c.hx, vmax, c.damp_R, c.dt, eta.data());
    damping_profile(c.ny, c.nbl, c.hy, vmax, c.damp_R, c.dt, eta.data() + c.nx);
    damping_profile(c.nz, c.nbl, c.hz, vmax, c.damp_R, c.dt, eta.data() + c.nx + c.ny);
    if (c.free_surface) clear_surface_layer(c.nz, c.nbl, eta.data() + c.nx + c.ny);
    std::vector<float> bg;
    if (is_cpml(h)) {   // the layers are a CPML: no damping term, per-cell b, g per axis
        std::fill(eta.begin(), eta.end(), 0.0f);
        bg.assign(2 * (size_t)(c.nx + c.ny + c.nz), 0.0f);
        const int n3[3] = {c.nx, c.ny, c.nz};
        const double h3[3] = {c.hx, c.hy, c.hz};
        size_t off = 0;
        for (int a = 0; a < 3; ++a) {
            cpml_profile(n3[a], c.nbl, h3[a], vmax, c.damp_R, c.cpml_f0, c.dt, a == 2 && c.free_surface,
                         bg.data() + off, bg.data() + (size_t)(c.nx + c.ny + c.nz) + off);
            off += n3[a];
        }
        MMOD_CK(h, cudaMemcpyAsync(h->cpml_bg, bg.data(), sizeof(float) * bg.size(), cudaMemcpyHostToDevice, s));
    }
    MMOD_CK(h, cudaMemcpyAsync(h->eta, eta.data(), sizeof(float) * eta.size(), cudaMemcpyHostToDevice, s));
    MMOD_CK(h, cudaStreamSynchronize(s));   // eta lives on the host stack
    h->vmax = vmax;
    h->model_set = true;
    return MMOD_OK;
}

MMOD_API mmod_status mmod_set_state(mmod_handle *h, const float *u_prev, const float *u_cur,
                                    mmod_stream stream) {
    if (!h) return MMOD_ERR_ARG;
    if (mmod_status st = check_latched(h)) return st;
    DeviceGuard guard(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    const float *src[2] = {u_prev, u_cur};
    for (int b = 0; b < 2; ++b) {
        const float *d = src[b];
        if (d && !is_device_ptr(d)) {
            if (!h->st_vol) MMOD_CK(h, cudaMalloc(&h->st_vol, sizeof(float) * (size_t)h->npts));
            MMOD_CK(h, cudaMemcpyAsync(h->st_vol, d, sizeof(float) * (size_t)h->npts, cudaMemcpyHostToDevice, s));
            d = h->st_vol;
        }
        // buffer 0 holds u^{n-1}, buffer 1 holds u^n at step 0
        MMOD_CK(h, launch_pack(d, h->cfg.nx, h->cfg.ny, h->cfg.nz, h->nxp, h->u[b], s));
        // a free surface holds p = 0 on its plane from the start
        if (h->cfg.free_surface) MMOD_CK(h, cudaMemsetAsync(h->u[b], 0, sizeof(float) * (size_t)h->plane, s));
    }
    h->state_pending = true;
    return MMOD_OK;
}

MMOD_API mmod_status mmod_get_state(mmod_handle *h, float *u_prev, float *u_cur, mmod_stream stream) {
    if (!h) return MMOD_ERR_ARG;
    if (mmod_status st = check_latched(h)) return st;
    if (!h->ran) return fail(h, MMOD_ERR_STATE, "no forward run yet");
    DeviceGuard guard(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int nt = h->cfg.nt;
    // after nt steps u^{nt} is in buffer (nt+1)&1 and u^{nt-1} in nt&1
    float *dst[2] = {u_prev, u_cur};
    const float *bufs[2] = {h->u[nt & 1], h->u[(nt + 1) & 1]};
    for (int b = 0; b < 2; ++b) {
        if (!dst[b]) continue;
        if (is_device_ptr(dst[b])) {
            MMOD_CK(h, launch_unpack(bufs[b], h->cfg.nx, h->cfg.ny, h->cfg.nz, h->nxp, dst[b], s));
        } else {
            if (!h->st_vol) MMOD_CK(h, cudaMalloc(&h->st_vol, sizeof(float) * (size_t)h->npts));
            MMOD_CK(h, launch_unpack(bufs[b], h->cfg.nx, h->cfg.ny, h->cfg.nz, h->nxp, h->st_vol, s));
            MMOD_CK(h, cudaMemcpyAsync(dst[b], h->st_vol, sizeof(float) * (size_t)h->npts, cudaMemcpyDeviceToHost, s));
            MMOD_CK(h, cudaStreamSynchronize(s));
        }
    }
    return MMOD_OK;
}

MMOD_API mmod_status mmod_forward(mmod_handle *h, const float *wavelet, float *traces, float *final_u,
                                  mmod_stream stream) {
    if (!h) return MMOD_ERR_ARG;
    if (mmod_status st = check_latched(h)) return st;
    if (!h->model_set) return fail(h, MMOD_ERR_STATE, "mmod_set_model has not succeeded");
    const auto &c = h->cfg;
    if (c.nsrc > 0 && c.nt > 0 && !wavelet) return fail(h, MMOD_ERR_ARG, "null wavelet with nsrc > 0");
    if (c.nrec > 0 && c.nt > 0 && !traces) return fail(h, MMOD_ERR_ARG, "null traces with nrec > 0");
    DeviceGuard guard(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    long long launches = 0;

    const float *dwav = wavelet;
    const size_t nwav = (size_t)c.nsrc * c.nt;
    if (c.nsrc > 0 && nwav > 0 && !is_device_ptr(wavelet)) {
        if (!h->st_wav) MMOD_CK(h, cudaMalloc(&h->st_wav, sizeof(float) * nwav));
        MMOD_CK(h, cudaMemcpyAsync(h->st_wav, wavelet, sizeof(float) * nwav, cudaMemcpyHostToDevice, s));
        dwav = h->st_wav;
    }
    float *dtr = traces;
    const bool host_tr = c.nrec > 0 && c.nt > 0 && !is_device_ptr(traces);
    const size_t ntr = (size_t)c.nrec * c.nt;
    if (host_tr) {
        if (!h->st_tr) MMOD_CK(h, cudaMalloc(&h->st_tr, sizeof(float) * ntr));
        dtr = h->st_tr;
    }
    if (!h->state_pending) {
        MMOD_CK(h, cudaMemsetAsync(h->u[0], 0, sizeof(float) * (size_t)h->vol, s));
        MMOD_CK(h, cudaMemsetAsync(h->u[1], 0, sizeof(float) * (size_t)h->vol, s));
    }
    if (is_cpml(h)) MMOD_CK(h, cudaMemsetAsync(h->cpml_mem, 0, 6 * sizeof(float) * (size_t)h->vol, s));
    if (h->cpml_xc)   // psi_x and zeta_x of the compact x layers (c_x stays)
        MMOD_CK(h, cudaMemsetAsync(h->cpml_xc, 0, sizeof(float) * (size_t)(h->cpml_xc_floats / 3 * 2), s));
    h->state_pending = false;
    // the loop runs as the captured graph (which records the trace-row
    // events) unless the persistent kernel takes it
    const bool looped_graph = c.nt > 0 && persistent_grid_of(h) == 0;
    if (c.nt > 0)
        if (mmod_status st = run_loop_graph(h, h->g_fwd, h->fwd, dwav, c.nrec > 0 ? dtr : nullptr, s, &launches))
            return st;
    h->ran = true;
    if (final_u) {
        const float *ufin = h->u[(c.nt + 1) & 1];
        if (is_device_ptr(final_u)) {
            MMOD_CK(h, launch_unpack(ufin, c.nx, c.ny, c.nz, h->nxp, final_u, s));
        } else {
            if (!h->st_vol) MMOD_CK(h, cudaMalloc(&h->st_vol, sizeof(float) * (size_t)h->npts));
            MMOD_CK(h, launch_unpack(ufin, c.nx, c.ny, c.nz, h->nxp, h->st_vol, s));
            MMOD_CK(h, cudaMemcpyAsync(final_u, h->st_vol, sizeof(float) * (size_t)h->npts, cudaMemcpyDeviceToHost, s));
        }
        ++launches;
    }
    if (host_tr) {
        if (looped_graph) {
            // rows of each chunk as soon as the loop graph has recorded them final
            long long r0 = 0;
            for (int i = 0; i < mmod_handle::kTraceChunks; ++i) {
                const long long r1 = h->rows_at[i];
                if (r1 <= r0) continue;
                MMOD_CK(h, cudaStreamWaitEvent(h->st_copy, h->ev_rows[i], 0));
                MMOD_CK(h, cudaMemcpyAsync(traces + r0 * c.nrec, dtr + r0 * c.nrec, sizeof(float) * (r1 - r0) * c.nrec,
                                           cudaMemcpyDeviceToHost, h->st_copy));
                r0 = r1;
            }
            MMOD_CK(h, cudaEventRecord(h->ev_copied, h->st_copy));
            MMOD_CK(h, cudaStreamWaitEvent(s, h->ev_copied, 0));
        } else {
            MMOD_CK(h, cudaMemcpyAsync(traces, dtr, sizeof(float) * ntr, cudaMemcpyDeviceToHost, s));
        }
    }
    if (host_tr || (final_u && !is_device_ptr(final_u))) MMOD_CK(h, cudaStreamSynchronize(s));
    h->last_launches = launches;
    return check_latched(h);
}

MMOD_API float mmod_last_loop_ms(mmod_handle *h) {
    if (!h || !h->ran || h->cfg.nt == 0) return -1.0f;
    DeviceGuard guard(h->device);
    float ms = -1.0f;
    if (cudaEventSynchronize(h->ev_t1) != cudaSuccess || cudaEventElapsedTime(&ms, h->ev_t0, h->ev_t1) != cudaSuccess) {
        cudaGetLastError();
        return -1.0f;
    }
    return ms;
}
