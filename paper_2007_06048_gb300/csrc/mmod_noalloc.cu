// mmod_forward_noalloc: the forward run of mmod_forward for callers that may
// not allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is off limits — inside a
// framework's memory pool that must account for every byte, in a process
// that pre-reserves all device memory at start-up, or under a real-time
// budget where an allocation's implicit synchronisation or failure at run
// time is not acceptable.  The handle API allocates its wavefields at
// mmod_create; this entry point instead works in one fixed block of device
// memory that is part of the loaded library (a file-scope __device__ array),
// so a call allocates nothing: no cudaMalloc, cudaFree, graph, event or
// library call that allocates.
//
// The block holds the two wavefields, the coefficient volume, the damping
// profiles and the source/receiver tables for grids up to the limits below
// (about 25 MB).  Every GPU that loads the library keeps that block until the
// process exits.  All calls share it: each call clears what must start at
// zero, and two calls that overlap on the GPU (other streams, other host
// threads) race on it — serialise them.
//
// In host code the array's name is only a stand-in for the device object, so
// every call looks up the device address with cudaGetSymbolAddress, with the
// call's device current (the lookup allocates nothing).  Looking it up per
// call keeps the address right when the array is instantiated again, e.g.
// after cudaDeviceReset or in another context.  The first call on a device
// may load the library's device code; make it before any stream capture.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>

#include "mmod_internal.h"
#include "tma_plan.h"

namespace {

using namespace mmod;

constexpr long long kMaxVolume = 1LL << 21;   // padded points (nx rounded up to 32) x ny x nz
constexpr int kMaxAxis = 4096;                // points per axis
constexpr int kMaxSrc = 64;
constexpr int kMaxRec = 65536;

constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kOffU0 = 0;
constexpr size_t kOffU1 = kOffU0 + align256(kMaxVolume * 4);
constexpr size_t kOffC = kOffU1 + align256(kMaxVolume * 4);
// Injection buckets: nz * ceil(nx / 64) * ceil(ny / 16).  ceil(nx / 64) <=
// nxp / 32 and ceil(ny / 16) <= ny, so the count never exceeds
// nxp * ny * nz / 32 <= 2^21 / 32 within the volume limit above (nx <= 32
// and ny = 1 reach it).
constexpr int kMaxBuckets = (int)(kMaxVolume / 32);
constexpr size_t kOffEta = kOffC + align256(kMaxVolume * 4);
constexpr size_t kOffTiles = kOffEta + align256(3 * kMaxAxis * 4);
constexpr size_t kOffTab = kOffTiles + align256((kMaxBuckets + 1) * 4);   // point and source tables
constexpr size_t kTabInts = 8 * kMaxSrc + 1;   // pt_i, pt_j, pt_k, pt_first(+1), src_row, src_i, src_j, src_k
constexpr size_t kOffPtOff = kOffTab + align256(kTabInts * 4);
constexpr size_t kOffScale = kOffPtOff + align256(kMaxSrc * 8);
constexpr size_t kOffRec = kOffScale + align256(kMaxSrc * 4);
constexpr size_t kOffMisc = kOffRec + align256((size_t)kMaxRec * 8);   // vmax bits, bad count, error word
constexpr size_t kScratchBytes = kOffMisc + 256;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of the block in the current context.
cudaError_t scratch_address(unsigned char **out) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    *out = static_cast<unsigned char *>(p);
    return cudaSuccess;
}

// Memory the kernels on `device` can dereference: device memory of that
// device, or managed memory.
bool on_device(const void *p, int device) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    return at.type == cudaMemoryTypeDevice && at.device == device;
}

mmod_status fail(mmod_status st, const char *msg) {
    set_thread_error(msg);
    return st;
}

mmod_status fail_cuda(cudaError_t e, const char *what) {
    char buf[200];
    std::snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorName(e));
    set_thread_error(buf);
    return MMOD_ERR_CUDA;
}

#define CKN(call)                                      \
    do {                                               \
        cudaError_t _e = (call);                       \
        if (_e != cudaSuccess) return fail_cuda(_e, #call); \
    } while (0)

// After the first enqueue: on a failure, wait (ignoring its status) for the
// work already queued on `s`, which still uses the block, before returning,
// so that a following call finds it idle.
#define CKS(call)                                      \
    do {                                               \
        cudaError_t _e = (call);                       \
        if (_e != cudaSuccess) {                       \
            cudaStreamSynchronize(s);                  \
            cudaGetLastError();                        \
            return fail_cuda(_e, #call);               \
        }                                              \
    } while (0)

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int d) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != d) cudaSetDevice(d);
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

}  // namespace

extern "C" __attribute__((visibility("default"))) mmod_status mmod_forward_noalloc(
    const mmod_config *cfg, int device, const float *vel, const float *wavelet, float *traces, float *final_u,
    mmod_stream stream) {
    set_thread_error("");
    // ---- configuration and limits (host only, nothing enqueued yet)
    if (!cfg) return fail(MMOD_ERR_ARG, "null config");
    const mmod_config &c = *cfg;
    if (c.order != 8) return fail(MMOD_ERR_UNSUPPORTED, "the GPU path implements order 8 only");
    if (c.nx < 1 || c.ny < 1 || c.nz < 1) return fail(MMOD_ERR_ARG, "grid sizes must be >= 1");
    if (!(c.hx > 0 && c.hy > 0 && c.hz > 0) || !std::isfinite(c.hx) || !std::isfinite(c.hy) || !std::isfinite(c.hz))
        return fail(MMOD_ERR_ARG, "grid spacings must be positive and finite");
    if (!(c.dt > 0) || !std::isfinite(c.dt)) return fail(MMOD_ERR_ARG, "dt must be positive and finite");
    if (c.nt < 0) return fail(MMOD_ERR_ARG, "nt must be >= 0");
    if (c.nbl < 0 || 2LL * c.nbl > c.nx || 2LL * c.nbl > c.ny || 2LL * c.nbl > c.nz)
        return fail(MMOD_ERR_ARG, "damping width must satisfy 0 <= 2*nbl <= n on every axis");
    if (c.nbl > 0 && !(c.damp_R > 0 && c.damp_R < 1)) return fail(MMOD_ERR_ARG, "damp_R must be in (0, 1)");
    if (c.free_surface != 0 && c.free_surface != 1) return fail(MMOD_ERR_ARG, "free_surface must be 0 or 1");
    if (c.boundary != MMOD_BOUNDARY_DAMPING)
        return fail(MMOD_ERR_UNSUPPORTED, "the allocation-free forward has damping layers only");
    if (c.free_surface && c.nz < kRadius + 1) return fail(MMOD_ERR_ARG, "a free surface needs nz >= 5");
    const int nxp = (c.nx + 31) / 32 * 32;
    const long long plane = (long long)nxp * c.ny, vol = plane * c.nz;
    if (c.nx > kMaxAxis || c.ny > kMaxAxis || c.nz > kMaxAxis || vol > kMaxVolume)
        return fail(MMOD_ERR_ARG,
                    "grid exceeds the allocation-free limits: each axis <= 4096 and "
                    "(nx rounded up to 32) * ny * nz <= 2097152 points; use mmod_create / mmod_forward");
    if (c.nsrc < 0 || c.nsrc > kMaxSrc) return fail(MMOD_ERR_ARG, "allocation-free forward takes 0..64 sources");
    if (c.nrec < 0 || c.nrec > kMaxRec) return fail(MMOD_ERR_ARG, "allocation-free forward takes 0..65536 receivers");
    if ((c.nsrc > 0 && !c.src_ijk) || (c.nrec > 0 && !c.rec_ijk)) return fail(MMOD_ERR_ARG, "null position list");
    for (int s = 0; s < c.nsrc; ++s) {
        const int *p = c.src_ijk + 3 * s;
        if (p[0] < 0 || p[0] >= c.nx || p[1] < 0 || p[1] >= c.ny || p[2] < 0 || p[2] >= c.nz)
            return fail(MMOD_ERR_ARG, "a source lies outside the grid");
    }
    for (int r = 0; r < c.nrec; ++r) {
        const int *p = c.rec_ijk + 3 * r;
        if (p[0] < 0 || p[0] >= c.nx || p[1] < 0 || p[1] >= c.ny || p[2] < 0 || p[2] >= c.nz)
            return fail(MMOD_ERR_ARG, "a receiver lies outside the grid");
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return fail(MMOD_ERR_CUDA, "CUDA device not available");
    }
    DeviceGuard guard(device);
    if (!vel || !on_device(vel, device)) return fail(MMOD_ERR_ARG, "vel must be a pointer to memory of `device`");
    if (c.nsrc > 0 && c.nt > 0 && (!wavelet || !on_device(wavelet, device)))
        return fail(MMOD_ERR_ARG, "wavelet must be a pointer to memory of `device`");
    if (c.nrec > 0 && c.nt > 0 && (!traces || !on_device(traces, device)))
        return fail(MMOD_ERR_ARG, "traces must be a pointer to memory of `device`");
    if (final_u && !on_device(final_u, device))
        return fail(MMOD_ERR_ARG, "final_u must be a pointer to memory of `device`");

    unsigned char *base = nullptr;
    CKN(scratch_address(&base));
    cudaStream_t s = (cudaStream_t)stream;
    float *u[2] = {reinterpret_cast<float *>(base + kOffU0), reinterpret_cast<float *>(base + kOffU1)};
    float *cvol = reinterpret_cast<float *>(base + kOffC);
    float *eta = reinterpret_cast<float *>(base + kOffEta);
    int *tiles_d = reinterpret_cast<int *>(base + kOffTiles);
    int *tab_d = reinterpret_cast<int *>(base + kOffTab);
    long long *pt_off_d = reinterpret_cast<long long *>(base + kOffPtOff);
    float *src_scale = reinterpret_cast<float *>(base + kOffScale);
    long long *rec_off = reinterpret_cast<long long *>(base + kOffRec);
    unsigned int *vmax_bits = reinterpret_cast<unsigned int *>(base + kOffMisc);
    unsigned long long *bad = reinterpret_cast<unsigned long long *>(base + kOffMisc + 8);
    int *err = reinterpret_cast<int *>(base + kOffMisc + 16);

    // ---- injection table (sources grouped by point, bucketed per tile and
    // 64 x 16 tile, as the handle API builds it) and receiver offsets
    const int tiles_x = (c.nx + kInjTileX - 1) / kInjTileX, tiles_y = (c.ny + kInjTileY - 1) / kInjTileY;
    const long long nbuckets = (long long)c.nz * tiles_x * tiles_y;
    if (nbuckets > kMaxBuckets) return fail(MMOD_ERR_ARG, "grid exceeds the allocation-free limits (tile buckets)");
    auto bucket = [&](int s) {
        const int *p = c.src_ijk + 3 * s;
        return ((long long)(p[1] / kInjTileY) * tiles_x + p[0] / kInjTileX) * c.nz + p[2];
    };
    auto before = [&](int a, int b) {   // strict order: bucket, j, i, then input order
        const long long ba = bucket(a), bb = bucket(b);
        if (ba != bb) return ba < bb;
        const int *pa = c.src_ijk + 3 * a, *pb = c.src_ijk + 3 * b;
        if (pa[1] != pb[1]) return pa[1] < pb[1];
        if (pa[0] != pb[0]) return pa[0] < pb[0];
        return a < b;
    };
    int order[kMaxSrc];
    int nkeep = 0;   // with a free surface, sources on the plane k = 0 inject nothing
    for (int t = 0; t < c.nsrc; ++t)
        if (!(c.free_surface && c.src_ijk[3 * t + 2] == 0)) order[nkeep++] = t;
    for (int t = 1; t < nkeep; ++t)   // insertion sort (at most 64 entries)
        for (int q = t; q > 0 && before(order[q], order[q - 1]); --q) {
            const int tmp = order[q];
            order[q] = order[q - 1];
            order[q - 1] = tmp;
        }
    int tab[kTabInts] = {0};
    int *pt_i = tab, *pt_j = tab + kMaxSrc, *pt_k = tab + 2 * kMaxSrc, *pt_first = tab + 3 * kMaxSrc;
    int *src_row = tab + 4 * kMaxSrc + 1, *src_i = src_row + kMaxSrc, *src_j = src_i + kMaxSrc, *src_k = src_j + kMaxSrc;
    long long pt_off[kMaxSrc] = {0}, pt_bucket[kMaxSrc] = {0};
    int npt = 0;
    for (int q = 0; q < nkeep; ++q) {
        const int sidx = order[q];
        const int *p = c.src_ijk + 3 * sidx;
        src_row[q] = sidx;
        src_i[q] = p[0];
        src_j[q] = p[1];
        src_k[q] = p[2];
        const bool same = q > 0 && std::memcmp(c.src_ijk + 3 * order[q - 1], p, 3 * sizeof(int)) == 0;
        if (!same) {
            pt_i[npt] = p[0];
            pt_j[npt] = p[1];
            pt_k[npt] = p[2];
            pt_off[npt] = (long long)p[2] * plane + (long long)p[1] * nxp + p[0];
            pt_bucket[npt] = bucket(sidx);
            pt_first[npt] = q;
            ++npt;
        }
    }
    pt_first[npt] = nkeep;
    CKS(cudaMemcpyAsync(tab_d, tab, sizeof(tab), cudaMemcpyHostToDevice, s));
    CKS(cudaMemcpyAsync(pt_off_d, pt_off, sizeof(pt_off), cudaMemcpyHostToDevice, s));
    CKS(cudaStreamSynchronize(s));   // the host tables above live on the stack
    {
        int chunk[1024];   // tile_start[b] = points in buckets < b
        int ptr = 0;
        for (long long b0 = 0; b0 <= nbuckets; b0 += 1024) {
            const int n = (int)std::min<long long>(1024, nbuckets + 1 - b0);
            for (int q = 0; q < n; ++q) {
                while (ptr < npt && pt_bucket[ptr] < b0 + q) ++ptr;
                chunk[q] = ptr;
            }
            CKS(cudaMemcpyAsync(tiles_d + b0, chunk, sizeof(int) * n, cudaMemcpyHostToDevice, s));
            CKS(cudaStreamSynchronize(s));   // the chunk buffer is reused
        }
    }
    {
        long long chunk[1024];
        for (int r0 = 0; r0 < c.nrec; r0 += 1024) {
            const int n = c.nrec - r0 < 1024 ? c.nrec - r0 : 1024;
            for (int r = 0; r < n; ++r) {
                const int *p = c.rec_ijk + 3 * (r0 + r);
                chunk[r] = (long long)p[2] * plane + (long long)p[1] * nxp + p[0];
            }
            CKS(cudaMemcpyAsync(rec_off + r0, chunk, sizeof(long long) * n, cudaMemcpyHostToDevice, s));
            CKS(cudaStreamSynchronize(s));   // the chunk buffer is reused
        }
    }

    // ---- model: scan, stability check, c = dt^2 v^2, profiles, source scales
    const long long npts = (long long)c.nx * c.ny * c.nz;
    CKS(cudaMemsetAsync(base + kOffMisc, 0, 256, s));
    CKS(launch_model_scan(vel, npts, vmax_bits, bad, s));
    unsigned int vbits = 0;
    unsigned long long nbad = 0;
    CKS(cudaMemcpyAsync(&vbits, vmax_bits, sizeof(vbits), cudaMemcpyDeviceToHost, s));
    CKS(cudaMemcpyAsync(&nbad, bad, sizeof(nbad), cudaMemcpyDeviceToHost, s));
    CKS(cudaStreamSynchronize(s));
    if (nbad) return fail(MMOD_ERR_ARG, "velocities must be positive and finite");
    float vmaxf;
    std::memcpy(&vmaxf, &vbits, sizeof(vmaxf));
    const double vmax = vmaxf;
    const double ksum = kSymbolMax8 * (1.0 / (c.hx * c.hx) + 1.0 / (c.hy * c.hy) + 1.0 / (c.hz * c.hz));
    if (c.dt * vmax * std::sqrt(ksum) > 2.0) return fail(MMOD_ERR_UNSTABLE, "dt too large for the model (CFL bound)");
    CKS(launch_model_fill(vel, c.nx, c.ny, c.nz, nxp, c.dt, cvol, s));
    {
        int *tab_src_i = tab_d + 4 * kMaxSrc + 1 + kMaxSrc;
        CKS(launch_source_scale(vel, c.nx, c.ny, nkeep, tab_src_i, tab_src_i + kMaxSrc, tab_src_i + 2 * kMaxSrc,
                                c.dt, c.hx * c.hy * c.hz, src_scale, s));
    }
    float eta_h[3 * kMaxAxis];
    damping_profile(c.nx, c.nbl, c.hx, vmax, c.damp_R, c.dt, eta_h);
    damping_profile(c.ny, c.nbl, c.hy, vmax, c.damp_R, c.dt, eta_h + c.nx);
    damping_profile(c.nz, c.nbl, c.hz, vmax, c.damp_R, c.dt, eta_h + c.nx + c.ny);
    if (c.free_surface) clear_surface_layer(c.nz, c.nbl, eta_h + c.nx + c.ny);
    CKS(cudaMemcpyAsync(eta, eta_h, sizeof(float) * (c.nx + c.ny + c.nz), cudaMemcpyHostToDevice, s));

    // ---- time loop: u^{-1} = u^0 = 0, one step kernel per step
    CKS(cudaMemsetAsync(u[0], 0, sizeof(float) * vol, s));
    CKS(cudaMemsetAsync(u[1], 0, sizeof(float) * vol, s));
    CUtensorMap cur_map[2], prev_map[2], c_map;
    TmaPlan plans[kMaxTmaVariants];
    const bool tma = make_tma_plan(c, nxp, u, cvol, cur_map, prev_map, &c_map, plans);
    StepArgs a{};
    a.nx = c.nx; a.ny = c.ny; a.nz = c.nz; a.nxp = nxp; a.plane = plane; a.nbl = c.nbl; a.nt = c.nt;
    for (int m = 0; m < kRadius; ++m) {
        a.w.x[m] = (float)(kTaylor8[m] / (c.hx * c.hx));
        a.w.y[m] = (float)(kTaylor8[m] / (c.hy * c.hy));
        a.w.z[m] = (float)(kTaylor8[m] / (c.hz * c.hz));
    }
    a.c = cvol;
    a.ex = eta; a.ey = eta + c.nx; a.ez = eta + c.nx + c.ny;
    a.inj.tile_start = tiles_d;
    a.inj.pt_i = tab_d; a.inj.pt_j = tab_d + kMaxSrc; a.inj.pt_k = tab_d + 2 * kMaxSrc;
    a.inj.pt_first = tab_d + 3 * kMaxSrc; a.inj.src_row = tab_d + 4 * kMaxSrc + 1;
    a.inj.pt_off = pt_off_d; a.inj.src_scale = src_scale;
    a.inj.tiles_x = tiles_x; a.inj.tiles_y = tiles_y; a.inj.npts = npt;
    a.wavelet = wavelet;
    a.wrs = c.nt;
    a.wcs = 1;
    a.fs = c.free_surface;
    a.pdl = 0;
    a.nrec = c.nrec; a.rec_off = rec_off;
    a.err = err;
    const bool want_tr = c.nrec > 0 && traces;
    for (int n = 0; n < c.nt; ++n) {
        a.n = n;
        a.ucur = u[(n + 1) & 1];
        a.uprev = u[n & 1];
        a.uout = u[n & 1];
        if (tma) {
            a.traces = (n >= 1 && want_tr) ? traces + (long long)(n - 1) * c.nrec : nullptr;
            CKS(launch_step_tma(a, &cur_map[(n + 1) & 1], &prev_map[n & 1], &c_map, plans[kTmaDefaultVariant], s));
        } else {
            a.traces = nullptr;
            CKS(launch_step_simple(a, s));
            if (npt > 0) CKS(launch_inject(a, s));
            if (want_tr) CKS(launch_gather(u[n & 1], rec_off, c.nrec, traces + (long long)n * c.nrec, s));
        }
    }
    if (tma && c.nt > 0 && want_tr)
        CKS(launch_gather(u[(c.nt - 1) & 1], rec_off, c.nrec, traces + (long long)(c.nt - 1) * c.nrec, s));
    if (final_u) CKS(launch_unpack(u[(c.nt + 1) & 1], c.nx, c.ny, c.nz, nxp, final_u, s));
    int err_h = 0;
    CKS(cudaMemcpyAsync(&err_h, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    CKS(cudaStreamSynchronize(s));
    if (err_h) return fail(MMOD_ERR_TIMEOUT, "a step kernel gave up waiting for its copies (device-side timeout)");
    return MMOD_OK;
}
