// Adjoint propagator, velocity gradient with checkpointing, FP64 dot product.
//
// Adjoint.  With D = 1 + e, E = 1 - e, C = dt^2 v^2, the transpose of the
// forward map wavelet -> traces runs backward as
//     D mu^n = 2 mu^{n+1} - E mu^{n+2} + L(C mu^{n+1}) + R^T r^{n-1}.
// Multiplying by C shows that psi = C mu obeys the forward recurrence
//     D psi^n = 2 psi^{n+1} - E psi^{n+2} + C L psi^{n+1} + C R^T r^{n-1},
// so the adjoint reuses the forward step kernels run backward in time: the
// receivers become injection points (scale c, no cell volume), the residual
// read backward in time is their wavelet (rows [nt][nrec] as given: one
// contiguous row per step), and the sources are gathered; the
// adjoint source is a[s][n] = psi^{n+1}(x_s) / (hx hy hz).
//
// Gradient.  dJ/dc(x) = sum_n mu^{n+1}(x) g^n(x), g^n = L u^n + s^n, so
// with mu = psi / c the kernels accumulate A = sum_n psi^{n+1} g^n (FP32)
// and dJ/dv = 2 dt^2 v A / c = 2 A / v.  g^n is written by the step kernel that
// advances u^n (the Laplacian it already holds, plus w[n] / (hx hy hz) at the
// sources): no difference of nearly equal wavefields is formed.  The forward
// states are recovered from checkpoints (u^{a-1}, u^a) (FP32, or BF16 / FP16
// with one scale per z plane) by one of two schemes:
//   segments: the first sweep stores a checkpoint at the start of each of S
//     segments of K steps; the backward sweep replays each segment from its
//     checkpoint, in place in two volumes, writing g^n into K more, and runs
//     the segment's adjoint steps against them.  Memory: 2 S checkpoint
//     volumes + K + 2; work: two forward sweeps and one adjoint (with FP32
//     checkpoints the first sweep writes g^n of the last segment itself,
//     which is then not replayed);
//   revolve: the binomial schedule of mmod_revolve.cu over S slots, with the
//     working state in the handle's two buffers, u^{n+1} and g^n of a
//     reversed step in two more volumes; the fewest replayed steps for S slots;
//   segments with S >= nt and FP32 storage keeps g^n of every step (nt + 2
//     volumes, written by the first sweep): no replay.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cfloat>
#include <cstring>

#include "mmod_handle.h"

#define MMOD_API extern "C" __attribute__((visibility("default")))

using namespace mmod;

namespace {

// ---- checkpoint storage: one scale per z plane, 16-bit values ------------

template <class T>
__device__ __forceinline__ T to_store(float v);
template <>
__device__ __forceinline__ __nv_bfloat16 to_store<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <>
__device__ __forceinline__ __half to_store<__half>(float v) { return __float2half_rn(v); }
__device__ __forceinline__ float from_store(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float from_store(__half v) { return __half2float(v); }

// One CTA per plane: scale = max(max |u| over the plane, FLT_MIN), stored =
// u / scale.
template <class T>
__global__ void compress_kernel(const float *__restrict__ u, long long plane, T *__restrict__ out,
                                float *__restrict__ scale) {
    const long long base = (long long)blockIdx.x * plane;
    float m = 0.0f;
    for (long long q = threadIdx.x; q < plane; q += blockDim.x) m = fmaxf(m, fabsf(u[base + q]));
    for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    __shared__ float part[32];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.0f;
        for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
        if (threadIdx.x == 0) part[0] = m;
    }
    __syncthreads();
    // A plane that holds only zeros and subnormals (the leading edge of a
    // wave, far planes early in a run) gets the smallest normal scale, so
    // 1/scale stays finite.
    const float s = fmaxf(part[0], FLT_MIN);
    if (threadIdx.x == 0) scale[blockIdx.x] = s;
    const float inv = 1.0f / s;
    for (long long q = threadIdx.x; q < plane; q += blockDim.x) out[base + q] = to_store<T>(u[base + q] * inv);
}

template <class T>
__global__ void decompress_kernel(const T *__restrict__ in, const float *__restrict__ scale, long long plane,
                                  float *__restrict__ u) {
    const long long base = (long long)blockIdx.x * plane;
    const float s = scale[blockIdx.x];
    for (long long q = threadIdx.x; q < plane; q += blockDim.x) u[base + q] = from_store(in[base + q]) * s;
}

// Block floating point (MMOD_CKPT_BFP16): per block of 32 consecutive x
// values of a padded row (rows are padded to 32, so blocks never straddle
// rows), scale s = max |u| over the block and q = round(u * 32767 / s) as
// int16; u is restored as q * (s / 32767), within s / 65534 of the stored
// value.  One warp per block, grid-stride over the volume's blocks.
constexpr int kBfpBlock = 32;
constexpr float kBfpMax = 32767.0f;

__global__ void compress_bfp_kernel(const float *__restrict__ u, long long nblocks, short *__restrict__ out,
                                    float *__restrict__ scale) {
    const int lane = threadIdx.x & 31;
    const long long warp0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long b = warp0; b < nblocks; b += nwarps) {
        const float v = u[b * kBfpBlock + lane];
        float m = fabsf(v);
        for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
        int q = 0;
        if (m > 0.0f) q = max(-32767, min(32767, __float2int_rn(v * (kBfpMax / m))));
        out[b * kBfpBlock + lane] = (short)q;
        if (lane == 0) scale[b] = m;
    }
}

__global__ void decompress_bfp_kernel(const short *__restrict__ in, const float *__restrict__ scale, long long nblocks,
                                      float *__restrict__ u) {
    const int lane = threadIdx.x & 31;
    const long long warp0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long b = warp0; b < nblocks; b += nwarps)
        u[b * kBfpBlock + lane] = (float)in[b * kBfpBlock + lane] * (scale[b] / kBfpMax);
}

int bfp_grid(long long nblocks) { return (int)std::min<long long>((nblocks + 7) / 8, 152LL * 16); }

size_t ckpt_elem_bytes(int dtype) { return dtype == MMOD_CKPT_FP32 ? 4 : 2; }

// Scales per checkpoint volume: one per z plane (BF16 / FP16), one per
// 32-value block (BFP16), none (FP32).
size_t ckpt_scales(const mmod_handle *h, int dtype) {
    if (dtype == MMOD_CKPT_BFP16) return (size_t)h->vol / kBfpBlock;
    return dtype == MMOD_CKPT_FP32 ? 0 : (size_t)h->cfg.nz;
}

// Save the volume u as checkpoint volume slot (FP32: copy; 16-bit: compress).
cudaError_t save_volume(mmod_handle *h, const float *u, int slot, cudaStream_t s) {
    auto &gw = h->gw;
    const size_t eb = ckpt_elem_bytes(gw.dtype);
    char *dst = static_cast<char *>(gw.ckpt) + (size_t)slot * h->vol * eb;
    if (gw.dtype == MMOD_CKPT_FP32)
        return cudaMemcpyAsync(dst, u, sizeof(float) * (size_t)h->vol, cudaMemcpyDeviceToDevice, s);
    float *sc = gw.ckpt_scale + (size_t)slot * ckpt_scales(h, gw.dtype);
    if (gw.dtype == MMOD_CKPT_BFP16) {
        const long long nb = h->vol / kBfpBlock;
        compress_bfp_kernel<<<bfp_grid(nb), 256, 0, s>>>(u, nb, reinterpret_cast<short *>(dst), sc);
    } else if (gw.dtype == MMOD_CKPT_BF16)
        compress_kernel<__nv_bfloat16><<<h->cfg.nz, 256, 0, s>>>(u, h->plane, reinterpret_cast<__nv_bfloat16 *>(dst), sc);
    else
        compress_kernel<__half><<<h->cfg.nz, 256, 0, s>>>(u, h->plane, reinterpret_cast<__half *>(dst), sc);
    return cudaGetLastError();
}

cudaError_t restore_volume(mmod_handle *h, int slot, float *u, cudaStream_t s) {
    auto &gw = h->gw;
    const size_t eb = ckpt_elem_bytes(gw.dtype);
    const char *src = static_cast<const char *>(gw.ckpt) + (size_t)slot * h->vol * eb;
    if (gw.dtype == MMOD_CKPT_FP32)
        return cudaMemcpyAsync(u, src, sizeof(float) * (size_t)h->vol, cudaMemcpyDeviceToDevice, s);
    const float *sc = gw.ckpt_scale + (size_t)slot * ckpt_scales(h, gw.dtype);
    if (gw.dtype == MMOD_CKPT_BFP16) {
        const long long nb = h->vol / kBfpBlock;
        decompress_bfp_kernel<<<bfp_grid(nb), 256, 0, s>>>(reinterpret_cast<const short *>(src), sc, nb, u);
    } else if (gw.dtype == MMOD_CKPT_BF16)
        decompress_kernel<__nv_bfloat16><<<h->cfg.nz, 256, 0, s>>>(reinterpret_cast<const __nv_bfloat16 *>(src), sc,
                                                                    h->plane, u);
    else
        decompress_kernel<__half><<<h->cfg.nz, 256, 0, s>>>(reinterpret_cast<const __half *>(src), sc, h->plane, u);
    return cudaGetLastError();
}

// Allocate (or keep) the gradient work space: nslot checkpoints of two
// volumes, nwork FP32 work volumes (with tensor maps), psi, grad_c.
mmod_status ensure_grad_work(mmod_handle *h, int nslot, int nwork, int dtype) {
    auto &gw = h->gw;
    if (gw.nslot == nslot && gw.nwork == nwork && gw.dtype == dtype) return MMOD_OK;
    free_grad_work(h);
    const size_t vb = sizeof(float) * (size_t)h->vol;
    gw.seg.assign(nwork, nullptr);
    gw.seg_cur.resize(nwork);
    gw.seg_prev.resize(nwork);
    for (int i = 0; i < nwork; ++i) {
        MMOD_CK(h, cudaMalloc(&gw.seg[i], vb));
        MMOD_CK(h, cudaMemset(gw.seg[i], 0, vb));
        if (h->tma_ok && !encode_maps(h->cfg, h->nxp, gw.seg[i], &gw.seg_cur[i], &gw.seg_prev[i]))
            return fail(h, MMOD_ERR_CUDA, "tensor map encoding failed for a work volume");
    }
    for (int b = 0; b < 2; ++b) {
        MMOD_CK(h, cudaMalloc(&gw.psi[b], vb));
        if (h->tma_ok && !encode_maps(h->cfg, h->nxp, gw.psi[b], &gw.psi_cur[b], &gw.psi_prev[b]))
            return fail(h, MMOD_ERR_CUDA, "tensor map encoding failed for an adjoint buffer");
    }
    MMOD_CK(h, cudaMalloc(&gw.gradc, vb));
    gw.ckpt_bytes = (size_t)nslot * 2 * (size_t)h->vol * ckpt_elem_bytes(dtype);
    if (nslot > 0) MMOD_CK(h, cudaMalloc(&gw.ckpt, gw.ckpt_bytes));
    if (nslot > 0 && dtype != MMOD_CKPT_FP32)
        MMOD_CK(h, cudaMalloc(&gw.ckpt_scale, sizeof(float) * (size_t)nslot * 2 * ckpt_scales(h, dtype)));
    gw.nslot = nslot;
    gw.nwork = nwork;
    gw.dtype = dtype;
    return MMOD_OK;
}

// Checkpoint layout of a gradient call: slots and FP32 work volumes.
// seglen = 0 with nslot = 0: every forward state is kept (FP32 checkpoints,
// ckpt_count >= nt), so nothing is replayed.
void grad_layout(const mmod_handle *h, int ckpt_count, int dtype, int *nslot, int *nwork, int *seglen) {
    const int nt = h->cfg.nt;
    if (h->ckpt_scheme == MMOD_SCHEME_SEGMENTS && dtype == MMOD_CKPT_FP32 && ckpt_count >= nt && nt > 0) {
        *seglen = 0;
        *nslot = 0;
        *nwork = nt + 2;
        return;
    }
    if (h->ckpt_scheme == MMOD_SCHEME_REVOLVE) {
        *seglen = 0;
        *nslot = std::max(1, std::min(ckpt_count, nt - 1));
        *nwork = 2;
    } else {
        *seglen = std::max(1, (nt + ckpt_count - 1) / ckpt_count);
        *nslot = nt > 0 ? (nt + *seglen - 1) / *seglen : 1;
        *nwork = *seglen + 2;
    }
}

// Device copy of an input array: device pointers pass through, host arrays go
// through the staging buffer *stage (allocated on first use, n floats).
mmod_status device_input(mmod_handle *h, const float *p, size_t n, float **stage, const float **out,
                         cudaStream_t s) {
    if (is_device_ptr(p)) {
        *out = p;
        return MMOD_OK;
    }
    if (!*stage) MMOD_CK(h, cudaMalloc(stage, sizeof(float) * std::max<size_t>(n, 1)));
    if (n) MMOD_CK(h, cudaMemcpyAsync(*stage, p, sizeof(float) * n, cudaMemcpyHostToDevice, s));
    *out = *stage;
    return MMOD_OK;
}

}  // namespace

namespace mmod {

void free_grad_work(mmod_handle *h) {
    auto &gw = h->gw;
    for (float *p : gw.seg)
        if (p) cudaFree(p);
    gw.seg.clear();
    gw.seg_cur.clear();
    gw.seg_prev.clear();
    for (float *&p : gw.psi) {
        if (p) cudaFree(p);
        p = nullptr;
    }
    if (gw.gradc) cudaFree(gw.gradc);
    if (gw.ckpt) cudaFree(gw.ckpt);
    if (gw.ckpt_scale) cudaFree(gw.ckpt_scale);
    gw.gradc = nullptr;
    gw.ckpt = nullptr;
    gw.ckpt_scale = nullptr;
    gw.nslot = gw.nwork = 0;
    gw.dtype = -1;
    gw.ckpt_bytes = 0;
}

}  // namespace mmod

MMOD_API mmod_status mmod_adjoint(mmod_handle *h, const float *resid, float *adj_src, mmod_stream stream) {
    if (!h) return MMOD_ERR_ARG;
    if (mmod_status st = check_latched(h)) return st;
    if (is_cpml(h)) return fail(h, MMOD_ERR_UNSUPPORTED, "the adjoint is built for the damping layers only");
    if (!h->model_set) return fail(h, MMOD_ERR_STATE, "mmod_set_model has not succeeded");
    const auto &c = h->cfg;
    if (c.nrec > 0 && c.nt > 0 && !resid) return fail(h, MMOD_ERR_ARG, "null residual with nrec > 0");
    if (c.nsrc > 0 && c.nt > 0 && !adj_src) return fail(h, MMOD_ERR_ARG, "null adjoint source with nsrc > 0");
    DeviceGuard guard(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t nres = (size_t)c.nt * c.nrec, nadj = (size_t)c.nt * c.nsrc;
    long long launches = 0;
    const float *dres = nullptr;
    if (mmod_status st = device_input(h, resid, nres, &h->st_tr, &dres, s)) return st;
    if (!h->st_adjw) MMOD_CK(h, cudaMalloc(&h->st_adjw, sizeof(float) * std::max<size_t>(nres, 1)));
    if (!h->st_adjg) MMOD_CK(h, cudaMalloc(&h->st_adjg, sizeof(float) * std::max<size_t>(nadj, 1)));
    if (nres) MMOD_CK(h, cudaMemcpyAsync(h->st_adjw, dres, sizeof(float) * nres, cudaMemcpyDeviceToDevice, s));
    MMOD_CK(h, cudaMemsetAsync(h->u[0], 0, sizeof(float) * (size_t)h->vol, s));
    MMOD_CK(h, cudaMemsetAsync(h->u[1], 0, sizeof(float) * (size_t)h->vol, s));
    h->state_pending = false;
    if (c.nt > 0)
        if (mmod_status st = run_loop_graph(h, h->g_adj, h->adj, h->st_adjw, c.nsrc > 0 ? h->st_adjg : nullptr, s,
                                            &launches))
            return st;
    h->ran = false;   // the wavefield buffers now hold the adjoint state
    if (nadj) {
        const bool dev_out = is_device_ptr(adj_src);
        float *dst = adj_src;
        if (!dev_out) {
            if (!h->st_adjo) MMOD_CK(h, cudaMalloc(&h->st_adjo, sizeof(float) * nadj));
            dst = h->st_adjo;
        }
        MMOD_CK(h, launch_unreverse_transpose(h->st_adjg, c.nt, c.nsrc, 1.0 / (c.hx * c.hy * c.hz), dst, s));
        ++launches;
        if (!dev_out) {
            MMOD_CK(h, cudaMemcpyAsync(adj_src, dst, sizeof(float) * nadj, cudaMemcpyDeviceToHost, s));
            MMOD_CK(h, cudaStreamSynchronize(s));
        }
    }
    h->last_launches = launches;
    return check_latched(h);
}

MMOD_API mmod_status mmod_gradient(mmod_handle *h, const float *wavelet, const float *resid, float *grad_v,
                                   int ckpt_count, int ckpt_dtype, mmod_stream stream) {
    if (!h) return MMOD_ERR_ARG;
    if (mmod_status st = check_latched(h)) return st;
    if (is_cpml(h)) return fail(h, MMOD_ERR_UNSUPPORTED, "the gradient is built for the damping layers only");
    if (!h->model_set) return fail(h, MMOD_ERR_STATE, "mmod_set_model has not succeeded");
    const auto &c = h->cfg;
    if (!grad_v) return fail(h, MMOD_ERR_ARG, "null gradient output");
    if (ckpt_count < 1) return fail(h, MMOD_ERR_ARG, "ckpt_count must be >= 1");
    if (ckpt_dtype != MMOD_CKPT_FP32 && ckpt_dtype != MMOD_CKPT_BF16 && ckpt_dtype != MMOD_CKPT_FP16 &&
        ckpt_dtype != MMOD_CKPT_BFP16)
        return fail(h, MMOD_ERR_ARG, "unknown checkpoint type");
    if (c.nsrc > 0 && c.nt > 0 && !wavelet) return fail(h, MMOD_ERR_ARG, "null wavelet with nsrc > 0");
    if (c.nrec > 0 && c.nt > 0 && !resid) return fail(h, MMOD_ERR_ARG, "null residual with nrec > 0");
    DeviceGuard guard(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int nt = c.nt;
    int nslot = 0, nwork = 0, seglen = 0;
    grad_layout(h, ckpt_count, ckpt_dtype, &nslot, &nwork, &seglen);
    if (mmod_status st = ensure_grad_work(h, nslot, nwork, ckpt_dtype)) return st;
    auto &gw = h->gw;
    const bool tma = use_tma(h);
    long long launches = 0;
    const size_t vb = sizeof(float) * (size_t)h->vol;

    const float *dwav = nullptr, *dres = nullptr;
    if (mmod_status st = device_input(h, wavelet, (size_t)c.nsrc * nt, &h->st_wav, &dwav, s)) return st;
    if (mmod_status st = device_input(h, resid, (size_t)c.nrec * nt, &h->st_tr, &dres, s)) return st;
    const size_t nres = (size_t)nt * c.nrec;
    if (!h->st_adjw) MMOD_CK(h, cudaMalloc(&h->st_adjw, sizeof(float) * std::max<size_t>(nres, 1)));
    if (nres) MMOD_CK(h, cudaMemcpyAsync(h->st_adjw, dres, sizeof(float) * nres, cudaMemcpyDeviceToDevice, s));

    MMOD_CK(h, cudaMemsetAsync(h->u[0], 0, vb, s));
    MMOD_CK(h, cudaMemsetAsync(h->u[1], 0, vb, s));
    h->state_pending = false;
    StepArgs fa = base_args(h, h->fwd, dwav);
    fa.nrec = 0;   // no receivers in the gradient's forward sweeps
    fa.inv_cell = (float)(1.0 / (c.hx * c.hy * c.hz));
    StepArgs aa = base_args(h, h->adj, h->st_adjw);
    aa.nrec = 0;
    // forward step n in place on the handle's buffers: u^{n-1} in u[n & 1],
    // u^n in u[(n + 1) & 1], u^{n+1} over u^{n-1}
    auto fwd_step_in_place = [&](int n) {
        fa.n = n;
        fa.ucur = h->u[(n + 1) & 1];
        fa.uprev = h->u[n & 1];
        fa.uout = h->u[n & 1];
        return enqueue_step(h, fa, &h->cur_map[(n + 1) & 1], &h->prev_map[n & 1], tma, nullptr, s, &launches);
    };
    // forward step n of a replay in the work volumes w0, w1 (u^{n-1} in w0,
    // u^n in w1, u^{n+1} over u^{n-1}), also writing g^n into gout
    auto fwd_step_g = [&](int n, int w0, int w1, float *gout) {
        fa.n = n;
        fa.ucur = gw.seg[w1];
        fa.uprev = gw.seg[w0];
        fa.uout = gw.seg[w0];
        fa.gout = gout;
        const cudaError_t e = enqueue_step(h, fa, tma ? &gw.seg_cur[w1] : nullptr, tma ? &gw.seg_prev[w0] : nullptr,
                                           tma, nullptr, s, &launches);
        fa.gout = nullptr;
        return e;
    };
    // adjoint step of forward step n: adjoint step m = nt-1-n produces
    // psi^{n+1} in psi[m & 1] (psi^{n+2} stays in the other buffer until the
    // next adjoint step)
    auto adj_step = [&](int n) {
        const int m = nt - 1 - n;
        aa.n = m;
        aa.ucur = gw.psi[(m + 1) & 1];
        aa.uprev = gw.psi[m & 1];
        aa.uout = gw.psi[m & 1];
        return enqueue_step(h, aa, tma ? &gw.psi_cur[(m + 1) & 1] : nullptr, tma ? &gw.psi_prev[m & 1] : nullptr,
                            tma, nullptr, s, &launches);
    };
    // imaging terms of forward steps n (and n - 1 when ns = 2) from g[t] =
    // g^{n-t}, after their adjoint steps: psi^{n+1} in psi[(nt-1-n) & 1],
    // psi^n in the other buffer
    auto image = [&](int n, const float *const *g, int ns) {
        const int m = nt - 1 - n;
        const float *ps[2] = {gw.psi[m & 1], gw.psi[(m + 1) & 1]};
        ++launches;
        return launch_imaging(ns, ps, g, c.nx, c.ny, c.nz, h->nxp, gw.gradc, s);
    };
    // steps hi down to lo with g^j in gof(j): two adjoint steps, then one
    // imaging pass over both (the same accumulation order as one pass per
    // step, the accumulator read and written once per pair)
    auto backward_range = [&](int hi, int lo, auto gof) -> cudaError_t {
        int n = hi;
        for (; n - 1 >= lo; n -= 2) {
            cudaError_t e = adj_step(n);
            if (e == cudaSuccess) e = adj_step(n - 1);
            if (e != cudaSuccess) return e;
            const float *g[2] = {gof(n), gof(n - 1)};
            if ((e = image(n, g, 2)) != cudaSuccess) return e;
        }
        if (n == lo) {
            cudaError_t e = adj_step(n);
            if (e != cudaSuccess) return e;
            const float *g[1] = {gof(n)};
            return image(n, g, 1);
        }
        return cudaSuccess;
    };

    if (seglen == 0 && nslot == 0) {
        // every step's g^n kept: seg[0], seg[1] hold the stepped state,
        // seg[2 + n] = g^n
        MMOD_CK(h, cudaMemsetAsync(gw.seg[0], 0, vb, s));
        MMOD_CK(h, cudaMemsetAsync(gw.seg[1], 0, vb, s));
        for (int n = 0; n < nt; ++n) MMOD_CK(h, fwd_step_g(n, n & 1, (n + 1) & 1, gw.seg[2 + n]));
        MMOD_CK(h, cudaMemsetAsync(gw.psi[0], 0, vb, s));
        MMOD_CK(h, cudaMemsetAsync(gw.psi[1], 0, vb, s));
        MMOD_CK(h, cudaMemsetAsync(gw.gradc, 0, vb, s));
        MMOD_CK(h, backward_range(nt - 1, 0, [&](int j) { return gw.seg[2 + j]; }));
    } else if (h->ckpt_scheme == MMOD_SCHEME_REVOLVE) {
        std::vector<RevAction> sched;
        revolve_schedule(nt, nslot, &sched);
        MMOD_CK(h, cudaMemsetAsync(gw.psi[0], 0, vb, s));
        MMOD_CK(h, cudaMemsetAsync(gw.psi[1], 0, vb, s));
        MMOD_CK(h, cudaMemsetAsync(gw.gradc, 0, vb, s));
        float *unext = gw.seg[0], *gn = gw.seg[1];
        for (const RevAction &act : sched) {
            switch (act.kind) {
                case MMOD_REV_ADVANCE:
                    for (int n = act.a; n < act.b; ++n) MMOD_CK(h, fwd_step_in_place(n));
                    break;
                case MMOD_REV_SAVE:   // state of step b: u^{b-1} in u[b & 1], u^b in u[(b + 1) & 1]
                    MMOD_CK(h, save_volume(h, h->u[act.b & 1], 2 * act.a, s));
                    MMOD_CK(h, save_volume(h, h->u[(act.b + 1) & 1], 2 * act.a + 1, s));
                    break;
                case MMOD_REV_RESTORE:
                    if (act.a < 0) {
                        MMOD_CK(h, cudaMemsetAsync(h->u[0], 0, vb, s));
                        MMOD_CK(h, cudaMemsetAsync(h->u[1], 0, vb, s));
                    } else {
                        MMOD_CK(h, restore_volume(h, 2 * act.a, h->u[act.b & 1], s));
                        MMOD_CK(h, restore_volume(h, 2 * act.a + 1, h->u[(act.b + 1) & 1], s));
                    }
                    break;
                case MMOD_REV_REVERSE: {   // g^n from the working state, then the adjoint step and its term
                    const int n = act.a;
                    fa.n = n;
                    fa.ucur = h->u[(n + 1) & 1];
                    fa.uprev = h->u[n & 1];
                    fa.uout = unext;
                    fa.gout = gn;
                    const cudaError_t e = enqueue_step(h, fa, &h->cur_map[(n + 1) & 1], &h->prev_map[n & 1], tma,
                                                       nullptr, s, &launches);
                    fa.gout = nullptr;
                    MMOD_CK(h, e);
                    MMOD_CK(h, adj_step(n));
                    const float *g[1] = {gn};
                    MMOD_CK(h, image(n, g, 1));
                    break;
                }
                default:
                    return fail(h, MMOD_ERR_CUDA, "invalid checkpoint schedule");
            }
        }
    } else {
        const int nseg = nt > 0 ? nslot : 0;
        // With FP32 checkpoints a replay reproduces the first sweep bit for
        // bit, so the first sweep writes g^n of the last segment straight into
        // the segment buffer and that segment is neither saved nor replayed.
        // (A 16-bit checkpoint would start its replay from the rounded state.)
        const bool keep_last = ckpt_dtype == MMOD_CKPT_FP32;
        // ---- sweep 1: forward with a checkpoint at the start of every segment
        for (int sg = 0; sg < nseg; ++sg) {
            const int a0 = sg * seglen, b0 = std::min(nt, a0 + seglen);
            const bool last = keep_last && sg == nseg - 1;
            if (!last) {   // at step a0: u^{a0-1} in u[a0 & 1], u^{a0} in u[(a0 + 1) & 1]
                MMOD_CK(h, save_volume(h, h->u[a0 & 1], 2 * sg, s));
                MMOD_CK(h, save_volume(h, h->u[(a0 + 1) & 1], 2 * sg + 1, s));
            }
            for (int n = a0; n < b0; ++n) {
                fa.gout = last ? gw.seg[2 + n - a0] : nullptr;
                const cudaError_t e = fwd_step_in_place(n);
                fa.gout = nullptr;
                MMOD_CK(h, e);
            }
        }
        // ---- backward: replay each segment (g^n of its steps), then its
        // adjoint steps + imaging
        MMOD_CK(h, cudaMemsetAsync(gw.psi[0], 0, vb, s));
        MMOD_CK(h, cudaMemsetAsync(gw.psi[1], 0, vb, s));
        MMOD_CK(h, cudaMemsetAsync(gw.gradc, 0, vb, s));
        for (int sg = nseg - 1; sg >= 0; --sg) {
            const int a0 = sg * seglen, b0 = std::min(nt, a0 + seglen);
            if (!(keep_last && sg == nseg - 1)) {
                MMOD_CK(h, restore_volume(h, 2 * sg, gw.seg[0], s));
                MMOD_CK(h, restore_volume(h, 2 * sg + 1, gw.seg[1], s));
                for (int n = a0; n < b0; ++n) {   // seg[2 + n - a0] receives g^n
                    const int j = n - a0;
                    MMOD_CK(h, fwd_step_g(n, j & 1, (j + 1) & 1, gw.seg[2 + j]));
                }
            }
            MMOD_CK(h, backward_range(b0 - 1, a0, [&](int j) { return gw.seg[2 + j - a0]; }));
        }
    }
    h->ran = false;
    // ---- dJ/dv = 2 dt^2 v dJ/dc = 2 A / v (FP32)
    const size_t npts = (size_t)h->npts;
    const bool dev_out = is_device_ptr(grad_v);
    float *dst = grad_v;
    if (!dev_out) {
        if (!h->st_vol) MMOD_CK(h, cudaMalloc(&h->st_vol, sizeof(float) * npts));
        dst = h->st_vol;
    }
    MMOD_CK(h, launch_grad_to_velocity(gw.gradc, h->vel_copy, c.nx, c.ny, c.nz, h->nxp, dst, s));
    ++launches;
    if (!dev_out) {
        MMOD_CK(h, cudaMemcpyAsync(grad_v, dst, sizeof(float) * npts, cudaMemcpyDeviceToHost, s));
        MMOD_CK(h, cudaStreamSynchronize(s));
    }
    h->last_launches = launches;
    return check_latched(h);
}

MMOD_API long long mmod_gradient_memory(const mmod_handle *h, int ckpt_count, int ckpt_dtype) {
    if (!h || ckpt_count < 1) return -1;
    if (ckpt_dtype != MMOD_CKPT_FP32 && ckpt_dtype != MMOD_CKPT_BF16 && ckpt_dtype != MMOD_CKPT_FP16 &&
        ckpt_dtype != MMOD_CKPT_BFP16)
        return -1;
    int nslot = 0, nwork = 0, seglen = 0;
    grad_layout(h, ckpt_count, ckpt_dtype, &nslot, &nwork, &seglen);
    const long long vb = 4LL * h->vol;
    const long long eb = ckpt_dtype == MMOD_CKPT_FP32 ? 4 : 2;
    return (long long)(nwork + 3) * vb + (long long)nslot * 2 * h->vol * eb +
           4LL * nslot * 2 * (long long)ckpt_scales(h, ckpt_dtype);
}

MMOD_API mmod_status mmod_dot(const float *a, const float *b, long long n, double *out, mmod_stream stream) {
    if (!a || !b || !out || n < 0) return MMOD_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    double *d = nullptr;
    if (cudaMallocAsync(&d, sizeof(double), s) != cudaSuccess) return MMOD_ERR_OOM;
    cudaError_t e = cudaMemsetAsync(d, 0, sizeof(double), s);
    if (e == cudaSuccess) e = launch_dot(a, b, n, d, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, d, sizeof(double), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(d, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? MMOD_OK : MMOD_ERR_CUDA;
}
