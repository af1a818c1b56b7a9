// Per-point arithmetic of the propagator, shared by every step kernel.
//
// Sec. 3 Laplacian in the paper's pair-difference form, per axis and offset m:
//     w_am * ((p(+m) + p(-m)) - 2p),   w_am = c_m / h_a^2,
// summed per axis in the order m = 1..4 (the first term is a product), then
// lap = (l_x + l_y) + l_z.  Three independent chains instead of one keep the
// FMA pipes busy with few warps.  In FP32 this form
// keeps the small Laplacian accurate (the differences are formed before the
// weights are applied); folding the centre weight -2 sum_m w_am into one term
// loses about a decimal digit over 1000 steps.
//
// Eq. 5 and the damping update (e = dt * eta, e = 0 inside):
//     num     = 2p - pp + e * pp + c * lap
//     r       = 1 / (1 + e): hardware approximate reciprocal refined by one
//               Newton-Raphson step r <- r + r (1 - d r); exactly 1 where e = 0
//     u^{n+1} = num * r  (+ (s * w[n]) * r at a source point)
// With e = 0 the multiply-add and the multiplication by r = 1 are exact, so a
// kernel may skip the damping arithmetic where e = 0 and get identical bits.
// The source term is added last so that kernels can apply it in a rare
// separate pass over the few source points.
//
// Explicit __fadd_rn / __fmaf_rn pin every rounding: the compiler cannot
// contract or reorder them, so all kernels produce the same bits per point.
#pragma once
#include <cuda_runtime.h>

namespace mmod {

constexpr int kRadius = 4;

struct Weights {
    float x[kRadius], y[kRadius], z[kRadius];   // c_m / h_a^2, m = 1..4
};

__device__ __forceinline__ float pair_first(float w, float a, float b, float two_p) {
    return __fmul_rn(w, __fsub_rn(__fadd_rn(a, b), two_p));
}

__device__ __forceinline__ float pair_acc(float acc, float w, float a, float b, float two_p) {
    return __fmaf_rn(w, __fsub_rn(__fadd_rn(a, b), two_p), acc);
}

__device__ __forceinline__ float lap_sum(float lx, float ly, float lz) {
    return __fadd_rn(__fadd_rn(lx, ly), lz);
}

// Undamped numerator 2p - pp + c * lap.
__device__ __forceinline__ float num_inner(float two_p, float pp, float c, float lap) {
    return __fmaf_rn(c, lap, __fsub_rn(two_p, pp));
}

// Damped numerator 2p - (1 - e) pp + c * lap.
__device__ __forceinline__ float num_damped(float two_p, float pp, float c, float lap, float e) {
    return __fmaf_rn(c, lap, __fmaf_rn(e, pp, __fsub_rn(two_p, pp)));
}

// 1 / d for d = 1 + e in [1, 8): rcp.approx (relative error below 2^-22) then
// one Newton-Raphson step for the reciprocal, r1 = r0 + r0 (1 - d r0), which
// squares the relative error.  For d = 1 both steps are exact (r = 1).
__device__ __forceinline__ float recip_nr(float d) {
    float r0;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r0) : "f"(d));
    return __fmaf_rn(r0, __fmaf_rn(-d, r0, 1.0f), r0);
}

__device__ __forceinline__ float damp_factor(float e) { return recip_nr(__fadd_rn(1.0f, e)); }

__device__ __forceinline__ float add_source(float out, float scale, float w, float r) {
    return __fmaf_rn(__fmul_rn(scale, w), r, out);
}

}  // namespace mmod
