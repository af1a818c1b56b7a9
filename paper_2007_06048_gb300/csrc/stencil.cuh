// Per-point arithmetic of the propagator, shared by every step kernel.
//
// Sec. 3 Laplacian in the paper's pair-difference form, per axis and offset m:
//     w_am * ((p(+m) + p(-m)) - 2p),   w_am = c_m / h_a^2,
// accumulated in the fixed order x1..x4, y1..y4, z1..z4.  In FP32 this form
// keeps the small Laplacian accurate (the differences are formed before the
// weights are applied); folding the centre weight -2 sum_m w_am into one term
// loses about a decimal digit over 1000 steps.
//
// Eq. 5 and the damping update (e = dt * eta, e = 0 inside):
//     num     = 2p - pp + e * pp + c * lap (+ s * w[n] at a source)
//     u^{n+1} = num / (1 + e)
// With e = 0 the multiply-add and the division by 1 are exact, so a kernel may
// use the undamped form in the inner region and get identical bits.
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

__device__ __forceinline__ float pair_acc(float acc, float w, float a, float b, float two_p) {
    return __fmaf_rn(w, __fsub_rn(__fadd_rn(a, b), two_p), acc);
}

// Undamped numerator 2p - pp + c * lap.
__device__ __forceinline__ float num_inner(float two_p, float pp, float c, float lap) {
    return __fmaf_rn(c, lap, __fsub_rn(two_p, pp));
}

// Damped numerator 2p - (1 - e) pp + c * lap.
__device__ __forceinline__ float num_damped(float two_p, float pp, float c, float lap, float e) {
    return __fmaf_rn(c, lap, __fmaf_rn(e, pp, __fsub_rn(two_p, pp)));
}

__device__ __forceinline__ float add_source(float num, float scale, float w) {
    return __fmaf_rn(scale, w, num);
}

__device__ __forceinline__ float finish_damped(float num, float e) {
    return __fdiv_rn(num, __fadd_rn(1.0f, e));
}

}  // namespace mmod
