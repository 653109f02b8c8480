// Device helpers shared by the step kernels and the diagnostics kernels.
#pragma once

#include "ann_internal.cuh"

namespace ann {

// One periodic shift into [0, L) (a step moves a particle far less than L); returns the shift
// count (-1, 0, +1) so that unwrapped = wrapped + count * L.
__device__ __forceinline__ int wrap_count(double &a, double L)
{
    int k = 0;
    if (a < 0.0) {
        a = a + L;
        k = -1;
    }
    if (a >= L) {
        a = a - L;
        k += 1;
    }
    return k;
}

__device__ __forceinline__ double wrap_d(double a, double L)
{
    if (a < 0.0) a = a + L;
    if (a >= L) a = a - L;
    return a;
}

// x in [+0, L)?  Non-negative doubles order like their bit patterns, so two integer compares decide
// it; negative values, -0, NaN and values >= L fail.
__device__ __forceinline__ bool in_box(double x, long long bitsL)
{
    long long bx = __double_as_longlong(x);
    return bx >= 0 && bx < bitsL;
}

// Two-lane FP32 arithmetic (one instruction issues both lanes, each lane rounded as the scalar
// operation).  The pair passes are issue-bound, and their x/y arithmetic pairs up naturally.
__device__ __forceinline__ float2 f2(float x, float y) { return make_float2(x, y); }
__device__ __forceinline__ float2 bc(float s) { return make_float2(s, s); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, f2(-b.x, -b.y)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// 1/sqrt(r2) by the hardware approximation (r2 is a squared pair distance: never subnormal
// unless two particles coincide, where both forms give +inf).
__device__ __forceinline__ float rsqrt_approx(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Quintic kernel of Eq. (18) in branch-free form: with t_k = max(k - b, 0),
//   W = a_d [t3^5 - 6 t2^5 + 15 t1^5],   F = W'(b) / (h r) = a_d/h [-5 t3^4 + 30 t2^4 - 75 t1^4] / r,
// so that grad_i W_ij = F d_ij.  The constants a_d, -6 a_d, ... are folded on the host.  For true
// neighbours b < 3 up to FP32 rounding, and t3 needs no clamp (a rounding-negative t3 gives
// |t3|^4 ~ 1e-28); `clamp3` keeps it for candidates that may lie beyond the support, where it
// makes W = F = 0 exactly.  (t3, t2) travel as one two-lane value.
struct KernelPowers {
    float2 t, q;     // (t3, t2), (t3^4, t2^4)
    float t1, q1;    // t1, t1^4
    float rinv, r;   // 1/|d| and |d|
};

template <bool clamp3>
__device__ __forceinline__ KernelPowers kernel_powers(float r2, const DevParams &P)
{
    KernelPowers k;
    k.rinv = rsqrt_approx(r2);
    k.r = r2 * k.rinv;
    float bq = k.r * P.inv_h;
    k.t = add2(f2(3.f, 2.f), bc(-bq));
    if (clamp3) k.t.x = fmaxf(k.t.x, 0.f);
    k.t.y = fmaxf(k.t.y, 0.f);
    k.t1 = fmaxf(1.f - bq, 0.f);
    float2 sq = mul2(k.t, k.t);
    float s1 = k.t1 * k.t1;
    k.q = mul2(sq, sq);
    k.q1 = s1 * s1;
    return k;
}

__device__ __forceinline__ float kernel_w_of(const KernelPowers &k, const DevParams &P)
{
    float2 w = mul2(k.q, k.t);   // (t3^5, t2^5)
    return fmaf(P.ad, w.x, fmaf(P.kw6, w.y, P.kw15 * (k.q1 * k.t1)));
}

__device__ __forceinline__ float kernel_f_of(const KernelPowers &k, const DevParams &P)
{
    float2 f = mul2(f2(P.kf5, P.kf30), k.q);
    return fmaf(P.kf75, k.q1, f.x + f.y) * k.rinv;
}

template <bool clamp3>
__device__ __forceinline__ void kernel_wf(float r2, const DevParams &P, float &W, float &F, float &rinv)
{
    KernelPowers k = kernel_powers<clamp3>(r2, P);
    W = kernel_w_of(k, P);
    F = kernel_f_of(k, P);
    rinv = k.rinv;
}

template <bool clamp3>
__device__ __forceinline__ float kernel_w(float r2, const DevParams &P)
{
    return kernel_w_of(kernel_powers<clamp3>(r2, P), P);
}

// Squared length, one rounding per product as the support-test band allows.
__device__ __forceinline__ float len2(float2 d) { return fmaf(d.x, d.x, d.y * d.y); }

}  // namespace ann
