// Generated by gen_poly.py (least-squares fit at Chebyshev nodes); do not edit.
// atan(t) = t * P(t^2), t in [0, 1]: max error 1.78e-07 rad evaluated in FP32.
// asin(c) = c * Q(c^2), |c| <= 1/2: max error 1.32e-07 rad evaluated in FP32.
#pragma once

namespace stsdf {

// P(s) and Q(s) by Horner's rule with fused multiply-adds
__host__ __device__ __forceinline__ float atan_p(float s) {
    float p = -4.668773152e-03f;
    p = fmaf(p, s, 2.416618913e-02f);
    p = fmaf(p, s, -5.936710164e-02f);
    p = fmaf(p, s, 9.906096756e-02f);
    p = fmaf(p, s, -1.401658505e-01f);
    p = fmaf(p, s, 1.996923536e-01f);
    p = fmaf(p, s, -3.333196044e-01f);
    p = fmaf(p, s, 9.999998808e-01f);
    return p;
}
__host__ __device__ __forceinline__ float asin_q(float s) {
    float q = 5.050536245e-02f;
    q = fmaf(q, s, 3.972113505e-02f);
    q = fmaf(q, s, 7.546479255e-02f);
    q = fmaf(q, s, 1.666516364e-01f);
    q = fmaf(q, s, 1.000000119e+00f);
    return q;
}

}  // namespace stsdf
