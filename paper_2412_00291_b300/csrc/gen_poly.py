"""Generate poly_approx.h: polynomial approximations used to find a voxel's pixel.

    python paper_2412_00291_b300/csrc/gen_poly.py

Method: least-squares fit at Chebyshev nodes (a near-minimax polynomial) of
  atan(t) / t  as a polynomial of degree 7 in s = t^2 on t in [0, 1], and
  asin(c) / c  as a polynomial of degree 4 in s = c^2 on c in [0, 1/2].
The script checks the error of each polynomial evaluated in IEEE single
precision (Horner in s, then one multiply by t or c) against numpy's double
precision arctan / arcsin on a dense grid and writes the bound into the header.
"""
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def cheb_nodes(a, b, n):
    k = np.arange(n)
    return 0.5 * (a + b) + 0.5 * (b - a) * np.cos((2 * k + 1) * np.pi / (2 * n))


def fit(ratio, a, b, deg, n=4000):
    s = cheb_nodes(a, b, n)
    A = np.vander(s, deg + 1, increasing=True)
    c, *_ = np.linalg.lstsq(A, ratio(s), rcond=None)
    return c.astype(np.float32)


def horner32(c, s):
    r = np.float32(c[-1]) * np.ones_like(s, dtype=np.float32)
    for ci in c[-2::-1]:
        r = (r * s + np.float32(ci)).astype(np.float32)
    return r


def max_err(c, x, ref):
    x32 = x.astype(np.float32)
    approx = (x32 * horner32(c, (x32 * x32).astype(np.float32))).astype(np.float64)
    return float(np.abs(approx - ref(x)).max())


def main():
    atan_c = fit(lambda s: np.arctan(np.sqrt(s)) / np.sqrt(np.maximum(s, 1e-300)), 0.0, 1.0, 7)
    asin_c = fit(lambda s: np.arcsin(np.sqrt(s)) / np.sqrt(np.maximum(s, 1e-300)), 0.0, 0.25, 4)
    t = np.linspace(0.0, 1.0, 2000001)
    x = np.linspace(0.0, 0.5, 2000001)
    e_atan = max_err(atan_c, t, np.arctan)
    e_asin = max_err(asin_c, x, np.arcsin)
    lines = [
        "// Generated by gen_poly.py (least-squares fit at Chebyshev nodes); do not edit.",
        "// atan(t) = t * P(t^2), t in [0, 1]: max error %.3g rad evaluated in FP32." % e_atan,
        "// asin(c) = c * Q(c^2), |c| <= 1/2: max error %.3g rad evaluated in FP32." % e_asin,
        "#pragma once",
        "",
        "namespace stsdf {",
        "",
        "// P(s) and Q(s) by Horner's rule with fused multiply-adds",
        "__host__ __device__ __forceinline__ float atan_p(float s) {",
        "    float p = %.9ef;" % atan_c[-1],
    ] + ["    p = fmaf(p, s, %.9ef);" % v for v in atan_c[-2::-1]] + [
        "    return p;",
        "}",
        "__host__ __device__ __forceinline__ float asin_q(float s) {",
        "    float q = %.9ef;" % asin_c[-1],
    ] + ["    q = fmaf(q, s, %.9ef);" % v for v in asin_c[-2::-1]] + [
        "    return q;",
        "}",
        "",
        "}  // namespace stsdf",
        "",
    ]
    with open(os.path.join(HERE, "poly_approx.h"), "w") as f:
        f.write("\n".join(lines))
    print("atan max err %.3g, asin max err %.3g" % (e_atan, e_asin))


if __name__ == "__main__":
    main()
