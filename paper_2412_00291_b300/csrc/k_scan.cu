// Measurement preprocessing (Sec. III-C.1): the scan's range image.
//
// Each point goes to pixel u = round((pi - atan2(y, x)) / dphi) mod W,
// v = round((acos(z / r) - theta0) / dtheta); the nearest point wins a pixel
// (equal ranges: lower index), decided by one 64-bit atomicMin on
// (range bits << 32 | index), ranges being non-negative floats.
#include "kernels.h"

namespace stsdf {

__global__ void __launch_bounds__(256) k_range_image(const float *__restrict__ pts, ScanConst sc, FrameDev fd) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int valid = 0, inpix = 0;
    if (i < sc.n) {
        const float x = pts[3 * i], y = pts[3 * i + 1], z = pts[3 * i + 2];
        if (isfinite(x) && isfinite(y) && isfinite(z)) {
            const float l = range_f32(x, y, z);
            if (l >= sc.r_min && l <= sc.r_max && l > 0.f) {
                valid = 1;
                const float uc = (PI_F - atan2f(y, x)) * sc.inv_dphi;
                const float vc = (acosf(fminf(fmaxf(z / l, -1.f), 1.f)) - sc.theta0) * sc.inv_dtheta;
                int u = (int)floorf(uc + 0.5f);
                const int v = (int)floorf(vc + 0.5f);
                if (u >= sc.W) u -= sc.W;
                if (u < 0) u += sc.W;
                if (v >= 0 && v < sc.H) {
                    inpix = 1;
                    atomicMin(&fd.win[v * sc.W + u], ((unsigned long long)__float_as_uint(l) << 32) | (unsigned)i);
                }
            }
        }
    }
    const unsigned mv = __ballot_sync(0xffffffffu, valid), mp = __ballot_sync(0xffffffffu, inpix);
    if ((threadIdx.x & 31) == 0 && (mv | mp)) {
        atomicAdd(&fd.ctr[CT_VALID], (unsigned long long)__popc(mv));
        atomicAdd(&fd.ctr[CT_PIXEL], (unsigned long long)__popc(mp));
    }
}

// Per pixel: the winner's range r, r^2 as an exact float pair, its index,
// and whether it carries a class likelihood.
__global__ void __launch_bounds__(256) k_pixels(const float *__restrict__ pts, const int32_t *__restrict__ labels,
                                                ScanConst sc, FrameDev fd) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= sc.H * sc.W) return;
    const unsigned long long key = fd.win[p];
    if (key == ~0ull) {
        fd.pix[p] = make_float4(-1.f, 0.f, 0.f, __int_as_float(-1));
        fd.sem_ok[p] = 0;
        return;
    }
    const int idx = (int)(key & 0xffffffffu);
    const float r = __uint_as_float((unsigned)(key >> 32));
    const float x = pts[3 * idx], y = pts[3 * idx + 1], z = pts[3 * idx + 2];
    float a, ae, b, be, c, ce, sh, sl;
    two_prod(x, x, a, ae);
    two_prod(y, y, b, be);
    two_prod(z, z, c, ce);
    df_add(a, ae, b, be, sh, sl);
    df_add(sh, sl, c, ce, sh, sl);
    fd.pix[p] = make_float4(r, sh, sl, __int_as_float(idx));
    int ok = 1;
    if (!sc.has_probs) {
        const int l = labels[idx];
        ok = (l >= 0 && l < sc.C);
    }
    fd.sem_ok[p] = (uint8_t)ok;
}

// Per (pixel, class): log P(O = l | I_k) of Eq. (bayesian_filter) for the winner.
__global__ void __launch_bounds__(256) k_loglik(const int32_t *__restrict__ labels, const float *__restrict__ probs,
                                                ScanConst sc, FrameDev fd) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long np = (long long)sc.H * sc.W;
    if (e >= np * sc.C) return;
    const int p = (int)(e / sc.C), c = (int)(e - (long long)p * sc.C);
    const unsigned long long key = fd.win[p];
    if (key == ~0ull) return;
    const int idx = (int)(key & 0xffffffffu);
    float v;
    if (sc.has_probs) {
        v = logf(fmaxf(probs[(long long)idx * sc.C + c], sc.lik_floor));
    } else {
        const int l = labels[idx];
        v = (l == c) ? sc.log_phit : sc.log_pmiss;
    }
    fd.logL[e] = v;
}

void launch_range_image(const float *pts, const ScanConst &sc, const FrameDev &fd, cudaStream_t s) {
    if (sc.n <= 0) return;
    k_range_image<<<(unsigned)((sc.n + 255) / 256), 256, 0, s>>>(pts, sc, fd);
}

void launch_pixels(const float *pts, const int32_t *labels, const float *probs, const ScanConst &sc,
                   const FrameDev &fd, cudaStream_t s) {
    const long long np = (long long)sc.H * sc.W;
    k_pixels<<<(unsigned)((np + 255) / 256), 256, 0, s>>>(pts, labels, sc, fd);
    const long long ne = np * sc.C;
    k_loglik<<<(unsigned)((ne + 255) / 256), 256, 0, s>>>(labels, probs, sc, fd);
}

}  // namespace stsdf
