// Measurement preprocessing (Sec. III-C.1), second half: the per-pixel table
// of the range image whose winners k_points (k_alloc.cu) decided.
#include "kernels.h"

namespace stsdf {

// Per pixel: the winner's range r, r^2 as an exact float pair, its index, and
// its class log-likelihood row log P(O = l | I_k) of Eq. (bayesian_filter)
// (or no likelihood when the winner carries no valid label).
__global__ void __launch_bounds__(256) k_pixels(const float *__restrict__ pts, const int32_t *__restrict__ labels,
                                                const float *__restrict__ probs, ScanConst sc, FrameDev fd) {
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
    const int C = sc.C;
    float *out = fd.logL + (long long)p * C;
    if (sc.has_probs) {
        const float *q = probs + (long long)idx * C;
        if (sc.probs_vec4) {
            for (int cc = 0; cc < C; cc += 4) {
                const float4 v = *reinterpret_cast<const float4 *>(q + cc);
                *reinterpret_cast<float4 *>(out + cc) =
                    make_float4(logf(fmaxf(v.x, sc.lik_floor)), logf(fmaxf(v.y, sc.lik_floor)),
                                logf(fmaxf(v.z, sc.lik_floor)), logf(fmaxf(v.w, sc.lik_floor)));
            }
        } else {
            for (int cc = 0; cc < C; ++cc) out[cc] = logf(fmaxf(q[cc], sc.lik_floor));
        }
        fd.sem_ok[p] = 1;
    } else {
        const int l = labels[idx];
        const int ok = (l >= 0 && l < C);
        if (ok)
            for (int cc = 0; cc < C; ++cc) out[cc] = (cc == l) ? sc.log_phit : sc.log_pmiss;
        fd.sem_ok[p] = (uint8_t)ok;
    }
}

void launch_pixels(const float *pts, const int32_t *labels, const float *probs, const ScanConst &sc,
                   const FrameDev &fd, cudaStream_t s) {
    const long long np = (long long)sc.H * sc.W;
    k_pixels<<<(unsigned)((np + 255) / 256), 256, 0, s>>>(pts, labels, probs, sc, fd);
}

}  // namespace stsdf
