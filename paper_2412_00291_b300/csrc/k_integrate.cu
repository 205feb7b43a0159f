// Projective TSDF update (Sec. III-C.2) fused with the recursive Bayesian
// class update (Sec. III-C.3, Eq. bayesian_filter), one CTA per touched block
// (persistent grid-stride over the device-side list U_k), one voxel per thread
// per step, 512 voxels per block.
//
// Per voxel v of block b:
//   x_l   = R^T (nu v - t)            (its direction picks the pixel)
//   psi   = r_pixel - |x_l|           (projective distance, > 0 in front)
//   skip when the pixel is empty or psi < -tau
//   w     = clamp((psi + tau) / (2 tau), 0, 1)   (or 1 in constant mode)
//   D     = (W D + w min(psi, tau)) / (W + w),  W = W + w
//   if |psi| <= tau and the pixel carries a class likelihood L:
//       logP_c = max(logP_c + log L_c - logsumexp_c(logP + log L), floor)
//       label  = argmax_c logP_c (lowest class on ties)
//
// psi is formed as (r^2 - rho^2) / (r + rho) with r^2 and rho^2 carried as
// unevaluated float pairs, and the voxel's offset from the sensor carried
// in voxel units as integer + float pair, so that a 100 m range costs no
// absolute accuracy near the surface.
#include "kernels.h"

namespace stsdf {

template <bool F16>
__device__ __forceinline__ float2 load_dw(const MapDev &md, long long vox) {
    if (F16) return __half22float2(md.dw16[vox]);
    return md.dw32[vox];
}
template <bool F16>
__device__ __forceinline__ void store_dw(const MapDev &md, long long vox, float D, float W) {
    if (F16) md.dw16[vox] = __floats2half2_rn(D, W);
    else md.dw32[vox] = make_float2(D, W);
}
template <bool F16>
__device__ __forceinline__ float load_lp(const MapDev &md, long long j) {
    if (F16) return __half2float(md.lp16[j]);
    return md.lp32[j];
}
template <bool F16>
__device__ __forceinline__ void store_lp(const MapDev &md, long long j, float v) {
    if (F16) md.lp16[j] = __float2half_rn(v);
    else md.lp32[j] = v;
}

// NC > 0: class count known at compile time (register array); NC == 0: any C.
template <bool F16, int NC>
__global__ void __launch_bounds__(256) k_integrate(ScanConst sc, MapDev md, FrameDev fd) {
    __shared__ long long s_red[8];
    constexpr int MAXC_RT = 64;
    const int C = NC > 0 ? NC : sc.C;
    long long n_upd = 0, n_sem = 0;
    unsigned long long nt = *(volatile unsigned long long *)&fd.ctr[CT_TOUCHED];
    if (nt > (unsigned long long)md.max_blocks) nt = md.max_blocks;
    const float tau = sc.tau;
    for (unsigned long long li = blockIdx.x; li < nt; li += gridDim.x) {
        const int h = fd.touched[li];
        const int slot = md.vals[h];
        if (slot < 0) continue;
        int bx, by, bz;
        unpack_block(md.keys[h], bx, by, bz);
        for (int r = 0; r < 2; ++r) {
            const int vi = threadIdx.x + 256 * r;
            const int lx = vi & 7, ly = (vi >> 3) & 7, lz = vi >> 6;
            // offset from the sensor in voxel units: integer part exact, fraction as a float pair
            float s0, s1, s2, e0, e1, e2;
            two_sum((float)(8 * bx + lx - sc.k[0]), -sc.fhi[0], s0, e0);
            two_sum((float)(8 * by + ly - sc.k[1]), -sc.fhi[1], s1, e1);
            two_sum((float)(8 * bz + lz - sc.k[2]), -sc.fhi[2], s2, e2);
            e0 = __fsub_rn(e0, sc.flo[0]);
            e1 = __fsub_rn(e1, sc.flo[1]);
            e2 = __fsub_rn(e2, sc.flo[2]);
            // direction in the LiDAR frame (scale-free) -> pixel (Sec. III-C.1)
            const float x0 = sc.Rt[0] * s0 + sc.Rt[1] * s1 + sc.Rt[2] * s2;
            const float x1 = sc.Rt[3] * s0 + sc.Rt[4] * s1 + sc.Rt[5] * s2;
            const float x2 = sc.Rt[6] * s0 + sc.Rt[7] * s1 + sc.Rt[8] * s2;
            const float rr2 = x0 * x0 + x1 * x1 + x2 * x2;
            if (!(rr2 > 0.f)) continue;
            const float uc = (PI_F - atan2f(x1, x0)) * sc.inv_dphi;
            const float cz = fminf(fmaxf(x2 * rsqrtf(rr2), -1.f), 1.f);
            const float vc = (acosf(cz) - sc.theta0) * sc.inv_dtheta;
            int u = (int)floorf(uc + 0.5f);
            const int v = (int)floorf(vc + 0.5f);
            if (v < 0 || v >= sc.H) continue;
            if (u >= sc.W) u -= sc.W;
            if (u < 0) u += sc.W;
            const int p = v * sc.W + u;
            const float4 px = fd.pix[p];
            if (__float_as_int(px.w) < 0) continue;
            // rho^2 in voxel units, then metres^2, as float pairs
            float a, ae, b, be, c, ce, qh, ql, mh, ml, dh, dl;
            two_prod(s0, s0, a, ae);
            two_prod(s1, s1, b, be);
            two_prod(s2, s2, c, ce);
            ae = __fmaf_rn(2.f * s0, e0, ae);
            be = __fmaf_rn(2.f * s1, e1, be);
            ce = __fmaf_rn(2.f * s2, e2, ce);
            df_add(a, ae, b, be, qh, ql);
            df_add(qh, ql, c, ce, qh, ql);
            df_mul(qh, ql, sc.nu2hi, sc.nu2lo, mh, ml);
            df_add(px.y, px.z, -mh, -ml, dh, dl);
            const float rho = __fsqrt_rn(mh);
            const float psi = __fdiv_rn(__fadd_rn(dh, dl), __fadd_rn(px.x, rho));
            if (psi < -tau) continue;
            float w = 1.f;
            if (sc.weight_mode == 0) w = fminf(fmaxf(__fdiv_rn(psi + tau, 2.f * tau), 0.f), 1.f);
            if (!(w > 0.f)) continue;
            const float sdf = fminf(psi, tau);
            const long long vox = (long long)slot * BV + vi;
            const float2 dw = load_dw<F16>(md, vox);
            const float Wn = dw.y + w;
            store_dw<F16>(md, vox, __fdiv_rn(dw.y * dw.x + w * sdf, Wn), Wn);
            ++n_upd;
            if (fabsf(psi) <= tau && fd.sem_ok[p]) {
                const float *lrow = fd.logL + (long long)p * C;
                const long long base = (long long)slot * C * BV + vi;
                float m = -INFINITY;
                if (NC > 0) {
                    float av[NC > 0 ? NC : 1];
#pragma unroll
                    for (int cc = 0; cc < (NC > 0 ? NC : 1); ++cc) {
                        av[cc] = load_lp<F16>(md, base + (long long)cc * BV) + lrow[cc];
                        m = fmaxf(m, av[cc]);
                    }
                    float ssum = 0.f;
#pragma unroll
                    for (int cc = 0; cc < (NC > 0 ? NC : 1); ++cc) ssum += expf(av[cc] - m);
                    const float lse = m + logf(ssum);
                    int best = 0;
                    float bv = -INFINITY;
#pragma unroll
                    for (int cc = 0; cc < (NC > 0 ? NC : 1); ++cc) {
                        const float nv = fmaxf(av[cc] - lse, sc.logp_floor);
                        store_lp<F16>(md, base + (long long)cc * BV, nv);
                        const float stored = F16 ? __half2float(__float2half_rn(nv)) : nv;
                        if (stored > bv) {
                            bv = stored;
                            best = cc;
                        }
                    }
                    md.label[vox] = (uint8_t)best;
                } else {
                    float av[MAXC_RT];
                    for (int cc = 0; cc < C; ++cc) {
                        av[cc] = load_lp<F16>(md, base + (long long)cc * BV) + lrow[cc];
                        m = fmaxf(m, av[cc]);
                    }
                    float ssum = 0.f;
                    for (int cc = 0; cc < C; ++cc) ssum += expf(av[cc] - m);
                    const float lse = m + logf(ssum);
                    int best = 0;
                    float bv = -INFINITY;
                    for (int cc = 0; cc < C; ++cc) {
                        const float nv = fmaxf(av[cc] - lse, sc.logp_floor);
                        store_lp<F16>(md, base + (long long)cc * BV, nv);
                        const float stored = F16 ? __half2float(__float2half_rn(nv)) : nv;
                        if (stored > bv) {
                            bv = stored;
                            best = cc;
                        }
                    }
                    md.label[vox] = (uint8_t)best;
                }
                ++n_sem;
            }
        }
    }
    n_upd = block_sum(n_upd, s_red);
    n_sem = block_sum(n_sem, s_red);
    if (threadIdx.x == 0) {
        if (n_upd) atomicAdd(&fd.ctr[CT_UPD], (unsigned long long)n_upd);
        if (n_sem) atomicAdd(&fd.ctr[CT_SEM], (unsigned long long)n_sem);
    }
}

template <bool F16, int NC>
static int bps() {
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_integrate<F16, NC>, 256, 0);
    return n > 0 ? n : 1;
}

int integrate_blocks_per_sm(int storage, int C) {
    if (storage == 0) return C == 20 ? bps<false, 20>() : bps<false, 0>();
    return C == 20 ? bps<true, 20>() : bps<true, 0>();
}

void launch_integrate(const ScanConst &sc, const MapDev &md, const FrameDev &fd, int grid, cudaStream_t s) {
    if (md.storage == 0) {
        if (sc.C == 20) k_integrate<false, 20><<<grid, 256, 0, s>>>(sc, md, fd);
        else k_integrate<false, 0><<<grid, 256, 0, s>>>(sc, md, fd);
    } else {
        if (sc.C == 20) k_integrate<true, 20><<<grid, 256, 0, s>>>(sc, md, fd);
        else k_integrate<true, 0><<<grid, 256, 0, s>>>(sc, md, fd);
    }
}

}  // namespace stsdf
