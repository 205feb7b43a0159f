// Projective TSDF update (Sec. III-C.2) and the recursive Bayesian class
// update (Sec. III-C.3, Eq. bayesian_filter).  k_tsdf: one CTA per touched
// block (persistent grid-stride over the device-side list U_k), one voxel per
// thread per step, 512 voxels per block; it lists the voxels whose class
// distribution must change, and k_semantic streams that list.
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

// Projective TSDF update of every voxel of the touched blocks, one warp per
// block (16 voxels per lane, no block-wide barriers).  Voxels that also need
// the class update (|psi| <= tau, pixel with a likelihood) are appended to a
// compact list (voxel, pixel), warp-aggregated so that the list keeps voxel
// order within each warp.  Each block also queues itself and its lower
// neighbours for re-meshing, and a block allocated in this frame links
// itself with its neighbours.
// Offsets o (bit o, e_o = (o & 1, o >> 1 & 1, o >> 2)) whose lower neighbour
// b - e_o reads a voxel of b: those with e_o inside the set Z of axes on which
// the voxel sits at local coordinate 0.  Byte Z of the table is that set of o.
constexpr unsigned long long remesh_table() {
    unsigned long long t = 0;
    for (int z = 0; z < 8; ++z)
        for (int o = 0; o < 8; ++o)
            if ((o & ~z) == 0) t |= 1ull << (8 * z + o);
    return t;
}
constexpr unsigned long long REMESH_TABLE = remesh_table();
static_assert(REMESH_TABLE == 0xFF5533110F050301ull, "re-mesh offset table");

__device__ __forceinline__ unsigned remesh_offsets(int vi) {
    const int z = ((vi & 7) == 0 ? 1 : 0) | (((vi >> 3) & 7) == 0 ? 2 : 0) | ((vi >> 6) == 0 ? 4 : 0);
    return (unsigned)(REMESH_TABLE >> (8 * z)) & 0xffu;
}

// One voxel of the block: pixel, projective psi, running-average update,
// and the class-update list entry.
template <bool F16>
__device__ __forceinline__ void tsdf_voxel(const ScanConst &sc, const MapDev &md, const FrameDev &fd, int slot,
                                           int bx, int by, int bz, int vi, long long &n_upd, unsigned &remesh,
                                           int2 *wbuf, int &wcount) {
    const int lane = threadIdx.x & 31;
    const float tau = sc.tau;
    const int lx = vi & 7, ly = (vi >> 3) & 7, lz = vi >> 6;
    // offset from the sensor in voxel units: exact integer part minus the fraction's high part
    const float m0 = (float)(8 * bx + lx - sc.k[0]), m1 = (float)(8 * by + ly - sc.k[1]),
                m2 = (float)(8 * bz + lz - sc.k[2]);
    const float s0 = m0 - sc.fhi[0], s1 = m1 - sc.fhi[1], s2 = m2 - sc.fhi[2];
    // direction in the LiDAR frame (scale-free) -> pixel (Sec. III-C.1)
    const float x0 = sc.Rt[0] * s0 + sc.Rt[1] * s1 + sc.Rt[2] * s2;
    const float x1 = sc.Rt[3] * s0 + sc.Rt[4] * s1 + sc.Rt[5] * s2;
    const float x2 = sc.Rt[6] * s0 + sc.Rt[7] * s1 + sc.Rt[8] * s2;
    const float rr2 = x0 * x0 + x1 * x1 + x2 * x2;
    bool upd = false, sem = false;
    int p = 0;
    if (rr2 > 0.f) {
        const float irr = rsqrtf(rr2);
        const float uc = (PI_F - atan2f(x1, x0)) * sc.inv_dphi;
        const float vc = (acosf(fminf(fmaxf(x2 * irr, -1.f), 1.f)) - sc.theta0) * sc.inv_dtheta;
        int u = (int)floorf(uc + 0.5f);
        const int v = (int)floorf(vc + 0.5f);
        if (u >= sc.W) u -= sc.W;
        if (u < 0) u += sc.W;
        if (v >= 0 && v < sc.H) {
            p = v * sc.W + u;
            const float4 px = fd.pix[p];
            if (__float_as_int(px.w) >= 0) {
                // plain FP32 psi is within ~1e-5 m of the exact value; away from +-tau it
                // decides the update exactly: beyond +tau (+1 mm) sdf = tau and w = 1, below
                // -tau (-1 mm) nothing; only the band in between needs the float-pair psi
                float psi = px.x - sc.nu * (rr2 * irr);
                float sdf = tau, w = 1.f;
                upd = psi >= -tau - 1e-3f;
                if (upd && psi <= tau + 1e-3f) {
                    float e0, e1, e2, t0, t1, t2;
                    two_sum(m0, -sc.fhi[0], t0, e0);
                    two_sum(m1, -sc.fhi[1], t1, e1);
                    two_sum(m2, -sc.fhi[2], t2, e2);
                    e0 = __fsub_rn(e0, sc.flo[0]);
                    e1 = __fsub_rn(e1, sc.flo[1]);
                    e2 = __fsub_rn(e2, sc.flo[2]);
                    // rho^2 in voxel units, then metres^2, as float pairs; psi = (r^2 - rho^2) / (r + rho)
                    float a, ae, b, be, c, ce, qh, ql, mh, ml, dh, dl;
                    two_prod(t0, t0, a, ae);
                    two_prod(t1, t1, b, be);
                    two_prod(t2, t2, c, ce);
                    ae = __fmaf_rn(2.f * t0, e0, ae);
                    be = __fmaf_rn(2.f * t1, e1, be);
                    ce = __fmaf_rn(2.f * t2, e2, ce);
                    df_add(a, ae, b, be, qh, ql);
                    df_add(qh, ql, c, ce, qh, ql);
                    df_mul(qh, ql, sc.nu2hi, sc.nu2lo, mh, ml);
                    df_add(px.y, px.z, -mh, -ml, dh, dl);
                    psi = __fdividef(dh + dl, px.x + mh * rsqrtf(mh));
                    sdf = fminf(psi, tau);
                    if (sc.weight_mode == 0) w = fminf(fmaxf((psi + tau) * sc.inv_2tau, 0.f), 1.f);
                    upd = psi >= -tau && w > 0.f;
                    sem = upd && fabsf(psi) <= tau && fd.sem_ok[p];
                }
                if (upd) {
                    const long long vox = (long long)slot * BV + vi;
                    const float2 dw = load_dw<F16>(md, vox);
                    const float Wn = dw.y + w;
                    store_dw<F16>(md, vox, __fdividef(dw.y * dw.x + w * sdf, Wn), Wn);
                    ++n_upd;
                    remesh |= remesh_offsets(vi);
                }
            }
        }
    }
    // class-update entries collect in the warp's shared buffer (one global append per block)
    const unsigned mk = __ballot_sync(0xffffffffu, sem);
    if (sem) wbuf[wcount + __popc(mk & ((1u << lane) - 1u))] = make_int2(slot * BV + vi, p);
    wcount += __popc(mk);
}

template <bool F16>
__global__ void __launch_bounds__(256, 6) k_tsdf(ScanConst sc, MapDev md, FrameDev fd) {
    __shared__ int2 s_buf[8][BV];   // per-warp class-update entries of the current block
    const int lane = threadIdx.x & 31;
    int2 *wbuf = s_buf[threadIdx.x >> 5];
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    long long n_upd = 0;
    unsigned long long nt = *(volatile unsigned long long *)&fd.ctr[CT_TOUCHED];
    if (nt > (unsigned long long)md.max_blocks) nt = md.max_blocks;
    for (long long li = warp; li < (long long)nt; li += nwarps) {
        const int h = fd.touched[li];
        const int slot = md.vals[h];
        if (slot < 0) continue;
        const uint64_t key = md.keys[h];
        int bx, by, bz;
        unpack_block(key, bx, by, bz);
        // a block allocated in this frame links itself with its neighbours
        if (lane >= 8 && lane < 15 && md.slot_frame[slot] == sc.frame) link_block(md, key, slot, lane - 7);
        unsigned remesh = 0;
        int wcount = 0;
#pragma unroll 1
        for (int vi = lane; vi < BV; vi += 32)
            tsdf_voxel<F16>(sc, md, fd, slot, bx, by, bz, vi, n_upd, remesh, wbuf, wcount);
        __syncwarp();
        // one append of the block's class-update entries
        if (wcount) {
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(&fd.ctr[CT_SEM], (unsigned long long)wcount);
            base = __shfl_sync(0xffffffffu, base, 0);
            for (int i = lane; i < wcount; i += 32) {
                if (base + i < (unsigned long long)fd.sem_cap) fd.sem_list[base + i] = wbuf[i];
                else atomicOr(&md.st->err, ERR_LIST_FULL);
            }
        }
        // queue for re-meshing this block (if any voxel changed) and each lower
        // neighbour b - e whose cubes read a changed voxel of b, once per frame each
        // (the block's own links: set before, or just above by this warp)
        remesh = __reduce_or_sync(0xffffffffu, remesh);
        bool q = false;
        int hs = -1;
        if (lane < 8 && ((remesh >> lane) & 1u)) {
            hs = lane == 0 ? slot : md.nbr[slot * 16 + 8 + lane];
            q = hs >= 0 && atomicExch(&md.dstamp_slot[hs], sc.frame) != sc.frame;
        }
        const unsigned mq = __ballot_sync(0xffffffffu, q);
        if (mq) {
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(&fd.ctr[CT_DIRTY], (unsigned long long)__popc(mq));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (q) {
                const unsigned long long idx = base + __popc(mq & ((1u << lane) - 1u));
                if (idx < (unsigned long long)md.max_blocks) fd.dirty[idx] = hs;
                else atomicOr(&md.st->err, ERR_LIST_FULL);
            }
        }
        __syncwarp();
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) n_upd += __shfl_xor_sync(0xffffffffu, n_upd, o);
    if (lane == 0 && n_upd) atomicAdd(&fd.ctr[CT_UPD], (unsigned long long)n_upd);
}

// Recursive Bayesian class update (Eq. bayesian_filter) of the listed voxels,
// one voxel per thread: logP_c += log L_c, renormalise by logsumexp, floor,
// and refresh the voxel's argmax label.  A voxel's classes form one record of
// whole 32-byte sectors (FP32: 24 floats, FP16: 32 halves for 20 classes),
// read and written with vector accesses, padding included.
template <bool F16, int NC>
__device__ __forceinline__ void load_record(const MapDev &md, long long vox, float *av) {
    if (F16) {
        const uint4 *q = reinterpret_cast<const uint4 *>(md.lp16 + lp_index(md, vox, 0));
#pragma unroll
        for (int j = 0; j < NC / 8; ++j) {
            const uint4 u = q[j];
            const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&u.x));
            const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&u.y));
            const float2 c = __half22float2(*reinterpret_cast<const __half2 *>(&u.z));
            const float2 d = __half22float2(*reinterpret_cast<const __half2 *>(&u.w));
            av[8 * j] = a.x; av[8 * j + 1] = a.y; av[8 * j + 2] = b.x; av[8 * j + 3] = b.y;
            av[8 * j + 4] = c.x; av[8 * j + 5] = c.y; av[8 * j + 6] = d.x; av[8 * j + 7] = d.y;
        }
#pragma unroll
        for (int cc = (NC / 8) * 8; cc < NC; ++cc) av[cc] = __half2float(md.lp16[lp_index(md, vox, cc)]);
    } else {
        const float4 *q = reinterpret_cast<const float4 *>(md.lp32 + lp_index(md, vox, 0));
#pragma unroll
        for (int j = 0; j < NC / 4; ++j) {
            const float4 v = q[j];
            av[4 * j] = v.x; av[4 * j + 1] = v.y; av[4 * j + 2] = v.z; av[4 * j + 3] = v.w;
        }
#pragma unroll
        for (int cc = (NC / 4) * 4; cc < NC; ++cc) av[cc] = md.lp32[lp_index(md, vox, cc)];
    }
}

// Store a full padded record (NCP elements, zeros beyond NC) so that every
// written sector is written whole.
template <bool F16, int NC, int NCP>
__device__ __forceinline__ void store_record(const MapDev &md, long long vox, const float *nv) {
    if (F16) {
        uint4 *q = reinterpret_cast<uint4 *>(md.lp16 + lp_index(md, vox, 0));
#pragma unroll
        for (int j = 0; j < NCP / 8; ++j) {
            float f[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) f[k] = (8 * j + k < NC) ? nv[8 * j + k] : 0.f;
            uint4 u;
            __half2 h0 = __floats2half2_rn(f[0], f[1]), h1 = __floats2half2_rn(f[2], f[3]);
            __half2 h2 = __floats2half2_rn(f[4], f[5]), h3 = __floats2half2_rn(f[6], f[7]);
            u.x = *reinterpret_cast<unsigned *>(&h0);
            u.y = *reinterpret_cast<unsigned *>(&h1);
            u.z = *reinterpret_cast<unsigned *>(&h2);
            u.w = *reinterpret_cast<unsigned *>(&h3);
            q[j] = u;
        }
    } else {
        float4 *q = reinterpret_cast<float4 *>(md.lp32 + lp_index(md, vox, 0));
#pragma unroll
        for (int j = 0; j < NCP / 4; ++j) {
            float f[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) f[k] = (4 * j + k < NC) ? nv[4 * j + k] : 0.f;
            q[j] = make_float4(f[0], f[1], f[2], f[3]);
        }
    }
}

template <bool F16, int NC>
__global__ void __launch_bounds__(256) k_semantic(ScanConst sc, MapDev md, FrameDev fd) {
    constexpr int MAXC_RT = 64;
    // padded record length for the compile-time class count (32-byte sectors)
    constexpr int NCP = NC > 0 ? (F16 ? ((NC + 15) / 16) * 16 : ((NC + 7) / 8) * 8) : 1;
    unsigned long long ns = *(volatile unsigned long long *)&fd.ctr[CT_SEM];
    if (ns > (unsigned long long)fd.sem_cap) ns = fd.sem_cap;
    const int C = NC > 0 ? NC : sc.C;
    for (unsigned long long e = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; e < ns;
         e += (unsigned long long)gridDim.x * blockDim.x) {
        const int2 ent = fd.sem_list[e];
        const long long vox = ent.x;
        const float *lrow = fd.logL + (long long)ent.y * C;
        float m = -INFINITY;
        if (NC > 0) {
            float av[NC > 0 ? NC : 1];
            load_record<F16, (NC > 0 ? NC : 1)>(md, vox, av);
            if (NC % 4 == 0) {
#pragma unroll
                for (int cc = 0; cc < (NC > 0 ? NC : 1); cc += 4) {
                    const float4 l4 = *reinterpret_cast<const float4 *>(lrow + cc);
                    av[cc] += l4.x;
                    av[cc + 1] += l4.y;
                    av[cc + 2] += l4.z;
                    av[cc + 3] += l4.w;
                }
            } else {
#pragma unroll
                for (int cc = 0; cc < (NC > 0 ? NC : 1); ++cc) av[cc] += lrow[cc];
            }
#pragma unroll
            for (int cc = 0; cc < (NC > 0 ? NC : 1); ++cc) m = fmaxf(m, av[cc]);
            float ssum = 0.f;
#pragma unroll
            for (int cc = 0; cc < (NC > 0 ? NC : 1); ++cc) ssum += expf(av[cc] - m);
            const float lse = m + logf(ssum);
            int best = 0;
            float bv = -INFINITY;
#pragma unroll
            for (int cc = 0; cc < (NC > 0 ? NC : 1); ++cc) {
                av[cc] = fmaxf(av[cc] - lse, sc.logp_floor);
                const float stored = F16 ? __half2float(__float2half_rn(av[cc])) : av[cc];
                if (stored > bv) {
                    bv = stored;
                    best = cc;
                }
            }
            store_record<F16, (NC > 0 ? NC : 1), NCP>(md, vox, av);
            md.label[vox] = (uint8_t)best;
        } else {
            float av[MAXC_RT];
            for (int cc = 0; cc < C; ++cc) {
                av[cc] = load_lp<F16>(md, lp_index(md, vox, cc)) + lrow[cc];
                m = fmaxf(m, av[cc]);
            }
            float ssum = 0.f;
            for (int cc = 0; cc < C; ++cc) ssum += expf(av[cc] - m);
            const float lse = m + logf(ssum);
            int best = 0;
            float bv = -INFINITY;
            for (int cc = 0; cc < C; ++cc) {
                const float nv = fmaxf(av[cc] - lse, sc.logp_floor);
                store_lp<F16>(md, lp_index(md, vox, cc), nv);
                const float stored = F16 ? __half2float(__float2half_rn(nv)) : nv;
                if (stored > bv) {
                    bv = stored;
                    best = cc;
                }
            }
            md.label[vox] = (uint8_t)best;
        }
    }
}

template <typename K>
static int occupancy(K kernel) {
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, 256, 0);
    return n > 0 ? n : 1;
}

int integrate_blocks_per_sm(int storage, int C) {
    (void)C;
    return storage == 0 ? occupancy(k_tsdf<false>) : occupancy(k_tsdf<true>);
}

int semantic_blocks_per_sm(int storage, int C) {
    if (storage == 0) return C == 20 ? occupancy(k_semantic<false, 20>) : occupancy(k_semantic<false, 0>);
    return C == 20 ? occupancy(k_semantic<true, 20>) : occupancy(k_semantic<true, 0>);
}

void launch_integrate(const ScanConst &sc, const MapDev &md, const FrameDev &fd, int grid, cudaStream_t s) {
    if (md.storage == 0) k_tsdf<false><<<grid, 256, 0, s>>>(sc, md, fd);
    else k_tsdf<true><<<grid, 256, 0, s>>>(sc, md, fd);
}

void launch_semantic(const ScanConst &sc, const MapDev &md, const FrameDev &fd, int grid, cudaStream_t s) {
    if (md.storage == 0) {
        if (sc.C == 20) k_semantic<false, 20><<<grid, 256, 0, s>>>(sc, md, fd);
        else k_semantic<false, 0><<<grid, 256, 0, s>>>(sc, md, fd);
    } else {
        if (sc.C == 20) k_semantic<true, 20><<<grid, 256, 0, s>>>(sc, md, fd);
        else k_semantic<true, 0><<<grid, 256, 0, s>>>(sc, md, fd);
    }
}

}  // namespace stsdf
