// Projective TSDF update (Sec. III-C.2) and the recursive Bayesian class
// update (Sec. III-C.3, Eq. bayesian_filter).  k_tsdf: one warp per half of
// a touched block (256 voxels; grid-stride over the device-side list U_k,
// 8 warps per CTA); it lists the voxels whose class distribution must change,
// and k_semantic streams that list, one voxel per thread.
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
//
// Non-projective mode (Sec. III-C.2, Eq. distance): k_normals first builds
// the scan's normal image from the range image; each updated voxel then
// folds its pixel's normal into its gradient g_i and fuses Gamma(d_i, tau)
// instead of min(psi, tau) (weight and skip still on psi).
#include "frame_bodies.cuh"

namespace stsdf {

__global__ void __launch_bounds__(256) k_normals(ScanConst sc, FrameDev fd) {
    pdl_wait();
    pdl_trigger();
    const int np = sc.H * sc.W;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < np; p += gridDim.x * blockDim.x) normal_item(sc, fd.win, p);
}

// Work unit: half a touched block (256 voxels, z < 4 or z >= 4), so that
// the ~1.4 blocks per resident warp of a 64 x 2048 scan become ~2.8 units
// and the last round of the grid-stride loop idles fewer warps.
constexpr int TSDF_PARTS = 2;

template <bool F16, bool DIST, bool DBG = false>
__global__ void __launch_bounds__(256, 4) k_tsdf(ScanConst sc, MapDev md, FrameDev fd) {
    __shared__ TsdfWarpSmem s_w[8];   // per-warp class-update entries and band queue
    TsdfWarpSmem &tw = s_w[threadIdx.x >> 5];
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    long long n_upd = 0;
    pdl_wait();      // the per-point grid's touched list and range image
    pdl_trigger();   // the re-meshing grid may be scheduled now
    unsigned long long nt = *(volatile unsigned long long *)&fd.ctr[CT_TOUCHED];
    if (nt > (unsigned long long)md.max_blocks) nt = md.max_blocks;
    constexpr int PV = BV / TSDF_PARTS;
    for (long long u = warp; u < (long long)nt * TSDF_PARTS; u += nwarps) {
        const int part = (int)(u % TSDF_PARTS);
        tsdf_block_warp<F16, DIST, DBG>(sc, md, fd, fd.touched[u / TSDF_PARTS], tw, n_upd, part * PV,
                                        part * PV + PV);
    }
    long long cnt[1] = {n_upd};
    cta_count<1>(fd.ctr, {CT_UPD}, cnt);
}

template <bool F16, int NC>
__global__ void __launch_bounds__(256) k_semantic(ScanConst sc, MapDev md, FrameDev fd) {
    unsigned long long ns = *(volatile unsigned long long *)&fd.ctr[CT_SEM];
    if (ns > (unsigned long long)fd.sem_cap) ns = fd.sem_cap;
    for (unsigned long long e = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; e < ns;
         e += (unsigned long long)gridDim.x * blockDim.x)
        semantic_item<F16, NC>(sc, md, fd, e);
}

// The class update of the listed voxels with 20 classes, staged warp by warp
// through shared memory.  A thread's own record (96 B FP32 / 64 B FP16) and
// its winner's probability row (80 B) are each spread over several cache
// lines per warp instruction when every lane loads its own (32 lines per
// 16-byte load instruction: the L1's tag lookups, not DRAM, set the pace);
// here the 32 lanes copy consecutive 16-byte chunks of the warp's 32 records
// and rows (cp.async, global to shared without registers), so one
// instruction covers about five records in a handful of lines.  Each lane
// then updates its voxel from shared memory (class_update, the body every
// other path runs, so the results are the same bits) and the lanes write the
// records back chunk by chunk.
constexpr int SEMC_NC = 20;
template <bool F16>
struct SemCoop {
    static constexpr int RC = F16 ? 4 : 6;   // 16-byte chunks per record (32 halves / 24 floats)
    static constexpr int QC = SEMC_NC / 4;   // 16-byte chunks per probability row
    static constexpr int RB = 16 * RC;
};

__device__ __forceinline__ void cp_async16(void *dst_smem, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst_smem)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

template <bool F16>
__global__ void __launch_bounds__(256, 4) k_semantic_coop(ScanConst sc, MapDev md, FrameDev fd) {
    using S = SemCoop<F16>;
    __shared__ __align__(16) unsigned char s_rec[8][32 * S::RB];
    __shared__ __align__(16) float s_q[8][32 * SEMC_NC];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char *R = s_rec[wid];
    float *Q = s_q[wid];
    unsigned long long ns = *(volatile unsigned long long *)&fd.ctr[CT_SEM];
    if (ns > (unsigned long long)fd.sem_cap) ns = fd.sem_cap;
    const bool probs = sc.has_probs != 0;
    auto rec = [&](long long vox) -> unsigned char * {
        return F16 ? reinterpret_cast<unsigned char *>(md.lp16 + lp_index(md, vox, 0))
                   : reinterpret_cast<unsigned char *>(md.lp32 + lp_index(md, vox, 0));
    };
    for (unsigned long long base = ((unsigned long long)blockIdx.x * 8 + wid) * 32; base < ns;
         base += (unsigned long long)gridDim.x * 256) {
        const int nact = (int)min(32ull, ns - base);
        const bool act = lane < nact;
        const int2 ent = act ? fd.sem_list[base + lane] : make_int2(0, 0);
        // chunk k of the warp's records: record k / RC, 16-byte chunk k % RC
#pragma unroll
        for (int j = 0; j < S::RC; ++j) {
            const int k = 32 * j + lane, r = k / S::RC, c = k - r * S::RC;
            const int vox = __shfl_sync(0xffffffffu, ent.x, r);
            if (r < nact) cp_async16(R + r * S::RB + 16 * c, rec(vox) + 16 * c);
        }
        if (probs) {
#pragma unroll
            for (int j = 0; j < S::QC; ++j) {
                const int k = 32 * j + lane, r = k / S::QC, c = k - r * S::QC;
                const int idx = __shfl_sync(0xffffffffu, ent.y, r);
                if (r < nact) cp_async16(Q + r * SEMC_NC + 4 * c, sc.probs + (long long)idx * SEMC_NC + 4 * c);
            }
        }
        cp_async_wait_all();
        __syncwarp();
        if (act) {
            float av[SEMC_NC];
            unsigned char *rr = R + lane * S::RB;
            if (F16) {
                const uint4 *q = reinterpret_cast<const uint4 *>(rr);
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    const uint4 u = q[j];
                    const float2 f0 = __half22float2(*reinterpret_cast<const __half2 *>(&u.x));
                    const float2 f1 = __half22float2(*reinterpret_cast<const __half2 *>(&u.y));
                    const float2 f2 = __half22float2(*reinterpret_cast<const __half2 *>(&u.z));
                    const float2 f3 = __half22float2(*reinterpret_cast<const __half2 *>(&u.w));
                    const float g[8] = {f0.x, f0.y, f1.x, f1.y, f2.x, f2.y, f3.x, f3.y};
#pragma unroll
                    for (int k = 0; k < 8; ++k)
                        if (8 * j + k < SEMC_NC) av[8 * j + k] = g[k];
                }
            } else {
                const float4 *q = reinterpret_cast<const float4 *>(rr);
#pragma unroll
                for (int j = 0; j < SEMC_NC / 4; ++j) {
                    const float4 v = q[j];
                    av[4 * j] = v.x;
                    av[4 * j + 1] = v.y;
                    av[4 * j + 2] = v.z;
                    av[4 * j + 3] = v.w;
                }
            }
            const int best =
                class_update<F16, SEMC_NC>(sc, av, probs ? Q + lane * SEMC_NC : nullptr, probs ? 0 : sc.labels[ent.y]);
            // the new record in place, padding zero
            if (F16) {
                uint4 *q = reinterpret_cast<uint4 *>(rr);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    float f[8];
#pragma unroll
                    for (int k = 0; k < 8; ++k) f[k] = (8 * j + k < SEMC_NC) ? av[8 * j + k] : 0.f;
                    __half2 h0 = __floats2half2_rn(f[0], f[1]), h1 = __floats2half2_rn(f[2], f[3]);
                    __half2 h2 = __floats2half2_rn(f[4], f[5]), h3 = __floats2half2_rn(f[6], f[7]);
                    uint4 u;
                    u.x = *reinterpret_cast<unsigned *>(&h0);
                    u.y = *reinterpret_cast<unsigned *>(&h1);
                    u.z = *reinterpret_cast<unsigned *>(&h2);
                    u.w = *reinterpret_cast<unsigned *>(&h3);
                    q[j] = u;
                }
            } else {
                float4 *q = reinterpret_cast<float4 *>(rr);
#pragma unroll
                for (int j = 0; j < 6; ++j) {
                    float f[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) f[k] = (4 * j + k < SEMC_NC) ? av[4 * j + k] : 0.f;
                    q[j] = make_float4(f[0], f[1], f[2], f[3]);
                }
            }
            md.label[ent.x] = (uint8_t)best;
        }
        __syncwarp();
        // the records back, chunk by chunk as they came
#pragma unroll
        for (int j = 0; j < S::RC; ++j) {
            const int k = 32 * j + lane, r = k / S::RC, c = k - r * S::RC;
            const int vox = __shfl_sync(0xffffffffu, ent.x, r);
            if (r < nact)
                *reinterpret_cast<uint4 *>(rec(vox) + 16 * c) = *reinterpret_cast<const uint4 *>(R + r * S::RB + 16 * c);
        }
        __syncwarp();
    }
}

template <typename K>
static int occupancy(K kernel) {
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, 256, 0);
    return n > 0 ? n : 1;
}

int integrate_blocks_per_sm(int storage, int C, int dist_mode) {
    (void)C;
    if (dist_mode) return storage == 0 ? occupancy(k_tsdf<false, true>) : occupancy(k_tsdf<true, true>);
    return storage == 0 ? occupancy(k_tsdf<false, false>) : occupancy(k_tsdf<true, false>);
}

int semantic_blocks_per_sm(int storage, int C) {
    if (storage == 0) return C == 20 ? occupancy(k_semantic_coop<false>) : occupancy(k_semantic<false, 0>);
    return C == 20 ? occupancy(k_semantic_coop<true>) : occupancy(k_semantic<true, 0>);
}

void launch_integrate(const ScanConst &sc, const MapDev &md, const FrameDev &fd, int grid, cudaStream_t s) {
    auto k = sc.dist_mode ? (md.storage == 0 ? k_tsdf<false, true> : k_tsdf<true, true>)
                          : (md.storage == 0 ? k_tsdf<false, false> : k_tsdf<true, false>);
    if (fd.dbg_vox)   // decision record on: the recording instantiations
        k = sc.dist_mode ? (md.storage == 0 ? k_tsdf<false, true, true> : k_tsdf<true, true, true>)
                         : (md.storage == 0 ? k_tsdf<false, false, true> : k_tsdf<true, false, true>);
    launch_pdl(k, dim3(grid), dim3(256), 0, s, sc, md, fd);
}

void launch_normals(const ScanConst &sc, const FrameDev &fd, cudaStream_t s) {
    const int np = sc.H * sc.W;
    int grid = (np + 255) / 256;
    if (grid > 148 * 8) grid = 148 * 8;
    launch_pdl(k_normals, dim3(grid), dim3(256), 0, s, sc, fd);
}

void launch_semantic(const ScanConst &sc, const MapDev &md, const FrameDev &fd, int grid, cudaStream_t s) {
    // 20 classes with a label or 16-byte-aligned probability rows: the warp-staged kernel
    if (sc.C == SEMC_NC && (!sc.has_probs || sc.probs_vec4)) {
        if (md.storage == 0) k_semantic_coop<false><<<grid, 256, 0, s>>>(sc, md, fd);
        else k_semantic_coop<true><<<grid, 256, 0, s>>>(sc, md, fd);
        return;
    }
    if (md.storage == 0) {
        if (sc.C == 20) k_semantic<false, 20><<<grid, 256, 0, s>>>(sc, md, fd);
        else k_semantic<false, 0><<<grid, 256, 0, s>>>(sc, md, fd);
    } else {
        if (sc.C == 20) k_semantic<true, 20><<<grid, 256, 0, s>>>(sc, md, fd);
        else k_semantic<true, 0><<<grid, 256, 0, s>>>(sc, md, fd);
    }
}

}  // namespace stsdf
