// Projective TSDF update (Sec. III-C.2) and the recursive Bayesian class
// update (Sec. III-C.3, Eq. bayesian_filter).  k_tsdf: one warp per half of
// a touched block (256 voxels; grid-stride over the device-side list U_k,
// 8 warps per CTA); it lists the voxels whose class distribution must change,
// and the class update works that list off: k_semantic_coop (20 classes)
// warp by warp through shared memory, k_semantic (any class count) one voxel
// per thread.
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
// through shared memory (class_update_warp in frame_bodies.cuh): per warp 32
// list entries, their class records and the winners' probability rows copied
// as consecutive 16-byte chunks (cp.async) rather than one voxel per lane; a
// row shared by several of the 32 voxels is copied, and turned into log2
// likelihoods, once.  Four warps per CTA (20 KB of staging in FP32): two
// such CTAs fit on an SM beside the four re-meshing CTAs that run at the same
// time.
constexpr int SEM_WARPS = 4;
template <bool F16>
__global__ void __launch_bounds__(32 * SEM_WARPS, 8) k_semantic_coop(ScanConst sc, MapDev md, FrameDev fd) {
    using S = SemStage<F16>;
    __shared__ __align__(16) unsigned char s_rec[SEM_WARPS][32 * S::RB];
    __shared__ __align__(16) float s_q[SEM_WARPS][32 * SEM_NC];
    __shared__ int s_pt[SEM_WARPS][32];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char *R = s_rec[wid];
    float *Q = s_q[wid];
    unsigned long long ns = *(volatile unsigned long long *)&fd.ctr[CT_SEM];
    if (ns > (unsigned long long)fd.sem_cap) ns = fd.sem_cap;
    const bool probs = sc.has_probs != 0;
    for (unsigned long long base = ((unsigned long long)blockIdx.x * SEM_WARPS + wid) * 32; base < ns;
         base += (unsigned long long)gridDim.x * 32 * SEM_WARPS) {
        const int nact = (int)min(32ull, ns - base);
        const bool act = lane < nact;
        const int2 ent = act ? fd.sem_list[base + lane] : make_int2(0, 0);
        const float *qrow = nullptr;
        int nlog = 0;
        if (probs) {
            // the distinct winner points' probability rows, chunk by chunk like the records,
            // each once however many of the round's voxels share it (one lane of each group
            // of lanes with the same point lists it)
            const unsigned grp = __match_any_sync(0xffffffffu, act ? ent.y : -1 - lane);
            const int lead = __ffs(grp) - 1;
            const bool leader = act && lead == lane;
            const unsigned lm = __ballot_sync(0xffffffffu, leader);
            const int nu = __popc(lm);
            const int row = __popc(lm & ((1u << lead) - 1u));
            if (leader) s_pt[wid][row] = ent.y;
            __syncwarp();
            for (int k = lane; k < nu * (SEM_NC / 4); k += 32) {
                const int u = k / (SEM_NC / 4), c = k - u * (SEM_NC / 4);
                cp_async16(Q + u * SEM_NC + 4 * c, sc.probs + (long long)s_pt[wid][u] * SEM_NC + 4 * c);
            }
            qrow = Q + row * SEM_NC;
            nlog = nu * SEM_NC;
        }
        class_update_warp<F16, true>(sc, md, act, ent, R, qrow, Q, nlog);
    }
}

template <typename K>
static int occupancy(K kernel, int threads = 256) {
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, 0);
    return n > 0 ? n : 1;
}

void integrate_kernel_attributes() {
    const auto max_shared = [](auto k) {
        cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    };
    max_shared(k_tsdf<false, false>);
    max_shared(k_tsdf<true, false>);
    max_shared(k_tsdf<false, true>);
    max_shared(k_tsdf<true, true>);
    max_shared(k_tsdf<false, false, true>);
    max_shared(k_tsdf<true, false, true>);
    max_shared(k_tsdf<false, true, true>);
    max_shared(k_tsdf<true, true, true>);
    max_shared(k_semantic_coop<false>);
    max_shared(k_semantic_coop<true>);
    max_shared(k_semantic<false, 0>);
    max_shared(k_semantic<true, 0>);
    max_shared(k_semantic<false, 20>);
    max_shared(k_semantic<true, 20>);
    max_shared(k_normals);
}

int integrate_blocks_per_sm(int storage, int C, int dist_mode) {
    (void)C;
    if (dist_mode) return storage == 0 ? occupancy(k_tsdf<false, true>) : occupancy(k_tsdf<true, true>);
    return storage == 0 ? occupancy(k_tsdf<false, false>) : occupancy(k_tsdf<true, false>);
}

int semantic_blocks_per_sm(int storage, int C) {
    // (in 256-thread equivalents, so that the grids span the same warps)
    constexpr int per = 256 / (32 * SEM_WARPS);
    if (storage == 0)
        return C == 20 ? (occupancy(k_semantic_coop<false>, 32 * SEM_WARPS) + per - 1) / per
                       : occupancy(k_semantic<false, 0>);
    return C == 20 ? (occupancy(k_semantic_coop<true>, 32 * SEM_WARPS) + per - 1) / per
                   : occupancy(k_semantic<true, 0>);
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
    if (sc.C == SEM_NC && (!sc.has_probs || sc.probs_vec4)) {
        // grid counts 256-thread CTAs
        const int g = grid * (256 / (32 * SEM_WARPS));
        if (md.storage == 0) k_semantic_coop<false><<<g, 32 * SEM_WARPS, 0, s>>>(sc, md, fd);
        else k_semantic_coop<true><<<g, 32 * SEM_WARPS, 0, s>>>(sc, md, fd);
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
