// Batched persistent integration: one cooperative launch fuses one scan into
// each of up to BATCH_MAX maps (uneven scan sizes, voxel sizes and storage).
//
// The kernel runs the per-frame phases back to back for all maps at once:
//   reset -> points -> TSDF -> class update and re-meshing together,
// separated by a grid-wide barrier.  Inside a phase, a flattened work index
// is mapped to (map, item) through prefix sums over the maps' item counts
// (each map's range padded to a multiple of 32, so that warp-level votes
// never mix two maps).  Work sizes of the later phases are read from the
// device counters the earlier phases produced, so nothing returns to the
// host between phases.  The barrier's spin is bounded: on timeout the kernel
// latches ERR_TIMEOUT and every CTA returns.
#include <cooperative_groups.h>

#include "batch.h"
#include "frame_bodies.cuh"

namespace stsdf {

constexpr unsigned long long SPIN_LIMIT_DEFAULT = 1ull << 22;   // a few seconds of polling

// Grid barrier for a cooperative (co-resident) grid; false after a timeout.
__device__ __forceinline__ bool grid_sync(BatchCtl *ctl, unsigned long long limit, unsigned &gen) {
    __syncthreads();
    int ok = 1;
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned nb = gridDim.x;
        if (atomicAdd(&ctl->bar_count, 1u) == nb - 1) {
            atomicExch(&ctl->bar_count, 0u);
            __threadfence();
            atomicExch(&ctl->bar_gen, gen + 1);
        } else {
            unsigned long long spins = 0;
            while (atomicAdd(&ctl->bar_gen, 0u) == gen) {
                if (++spins > limit || atomicAdd(&ctl->err, 0u)) {
                    atomicOr(&ctl->err, ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(128);
            }
        }
        __threadfence();
    }
    ++gen;
    return __syncthreads_and(ok) != 0;
}

// Map index of flattened item e given the inclusive prefix pre[0..n] (pre[0] = 0).
__device__ __forceinline__ int find_map(const long long *pre, int n, long long e) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= e) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ long long pad32(long long x) { return (x + 31) & ~31ll; }

template <int WARPS>
struct BatchSmem {
    union {
        TsdfWarpSmem tsdf[WARPS];
        struct {
            int8_t tri[256 * MC_MAXTRI * 3];
            uint8_t ntri[256];
            MeshWarpSmem w[WARPS];
        } mesh;
    } u;
    long long pre[BATCH_MAX + 1];
    long long pre2[BATCH_MAX + 1];
    uint8_t lead[WARPS][32];   // warp-staged class update: the lane that lists each staged row
};

template <int WARPS, int VPT>
__global__ void __launch_bounds__(32 * WARPS, 32 / WARPS) k_batch(const __grid_constant__ BatchArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BatchSmem<WARPS> &S = *reinterpret_cast<BatchSmem<WARPS> *>(smem_raw);
    BatchCtl *ctl = a.ctl;
    const int n = a.n;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nthreads = (long long)gridDim.x * blockDim.x;
    const long long gwarp = (long long)blockIdx.x * WARPS + wid, nwarps = (long long)gridDim.x * WARPS;
    const unsigned long long limit = a.spin_limit ? a.spin_limit : SPIN_LIMIT_DEFAULT;
    unsigned gen = 0;
    if (a.fault_skip_cta0 && blockIdx.x == 0) return;   // test hook: the barrier must time out

    // ---- reset: range-image winners and counters ------------------------------
    if (threadIdx.x == 0) {
        S.pre[0] = 0;
        S.pre2[0] = 0;
        for (int i = 0; i < n; ++i) S.pre[i + 1] = S.pre[i] + (long long)a.it[i].sc.H * a.it[i].sc.W;
    }
    __syncthreads();
    for (long long e = tid; e < S.pre[n]; e += nthreads) {
        const int i = find_map(S.pre, n, e);
        a.it[i].fd.win[e - S.pre[i]] = ~0ull;
    }
    for (long long e = tid; e < (long long)n * CT_COUNT; e += nthreads) a.it[e / CT_COUNT].fd.ctr[e % CT_COUNT] = 0ull;
    if (!grid_sync(ctl, limit, gen)) return;

    // ---- points: range-image winner + band allocation ------------------------
    if (threadIdx.x == 0) {
        for (int i = 0; i < n; ++i) S.pre[i + 1] = S.pre[i] + pad32(a.it[i].sc.n);
    }
    __syncthreads();
    for (long long base = tid - lane; base < S.pre[n]; base += nthreads * VPT) {
#pragma unroll
        for (int k = 0; k < VPT; ++k) {
            const long long wb = base + (long long)k * nthreads;   // warp-uniform
            if (wb >= S.pre[n]) break;
            const int i = find_map(S.pre, n, wb);
            long long cnt[3] = {0, 0, 0};
            points_item(a.it[i].sc.pts, a.it[i].sc, a.it[i].md, a.it[i].fd, wb - S.pre[i] + lane, cnt);
            // the warp's items all belong to map i: one add per counter and warp
#pragma unroll
            for (int c = 0; c < 3; ++c) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) cnt[c] += __shfl_xor_sync(0xffffffffu, cnt[c], o);
            }
            if (lane == 0) {
                if (cnt[0]) atomicAdd(&a.it[i].fd.ctr[CT_VALID], (unsigned long long)cnt[0]);
                if (cnt[1]) atomicAdd(&a.it[i].fd.ctr[CT_PIXEL], (unsigned long long)cnt[1]);
                if (cnt[2]) atomicAdd(&a.it[i].fd.ctr[CT_NEW], (unsigned long long)cnt[2]);
            }
        }
    }
    if (!grid_sync(ctl, limit, gen)) return;

    // ---- TSDF: one warp per half of a touched block ---------------------------
    if (threadIdx.x == 0) {
        for (int i = 0; i < n; ++i) {
            unsigned long long t = *(volatile unsigned long long *)&a.it[i].fd.ctr[CT_TOUCHED];
            if (t > (unsigned long long)a.it[i].md.max_blocks) t = a.it[i].md.max_blocks;
            S.pre[i + 1] = S.pre[i] + (long long)t;
        }
    }
    __syncthreads();
    // (half blocks, as the per-phase kernel: 256 voxels per unit)
    for (long long u = gwarp; u < 2 * S.pre[n]; u += nwarps) {
        const long long e = u >> 1;
        const int v0 = (int)(u & 1) * (BV / 2);
        const int i = find_map(S.pre, n, e);
        const BatchItem &it = a.it[i];
        long long n_upd = 0;
        const int h = it.fd.touched[e - S.pre[i]];
        if (it.md.storage == 0) tsdf_block_warp<false>(it.sc, it.md, it.fd, h, S.u.tsdf[wid], n_upd, v0, v0 + BV / 2);
        else tsdf_block_warp<true>(it.sc, it.md, it.fd, h, S.u.tsdf[wid], n_upd, v0, v0 + BV / 2);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) n_upd += __shfl_xor_sync(0xffffffffu, n_upd, o);
        if (lane == 0 && n_upd) atomicAdd(&it.fd.ctr[CT_UPD], (unsigned long long)n_upd);
    }
    if (!grid_sync(ctl, limit, gen)) return;

    // ---- class update and re-meshing (independent: the mesh reads no labels) --
    for (int k = threadIdx.x; k < 256 * MC_MAXTRI * 3; k += blockDim.x) S.u.mesh.tri[k] = a.tri[k];
    for (int k = threadIdx.x; k < 256; k += blockDim.x) S.u.mesh.ntri[k] = a.ntri[k];
    if (threadIdx.x == 0) {
        for (int i = 0; i < n; ++i) {
            unsigned long long t = *(volatile unsigned long long *)&a.it[i].fd.ctr[CT_SEM];
            if (t > (unsigned long long)a.it[i].fd.sem_cap) t = a.it[i].fd.sem_cap;
            S.pre[i + 1] = S.pre[i] + (long long)t;
            t = *(volatile unsigned long long *)&a.it[i].fd.ctr[CT_DIRTY];
            if (t > (unsigned long long)a.it[i].md.max_blocks) t = a.it[i].md.max_blocks;
            S.pre2[i + 1] = S.pre2[i] + (long long)t;
        }
    }
    __syncthreads();
    if (a.sem_staged) {
        // warp-staged: 32 consecutive entries of the maps' concatenated lists per warp, the records
        // staged in the warp's re-meshing slot (free until this warp meshes); probability rows
        // read by each lane
        static_assert(sizeof(MeshWarpSmem) >= 32 * SemStage<false>::RB + 32 * SEM_NC * 4,
                      "records and rows fit the warp's slot");
        unsigned char *R = reinterpret_cast<unsigned char *>(&S.u.mesh.w[wid]);
        float *Q = reinterpret_cast<float *>(R + 32 * SemStage<false>::RB);
        for (long long base = gwarp * 32; base < S.pre[n]; base += nwarps * 32) {
            const long long e = base + lane;
            const bool act = e < S.pre[n];
            const int i = act ? find_map(S.pre, n, e) : 0;
            const BatchItem &it = a.it[i];
            const int2 ent = act ? it.fd.sem_list[e - S.pre[i]] : make_int2(0, 0);
            const float *qrow = act && it.sc.has_probs ? it.sc.probs + (long long)ent.y * SEM_NC : nullptr;
            if (a.sem_rows_once) {
                // the round's distinct (map, point) rows, staged once each (one lane of each group
                // lists it) and taken to log2 once
                const bool pr = qrow != nullptr;
                const unsigned long long kv = pr ? ((unsigned long long)i << 32) | (unsigned)ent.y : ~0ull - lane;
                const unsigned grp = __match_any_sync(0xffffffffu, kv);
                const int lead = __ffs(grp) - 1;
                const bool leader = pr && lead == lane;
                const unsigned lm = __ballot_sync(0xffffffffu, leader);
                const int nu = __popc(lm);
                const int row = __popc(lm & ((1u << lead) - 1u));
                if (leader) S.lead[wid][row] = (uint8_t)lane;
                __syncwarp();
                const unsigned long long rp = reinterpret_cast<unsigned long long>(qrow);
#pragma unroll
                for (int j = 0; j < SEM_NC / 4; ++j) {
                    const int k = 32 * j + lane, u = k / (SEM_NC / 4), c = k - u * (SEM_NC / 4);
                    const unsigned long long p = __shfl_sync(0xffffffffu, rp, S.lead[wid][u < nu ? u : 0]);
                    if (u < nu) cp_async16(Q + u * SEM_NC + 4 * c, reinterpret_cast<const float *>(p) + 4 * c);
                }
                qrow = pr ? Q + row * SEM_NC : nullptr;
                if (a.sem_staged == 2) class_update_warp<true, true>(it.sc, it.md, act, ent, R, qrow, Q, nu * SEM_NC);
                else class_update_warp<false, true>(it.sc, it.md, act, ent, R, qrow, Q, nu * SEM_NC);
            } else {
                if (a.sem_staged == 2) class_update_warp<true>(it.sc, it.md, act, ent, R, qrow);
                else class_update_warp<false>(it.sc, it.md, act, ent, R, qrow);
            }
        }
    }
    for (long long base = tid; !a.sem_staged && base < S.pre[n]; base += nthreads * VPT) {
#pragma unroll
        for (int k = 0; k < VPT; ++k) {
            const long long e = base + (long long)k * nthreads;
            if (e >= S.pre[n]) break;
            const int i = find_map(S.pre, n, e);
            const BatchItem &it = a.it[i];
            const unsigned long long j = (unsigned long long)(e - S.pre[i]);
            if (it.md.storage == 0) {
                if (it.sc.C == 20) semantic_item<false, 20>(it.sc, it.md, it.fd, j);
                else semantic_item<false, 0>(it.sc, it.md, it.fd, j);
            } else {
                if (it.sc.C == 20) semantic_item<true, 20>(it.sc, it.md, it.fd, j);
                else semantic_item<true, 0>(it.sc, it.md, it.fd, j);
            }
        }
    }
    const int part = (int)(gwarp % ARENA_PARTS);
    for (long long e = gwarp; e < S.pre2[n]; e += nwarps) {
        const int i = find_map(S.pre2, n, e);
        const BatchItem &it = a.it[i];
        long long n_v = 0, n_t = 0;
        mesh_block_warp(it.md, it.fd, S.u.mesh.tri, S.u.mesh.ntri, S.u.mesh.w[wid], it.fd.dirty[e - S.pre2[i]], part,
                        n_v, n_t);
        if (lane == 0) {
            if (n_v) atomicAdd(&it.fd.ctr[CT_MV], (unsigned long long)n_v);
            if (n_t) atomicAdd(&it.fd.ctr[CT_MT], (unsigned long long)n_t);
        }
    }
    if (!grid_sync(ctl, limit, gen)) return;

    // ---- per-map state for the host --------------------------------------------
    for (long long e = tid; e < n; e += nthreads) {
        BatchState &bs = a.out[e];
        bs.st = *a.it[e].md.st;
        for (int c = 0; c < CT_COUNT; ++c) bs.ctr[c] = a.it[e].fd.ctr[c];
    }
}

template <int WARPS, int VPT>
static cudaError_t setup_one(int &blocks_per_sm) {
    const int smem = (int)sizeof(BatchSmem<WARPS>);
    cudaError_t e = cudaFuncSetAttribute(k_batch<WARPS, VPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, k_batch<WARPS, VPT>, 32 * WARPS, smem);
}

const BatchConfig kBatchConfigs[kNumBatchConfigs] = {{4, 1}, {4, 2}, {4, 4}, {8, 1}, {8, 2}, {8, 4}};

cudaError_t batch_occupancy(int cfg, int &blocks_per_sm) {
    switch (cfg) {
        case 0: return setup_one<4, 1>(blocks_per_sm);
        case 1: return setup_one<4, 2>(blocks_per_sm);
        case 2: return setup_one<4, 4>(blocks_per_sm);
        case 3: return setup_one<8, 1>(blocks_per_sm);
        case 4: return setup_one<8, 2>(blocks_per_sm);
        default: return setup_one<8, 4>(blocks_per_sm);
    }
}

// Cooperative launch of configuration cfg on `grid` CTAs (capturable).
cudaError_t launch_batch(int cfg, int grid, const BatchArgs &args, cudaStream_t s) {
    void *params[] = {(void *)&args};
    const dim3 g(grid);
    switch (cfg) {
        case 0: return cudaLaunchCooperativeKernel((void *)k_batch<4, 1>, g, dim3(128), params, sizeof(BatchSmem<4>), s);
        case 1: return cudaLaunchCooperativeKernel((void *)k_batch<4, 2>, g, dim3(128), params, sizeof(BatchSmem<4>), s);
        case 2: return cudaLaunchCooperativeKernel((void *)k_batch<4, 4>, g, dim3(128), params, sizeof(BatchSmem<4>), s);
        case 3: return cudaLaunchCooperativeKernel((void *)k_batch<8, 1>, g, dim3(256), params, sizeof(BatchSmem<8>), s);
        case 4: return cudaLaunchCooperativeKernel((void *)k_batch<8, 2>, g, dim3(256), params, sizeof(BatchSmem<8>), s);
        default: return cudaLaunchCooperativeKernel((void *)k_batch<8, 4>, g, dim3(256), params, sizeof(BatchSmem<8>), s);
    }
}

}  // namespace stsdf
