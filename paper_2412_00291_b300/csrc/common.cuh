// Internal definitions shared by the CUDA kernels and the host orchestration
// of libsemtsdf.  Not part of the public C ABI (see include/semtsdf.h).
#pragma once

#include <utility>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace stsdf {

constexpr int BS = 8;                 // voxels per block side (Sec. III-C.2: 8x8x8 VoxelBlocks)
constexpr int BV = BS * BS * BS;
constexpr uint64_t EMPTY_KEY = ~0ull;
constexpr int MAX_PROBES = 256;       // linear-probing bound of the block hash
constexpr int MAX_AXIS_CROSS = 4;     // band may cross <= 4 block planes per axis (tau <= 16 nu)
constexpr int MC_MAXTRI = 5;          // triangles per cube case in the device copy of the generated table
                                       // (its largest case; the C-ABI table has MAP_MC_MAXTRI slots)
constexpr float PI_F = 3.14159265358979f;

// latched device error bits
enum : unsigned {
    ERR_POOL_FULL = 1u,
    ERR_HASH_PROBES = 2u,
    ERR_LIST_FULL = 4u,
    ERR_ARENA_FULL = 8u,
    ERR_TIMEOUT = 16u,
};

// per-frame counters (indices match MAP_STAT_* of the C ABI)
enum : int {
    CT_VALID = 0, CT_PIXEL, CT_TOUCHED, CT_NEW, CT_UPD, CT_SEM, CT_DIRTY, CT_MV, CT_MT,
    CT_COUNT = 16
};

// The mesh arena is split into ARENA_PARTS partitions with their own append
// cursors, so that concurrent meshing warps do not all contend for one atomic.
constexpr int ARENA_PARTS = 16;

// Persistent device scalars of a map.
struct DevState {
    unsigned long long pool_count;               // blocks allocated so far
    unsigned long long arena_v[ARENA_PARTS];     // vertex append cursor of each partition
    unsigned long long arena_t[ARENA_PARTS];     // triangle append cursor of each partition
    unsigned long long arena_v_base[ARENA_PARTS], arena_v_end[ARENA_PARTS];
    unsigned long long arena_t_base[ARENA_PARTS], arena_t_end[ARENA_PARTS];
    unsigned int err;                            // latched ERR_* bits
    unsigned int pad;
};

// Partition p of [live, cap): base and end.
__host__ __device__ inline void arena_partition(unsigned long long live, unsigned long long cap, int p,
                                                unsigned long long &base, unsigned long long &end) {
    const unsigned long long free_ = cap > live ? cap - live : 0;
    base = live + free_ / ARENA_PARTS * p;
    end = p == ARENA_PARTS - 1 ? cap : live + free_ / ARENA_PARTS * (p + 1);
}

// Largest |voxel coordinate| a map can hold on any axis: mesh edge keys keep
// 20 bits per voxel coordinate (biased by 2^19), block keys 21 bits per block
// coordinate; the margin covers a cube's upper corner and a band's rounding.
constexpr int MAX_VOXEL_COORD = (1 << 19) - 16;

// Block key: 21 bits per block coordinate, biased by 2^20.
__host__ __device__ inline uint64_t pack_block(int x, int y, int z) {
    return ((uint64_t)(uint32_t)(x + (1 << 20)) << 42) | ((uint64_t)(uint32_t)(y + (1 << 20)) << 21) |
           (uint64_t)(uint32_t)(z + (1 << 20));
}
__host__ __device__ inline void unpack_block(uint64_t k, int &x, int &y, int &z) {
    x = (int)((k >> 42) & 0x1FFFFF) - (1 << 20);
    y = (int)((k >> 21) & 0x1FFFFF) - (1 << 20);
    z = (int)(k & 0x1FFFFF) - (1 << 20);
}
// MurmurHash3 64-bit finaliser (Appleby), used as the table's hash function.
__host__ __device__ inline uint64_t fmix64(uint64_t k) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdULL;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ULL;
    k ^= k >> 33;
    return k;
}
// Lattice-edge key of a mesh vertex: axis | x, y, z of its lower voxel, 20 bits each.
__host__ __device__ inline int64_t edge_key(int x, int y, int z, int axis) {
    const int64_t b = (int64_t)1 << 19;
    return (int64_t)axis | (((int64_t)x + b) << 2) | (((int64_t)y + b) << 22) | (((int64_t)z + b) << 42);
}

// Everything a kernel needs about one scan (passed by value).
struct ScanConst {
    int H, W, C, n;
    float inv_dphi, inv_dtheta, theta0;
    float r_min, r_max;
    // band endpoints, IEEE single precision recipe: R / nu and t / nu + 1/2
    float Rv[9], tv[3], tau, inv_2tau;
    // world-to-LiDAR rotation R^T (row-major), used to find a voxel's pixel
    float Rt[9];
    // sensor position in voxel units = k + (fhi + flo), k integer, 0 <= f < 1
    int k[3];
    float fhi[3], flo[3];
    float nu, nu2hi, nu2lo;         // nu and nu^2 as an unevaluated float pair
    float log_phit, log_pmiss, lik_floor, logp_floor;
    int weight_mode;
    int frame;
    int has_probs;
    int probs_vec4;       // probability rows can be read as float4 (C % 4 == 0, 16-byte aligned)
    // the scan: points [n][3], and per point a label [n] or class probabilities [n][C]
    const float *pts;
    const int32_t *labels;
    const float *probs;
    // non-projective distance (Sec. III-C.2, Eq. distance): 0 off, 1 on
    int dist_mode;
    const float4 *row_dir;   // [H] beam v: {sin hi, sin lo, cos hi, cos lo} of its polar angle
    const float4 *col_dir;   // [W] column u: {cos hi, cos lo, sin hi, sin lo} of its azimuth
    float4 *nrm;             // [H*W] normal image, world frame; w = 1 where the pixel has a normal
};

// One slot of the block hash: key (EMPTY_KEY when free), pool slot of the
// block (-1: the pool was full), last frame the block was touched.  16 bytes,
// so a probe brings the pool slot and the stamp into the same 32-byte sector.
struct __align__(16) HashSlot {
    uint64_t key;
    int val;
    int stamp;
};

// Device pointers of one map.
struct MapDev {
    HashSlot *hs;        // [cap] the block hash
    int *dstamp_slot;    // [slot] last frame the block was queued for meshing
    uint64_t mask;       // cap - 1
    int max_blocks;
    int C;
    int storage;         // 0 FP32, 1 FP16
    float2 *dw32;        // [slot][512] {D, W}
    __half2 *dw16;
    float *lp32;         // [slot][512][CP] log-probabilities, one record per voxel
    __half *lp16;
    int CP;              // record stride in elements: C rounded up to whole 16-byte chunks
    uint8_t *label;      // [slot][512] most probable class
    const uchar4 *pal;   // [256] class colours (rgb)
    uint64_t *slot_key;  // [slot] block key owning the pool slot
    int *slot_frame;     // [slot] frame in which the slot was allocated
    int *nbr;            // [slot][16] slots of the blocks b + e_o (o = 1..7) and b - e_o (8 + o), -1 if none
    int4 *seg;           // [slot] mesh segment: vertex offset, count, triangle offset, count
    float4 *av;          // mesh arena: vertex {x, y, z, bits of its source pool voxel (class at extraction)}
    int64_t *ak;         // mesh arena: vertex edge keys
    ushort4 *at;         // mesh arena: triangle {i0, i1, i2, cube anchor (local)}
    long long av_cap, at_cap;
    DevState *st;
    float nu;
    float *g32;          // non-projective mode: [slot][3][512] gradient g_i (x, y, z planes), FP32 storage
    __half *g16;         //   the same in FP16 storage
};

// Per-frame scratch of one map.
struct FrameDev {
    unsigned long long *win;   // [H*W] range-image winner: (float bits of range << 32) | point index, ~0 if none
    int *touched;              // [max_blocks] hash slots of U_k
    int *dirty;                // [max_blocks] pool slots to re-mesh
    int2 *sem_list;            // [sem_cap] {pool voxel index, winner point index} awaiting the class update
    long long sem_cap;
    unsigned long long *ctr;   // [CT_COUNT]
    // the other range-image and counter buffers (the next scan's), which the
    // per-point kernel resets on the way: win_next[0, win_next_n) to ~0 and
    // ctr_next to 0 (null in paths that reset their own buffers)
    unsigned long long *win_next;
    long long win_next_n;
    unsigned long long *ctr_next;
    // parity instrumentation (null on the product path): the scan's choices,
    // for comparison with an FP64 reference
    int *dbg_point;            // [n] pixel of each point, -1 valid without a pixel, -2 invalid
    int *dbg_vox;              // [slot][512] pixel + 1 (0: none) | updated << 28 | class update << 29
};

// --- error-free transformations (Knuth TwoSum, Dekker/FMA TwoProduct) ----
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}
// (ah + al) + (bh + bl) as an unevaluated pair
__device__ __forceinline__ void df_add(float ah, float al, float bh, float bl, float &sh, float &sl) {
    float s, e;
    two_sum(ah, bh, s, e);
    e = __fadd_rn(e, __fadd_rn(al, bl));
    sh = __fadd_rn(s, e);
    sl = __fsub_rn(e, __fsub_rn(sh, s));
}
__device__ __forceinline__ void df_mul(float ah, float al, float bh, float bl, float &ph, float &pl) {
    float p, e;
    two_prod(ah, bh, p, e);
    e = __fmaf_rn(ah, bl, __fmaf_rn(al, bh, e));
    ph = __fadd_rn(p, e);
    pl = __fsub_rn(e, __fsub_rn(ph, p));
}
// sqrt(ah + al), ah > 0, as a pair: one Newton correction of the single-precision
// root (Dekker 1971, double-length square root), the residual ah - s^2 exact by FMA
__device__ __forceinline__ void df_sqrt(float ah, float al, float &sh, float &sl) {
    const float s = __fsqrt_rn(ah);
    const float r = __fadd_rn(__fmaf_rn(-s, s, ah), al);
    const float c = __fdiv_rn(r, __fmul_rn(2.f, s));
    sh = __fadd_rn(s, c);
    sl = __fsub_rn(c, __fsub_rn(sh, s));
}
// a b - c d with one rounding error at most beyond the result's (Kahan's FMA scheme)
__device__ __forceinline__ float diff_of_products(float a, float b, float c, float d) {
    const float w = __fmul_rn(c, d);
    const float e = __fmaf_rn(-c, d, w);
    const float f = __fmaf_rn(a, b, -w);
    return __fadd_rn(f, e);
}

// Offset of class c of pool voxel vox (= slot * 512 + voxel index) in the log-probability array.
__host__ __device__ inline long long lp_index(const MapDev &md, long long vox, int c) {
    return vox * md.CP + c;
}

// Range of a point exactly as the allocation recipe defines it.
__device__ __forceinline__ float range_f32(float x, float y, float z) {
    float s = __fmul_rn(x, x);
    s = __fadd_rn(s, __fmul_rn(y, y));
    s = __fadd_rn(s, __fmul_rn(z, z));
    return __fsqrt_rn(s);
}

__device__ __forceinline__ int hash_find(const HashSlot *__restrict__ hs, uint64_t mask, uint64_t key) {
    uint64_t h = fmix64(key) & mask;
    for (int p = 0; p < MAX_PROBES; ++p) {
        uint64_t k = hs[h].key;
        if (k == key) return (int)h;
        if (k == EMPTY_KEY) return -1;
        h = (h + 1) & mask;
    }
    return -1;
}

// Neighbour links of block `key` (pool slot s) with its 14 face/edge/corner
// neighbours b +- e_o, both directions; every block is in the hash already.
__device__ __forceinline__ void link_block(const MapDev &md, uint64_t key, int s, int o) {
    int x, y, z;
    unpack_block(key, x, y, z);
    const int dx = o & 1, dy = (o >> 1) & 1, dz = o >> 2;
    const int hp = hash_find(md.hs, md.mask, pack_block(x + dx, y + dy, z + dz));
    const int np = hp < 0 ? -1 : md.hs[hp].val;
    md.nbr[s * 16 + o] = np;
    if (np >= 0) md.nbr[np * 16 + 8 + o] = s;
    const int hm = hash_find(md.hs, md.mask, pack_block(x - dx, y - dy, z - dz));
    const int nm = hm < 0 ? -1 : md.hs[hm].val;
    md.nbr[s * 16 + 8 + o] = nm;
    if (nm >= 0) md.nbr[nm * 16 + o] = s;
}

// Block-wide exclusive scan of one int per thread (blockDim.x multiple of 32, <= 1024).
__device__ __forceinline__ int block_exclusive_scan(int v, int *s_warp, int &total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int t = lane < nw ? s_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < nw) s_warp[lane] = t;   // inclusive warp prefix
    }
    __syncthreads();
    int base = wid > 0 ? s_warp[wid - 1] : 0;
    total = s_warp[nw - 1];
    __syncthreads();
    return base + x - v;
}

// Exclusive scan over the 32 lanes of a warp; total returned in every lane.
__device__ __forceinline__ int warp_exclusive_scan(int v, int &total) {
    const int lane = threadIdx.x & 31;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    total = __shfl_sync(0xffffffffu, x, 31);
    return x - v;
}

// Per-CTA totals of per-thread statistics, added to the frame counters by
// thread 0 (one atomic per counter and CTA instead of one per warp: the
// counters share a cache line, whose atomics the L2 serialises).
template <int N>
__device__ __forceinline__ void cta_count(unsigned long long *ctr, const int (&idx)[N], long long (&v)[N]) {
    __shared__ long long s_part[N][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < N; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
        if (lane == 0) s_part[k][wid] = v[k];
    }
    __syncthreads();
    if (threadIdx.x < N) {
        long long t = 0;
        for (int i = 0; i < nw; ++i) t += s_part[threadIdx.x][i];
        if (t) atomicAdd(&ctr[idx[threadIdx.x]], (unsigned long long)t);
    }
}

// Programmatic dependent launch (PTX griddepcontrol): a kernel launched with
// the programmatic-stream-serialization attribute may be scheduled while its
// predecessor in the stream is still running.  pdl_wait() blocks until the
// predecessor has completed and its writes are visible (a no-op for a kernel
// launched without the attribute); pdl_trigger() lets the successor be
// scheduled before this grid ends.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Launch with programmatic stream serialization (the kernel calls pdl_wait()
// before it reads or writes anything its predecessor touches).
template <typename... P, typename... A>
inline cudaError_t launch_pdl(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, A &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...);
}

}  // namespace stsdf
