// Incremental marching cubes (Sec. III-C.3) over the blocks to re-mesh, and
// gathering of per-block mesh segments (mesh extraction, arena compaction).
//
// One warp per block (persistent over the device-side list, 8 blocks in
// flight per CTA, no block-wide barriers).  The block and the +x/+y/+z faces
// of its 7 upper neighbours (found through the per-slot neighbour links) are
// staged in shared memory as a 9x9x9 voxel region and packed into per-row
// bit masks; cube a (anchored at voxel a of the block) is meshed when all 8
// corners are observed (W > 0).  Meshed cubes mark their crossing lattice
// edges in a bitmap; vertices are numbered by popcount prefix, triangles by a
// warp scan, and both are appended to the map's mesh arena with one atomic
// each per block.
// Each vertex carries the most probable class of the edge endpoint nearer
// the surface (lower endpoint on ties) and that class's palette colour.
#include "batch.h"
#include "frame_bodies.cuh"
#include "semtsdf.h"

namespace stsdf {

// generated case table, shared by every map of the process
static int8_t *h_tri_dev = nullptr;      // [256][MC_MAXTRI][3] cube-edge ids
static uint8_t *h_ntri_dev = nullptr;    // [256] triangles per case

__global__ void __launch_bounds__(32 * MESH_WARPS, 5) k_mesh(MapDev md, FrameDev fd, const int8_t *__restrict__ ttri,
                                                           const uint8_t *__restrict__ tntri) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    MeshCtaSmem &S = *reinterpret_cast<MeshCtaSmem *>(smem_raw);
    for (int i = threadIdx.x; i < 256 * MC_MAXTRI * 3; i += blockDim.x) S.tri[i] = ttri[i];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) S.ntri[i] = tntri[i];
    __syncthreads();
    pdl_wait();   // the TSDF grid's re-mesh list and voxel values
    const int wid = threadIdx.x >> 5;
    unsigned long long nd = *(volatile unsigned long long *)&fd.ctr[CT_DIRTY];
    if (nd > (unsigned long long)md.max_blocks) nd = md.max_blocks;
    const long long nwarps = (long long)gridDim.x * MESH_WARPS;
    const int part = (int)((blockIdx.x * MESH_WARPS + wid) % ARENA_PARTS);
    long long n_v = 0, n_t = 0;
    for (long long li = (long long)blockIdx.x * MESH_WARPS + wid; li < (long long)nd; li += nwarps)
        mesh_block_warp(md, fd, S.tri, S.ntri, S.w[wid], fd.dirty[li], part, n_v, n_t);
    long long cnt[2] = {n_v, n_t};
    cta_count<2>(fd.ctr, {CT_MV, CT_MT}, cnt);
}

int mesh_upload_tables(const int8_t *tri_abi, const uint8_t *ntri) {
    // the device copy keeps MC_MAXTRI of the table's MAP_MC_MAXTRI slots per case
    int8_t tri[256 * MC_MAXTRI * 3];
    for (int c = 0; c < 256; ++c) {
        if (ntri[c] > MC_MAXTRI) return -1;
        for (int k = 0; k < MC_MAXTRI * 3; ++k) tri[c * MC_MAXTRI * 3 + k] = tri_abi[c * MAP_MC_MAXTRI * 3 + k];
    }
    if (!h_tri_dev) {
        if (cudaMalloc(&h_tri_dev, 256 * MC_MAXTRI * 3) != cudaSuccess) return -1;
        if (cudaMalloc(&h_ntri_dev, 256) != cudaSuccess) return -1;
        if (cudaMemcpy(h_tri_dev, tri, 256 * MC_MAXTRI * 3, cudaMemcpyHostToDevice) != cudaSuccess) return -1;
        if (cudaMemcpy(h_ntri_dev, ntri, 256, cudaMemcpyHostToDevice) != cudaSuccess) return -1;
    }
    return 0;
}

const int8_t *mesh_table_tri() { return h_tri_dev; }
const uint8_t *mesh_table_ntri() { return h_ntri_dev; }

// Shared memory per CTA, padded to 45 KB: four CTAs (4 x 46 KB with the
// per-CTA reserve) and two four-warp class-update CTAs (2 x 21 KB) fit in an
// SM's 228 KB, five CTAs do not, so the class update running beside the
// re-meshing always has room on every SM.
constexpr int MESH_SMEM_BYTES = 45 * 1024;
static_assert(sizeof(MeshCtaSmem) <= MESH_SMEM_BYTES, "the staging fits the padded size");

void mesh_kernel_attributes() {
    cudaFuncSetAttribute(k_mesh, cudaFuncAttributeMaxDynamicSharedMemorySize, MESH_SMEM_BYTES);
    cudaFuncSetAttribute(k_mesh, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
}

int mesh_blocks_per_sm() {
    const int bytes = MESH_SMEM_BYTES;
    mesh_kernel_attributes();
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_mesh, 32 * MESH_WARPS, bytes);
    return n > 0 ? n : 1;
}

void launch_mesh(const MapDev &md, const FrameDev &fd, int grid, cudaStream_t s) {
    launch_pdl(k_mesh, dim3(grid), dim3(32 * MESH_WARPS), MESH_SMEM_BYTES, s, md, fd,
               (const int8_t *)h_tri_dev, (const uint8_t *)h_ntri_dev);
}

// ---------------------------------------------------------------------------
// gathering segments: scan over pool slots, then copy
// ---------------------------------------------------------------------------
constexpr int SCAN_CHUNK = 1024;   // slots per CTA of the first scan pass (256 threads x 4)

__global__ void __launch_bounds__(256) k_seg_scan1(MapDev md, GatherBufs g) {
    __shared__ int s_warp[8];
    unsigned long long pc = md.st->pool_count;
    if (pc > (unsigned long long)md.max_blocks) pc = md.max_blocks;
    const long long base = (long long)blockIdx.x * SCAN_CHUNK;
    if (base >= (long long)pc) {
        if (threadIdx.x == 0) {
            g.bsum_v[blockIdx.x] = 0;
            g.bsum_t[blockIdx.x] = 0;
        }
        return;
    }
    int cv = 0, ct = 0;
    int4 sg[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const long long s = base + 4 * threadIdx.x + q;
        sg[q] = s < (long long)pc ? md.seg[s] : make_int4(0, 0, 0, 0);
        cv += sg[q].y;
        ct += sg[q].w;
    }
    int tv, tt;
    int ov = block_exclusive_scan(cv, s_warp, tv);
    int ot = block_exclusive_scan(ct, s_warp, tt);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const long long s = base + 4 * threadIdx.x + q;
        if (s < (long long)pc) {
            g.voff[s] = ov;
            g.toff[s] = ot;
        }
        ov += sg[q].y;
        ot += sg[q].w;
    }
    if (threadIdx.x == 0) {
        g.bsum_v[blockIdx.x] = tv;
        g.bsum_t[blockIdx.x] = tt;
    }
}

// exclusive scan of the chunk sums (serial per thread over a strided range, then combine)
__global__ void __launch_bounds__(1024) k_seg_scan2(GatherBufs g, int nchunks) {
    __shared__ long long sv[1024], st[1024];
    const int t = threadIdx.x;
    const int per = (nchunks + 1023) / 1024;
    long long av = 0, at = 0;
    for (int i = 0; i < per; ++i) {
        const int c = t * per + i;
        if (c < nchunks) {
            av += g.bsum_v[c];
            at += g.bsum_t[c];
        }
    }
    sv[t] = av;
    st[t] = at;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        long long xv = t >= o ? sv[t - o] : 0, xt = t >= o ? st[t - o] : 0;
        __syncthreads();
        sv[t] += xv;
        st[t] += xt;
        __syncthreads();
    }
    long long rv = sv[t] - av, rt = st[t] - at;
    for (int i = 0; i < per; ++i) {
        const int c = t * per + i;
        if (c < nchunks) {
            const long long bv = g.bsum_v[c], bt = g.bsum_t[c];
            g.bsum_v[c] = rv;
            g.bsum_t[c] = rt;
            rv += bv;
            rt += bt;
        }
    }
    if (t == 1023) {
        g.totals[0] = sv[1023];
        g.totals[1] = st[1023];
    }
}

// one warp per slot
__global__ void __launch_bounds__(256) k_seg_gather(MapDev md, GatherBufs g, int mode, float4 *av2, int64_t *ak2,
                                                    ushort4 *at2, float *pos, uint8_t *col, int64_t *keys,
                                                    int32_t *tri, int32_t *anchors) {
    unsigned long long pc = md.st->pool_count;
    if (pc > (unsigned long long)md.max_blocks) pc = md.max_blocks;
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long s = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); s < (long long)pc;
         s += warps) {
        const int4 sg = md.seg[s];
        const long long ov = g.voff[s] + g.bsum_v[s / SCAN_CHUNK];
        const long long ot = g.toff[s] + g.bsum_t[s / SCAN_CHUNK];
        if (mode == 0) {
            for (int i = lane; i < sg.y; i += 32) {
                av2[ov + i] = md.av[sg.x + i];
                ak2[ov + i] = md.ak[sg.x + i];
            }
            for (int i = lane; i < sg.w; i += 32) at2[ot + i] = md.at[sg.z + i];
            __syncwarp();
            if (lane == 0) md.seg[s] = make_int4((int)ov, sg.y, (int)ot, sg.w);
        } else {
            int bx = 0, by = 0, bz = 0;
            if (sg.w > 0) unpack_block(md.slot_key[s], bx, by, bz);
            for (int i = lane; i < sg.y; i += 32) {
                const float4 v = md.av[sg.x + i];
                // class of the vertex's source voxel, and its palette colour
                const unsigned src = __float_as_uint(v.w);
                const int lab = src == 0xffffffffu ? 0 : md.label[src];
                const uchar4 c = md.pal[lab];
                pos[3 * (ov + i)] = v.x;
                pos[3 * (ov + i) + 1] = v.y;
                pos[3 * (ov + i) + 2] = v.z;
                col[4 * (ov + i)] = c.x;
                col[4 * (ov + i) + 1] = c.y;
                col[4 * (ov + i) + 2] = c.z;
                col[4 * (ov + i) + 3] = (uint8_t)lab;
                keys[ov + i] = md.ak[sg.x + i];
            }
            for (int i = lane; i < sg.w; i += 32) {
                const ushort4 tr = md.at[sg.z + i];
                tri[3 * (ot + i)] = (int32_t)(ov + tr.x);
                tri[3 * (ot + i) + 1] = (int32_t)(ov + tr.y);
                tri[3 * (ot + i) + 2] = (int32_t)(ov + tr.z);
                anchors[3 * (ot + i)] = 8 * bx + (tr.w & 7);
                anchors[3 * (ot + i) + 1] = 8 * by + ((tr.w >> 3) & 7);
                anchors[3 * (ot + i) + 2] = 8 * bz + (tr.w >> 6);
            }
        }
    }
}

// After compaction: the live mesh fills [0, totals); split the rest into partitions.
__global__ void k_set_cursors(MapDev md, GatherBufs g) {
    for (int p = 0; p < ARENA_PARTS; ++p) {
        unsigned long long b, e;
        arena_partition((unsigned long long)g.totals[0], (unsigned long long)md.av_cap, p, b, e);
        md.st->arena_v[p] = b;
        md.st->arena_v_base[p] = b;
        md.st->arena_v_end[p] = e;
        arena_partition((unsigned long long)g.totals[1], (unsigned long long)md.at_cap, p, b, e);
        md.st->arena_t[p] = b;
        md.st->arena_t_base[p] = b;
        md.st->arena_t_end[p] = e;
    }
}

void launch_seg_scan(const MapDev &md, const GatherBufs &g, int max_blocks, cudaStream_t s) {
    const int nchunks = (max_blocks + SCAN_CHUNK - 1) / SCAN_CHUNK;
    k_seg_scan1<<<nchunks, 256, 0, s>>>(md, g);
    k_seg_scan2<<<1, 1024, 0, s>>>(g, nchunks);
}

void launch_seg_gather(const MapDev &md, const GatherBufs &g, int max_blocks, int mode, float4 *av2, int64_t *ak2,
                       ushort4 *at2, float *pos, uint8_t *col, int64_t *keys, int32_t *tri, int32_t *anchors,
                       cudaStream_t s) {
    int grid = (max_blocks + 7) / 8;
    if (grid > 148 * 16) grid = 148 * 16;
    if (grid < 1) grid = 1;
    k_seg_gather<<<grid, 256, 0, s>>>(md, g, mode, av2, ak2, at2, pos, col, keys, tri, anchors);
}

void launch_set_cursors(const MapDev &md, const GatherBufs &g, cudaStream_t s) {
    k_set_cursors<<<1, 1, 0, s>>>(md, g);
}

}  // namespace stsdf
