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
#include "kernels.h"

namespace stsdf {

// generated case table, shared by every map of the process
static int8_t *h_tri_dev = nullptr;      // [256][MC_MAXTRI][3] cube-edge ids
static uint8_t *h_ntri_dev = nullptr;    // [256] triangles per case

constexpr int EDGE_WORDS = (MC_EDGES + 31) / 32;   // 61 words of lattice-edge bits per block
constexpr int MESH_WARPS = 8;                       // warps (blocks in flight) per CTA

// Local index of the lattice edge that cube edge ce of the cube anchored at
// (ax, ay, az) lies on: axis * 648 + a + 8 (b + 9 c), with a the coordinate
// along the axis and b, c the coordinates along the next two axes cyclically.
__device__ __forceinline__ int cube_edge_index(int ce, int ax, int ay, int az) {
    const int axis = ce >> 2;
    const int pa = axis == 0 ? ax : (axis == 1 ? ay : az);
    const int pb = (axis == 0 ? ay : (axis == 1 ? az : ax)) + (ce & 1);
    const int pc = (axis == 0 ? az : (axis == 1 ? ax : ay)) + ((ce >> 1) & 1);
    return axis * 648 + pa + 8 * (pb + 9 * pc);
}

// Per-warp staging of one block: the 9^3 region (block + upper faces).
struct MeshWarpSmem {
    float D[729];
    uint32_t rowm[81];        // per (y, z) row of 9 voxels: bits 0..8 observed, bits 16..24 D < 0
    unsigned edge[64];        // lattice-edge bitmap (61 words used)
    int woff[64];             // vertex number of each word's first set bit
    int nb[8];                // slots of this block (0) and its 7 upper neighbours, -1 if none
    uint8_t F[729];           // bit 0 observed (W > 0), bit 1 D < 0
    uint8_t lab[729];
    uint8_t cs[512];          // cube case
};

struct MeshCtaSmem {
    int8_t tri[256 * MC_MAXTRI * 3];
    uint8_t ntri[256];
    uchar4 pal[256];
    MeshWarpSmem w[MESH_WARPS];
};

__device__ __forceinline__ int face_pos(int j, int &nbi) {
    // the 217 voxels of the region outside the block: x = 8 face, then y = 8, then z = 8
    int x, y, z;
    if (j < 81) {
        x = 8; y = j % 9; z = j / 9;
    } else if (j < 153) {
        const int k = j - 81;
        x = k & 7; y = 8; z = k >> 3;
    } else {
        const int k = j - 153;
        x = k & 7; y = k >> 3; z = 8;
    }
    nbi = (x >> 3) | ((y >> 3) << 1) | ((z >> 3) << 2);
    return x + 9 * (y + 9 * z);
}

__global__ void __launch_bounds__(32 * MESH_WARPS) k_mesh(MapDev md, FrameDev fd, const int8_t *__restrict__ ttri,
                                                           const uint8_t *__restrict__ tntri,
                                                           const uchar4 *__restrict__ tpal) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    MeshCtaSmem &S = *reinterpret_cast<MeshCtaSmem *>(smem_raw);
    for (int i = threadIdx.x; i < 256 * MC_MAXTRI * 3; i += blockDim.x) S.tri[i] = ttri[i];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) {
        S.ntri[i] = tntri[i];
        S.pal[i] = tpal[i];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    MeshWarpSmem &W = S.w[wid];
    unsigned long long nd = *(volatile unsigned long long *)&fd.ctr[CT_DIRTY];
    if (nd > (unsigned long long)md.max_blocks) nd = md.max_blocks;
    const long long nwarps = (long long)gridDim.x * MESH_WARPS;
    long long n_v = 0, n_t = 0;
    const bool f32 = md.storage == 0;
    for (long long li = (long long)blockIdx.x * MESH_WARPS + wid; li < (long long)nd; li += nwarps) {
        const int slot = fd.dirty[li];
        int bx, by, bz;
        unpack_block(md.slot_key[slot], bx, by, bz);
        // slots of the 7 upper neighbours, from the per-slot links
        if (lane < 8) W.nb[lane] = lane == 0 ? slot : md.nbr[slot * 16 + lane];
        int seen = 0;   // bit 0: an observed voxel with D < 0, bit 1: one with D >= 0
#pragma unroll 4
        for (int v = lane; v < BV; v += 32) {
            const int r = (v & 7) + 9 * (((v >> 3) & 7) + 9 * (v >> 6));
            const long long vox = (long long)slot * BV + v;
            const float2 dw = f32 ? md.dw32[vox] : __half22float2(md.dw16[vox]);
            const int f = (dw.y > 0.f ? 1 : 0) | (dw.x < 0.f ? 2 : 0);
            W.D[r] = dw.x;
            W.F[r] = (uint8_t)f;
            W.lab[r] = md.label[vox];
            if (f & 1) seen |= (f & 2) ? 1 : 2;
        }
        __syncwarp();
#pragma unroll 2
        for (int j = lane; j < 217; j += 32) {
            int nbi;
            const int r = face_pos(j, nbi);
            const int s = W.nb[nbi];
            float D = 0.f;
            int f = 0;
            uint8_t lab = 0;
            if (s >= 0) {
                const int x = r % 9, y = (r / 9) % 9, z = r / 81;
                const long long vox = (long long)s * BV + (x & 7) + 8 * (y & 7) + 64 * (z & 7);
                const float2 dw = f32 ? md.dw32[vox] : __half22float2(md.dw16[vox]);
                D = dw.x;
                f = (dw.y > 0.f ? 1 : 0) | (dw.x < 0.f ? 2 : 0);
                lab = md.label[vox];
            }
            W.D[r] = D;
            W.F[r] = (uint8_t)f;
            W.lab[r] = lab;
            if (f & 1) seen |= (f & 2) ? 1 : 2;
        }
        const bool any_neg = __any_sync(0xffffffffu, seen & 1), any_pos = __any_sync(0xffffffffu, seen & 2);
        if (!(any_neg && any_pos)) {
            // no sign change among observed voxels: no cube can cross; drop the old segment
            if (lane == 0) {
                const int4 old = md.seg[slot];
                if (old.y | old.w) md.seg[slot] = make_int4(0, 0, 0, 0);
            }
            __syncwarp();
            continue;
        }
        __syncwarp();
        // packed row masks of the 81 (y, z) rows
        for (int rw = lane; rw < 81; rw += 32) {
            uint32_t m = 0;
#pragma unroll
            for (int x = 0; x < 9; ++x) {
                const uint32_t f = W.F[x + 9 * rw];
                m |= ((f & 1u) << x) | (((f >> 1) & 1u) << (16 + x));
            }
            W.rowm[rw] = m;
        }
        for (int k = lane; k < 64; k += 32) W.edge[k] = 0u;
        __syncwarp();
        // cube rows (ay, az) = lane and lane + 32: eight cubes along x from four row masks
        int cnt_t = 0;
#pragma unroll 1
        for (int q = 0; q < 2; ++q) {
            const int cr = lane + 32 * q, ay = cr & 7, az = cr >> 3;
            const uint32_t m00 = W.rowm[ay + 9 * az], m10 = W.rowm[ay + 1 + 9 * az];
            const uint32_t m01 = W.rowm[ay + 9 * (az + 1)], m11 = W.rowm[ay + 1 + 9 * (az + 1)];
            const uint32_t okm = m00 & m10 & m01 & m11;
#pragma unroll 1
            for (int ax = 0; ax < 8; ++ax) {
                const bool ok = ((okm >> ax) & 3u) == 3u;
                const int cs = (int)(((m00 >> (16 + ax)) & 3u) | (((m10 >> (16 + ax)) & 3u) << 2) |
                                     (((m01 >> (16 + ax)) & 3u) << 4) | (((m11 >> (16 + ax)) & 3u) << 6));
                const int nt = ok ? S.ntri[cs] : 0;
                W.cs[ax + 8 * cr] = (uint8_t)(nt ? cs : 0);
                cnt_t += nt;
                if (nt) {
#pragma unroll
                    for (int ce = 0; ce < 12; ++ce) {
                        const int axis = ce >> 2, a1 = axis == 2 ? 0 : axis + 1, a2 = axis == 0 ? 2 : axis - 1;
                        const int clo = ((ce & 1) << a1) | (((ce >> 1) & 1) << a2);
                        if (((cs >> clo) ^ (cs >> (clo | (1 << axis)))) & 1) {
                            const int e = cube_edge_index(ce, ax, ay, az);
                            atomicOr(&W.edge[e >> 5], 1u << (e & 31));
                        }
                    }
                }
            }
        }
        int tot_t;
        const int toff = warp_exclusive_scan(cnt_t, tot_t);
        if (tot_t == 0) {
            if (lane == 0) {
                const int4 old = md.seg[slot];
                if (old.y | old.w) md.seg[slot] = make_int4(0, 0, 0, 0);
            }
            __syncwarp();
            continue;
        }
        __syncwarp();
        // vertex numbering: popcount prefix over the bitmap (words lane, lane + 32)
        const int c0 = __popc(W.edge[lane]), c1 = lane + 32 < EDGE_WORDS ? __popc(W.edge[lane + 32]) : 0;
        int tot_lo, tot_v;
        const int off_lo = warp_exclusive_scan(c0, tot_lo);
        const int off_hi = warp_exclusive_scan(c1, tot_v);
        W.woff[lane] = off_lo;
        W.woff[lane + 32] = tot_lo + off_hi;
        tot_v += tot_lo;
        // reserve arena space in this warp's partition (two lanes, two cursors)
        const int part = (int)((blockIdx.x * MESH_WARPS + wid) % ARENA_PARTS);
        unsigned long long res = 0, lim = 0;
        if (lane == 0) {
            res = atomicAdd(&md.st->arena_v[part], (unsigned long long)tot_v);
            lim = md.st->arena_v_end[part];
        }
        if (lane == 1) {
            res = atomicAdd(&md.st->arena_t[part], (unsigned long long)tot_t);
            lim = md.st->arena_t_end[part];
        }
        const long long vo = (long long)__shfl_sync(0xffffffffu, res, 0);
        const long long to = (long long)__shfl_sync(0xffffffffu, res, 1);
        const bool fits = (unsigned long long)vo + tot_v <= __shfl_sync(0xffffffffu, lim, 0) &&
                          (unsigned long long)to + tot_t <= __shfl_sync(0xffffffffu, lim, 1);
        if (lane == 0) {
            if (fits) {
                md.seg[slot] = make_int4((int)vo, tot_v, (int)to, tot_t);
            } else {
                atomicOr(&md.st->err, ERR_ARENA_FULL);
                md.seg[slot] = make_int4(0, 0, 0, 0);
            }
            n_v += tot_v;
            n_t += tot_t;
        }
        __syncwarp();
        if (fits) {
            // vertices: bytes b = lane + 32 k of the bitmap, edges 8 b .. 8 b + 7
            for (int b = lane; b < 4 * EDGE_WORDS; b += 32) {
                const unsigned word = W.edge[b >> 2];
                unsigned bits = (word >> ((b & 3) * 8)) & 0xffu;
                while (bits) {
                    const int q = __ffs(bits) - 1;
                    bits &= bits - 1;
                    const int e = 8 * b + q;
                    const int vid = W.woff[b >> 2] + __popc(word & ((1u << (e & 31)) - 1u));
                    const int axis = e / 648, rem = e - 648 * axis;
                    const int ca = rem & 7, cb = (rem >> 3) % 9, cc = (rem >> 3) / 9;
                    const int x = axis == 0 ? ca : (axis == 1 ? cc : cb);
                    const int y = axis == 0 ? cb : (axis == 1 ? ca : cc);
                    const int z = axis == 0 ? cc : (axis == 1 ? cb : ca);
                    const int r0 = x + 9 * (y + 9 * z);
                    const int r1 = r0 + (axis == 0 ? 1 : (axis == 1 ? 9 : 81));
                    const float D0 = W.D[r0], D1 = W.D[r1];
                    const float t = D0 / (D0 - D1);
                    const int gx = 8 * bx + x, gy = 8 * by + y, gz = 8 * bz + z;
                    float px = md.nu * (float)gx, py = md.nu * (float)gy, pz = md.nu * (float)gz;
                    if (axis == 0) px = md.nu * ((float)gx + t);
                    else if (axis == 1) py = md.nu * ((float)gy + t);
                    else pz = md.nu * ((float)gz + t);
                    // label of the endpoint nearer the surface (lower endpoint on ties)
                    const int lab = fabsf(D1) < fabsf(D0) ? W.lab[r1] : W.lab[r0];
                    const uchar4 col = S.pal[lab];
                    const unsigned packed = (unsigned)col.x | ((unsigned)col.y << 8) | ((unsigned)col.z << 16) |
                                            ((unsigned)lab << 24);
                    md.av[vo + vid] = make_float4(px, py, pz, __uint_as_float(packed));
                    md.ak[vo + vid] = edge_key(gx, gy, gz, axis);
                }
            }
            // triangles of this lane's cubes, in counting order
            long long tb = to + toff;
#pragma unroll 1
            for (int q = 0; q < 2; ++q) {
                const int cr = lane + 32 * q, ay = cr & 7, az = cr >> 3;
#pragma unroll 1
                for (int ax = 0; ax < 8; ++ax) {
                    const int a = ax + 8 * cr;
                    const int cs = W.cs[a];
                    const int nt = cs ? S.ntri[cs] : 0;
                    for (int j = 0; j < nt; ++j) {
                        int vid[3];
#pragma unroll
                        for (int k = 0; k < 3; ++k) {
                            const int e = cube_edge_index(S.tri[(cs * MC_MAXTRI + j) * 3 + k], ax, ay, az);
                            vid[k] = W.woff[e >> 5] + __popc(W.edge[e >> 5] & ((1u << (e & 31)) - 1u));
                        }
                        md.at[tb + j] = make_ushort4((unsigned short)vid[0], (unsigned short)vid[1],
                                                     (unsigned short)vid[2], (unsigned short)a);
                    }
                    tb += nt;
                }
            }
        }
        __syncwarp();
    }
    if (lane == 0) {
        if (n_v) atomicAdd(&fd.ctr[CT_MV], (unsigned long long)n_v);
        if (n_t) atomicAdd(&fd.ctr[CT_MT], (unsigned long long)n_t);
    }
}

int mesh_upload_tables(const int8_t *tri, const uint8_t *ntri) {
    if (!h_tri_dev) {
        if (cudaMalloc(&h_tri_dev, 256 * MC_MAXTRI * 3) != cudaSuccess) return -1;
        if (cudaMalloc(&h_ntri_dev, 256) != cudaSuccess) return -1;
        if (cudaMemcpy(h_tri_dev, tri, 256 * MC_MAXTRI * 3, cudaMemcpyHostToDevice) != cudaSuccess) return -1;
        if (cudaMemcpy(h_ntri_dev, ntri, 256, cudaMemcpyHostToDevice) != cudaSuccess) return -1;
    }
    return 0;
}

int mesh_blocks_per_sm() {
    const int bytes = (int)sizeof(MeshCtaSmem);
    cudaFuncSetAttribute(k_mesh, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_mesh, 32 * MESH_WARPS, bytes);
    return n > 0 ? n : 1;
}

void launch_mesh(const MapDev &md, const FrameDev &fd, const uchar4 *palette, int grid, cudaStream_t s) {
    k_mesh<<<grid, 32 * MESH_WARPS, sizeof(MeshCtaSmem), s>>>(md, fd, h_tri_dev, h_ntri_dev, palette);
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
                const unsigned pk = __float_as_uint(v.w);
                pos[3 * (ov + i)] = v.x;
                pos[3 * (ov + i) + 1] = v.y;
                pos[3 * (ov + i) + 2] = v.z;
                col[4 * (ov + i)] = pk & 0xff;
                col[4 * (ov + i) + 1] = (pk >> 8) & 0xff;
                col[4 * (ov + i) + 2] = (pk >> 16) & 0xff;
                col[4 * (ov + i) + 3] = (pk >> 24) & 0xff;
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
