// Incremental marching cubes (Sec. III-C.3) over the blocks to re-mesh, and
// gathering of per-block mesh segments (mesh extraction, arena compaction).
//
// One CTA per block (persistent over the device-side list).  The block and
// the +x/+y/+z faces of its 7 upper neighbours are staged in shared memory
// as a 9x9x9 voxel region; cube a (anchored at voxel a of the block) is
// meshed when all 8 corners are observed (W > 0).  A lattice edge gets a
// vertex when its endpoints differ in sign and a meshed cube of the block
// uses it; vertices and triangles are compacted with warp-ballot/shuffle
// scans and appended to the map's mesh arena with one atomic per block.
// Each vertex carries the most probable class of the edge endpoint nearer
// the surface (lower endpoint on ties) and that class's palette colour.
#include "kernels.h"

namespace stsdf {

// generated case table, shared by every map of the process
static int8_t *h_tri_dev = nullptr;      // [256][MC_MAXTRI][3] cube-edge ids
static uint8_t *h_ntri_dev = nullptr;    // [256] triangles per case

constexpr int EDGE_WORDS = (MC_EDGES + 31) / 32;   // 61 words of lattice-edge bits per block

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

__global__ void __launch_bounds__(256, 6) k_mesh(MapDev md, FrameDev fd, const int8_t *__restrict__ ttri,
                                                 const uint8_t *__restrict__ tntri, const uchar4 *__restrict__ tpal) {
    __shared__ int8_t s_tri[256 * MC_MAXTRI * 3];
    __shared__ uint8_t s_ntri[256];
    __shared__ uchar4 s_pal[256];
    __shared__ float sD[729];
    __shared__ uint8_t sF[729];        // bit 0: observed (W > 0), bit 1: inside (D < 0)
    __shared__ uint8_t sLab[729];
    __shared__ uint8_t sCase[512];
    __shared__ unsigned sEdge[EDGE_WORDS];
    __shared__ int sWordOff[EDGE_WORDS];
    __shared__ int s_nb[8];
    __shared__ int s_warp[8];
    __shared__ long long s_hdr[2];
    const int tid = threadIdx.x;
    for (int i = tid; i < 256 * MC_MAXTRI * 3; i += blockDim.x) s_tri[i] = ttri[i];
    for (int i = tid; i < 256; i += blockDim.x) {
        s_ntri[i] = tntri[i];
        s_pal[i] = tpal[i];
    }
    unsigned long long nd = *(volatile unsigned long long *)&fd.ctr[CT_DIRTY];
    if (nd > (unsigned long long)md.max_blocks) nd = md.max_blocks;
    long long n_v = 0, n_t = 0;
    const bool f32 = md.storage == 0;
    __syncthreads();
    for (unsigned long long li = blockIdx.x; li < nd; li += gridDim.x) {
        const int h = fd.dirty[li];
        const int slot = md.vals[h];
        int bx, by, bz;
        unpack_block(md.keys[h], bx, by, bz);
        // neighbour slots (lanes 1..7 of warp 0) overlap with the block's own 512 voxels
        if (tid >= 1 && tid < 8) {
            const int hh =
                hash_find(md.keys, md.mask, pack_block(bx + (tid & 1), by + ((tid >> 1) & 1), bz + (tid >> 2)));
            s_nb[tid] = hh < 0 ? -1 : md.vals[hh];
        }
        if (tid < EDGE_WORDS) sEdge[tid] = 0u;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int v = tid + 256 * q;
            const int r = (v & 7) + 9 * (((v >> 3) & 7) + 9 * (v >> 6));
            const long long vox = (long long)slot * BV + v;
            const float2 dw = f32 ? md.dw32[vox] : __half22float2(md.dw16[vox]);
            sD[r] = dw.x;
            sF[r] = (dw.y > 0.f ? 1 : 0) | (dw.x < 0.f ? 2 : 0);
            sLab[r] = md.label[vox];
        }
        __syncthreads();
        // the +x / +y / +z faces, edges and corner from the upper neighbours
        for (int r = tid; r < 729; r += blockDim.x) {
            const int x = r % 9, y = (r / 9) % 9, z = r / 81;
            const int nbi = (x >> 3) | ((y >> 3) << 1) | ((z >> 3) << 2);
            if (nbi == 0) continue;
            const int s = s_nb[nbi];
            float D = 0.f;
            uint8_t f = 0, lab = 0;
            if (s >= 0) {
                const long long vox = (long long)s * BV + (x & 7) + 8 * (y & 7) + 64 * (z & 7);
                const float2 dw = f32 ? md.dw32[vox] : __half22float2(md.dw16[vox]);
                D = dw.x;
                f = (dw.y > 0.f ? 1 : 0) | (dw.x < 0.f ? 2 : 0);
                lab = md.label[vox];
            }
            sD[r] = D;
            sF[r] = f;
            sLab[r] = lab;
        }
        __syncthreads();
        // cubes 2t, 2t+1: validity, case, triangle count; mark their crossing edges
        int nt_q[2];
        int cnt_t = 0;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int a = 2 * tid + q;
            const int ax = a & 7, ay = (a >> 3) & 7, az = a >> 6;
            const int r0 = ax + 9 * (ay + 9 * az);
            int ok = 1, cs = 0;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int f = sF[r0 + (c & 1) + 9 * ((c >> 1) & 1) + 81 * (c >> 2)];
                ok &= f;
                cs |= ((f >> 1) & 1) << c;
            }
            const int nt = ok ? s_ntri[cs] : 0;
            sCase[a] = (uint8_t)cs;
            nt_q[q] = nt;
            cnt_t += nt;
            if (nt) {
#pragma unroll
                for (int ce = 0; ce < 12; ++ce) {
                    const int axis = ce >> 2, a1 = axis == 2 ? 0 : axis + 1, a2 = axis == 0 ? 2 : axis - 1;
                    const int clo = ((ce & 1) << a1) | (((ce >> 1) & 1) << a2);
                    if (((cs >> clo) ^ (cs >> (clo | (1 << axis)))) & 1) {
                        const int e = cube_edge_index(ce, ax, ay, az);
                        atomicOr(&sEdge[e >> 5], 1u << (e & 31));
                    }
                }
            }
        }
        int tot_t;
        const int toff = block_exclusive_scan(cnt_t, s_warp, tot_t);
        if (tot_t == 0) {
            // nothing to mesh: drop the block's old segment
            if (tid == 0) {
                const int4 old = md.seg[slot];
                if (old.y | old.w) md.seg[slot] = make_int4(0, 0, 0, 0);
            }
            continue;   // tot_t is uniform; the scan's barriers protect shared memory reuse
        }
        // vertex numbering: popcount prefix over the edge bitmap
        const int wc = tid < EDGE_WORDS ? __popc(sEdge[tid]) : 0;
        int tot_v;
        const int woff = block_exclusive_scan(wc, s_warp, tot_v);
        if (tid < EDGE_WORDS) sWordOff[tid] = woff;
        // reserve arena space: vertex and triangle cursors advanced by two warps at once
        if (tid == 0) s_hdr[0] = (long long)atomicAdd(&md.st->arena_v, (unsigned long long)tot_v);
        if (tid == 32) s_hdr[1] = (long long)atomicAdd(&md.st->arena_t, (unsigned long long)tot_t);
        __syncthreads();
        const bool fits = s_hdr[0] + tot_v <= md.av_cap && s_hdr[1] + tot_t <= md.at_cap;
        if (tid == 0) {
            if (fits) {
                md.seg[slot] = make_int4((int)s_hdr[0], tot_v, (int)s_hdr[1], tot_t);
            } else {
                atomicOr(&md.st->err, ERR_ARENA_FULL);
                md.seg[slot] = make_int4(0, 0, 0, 0);
            }
            n_v += tot_v;
            n_t += tot_t;
        }
        if (fits) {
            const long long vo = s_hdr[0], to = s_hdr[1];
            // vertices of the marked edges 8t .. 8t+7 (one byte of one bitmap word)
            const int w = tid >> 2;
            if (w < EDGE_WORDS) {
                const unsigned word = sEdge[w];
                unsigned bits = (word >> ((tid & 3) * 8)) & 0xffu;
                while (bits) {
                    const int q = __ffs(bits) - 1;
                    bits &= bits - 1;
                    const int e = 8 * tid + q;
                    const int vid = sWordOff[w] + __popc(word & ((1u << (e & 31)) - 1u));
                    const int axis = e / 648, rem = e - 648 * axis;
                    const int ca = rem & 7, cb = (rem >> 3) % 9, cc = (rem >> 3) / 9;
                    const int x = axis == 0 ? ca : (axis == 1 ? cc : cb);
                    const int y = axis == 0 ? cb : (axis == 1 ? ca : cc);
                    const int z = axis == 0 ? cc : (axis == 1 ? cb : ca);
                    const int r0 = x + 9 * (y + 9 * z);
                    const int r1 = r0 + (axis == 0 ? 1 : (axis == 1 ? 9 : 81));
                    const float D0 = sD[r0], D1 = sD[r1];
                    const float t = D0 / (D0 - D1);
                    const int gx = 8 * bx + x, gy = 8 * by + y, gz = 8 * bz + z;
                    float px = md.nu * (float)gx, py = md.nu * (float)gy, pz = md.nu * (float)gz;
                    if (axis == 0) px = md.nu * ((float)gx + t);
                    else if (axis == 1) py = md.nu * ((float)gy + t);
                    else pz = md.nu * ((float)gz + t);
                    const int lab = fabsf(D1) < fabsf(D0) ? sLab[r1] : sLab[r0];
                    const uchar4 col = s_pal[lab];
                    const unsigned packed = (unsigned)col.x | ((unsigned)col.y << 8) | ((unsigned)col.z << 16) |
                                            ((unsigned)lab << 24);
                    md.av[vo + vid] = make_float4(px, py, pz, __uint_as_float(packed));
                    md.ak[vo + vid] = edge_key(gx, gy, gz, axis);
                }
            }
            long long tb = to + toff;
#pragma unroll 1
            for (int q = 0; q < 2; ++q) {
                const int a = 2 * tid + q;
                const int nt = nt_q[q];
                if (nt == 0) continue;
                const int cs = sCase[a];
                const int ax = a & 7, ay = (a >> 3) & 7, az = a >> 6;
                for (int j = 0; j < nt; ++j) {
                    int vid[3];
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        const int e = cube_edge_index(s_tri[(cs * MC_MAXTRI + j) * 3 + k], ax, ay, az);
                        vid[k] = sWordOff[e >> 5] + __popc(sEdge[e >> 5] & ((1u << (e & 31)) - 1u));
                    }
                    md.at[tb + j] = make_ushort4((unsigned short)vid[0], (unsigned short)vid[1],
                                                 (unsigned short)vid[2], (unsigned short)a);
                }
                tb += nt;
            }
        }
        __syncthreads();
    }
    if (tid == 0) {
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
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_mesh, 256, 0);
    return n > 0 ? n : 1;
}

void launch_mesh(const MapDev &md, const FrameDev &fd, const uchar4 *palette, int grid, cudaStream_t s) {
    k_mesh<<<grid, 256, 0, s>>>(md, fd, h_tri_dev, h_ntri_dev, palette);
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

__global__ void k_set_cursors(MapDev md, GatherBufs g) {
    md.st->arena_v = (unsigned long long)g.totals[0];
    md.st->arena_t = (unsigned long long)g.totals[1];
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
