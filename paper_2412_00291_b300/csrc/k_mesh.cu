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

__global__ void __launch_bounds__(256) k_mesh(MapDev md, FrameDev fd, const int8_t *__restrict__ ttri,
                                              const uint8_t *__restrict__ tntri, const uchar4 *__restrict__ tpal) {
    __shared__ int8_t s_tri[256 * MC_MAXTRI * 3];
    __shared__ uint8_t s_ntri[256];
    __shared__ uchar4 s_pal[256];
    __shared__ float sD[729];
    __shared__ uint8_t sOk[729];
    __shared__ uint8_t sLab[729];
    __shared__ uint16_t sCase[512];
    __shared__ int16_t sVid[MC_EDGES];
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
    __syncthreads();
    for (unsigned long long li = blockIdx.x; li < nd; li += gridDim.x) {
        const int h = fd.dirty[li];
        const int slot = md.vals[h];
        int bx, by, bz;
        unpack_block(md.keys[h], bx, by, bz);
        if (tid < 8) {
            int s = slot;
            if (tid) {
                const int hh =
                    hash_find(md.keys, md.mask, pack_block(bx + (tid & 1), by + ((tid >> 1) & 1), bz + (tid >> 2)));
                s = hh < 0 ? -1 : md.vals[hh];
            }
            s_nb[tid] = s;
        }
        __syncthreads();
        for (int r = tid; r < 729; r += blockDim.x) {
            const int x = r % 9, y = (r / 9) % 9, z = r / 81;
            const int s = s_nb[(x >> 3) | ((y >> 3) << 1) | ((z >> 3) << 2)];
            float D = 0.f;
            uint8_t ok = 0, lab = 0;
            if (s >= 0) {
                const long long vox = (long long)s * BV + (x & 7) + 8 * (y & 7) + 64 * (z & 7);
                const float2 dw = md.storage == 0 ? md.dw32[vox] : __half22float2(md.dw16[vox]);
                D = dw.x;
                ok = dw.y > 0.f;
                lab = md.label[vox];
            }
            sD[r] = D;
            sOk[r] = ok;
            sLab[r] = lab;
        }
        __syncthreads();
        // cubes 2t, 2t+1: validity, case, triangle count
        int nt_q[2];
        int cnt_t = 0;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int a = 2 * tid + q;
            const int ax = a & 7, ay = (a >> 3) & 7, az = a >> 6;
            bool valid = true;
            int cs = 0;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int r = (ax + (c & 1)) + 9 * ((ay + ((c >> 1) & 1)) + 9 * (az + (c >> 2)));
                valid = valid && sOk[r];
                cs |= (sD[r] < 0.f ? 1 : 0) << c;
            }
            const int nt = valid ? s_ntri[cs] : 0;
            sCase[a] = valid ? (uint16_t)(0x100 | cs) : (uint16_t)0;
            nt_q[q] = nt;
            cnt_t += nt;
        }
        int tot_t;
        const int toff = block_exclusive_scan(cnt_t, s_warp, tot_t);
        // lattice edges 8t .. 8t+7: crossing and used by a meshed cube of this block
        unsigned flags = 0;
        int cnt_v = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int e = 8 * tid + q;
            if (e >= MC_EDGES) break;
            const int axis = e / 648, rem = e % 648;
            const int a1 = (axis + 1) % 3, a2 = (axis + 2) % 3;
            int p[3];
            p[axis] = rem & 7;
            p[a1] = (rem >> 3) % 9;
            p[a2] = (rem >> 3) / 9;
            const int r0 = p[0] + 9 * (p[1] + 9 * p[2]);
            const int r1 = r0 + (axis == 0 ? 1 : (axis == 1 ? 9 : 81));
            if (!(sOk[r0] && sOk[r1] && ((sD[r0] < 0.f) != (sD[r1] < 0.f)))) continue;
            bool used = false;
#pragma unroll
            for (int d = 0; d < 4; ++d) {
                int an[3] = {p[0], p[1], p[2]};
                an[a1] -= d & 1;
                an[a2] -= d >> 1;
                if (an[a1] < 0 || an[a1] > 7 || an[a2] < 0 || an[a2] > 7) continue;
                if (sCase[an[0] + 8 * an[1] + 64 * an[2]] & 0x100) used = true;
            }
            if (used) {
                flags |= 1u << q;
                ++cnt_v;
            }
        }
        int tot_v;
        const int voff = block_exclusive_scan(cnt_v, s_warp, tot_v);
        {
            int k = voff;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int e = 8 * tid + q;
                if (e < MC_EDGES) sVid[e] = ((flags >> q) & 1) ? (int16_t)(k++) : (int16_t)-1;
            }
        }
        if (tid == 0) {
            const unsigned long long vo = atomicAdd(&md.st->arena_v, (unsigned long long)tot_v);
            const unsigned long long to = atomicAdd(&md.st->arena_t, (unsigned long long)tot_t);
            if (vo + tot_v > (unsigned long long)md.av_cap || to + tot_t > (unsigned long long)md.at_cap) {
                atomicOr(&md.st->err, ERR_ARENA_FULL);
                md.seg[slot] = make_int4(0, 0, 0, 0);
                s_hdr[0] = -1;
            } else {
                md.seg[slot] = make_int4((int)vo, tot_v, (int)to, tot_t);
                s_hdr[0] = (long long)vo;
                s_hdr[1] = (long long)to;
            }
            n_v += tot_v;
            n_t += tot_t;
        }
        __syncthreads();
        if (s_hdr[0] >= 0) {
            const long long vo = s_hdr[0], to = s_hdr[1];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                if (!((flags >> q) & 1)) continue;
                const int e = 8 * tid + q;
                const int axis = e / 648, rem = e % 648;
                const int a1 = (axis + 1) % 3, a2 = (axis + 2) % 3;
                int p[3];
                p[axis] = rem & 7;
                p[a1] = (rem >> 3) % 9;
                p[a2] = (rem >> 3) / 9;
                const int r0 = p[0] + 9 * (p[1] + 9 * p[2]);
                const int r1 = r0 + (axis == 0 ? 1 : (axis == 1 ? 9 : 81));
                const float D0 = sD[r0], D1 = sD[r1];
                const float t = D0 / (D0 - D1);
                const int g[3] = {8 * bx + p[0], 8 * by + p[1], 8 * bz + p[2]};
                float pos[3];
#pragma unroll
                for (int k = 0; k < 3; ++k) pos[k] = md.nu * (float)g[k];
                pos[axis] = md.nu * ((float)g[axis] + t);
                const int lab = fabsf(D1) < fabsf(D0) ? sLab[r1] : sLab[r0];
                const uchar4 col = s_pal[lab];
                const unsigned packed = (unsigned)col.x | ((unsigned)col.y << 8) | ((unsigned)col.z << 16) |
                                        ((unsigned)lab << 24);
                const long long o = vo + sVid[e];
                md.av[o] = make_float4(pos[0], pos[1], pos[2], __uint_as_float(packed));
                md.ak[o] = edge_key(g[0], g[1], g[2], axis);
            }
            long long tb = to + toff;
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int a = 2 * tid + q;
                const int nt = nt_q[q];
                if (nt == 0) continue;
                const int cs = sCase[a] & 0xff;
                const int an[3] = {a & 7, (a >> 3) & 7, a >> 6};
                for (int j = 0; j < nt; ++j) {
                    int vid[3];
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        const int ce = s_tri[(cs * MC_MAXTRI + j) * 3 + k];
                        const int axis = ce >> 2, a1 = (axis + 1) % 3, a2 = (axis + 2) % 3;
                        const int pa = an[axis], pb = an[a1] + (ce & 1), pc = an[a2] + ((ce >> 1) & 1);
                        vid[k] = sVid[axis * 648 + pa + 8 * (pb + 9 * pc)];
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
