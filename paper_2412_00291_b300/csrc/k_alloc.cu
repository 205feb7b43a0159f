// Per-point work of a scan (range-image winners and block allocation along
// each point's truncation band, the touched-block list U_k); plus pool
// initialisation and the block read/write helpers.
//
// Band of a valid point (range r in [r_min, r_max]): the world segment
// [p - tau d, p + tau d] (start clipped to the sensor when r < tau), d the
// ray direction, in "voxel units plus one half" so that block b occupies
// [8b, 8b + 8) on every axis.  Endpoints and crossing parameters follow a
// fixed IEEE single-precision recipe (correctly rounded intrinsics, no
// contraction), which makes the allocated block set reproducible bit for bit.
#include <algorithm>

#include "frame_bodies.cuh"

namespace stsdf {

__global__ void __launch_bounds__(128) k_points(const float *__restrict__ pts, ScanConst sc, MapDev md, FrameDev fd) {
    long long cnt[3] = {0, 0, 0};
    pdl_trigger();   // the TSDF grid may be scheduled now; it waits for this grid's end
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    // the next scan's buffers (no kernel of this scan reads them; the grid covers win_next_n)
    if (fd.win_next && i < fd.win_next_n) fd.win_next[i] = ~0ull;
    if (fd.ctr_next && i < CT_COUNT) fd.ctr_next[i] = 0ull;
    points_item(pts, sc, md, fd, i, cnt);
    cta_count<3>(fd.ctr, {CT_VALID, CT_PIXEL, CT_NEW}, cnt);
}

// Parity instrumentation: for each block of the touched list U_k (hash slots),
// its coordinates and the 512 voxel decision records the TSDF kernel wrote.
__global__ void k_dbg_gather(MapDev md, const int *__restrict__ touched, long long nt, const int *__restrict__ vrec,
                             int32_t *coords, int32_t *out) {
    for (long long j = blockIdx.x; j < nt; j += gridDim.x) {
        const int h = touched[j];
        const int slot = md.hs[h].val;
        if (threadIdx.x == 0) {
            int x, y, z;
            unpack_block(md.hs[h].key, x, y, z);
            coords[3 * j] = x;
            coords[3 * j + 1] = y;
            coords[3 * j + 2] = z;
        }
        for (int v = threadIdx.x; v < BV; v += blockDim.x)
            out[j * BV + v] = slot < 0 ? 0 : vrec[(long long)slot * BV + v];
    }
}

void launch_dbg_gather(const MapDev &md, const int *touched, long long nt, const int *vrec, int32_t *coords,
                       int32_t *out, cudaStream_t s) {
    if (nt <= 0) return;
    const int grid = (int)std::min<long long>(nt, 148 * 16);
    k_dbg_gather<<<grid, 128, 0, s>>>(md, touched, nt, vrec, coords, out);
}

// A scan's counters and the device state, copied after the scan's last kernel
// into one record [counters | state] for the host to download.
__global__ void k_snapshot(const unsigned long long *__restrict__ ctr, const DevState *__restrict__ st,
                           unsigned long long *__restrict__ rec) {
    constexpr int nst = (int)(sizeof(DevState) / sizeof(unsigned long long));
    const unsigned long long *sw = reinterpret_cast<const unsigned long long *>(st);
    for (int i = threadIdx.x; i < CT_COUNT + nst; i += blockDim.x) rec[i] = i < CT_COUNT ? ctr[i] : sw[i - CT_COUNT];
}

// Link every allocated block (after host-side writes).
__global__ void k_link_all(MapDev md) {
    unsigned long long pc = md.st->pool_count;
    if (pc > (unsigned long long)md.max_blocks) pc = md.max_blocks;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < (long long)pc * 7;
         e += (long long)gridDim.x * blockDim.x) {
        const int s = (int)(e / 7), o = 1 + (int)(e % 7);
        link_block(md, md.slot_key[s], s, o);
    }
}

// Every allocated pool slot, in slot order, into the re-mesh list (full re-mesh).
__global__ void k_list_all(MapDev md, FrameDev fd) {
    unsigned long long pc = md.st->pool_count;
    if (pc > (unsigned long long)md.max_blocks) pc = md.max_blocks;
    if (blockIdx.x == 0 && threadIdx.x == 0) fd.ctr[CT_DIRTY] = pc;
    for (unsigned long long s = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; s < pc;
         s += (unsigned long long)gridDim.x * blockDim.x)
        fd.dirty[s] = (int)s;
}

// D = 0, W = 0, uniform class distribution, label 0, empty mesh segment.
__global__ void k_init_pool(MapDev md) {
    const long long nvox = (long long)md.max_blocks * BV;
    const float lp0 = -logf((float)md.C);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nvox;
         i += (long long)gridDim.x * blockDim.x) {
        if (md.storage == 0) md.dw32[i] = make_float2(0.f, 0.f);
        else md.dw16[i] = __floats2half2_rn(0.f, 0.f);
        md.label[i] = 0;
        const long long slot = i / BV, v = i - slot * BV;
        for (int c = 0; c < md.CP; ++c) {
            const long long j = lp_index(md, i, c);
            const float val = c < md.C ? lp0 : 0.f;   // padding of the record stays zero
            if (md.storage == 0) md.lp32[j] = val;
            else md.lp16[j] = __float2half_rn(val);
        }
        if (v == 0) md.seg[slot] = make_int4(0, 0, 0, 0);
    }
}

// Write one block (host test fixtures / checkpoint load); allocates it when new.
__global__ void k_write_block(MapDev md, uint64_t key, const float *D, const float *W, const float *logP) {
    __shared__ int s_slot;
    if (threadIdx.x == 0) {
        int is_new = 0;
        const int h = hash_insert(md, key, is_new);
        s_slot = h < 0 ? -1 : md.hs[h].val;
        if (s_slot >= 0) {
            md.slot_key[s_slot] = key;
            if (is_new) md.slot_frame[s_slot] = -2;
        }
    }
    __syncthreads();
    const int slot = s_slot;
    if (slot < 0) return;
    for (int v = threadIdx.x; v < BV; v += blockDim.x) {
        const long long vox = (long long)slot * BV + v;
        if (md.storage == 0) md.dw32[vox] = make_float2(D[v], W[v]);
        else md.dw16[vox] = __floats2half2_rn(D[v], W[v]);
        int best = 0;
        float bv = -INFINITY;
        for (int c = 0; c < md.C; ++c) {
            const float lp = logP ? logP[c * BV + v] : -logf((float)md.C);
            const long long j = lp_index(md, vox, c);
            if (md.storage == 0) md.lp32[j] = lp;
            else md.lp16[j] = __float2half_rn(lp);
            const float stored = md.storage == 0 ? lp : __half2float(__float2half_rn(lp));
            if (stored > bv) {
                bv = stored;
                best = c;
            }
        }
        md.label[vox] = (uint8_t)best;
    }
}

__global__ void k_read_blocks(MapDev md, const uint64_t *keys, int n, float *D, float *W, float *logP,
                              uint8_t *label, uint8_t *found, float *G) {
    const int b = blockIdx.x;
    if (b >= n) return;
    __shared__ int s_slot;
    if (threadIdx.x == 0) {
        const int h = hash_find(md.hs, md.mask, keys[b]);
        s_slot = h < 0 ? -1 : md.hs[h].val;
        if (found) found[b] = s_slot >= 0;
    }
    __syncthreads();
    const int slot = s_slot;
    for (int v = threadIdx.x; v < BV; v += blockDim.x) {
        const long long o = (long long)b * BV + v;
        float d = 0.f, w = 0.f;
        if (slot >= 0) {
            const long long vox = (long long)slot * BV + v;
            if (md.storage == 0) {
                const float2 q = md.dw32[vox];
                d = q.x;
                w = q.y;
            } else {
                const float2 q = __half22float2(md.dw16[vox]);
                d = q.x;
                w = q.y;
            }
            if (label) label[o] = md.label[vox];
        } else if (label) {
            label[o] = 0;
        }
        if (D) D[o] = d;
        if (W) W[o] = w;
        if (logP) {
            for (int c = 0; c < md.C; ++c) {
                float lp = -logf((float)md.C);
                if (slot >= 0) {
                    const long long j = lp_index(md, (long long)slot * BV + v, c);
                    lp = md.storage == 0 ? md.lp32[j] : __half2float(md.lp16[j]);
                }
                logP[((long long)b * md.C + c) * BV + v] = lp;
            }
        }
        if (G) {
            // gradient planes of the non-projective mode, [b][3][512]
            for (int k = 0; k < 3; ++k) {
                float g = 0.f;
                if (slot >= 0) {
                    const long long j = ((long long)slot * 3 + k) * BV + v;
                    g = md.storage == 0 ? md.g32[j] : __half2float(md.g16[j]);
                }
                G[((long long)b * 3 + k) * BV + v] = g;
            }
        }
    }
}

__global__ void k_collect_blocks(MapDev md, int32_t *coords, unsigned long long *count) {
    for (unsigned long long h = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; h <= md.mask;
         h += (unsigned long long)gridDim.x * blockDim.x) {
        const uint64_t k = md.hs[h].key;
        if (k == EMPTY_KEY || md.hs[h].val < 0) continue;
        const unsigned long long i = atomicAdd(count, 1ull);
        if (coords && i < (unsigned long long)md.max_blocks) {
            int x, y, z;
            unpack_block(k, x, y, z);
            coords[3 * i] = x;
            coords[3 * i + 1] = y;
            coords[3 * i + 2] = z;
        }
    }
}

void launch_points(const float *pts, const ScanConst &sc, const MapDev &md, const FrameDev &fd, cudaStream_t s) {
    // 128-thread CTAs: ~7 per SM for a 131,072-point scan, evenly spread; at least
    // one CTA, and enough to reset the next scan's range image
    const long long n = std::max<long long>({(long long)sc.n, fd.win_next ? fd.win_next_n : 0ll, 1ll});
    k_points<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(pts, sc, md, fd);
}
void alloc_kernel_attributes() {
    cudaFuncSetAttribute(k_points, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    cudaFuncSetAttribute(k_snapshot, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
}
void launch_snapshot(const unsigned long long *ctr, const DevState *st, unsigned char *rec, cudaStream_t s) {
    static_assert(sizeof(DevState) % sizeof(unsigned long long) == 0, "DevState is a whole number of words");
    k_snapshot<<<1, 128, 0, s>>>(ctr, st, reinterpret_cast<unsigned long long *>(rec));
}
void launch_list_all(const MapDev &md, const FrameDev &fd, int, cudaStream_t s) {
    k_list_all<<<1024, 256, 0, s>>>(md, fd);
}
void launch_init_pool(const MapDev &md, cudaStream_t s) { k_init_pool<<<2048, 256, 0, s>>>(md); }
void launch_link_all(const MapDev &md, cudaStream_t s) { k_link_all<<<1024, 256, 0, s>>>(md); }
void launch_write_block(const MapDev &md, uint64_t key, const float *D, const float *W, const float *logP,
                        cudaStream_t s) {
    k_write_block<<<1, 256, 0, s>>>(md, key, D, W, logP);
}
void launch_read_blocks(const MapDev &md, const uint64_t *keys, int n, float *D, float *W, float *logP,
                        uint8_t *label, uint8_t *found, float *G, cudaStream_t s) {
    if (n > 0) k_read_blocks<<<n, 256, 0, s>>>(md, keys, n, D, W, logP, label, found, G);
}
void launch_collect_blocks(const MapDev &md, int32_t *coords, unsigned long long *count, cudaStream_t s) {
    k_collect_blocks<<<1024, 256, 0, s>>>(md, coords, count);
}

}  // namespace stsdf
