// Map quality against a ground-truth point cloud (Sec. IV-B.1, "Evaluation
// Metrics"): the welded mesh vertices M and the ground-truth points G are each
// sorted into a hash of cells of edge ~2 nu (the truncation), and every point
// of one cloud finds its nearest point of the other among the 27 cells around
// it.  Per point: d = min(2 nu, nearest distance); the sums of d and d^2 over
// M, of d over G, the points of G with a point of M within 2 nu, and for the
// vertices with a ground-truth point within 2 nu the class confusion
// (ground-truth class of the nearest point, vertex class) accumulate per CTA
// and reach global memory with one atomic per CTA and quantity.
#include "kernels.h"

namespace stsdf {

__device__ __forceinline__ int grid_slot_insert(uint64_t *keys, uint64_t mask, uint64_t key, unsigned *err) {
    uint64_t h = fmix64(key) & mask;
    for (int p = 0; p < MAX_PROBES; ++p) {
        const unsigned long long k =
            atomicCAS((unsigned long long *)&keys[h], (unsigned long long)EMPTY_KEY, (unsigned long long)key);
        if (k == EMPTY_KEY || k == key) return (int)h;
        h = (h + 1) & mask;
    }
    atomicOr(err, ERR_HASH_PROBES);
    return -1;
}

__device__ __forceinline__ int grid_slot_find(const uint64_t *keys, uint64_t mask, uint64_t key) {
    uint64_t h = fmix64(key) & mask;
    for (int p = 0; p < MAX_PROBES; ++p) {
        const uint64_t k = keys[h];
        if (k == key) return (int)h;
        if (k == EMPTY_KEY) return -1;
        h = (h + 1) & mask;
    }
    return -1;
}

__device__ __forceinline__ uint64_t grid_key(const GridDev &g, float x, float y, float z, int dx = 0, int dy = 0,
                                             int dz = 0) {
    return pack_block((int)floorf(x * g.inv_cell) + dx, (int)floorf(y * g.inv_cell) + dy,
                      (int)floorf(z * g.inv_cell) + dz);
}

// Cells of the points (rep: only points with rep[i] == i take part; null: all); slot per point in `slot`.
__global__ void k_grid_count(GridDev g, const float *__restrict__ pts, const int *__restrict__ rep, long long n,
                             int *slot) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        if (rep && rep[i] != (int)i) {
            slot[i] = -1;
            continue;
        }
        const int h = grid_slot_insert(g.ckeys, g.cmask, grid_key(g, pts[3 * i], pts[3 * i + 1], pts[3 * i + 2]), g.err);
        slot[i] = h;
        if (h >= 0) atomicAdd(&g.ccount[h], 1);
    }
}

__global__ void __launch_bounds__(256) k_grid_alloc(GridDev g) {
    __shared__ int s_warp[8];
    __shared__ unsigned long long s_base;
    const long long base = (long long)blockIdx.x * 1024 + 4 * threadIdx.x;
    int c[4], sum = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        c[q] = base + q <= (long long)g.cmask ? g.ccount[base + q] : 0;
        sum += c[q];
    }
    int total;
    int off = block_exclusive_scan(sum, s_warp, total);
    if (threadIdx.x == 0) s_base = atomicAdd(g.cursor, (unsigned long long)total);
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if (base + q <= (long long)g.cmask) g.cstart[base + q] = (int)(s_base + off);
        off += c[q];
    }
}

// class: from the mesh colours (byte 3 of 4) or from an int32 array
__global__ void k_grid_scatter(GridDev g, const float *__restrict__ pts, const int *__restrict__ slot,
                               const uint8_t *__restrict__ col, const int32_t *__restrict__ lab, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int h = slot[i];
        if (h < 0) continue;
        const int k = g.cstart[h] + atomicAdd(&g.cfill[h], 1);
        const int c = col ? (int)col[4 * i + 3] : lab[i];
        g.spts[k] = make_float4(pts[3 * i], pts[3 * i + 1], pts[3 * i + 2], __int_as_float(c));
    }
}

// Nearest point of grid `g` to (x, y, z) within sqrt(t2): squared distance (or > t2) and its class.
__device__ __forceinline__ float grid_nearest(const GridDev &g, float x, float y, float z, float t2, int &cls) {
    float best = t2 * 2.f + 1.f;
    cls = -1;
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                const int h = grid_slot_find(g.ckeys, g.cmask, grid_key(g, x, y, z, dx, dy, dz));
                if (h < 0) continue;
                const int k0 = g.cstart[h], k1 = k0 + g.ccount[h];
                for (int k = k0; k < k1; ++k) {
                    const float4 q = g.spts[k];
                    const float ex = q.x - x, ey = q.y - y, ez = q.z - z;
                    const float d2 = ex * ex + ey * ey + ez * ez;
                    if (d2 < best) {
                        best = d2;
                        cls = __float_as_int(q.w);
                    }
                }
            }
    return best;
}

template <typename T>
__device__ __forceinline__ T block_sum(T v, T *s) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) s[wid] = v;
    __syncthreads();
    T t = 0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s[w];
    __syncthreads();
    return t;
}

// M -> G: distances of the welded vertices, and the class confusion of those within the truncation
__global__ void __launch_bounds__(256) k_quality_map(GridDev ggt, const int *__restrict__ rep,
                                                     const float *__restrict__ mpos, const uint8_t *__restrict__ mcol,
                                                     long long nv, float trunc, int C, QualityAcc *acc,
                                                     unsigned long long *conf) {
    __shared__ double s_d[8];
    __shared__ unsigned long long s_u[8];
    const float t2 = trunc * trunc;
    double sd = 0.0, sd2 = 0.0;
    unsigned long long nm = 0, nl = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (long long)gridDim.x * blockDim.x) {
        if (rep[i] != (int)i) continue;
        int cls;
        const float d2 = grid_nearest(ggt, mpos[3 * i], mpos[3 * i + 1], mpos[3 * i + 2], t2, cls);
        const float d = d2 <= t2 ? sqrtf(d2) : trunc;
        sd += d;
        sd2 += (double)d * d;
        ++nm;
        if (d2 <= t2) {
            ++nl;
            const int mc = (int)mcol[4 * i + 3];
            if (cls >= 0 && cls < C && mc < C) atomicAdd(&conf[cls * C + mc], 1ull);
        }
    }
    sd = block_sum(sd, s_d);
    if (threadIdx.x == 0) atomicAdd(&acc->sum_d_map, sd);
    sd2 = block_sum(sd2, s_d);
    if (threadIdx.x == 0) atomicAdd(&acc->sum_d2_map, sd2);
    nm = block_sum(nm, s_u);
    if (threadIdx.x == 0) atomicAdd(&acc->n_map, nm);
    nl = block_sum(nl, s_u);
    if (threadIdx.x == 0) atomicAdd(&acc->n_labeled, nl);
}

// G -> M: distances of the ground-truth points, and how many have a vertex within the truncation
__global__ void __launch_bounds__(256) k_quality_gt(GridDev gmap, const float *__restrict__ gpos, long long ng,
                                                    float trunc, QualityAcc *acc) {
    __shared__ double s_d[8];
    __shared__ unsigned long long s_u[8];
    const float t2 = trunc * trunc;
    double sd = 0.0;
    unsigned long long nc = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < ng; i += (long long)gridDim.x * blockDim.x) {
        int cls;
        const float d2 = grid_nearest(gmap, gpos[3 * i], gpos[3 * i + 1], gpos[3 * i + 2], t2, cls);
        sd += d2 <= t2 ? sqrtf(d2) : trunc;
        if (d2 <= t2) ++nc;
    }
    sd = block_sum(sd, s_d);
    if (threadIdx.x == 0) atomicAdd(&acc->sum_d_gt, sd);
    nc = block_sum(nc, s_u);
    if (threadIdx.x == 0) atomicAdd(&acc->n_gt_covered, nc);
    if (blockIdx.x == 0 && threadIdx.x == 0) acc->n_gt = (unsigned long long)ng;
}

static int grid_for(long long n, int per) {
    long long g = (n + per - 1) / per;
    if (g > 148 * 16) g = 148 * 16;
    return (int)(g < 1 ? 1 : g);
}

static void build_grid(const GridDev &g, const float *pts, const int *rep, const uint8_t *col, const int32_t *lab,
                       long long n, int *slot, cudaStream_t s) {
    k_grid_count<<<grid_for(n, 256), 256, 0, s>>>(g, pts, rep, n, slot);
    k_grid_alloc<<<(unsigned)((g.cmask + 1 + 1023) / 1024), 256, 0, s>>>(g);
    k_grid_scatter<<<grid_for(n, 256), 256, 0, s>>>(g, pts, slot, col, lab, n);
}

void launch_quality(const GridDev &gmap, const GridDev &ggt, const int *rep, const float *mpos, const uint8_t *mcol,
                    long long nv, const float *gpos, const int32_t *glab, long long ng, float trunc, int C,
                    QualityAcc *acc, unsigned long long *conf, cudaStream_t s) {
    if (nv > 0) build_grid(gmap, mpos, rep, mcol, nullptr, nv, gmap.slot, s);
    if (ng > 0) build_grid(ggt, gpos, nullptr, nullptr, glab, ng, ggt.slot, s);
    if (nv > 0 && ng > 0) {
        k_quality_map<<<grid_for(nv, 256), 256, 0, s>>>(ggt, rep, mpos, mcol, nv, trunc, C, acc, conf);
        k_quality_gt<<<grid_for(ng, 256), 256, 0, s>>>(gmap, gpos, ng, trunc, acc);
    }
}

}  // namespace stsdf
