// Mesh traversability (Sec. III-D, "Traversability Extraction"; Table II
// parameters) over the mesh last extracted from a map.
//
// For every extracted vertex, within the ball B of radius r around it:
//   v_hd = max z - min z over B (height difference),
//   v_s  = angle of the vertex normal from the vertical (steepness),
//   v_r  = angle between the vertex normal and the mean normal of B (roughness),
// traversable when all three are below their thresholds and the vertex's class
// is in the allowed set.  Vertices are welded by lattice-edge key (seam copies
// in different blocks are one vertex); a vertex normal is the area-weighted sum
// of its triangles' normals.
//
// Pipeline (all device-side, one stream):
//   k_trav_weld    open-addressing hash of vertex keys; each key's lowest
//                  vertex index becomes the representative of its copies;
//   k_trav_rep     every vertex learns its representative;
//   k_trav_face    per triangle, (b - a) x (c - a) added to its three
//                  representatives (vector atomics; FMA difference of
//                  products per component, so slivers keep their direction);
//   k_trav_cells   representatives: unit normal; a hash of cells of edge ~r
//                  counts the vertices per cell;
//   k_trav_alloc   cell ranges: block-wide scan of the counts, one atomic per
//                  CTA for the block's base;
//   k_trav_scatter representatives into their cell's range (position, label,
//                  normal contiguous per cell);
//   k_trav_query   per vertex: the 27 cells around it, candidates within r.
// Angles use atan2(|a x b|, a . b), accurate for small angles in FP32.
#include "kernels.h"

namespace stsdf {

__device__ __forceinline__ int trav_slot_insert(uint64_t *keys, uint64_t mask, uint64_t key, unsigned *err) {
    uint64_t h = fmix64(key) & mask;
    for (int p = 0; p < MAX_PROBES; ++p) {
        const unsigned long long k =
            atomicCAS((unsigned long long *)&keys[h], (unsigned long long)EMPTY_KEY, (unsigned long long)key);
        if (k == EMPTY_KEY || k == key) return (int)h;
        h = (h + 1) & mask;
    }
    atomicOr(err, 1u);
    return -1;
}

__device__ __forceinline__ int trav_slot_find(const uint64_t *keys, uint64_t mask, uint64_t key) {
    uint64_t h = fmix64(key) & mask;
    for (int p = 0; p < MAX_PROBES; ++p) {
        const uint64_t k = keys[h];
        if (k == key) return (int)h;
        if (k == EMPTY_KEY) return -1;
        h = (h + 1) & mask;
    }
    return -1;
}

__device__ __forceinline__ void trav_cell(const TravDev &b, float x, float y, float z, int &cx, int &cy, int &cz) {
    cx = (int)floorf(x * b.inv_cell);
    cy = (int)floorf(y * b.inv_cell);
    cz = (int)floorf(z * b.inv_cell);
}

__global__ void k_trav_weld(TravDev b, const int64_t *__restrict__ vkey, long long nv) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (long long)gridDim.x * blockDim.x) {
        const int h = trav_slot_insert(b.vkeys, b.vmask, (uint64_t)vkey[i], b.err);
        b.rep[i] = h;
        if (h >= 0) atomicMin(&b.vfirst[h], (int)i);
    }
}

__global__ void k_trav_rep(TravDev b, long long nv) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (long long)gridDim.x * blockDim.x) {
        const int h = b.rep[i];
        b.rep[i] = h >= 0 ? b.vfirst[h] : (int)i;
    }
}

__global__ void k_trav_face(TravDev b, const float *__restrict__ pos, const int32_t *__restrict__ tri, long long nt) {
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += (long long)gridDim.x * blockDim.x) {
        const int ia = tri[3 * t], ib = tri[3 * t + 1], ic = tri[3 * t + 2];
        const float ax = pos[3 * ia], ay = pos[3 * ia + 1], az = pos[3 * ia + 2];
        const float ux = pos[3 * ib] - ax, uy = pos[3 * ib + 1] - ay, uz = pos[3 * ib + 2] - az;
        const float vx = pos[3 * ic] - ax, vy = pos[3 * ic + 1] - ay, vz = pos[3 * ic + 2] - az;
        // each component with Kahan's FMA difference of products: accurate to a few ulp
        // of the component itself, also for sliver triangles (|u x v| << |u| |v|)
        const float4 n = make_float4(diff_of_products(uy, vz, uz, vy), diff_of_products(uz, vx, ux, vz),
                                     diff_of_products(ux, vy, uy, vx), 0.f);
        atomicAdd(&b.nacc[b.rep[ia]], n);
        atomicAdd(&b.nacc[b.rep[ib]], n);
        atomicAdd(&b.nacc[b.rep[ic]], n);
    }
}

__global__ void k_trav_cells(TravDev b, const float *__restrict__ pos, long long nv) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (long long)gridDim.x * blockDim.x) {
        if (b.rep[i] != (int)i) {
            b.vcell[i] = -1;
            continue;
        }
        float4 n = b.nacc[i];
        const float l2 = n.x * n.x + n.y * n.y + n.z * n.z;
        if (l2 > 0.f) {
            const float il = rsqrtf(l2);
            n = make_float4(n.x * il, n.y * il, n.z * il, 1.f);
        } else {
            n = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        b.nacc[i] = n;
        int cx, cy, cz;
        trav_cell(b, pos[3 * i], pos[3 * i + 1], pos[3 * i + 2], cx, cy, cz);
        const int h = trav_slot_insert(b.ckeys, b.cmask, pack_block(cx, cy, cz), b.err);
        b.vcell[i] = h;
        if (h >= 0) atomicAdd(&b.ccount[h], 1);
    }
}

// 1024 cell slots per CTA (256 threads x 4): exclusive offsets within the CTA,
// one atomic for the CTA's base in the sorted arrays.
__global__ void __launch_bounds__(256) k_trav_alloc(TravDev b) {
    __shared__ int s_warp[8];
    __shared__ unsigned long long s_base;
    const long long base = (long long)blockIdx.x * 1024 + 4 * threadIdx.x;
    int c[4], sum = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        c[q] = base + q <= (long long)b.cmask ? b.ccount[base + q] : 0;
        sum += c[q];
    }
    int total;
    int off = block_exclusive_scan(sum, s_warp, total);
    if (threadIdx.x == 0) s_base = atomicAdd(b.cursor, (unsigned long long)total);
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if (base + q <= (long long)b.cmask) b.cstart[base + q] = (int)(s_base + off);
        off += c[q];
    }
}

__global__ void k_trav_scatter(TravDev b, const float *__restrict__ pos, const uint8_t *__restrict__ col, long long nv) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (long long)gridDim.x * blockDim.x) {
        const int h = b.vcell[i];
        if (h < 0) continue;
        const int k = b.cstart[h] + atomicAdd(&b.cfill[h], 1);
        b.spos[k] = make_float4(pos[3 * i], pos[3 * i + 1], pos[3 * i + 2], __int_as_float((int)col[4 * i + 3]));
        b.snrm[k] = b.nacc[i];
    }
}

__global__ void __launch_bounds__(256) k_trav_query(TravDev b, TravParamsDev p, const float *__restrict__ pos,
                                                    const uint8_t *__restrict__ col, long long nv, float4 *props,
                                                    uint8_t *trav) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (long long)gridDim.x * blockDim.x) {
        const float px = pos[3 * i], py = pos[3 * i + 1], pz = pos[3 * i + 2];
        const float4 n = b.nacc[b.rep[i]];
        int cx, cy, cz;
        trav_cell(b, px, py, pz, cx, cy, cz);
        float zmin = pz, zmax = pz, mx = 0.f, my = 0.f, mz = 0.f;
        int cnt = 0;
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const int h = trav_slot_find(b.ckeys, b.cmask, pack_block(cx + dx, cy + dy, cz + dz));
                    if (h < 0) continue;
                    const int k0 = b.cstart[h], k1 = k0 + b.ccount[h];
                    for (int k = k0; k < k1; ++k) {
                        const float4 q = b.spos[k];
                        const float ex = q.x - px, ey = q.y - py, ez = q.z - pz;
                        if (ex * ex + ey * ey + ez * ez > p.r2) continue;
                        zmin = fminf(zmin, q.z);
                        zmax = fmaxf(zmax, q.z);
                        const float4 m = b.snrm[k];
                        mx += m.x;
                        my += m.y;
                        mz += m.z;
                        ++cnt;
                    }
                }
        const float hd = zmax - zmin;
        float s, r;
        if (n.w > 0.f) {
            s = atan2f(sqrtf(n.x * n.x + n.y * n.y), n.z);
            const float c0 = n.y * mz - n.z * my, c1 = n.z * mx - n.x * mz, c2 = n.x * my - n.y * mx;
            const float ml2 = mx * mx + my * my + mz * mz;
            r = ml2 > 0.f ? atan2f(sqrtf(c0 * c0 + c1 * c1 + c2 * c2), n.x * mx + n.y * my + n.z * mz) : 0.f;
        } else {
            // no normal: steepness and roughness of a vertical normal (never traversable)
            s = 1.57079632679489662f;
            r = (mx * mx + my * my + mz * mz) > 0.f ? 1.57079632679489662f : 0.f;
        }
        const int lab = (int)col[4 * i + 3];
        const bool cls = lab < 64 && ((p.class_mask >> lab) & 1ull);
        props[i] = make_float4(hd, s, r, (float)cnt);
        trav[i] = (uint8_t)(hd < p.t_hd && s < p.t_s && r < p.t_r && cls);
    }
}

void launch_weld(const TravDev &b, const int64_t *vkey, long long nv, cudaStream_t s);

static int grid_for(long long n, int per) {
    long long g = (n + per - 1) / per;
    if (g > 148 * 16) g = 148 * 16;
    return (int)(g < 1 ? 1 : g);
}

void launch_weld(const TravDev &b, const int64_t *vkey, long long nv, cudaStream_t s) {
    if (nv <= 0) return;
    k_trav_weld<<<grid_for(nv, 256), 256, 0, s>>>(b, vkey, nv);
    k_trav_rep<<<grid_for(nv, 256), 256, 0, s>>>(b, nv);
}

void launch_traversability(const TravDev &b, const TravParamsDev &p, const float *pos, const uint8_t *col,
                           const int64_t *vkey, const int32_t *tri, long long nv, long long nt, float4 *props,
                           uint8_t *trav, cudaStream_t s) {
    if (nv <= 0) return;
    k_trav_weld<<<grid_for(nv, 256), 256, 0, s>>>(b, vkey, nv);
    k_trav_rep<<<grid_for(nv, 256), 256, 0, s>>>(b, nv);
    if (nt > 0) k_trav_face<<<grid_for(nt, 256), 256, 0, s>>>(b, pos, tri, nt);
    k_trav_cells<<<grid_for(nv, 256), 256, 0, s>>>(b, pos, nv);
    k_trav_alloc<<<(unsigned)((b.cmask + 1 + 1023) / 1024), 256, 0, s>>>(b);
    k_trav_scatter<<<grid_for(nv, 256), 256, 0, s>>>(b, pos, col, nv);
    k_trav_query<<<grid_for(nv, 256), 256, 0, s>>>(b, p, pos, col, nv, props, trav);
}

}  // namespace stsdf
