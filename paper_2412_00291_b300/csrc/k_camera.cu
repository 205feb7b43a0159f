// Class update from a camera label image (Sec. III-C.3): only visible,
// observed voxels (W > 0) inside the camera frustum take the image's class
// likelihood, found by ray casting the TSDF, and the distribution is updated
// by the recursive Bayesian filter (Eq. bayesian_filter).
//
//   k_block_bounds the bounding box of the allocated blocks;
//   k_cam_raycast  per pixel: the voxels the pixel's ray passes through, in
//                  order (exact cell traversal from the camera centre up to
//                  r_max, or to where the ray leaves the box); the first pair of consecutive observed voxels with
//                  D >= 0 then D < 0 is the visible surface, its range along
//                  the ray interpolated between the two centres' ranges;
//   k_cam_select   one warp per allocated block (blocks wholly behind the
//                  camera or out of range skipped): every observed voxel that
//                  projects to a pixel with a hit and lies within tau of the
//                  hit range (|psi| <= tau, psi = hit range - distance from
//                  the camera) is listed with its pixel;
//   k_semantic     the listed voxels' Bayesian update (the per-scan kernel,
//                  reading the likelihood of each voxel's pixel).
#include "frame_bodies.cuh"
#include "kernels.h"

namespace stsdf {

// Bounding box of the allocated blocks, in block coordinates: bounds[0..2] min, [3..5] max
// (initialised to +- large by the caller).  One atomic per warp and bound.
__global__ void __launch_bounds__(256) k_block_bounds(MapDev md, int *bounds) {
    unsigned long long pc = md.st->pool_count;
    if (pc > (unsigned long long)md.max_blocks) pc = md.max_blocks;
    int lo[3] = {0x7fffffff, 0x7fffffff, 0x7fffffff}, hi[3] = {-0x7fffffff, -0x7fffffff, -0x7fffffff};
    for (unsigned long long s = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; s < pc;
         s += (unsigned long long)gridDim.x * blockDim.x) {
        int b[3];
        unpack_block(md.slot_key[s], b[0], b[1], b[2]);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            lo[k] = min(lo[k], b[k]);
            hi[k] = max(hi[k], b[k]);
        }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int l = __reduce_min_sync(0xffffffffu, lo[k]), h = __reduce_max_sync(0xffffffffu, hi[k]);
        if ((threadIdx.x & 31) == 0) {
            atomicMin(&bounds[k], l);
            atomicMax(&bounds[3 + k], h);
        }
    }
}

__global__ void __launch_bounds__(256) k_cam_raycast(CamConst cc, MapDev md, const int *__restrict__ bounds,
                                                     float *range) {
    const int np = cc.W * cc.H;
    // the allocated blocks' box in metres: cells [nu (8 b - 1/2), nu (8 b + 7 + 1/2))
    float blo[3], bhi[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        // (in float: an empty map leaves the bounds at +-2^31 and an empty box)
        blo[k] = ((float)bounds[k] * BS - 0.5f) * cc.nu;
        bhi[k] = ((float)bounds[3 + k] * BS + (BS - 0.5f)) * cc.nu;
    }
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < np; p += gridDim.x * blockDim.x) {
        const int u = p % cc.W, v = p / cc.W;
        float d0 = ((float)u - cc.cx) * cc.inv_fx, d1 = ((float)v - cc.cy) * cc.inv_fy, d2 = 1.f;
        const float il = 1.f / sqrtf(d0 * d0 + d1 * d1 + 1.f);
        d0 *= il;
        d1 *= il;
        d2 *= il;
        const float d[3] = {cc.R[0] * d0 + cc.R[1] * d1 + cc.R[2] * d2, cc.R[3] * d0 + cc.R[4] * d1 + cc.R[5] * d2,
                            cc.R[6] * d0 + cc.R[7] * d1 + cc.R[8] * d2};
        int vx[3], step[3];
        float tmax[3], tdel[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            vx[k] = (int)floorf(cc.c[k] * cc.inv_nu + 0.5f);
            step[k] = 0;
            tmax[k] = INFINITY;
            tdel[k] = INFINITY;
            if (d[k] > 0.f) {
                step[k] = 1;
                tmax[k] = (((float)vx[k] + 0.5f) * cc.nu - cc.c[k]) / d[k];
                tdel[k] = cc.nu / d[k];
            } else if (d[k] < 0.f) {
                step[k] = -1;
                tmax[k] = (((float)vx[k] - 0.5f) * cc.nu - cc.c[k]) / d[k];
                tdel[k] = -cc.nu / d[k];
            }
        }
        // no observed voxel lies outside the box: the traversal ends where the ray leaves it
        // (a voxel's cells are entered before that, so the visited cells up to then are unchanged)
        float t_end = cc.r_max;
        {
            float t_in = 0.f, t_out = cc.r_max;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                if (d[k] != 0.f) {
                    const float a = (blo[k] - cc.c[k]) / d[k], b = (bhi[k] - cc.c[k]) / d[k];
                    t_in = fmaxf(t_in, fminf(a, b));
                    t_out = fminf(t_out, fmaxf(a, b));
                } else if (cc.c[k] < blo[k] || cc.c[k] > bhi[k]) {
                    t_out = -1.f;
                }
            }
            t_end = t_in > t_out ? -1.f : fminf(cc.r_max, t_out + cc.nu);
        }
        float hit = NAN, t = 0.f, pt = 0.f, pD = 0.f;
        bool prev = false;
        int bk[3] = {0x7fffffff, 0x7fffffff, 0x7fffffff}, slot = -1;   // no block yet
        for (int it = 0; it < cc.max_steps && t <= t_end; ++it) {
            int b[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) b[k] = vx[k] >= 0 ? vx[k] / BS : -((-vx[k] + BS - 1) / BS);
            if (b[0] != bk[0] || b[1] != bk[1] || b[2] != bk[2]) {
                bk[0] = b[0];
                bk[1] = b[1];
                bk[2] = b[2];
                const int h = hash_find(md.hs, md.mask, pack_block(b[0], b[1], b[2]));
                slot = h < 0 ? -1 : md.hs[h].val;
            }
            bool cur = false;
            float ct = 0.f, cD = 0.f;
            if (slot >= 0) {
                const int li = (vx[0] - BS * b[0]) + BS * ((vx[1] - BS * b[1]) + BS * (vx[2] - BS * b[2]));
                const long long vox = (long long)slot * BV + li;
                const float2 dw = md.storage == 0 ? md.dw32[vox] : __half22float2(md.dw16[vox]);
                if (dw.y > 0.f) {
                    cur = true;
                    cD = dw.x;
                    ct = ((float)vx[0] * cc.nu - cc.c[0]) * d[0] + ((float)vx[1] * cc.nu - cc.c[1]) * d[1] +
                         ((float)vx[2] * cc.nu - cc.c[2]) * d[2];
                }
            }
            if (prev && cur && pD >= 0.f && cD < 0.f) {
                hit = pt + (ct - pt) * pD / (pD - cD);
                break;
            }
            prev = cur;
            pt = ct;
            pD = cD;
            // the nearest cell face (the lowest axis on ties)
            const int k = (tmax[0] <= tmax[1] && tmax[0] <= tmax[2]) ? 0 : (tmax[1] <= tmax[2] ? 1 : 2);
            t = tmax[k];
            vx[k] += step[k];
            tmax[k] += tdel[k];
        }
        range[p] = hit;
    }
}

__global__ void __launch_bounds__(256) k_cam_select(CamConst cc, ScanConst sc, MapDev md, FrameDev fd,
                                                    const float *__restrict__ range) {
    const int lane = threadIdx.x & 31;
    unsigned long long pc = md.st->pool_count;
    if (pc > (unsigned long long)md.max_blocks) pc = md.max_blocks;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const float brad = 0.8660254f * BS * cc.nu;    // half the block's diagonal
    for (long long s = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < (long long)pc; s += nwarps) {
        int bx, by, bz;
        unpack_block(md.slot_key[s], bx, by, bz);
        {
            const float e0 = ((float)(BS * bx) + 3.5f) * cc.nu - cc.c[0];
            const float e1 = ((float)(BS * by) + 3.5f) * cc.nu - cc.c[1];
            const float e2 = ((float)(BS * bz) + 3.5f) * cc.nu - cc.c[2];
            const float z = cc.R[2] * e0 + cc.R[5] * e1 + cc.R[8] * e2;
            if (z < -brad || e0 * e0 + e1 * e1 + e2 * e2 > (cc.r_max + brad) * (cc.r_max + brad)) continue;
        }
        for (int vi = lane; vi < BV; vi += 32) {
            bool sel = false;
            int pix = 0;
            const long long vox = s * BV + vi;
            const float2 dw = md.storage == 0 ? md.dw32[vox] : __half22float2(md.dw16[vox]);
            if (dw.y > 0.f) {
                const float e0 = (float)(BS * bx + (vi & 7)) * cc.nu - cc.c[0];
                const float e1 = (float)(BS * by + ((vi >> 3) & 7)) * cc.nu - cc.c[1];
                const float e2 = (float)(BS * bz + (vi >> 6)) * cc.nu - cc.c[2];
                // camera frame: R^T e
                const float x = cc.R[0] * e0 + cc.R[3] * e1 + cc.R[6] * e2;
                const float y = cc.R[1] * e0 + cc.R[4] * e1 + cc.R[7] * e2;
                const float z = cc.R[2] * e0 + cc.R[5] * e1 + cc.R[8] * e2;
                if (z > 0.f) {
                    const int u = (int)floorf(cc.fx * x / z + cc.cx + 0.5f);
                    const int v = (int)floorf(cc.fy * y / z + cc.cy + 0.5f);
                    if (u >= 0 && u < cc.W && v >= 0 && v < cc.H) {
                        pix = v * cc.W + u;
                        const float r = range[pix];
                        const float psi = r - sqrtf(e0 * e0 + e1 * e1 + e2 * e2);
                        if (fabsf(psi) <= sc.tau) {     // NaN (no hit) compares false
                            if (sc.has_probs) sel = true;
                            else {
                                const int l = sc.labels[pix];
                                sel = l >= 0 && l < sc.C;
                            }
                        }
                    }
                }
            }
            const unsigned mk = __ballot_sync(0xffffffffu, sel);
            if (mk) {
                unsigned long long base = 0;
                if (lane == 0) base = atomicAdd(&fd.ctr[CT_SEM], (unsigned long long)__popc(mk));
                base = __shfl_sync(0xffffffffu, base, 0);
                if (sel) {
                    const unsigned long long i = base + __popc(mk & ((1u << lane) - 1u));
                    if (i < (unsigned long long)fd.sem_cap) fd.sem_list[i] = make_int2((int)vox, pix);
                    else atomicOr(&md.st->err, ERR_LIST_FULL);
                }
            }
        }
    }
}

void launch_camera(const CamConst &cc, const ScanConst &sc, const MapDev &md, const FrameDev &fd, float *range,
                   int *bounds, int grid_semantic, cudaStream_t s) {
    const int np = cc.W * cc.H;
    int g = (np + 255) / 256;
    if (g > 148 * 16) g = 148 * 16;
    int gb = (md.max_blocks + 255) / 256;
    if (gb > 148 * 4) gb = 148 * 4;
    if (gb < 1) gb = 1;
    k_block_bounds<<<gb, 256, 0, s>>>(md, bounds);
    k_cam_raycast<<<g, 256, 0, s>>>(cc, md, bounds, range);
    int gs = (md.max_blocks + 7) / 8;
    if (gs > 148 * 8) gs = 148 * 8;
    if (gs < 1) gs = 1;
    k_cam_select<<<gs, 256, 0, s>>>(cc, sc, md, fd, range);
    launch_semantic(sc, md, fd, grid_semantic, s);
}

}  // namespace stsdf
