// Device bodies of the per-frame pipeline, shared by the single-map kernels
// (k_alloc.cu, k_integrate.cu, k_mesh.cu, k_camera.cu) and the batched
// persistent kernel (k_batch.cu).  Each body processes one work item: a point,
// a pixel of the normal image, half of a touched block (one warp), a
// class-update entry, a block to re-mesh (one warp).
#pragma once

#include "kernels.h"
#include "poly_approx.h"

namespace stsdf {

// atan2(y, x) in (-pi, pi] from the atan polynomial on [0, 1] and the octant
// symmetries; error below 5e-7 rad (polynomial 1.8e-7, the quotient and the
// octant subtractions one rounding each), atan2(+-0, x < 0) = +-pi as atan2f.
__device__ __forceinline__ float atan2_poly(float y, float x) {
    const float ax = fabsf(x), ay = fabsf(y);
    const float mx = fmaxf(ax, ay), mn = fminf(ax, ay);
    const float t = mx > 0.f ? __fdividef(mn, mx) : 0.f;
    const float p = atan_p(__fmul_rn(t, t));
    float a = ay > ax ? __fmaf_rn(-t, p, 1.57079632679489662f) : __fmul_rn(t, p);
    if (x < 0.f) a = __fsub_rn(PI_F, a);
    return copysignf(a, y);
}

// acos(c) for c in [-1, 1]: pi/2 - asin(c) from the asin polynomial when
// |c| <= 1/2 (error below 3e-7 rad), acosf beyond.
__device__ __forceinline__ float acos_poly(float c) {
    if (fabsf(c) > 0.5f) return acosf(c);
    return __fmaf_rn(-c, asin_q(__fmul_rn(c, c)), 1.57079632679489662f);
}

// Blocks met by the band of one point, visited in path order without storing
// them (registers only): a 3-D digital differential analyser over the lattice
// of 8-voxel blocks.  The band [p - tau d, p + tau d] (start clipped to the
// sensor when r < tau) is taken in voxel units plus one half, so that block b
// occupies [8 b, 8 b + 8) on every axis: e = t / nu + 1/2 + (R x / nu) f with
// f = max(0, 1 - tau / r) and 1 + tau / r at the two ends, each operation one
// IEEE single-precision rounding.  From the block of e0, each step crosses
// the block plane (or, on equal parameters, the planes) that the segment
// reaches first, t = (plane - e0) / (e1 - e0), until the block of e1.
struct BandWalk {
    float e0[3], d[3];
    float tn[3];      // parameter of the next plane crossing on each axis (infinite: none left)
    int cur[3];       // current block
    int rem[3];       // planes still to cross on each axis
    int step[3];      // direction of the crossings (+1 / -1)
    bool fresh;       // cur not yet yielded
    bool live;        // blocks left to yield
};

__device__ __forceinline__ void band_begin(const ScanConst &sc, float x0, float x1, float x2, float l, BandWalk &w) {
    const float q = __fdiv_rn(sc.tau, l);
    float f0 = __fsub_rn(1.f, q);
    if (f0 < 0.f) f0 = 0.f;
    const float f1 = __fadd_rn(1.f, q);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float s = __fmul_rn(sc.Rv[3 * k], x0);
        s = __fadd_rn(s, __fmul_rn(sc.Rv[3 * k + 1], x1));
        s = __fadd_rn(s, __fmul_rn(sc.Rv[3 * k + 2], x2));
        const float a = __fadd_rn(sc.tv[k], __fmul_rn(s, f0));
        const float e = __fadd_rn(sc.tv[k], __fmul_rn(s, f1));
        const int b0 = (int)floorf(__fmul_rn(a, 0.125f));
        const int b1 = (int)floorf(__fmul_rn(e, 0.125f));
        w.e0[k] = a;
        w.d[k] = __fsub_rn(e, a);
        w.cur[k] = b0;
        w.step[k] = b1 >= b0 ? 1 : -1;
        w.rem[k] = min(abs(b1 - b0), MAX_AXIS_CROSS);
        // first plane: 8 (b0 + 1) going up, 8 b0 going down
        const float plane = (float)(8 * (b1 > b0 ? b0 + 1 : b0));
        w.tn[k] = w.rem[k] > 0 ? __fdiv_rn(__fsub_rn(plane, a), w.d[k]) : INFINITY;
    }
    w.fresh = true;
    w.live = true;
}

// The next block of the walk; false when none is left.
__device__ __forceinline__ bool band_next(BandWalk &w, int &bx, int &by, int &bz) {
    if (!w.live) return false;
    if (!w.fresh) {
        const float t = fminf(w.tn[0], fminf(w.tn[1], w.tn[2]));
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            if (w.rem[k] > 0 && w.tn[k] == t) {
                w.cur[k] += w.step[k];
                --w.rem[k];
                const int next = w.step[k] > 0 ? w.cur[k] + 1 : w.cur[k];
                w.tn[k] = w.rem[k] > 0 ? __fdiv_rn(__fsub_rn((float)(8 * next), w.e0[k]), w.d[k]) : INFINITY;
            }
        }
    }
    w.fresh = false;
    bx = w.cur[0];
    by = w.cur[1];
    bz = w.cur[2];
    if (w.rem[0] == 0 && w.rem[1] == 0 && w.rem[2] == 0) w.live = false;
    return true;
}

// Pixel of a valid LiDAR-frame point with range l (Sec. III-C.1), -1 when its
// beam row is outside [0, H): polynomial atan2 / acos (error < 5e-7 rad, far
// inside the 1e-3-pixel band within which FP32 and FP64 choices may differ).
__device__ __forceinline__ int point_pixel_poly(const ScanConst &sc, float x, float y, float z, float l) {
    const float uc = __fmul_rn(__fsub_rn(PI_F, atan2_poly(y, x)), sc.inv_dphi);
    const float vc =
        __fmul_rn(__fsub_rn(acos_poly(fminf(fmaxf(__fdiv_rn(z, l), -1.f), 1.f)), sc.theta0), sc.inv_dtheta);
    int u = (int)floorf(__fadd_rn(uc, 0.5f));
    const int v = (int)floorf(__fadd_rn(vc, 0.5f));
    if (u >= sc.W) u -= sc.W;
    if (u < 0) u += sc.W;
    return (v >= 0 && v < sc.H) ? v * sc.W + u : -1;
}

// Find or insert a block key; lock-free (compare-and-swap on the key slot).
// The inserting thread takes the next pool slot; readers of vals[] run in
// later kernels only, so no thread waits on another.
__device__ __forceinline__ int hash_insert(const MapDev &md, uint64_t key, int &is_new) {
    uint64_t h = fmix64(key) & md.mask;
    for (int p = 0; p < MAX_PROBES; ++p) {
        const uint64_t k = md.hs[h].key;
        if (k == key) {
            is_new = 0;
            return (int)h;
        }
        if (k == EMPTY_KEY) {
            const uint64_t old = atomicCAS((unsigned long long *)&md.hs[h].key, EMPTY_KEY, key);
            if (old == EMPTY_KEY) {
                const unsigned long long s = atomicAdd(&md.st->pool_count, 1ull);
                if (s < (unsigned long long)md.max_blocks) {
                    md.hs[h].val = (int)s;
                } else {
                    md.hs[h].val = -1;
                    atomicOr(&md.st->err, ERR_POOL_FULL);
                }
                is_new = 1;
                return (int)h;
            }
            if (old == key) {
                is_new = 0;
                return (int)h;
            }
        }
        h = (h + 1) & md.mask;
    }
    atomicOr(&md.st->err, ERR_HASH_PROBES);
    return -1;
}

// One thread per point: validity, the range-image winner of its pixel
// (u = round((pi - atan2(y, x)) / dphi) mod W, v = round((acos(z / r) -
// theta0) / dtheta); nearest point wins, equal ranges the lower index, by one
// 64-bit atomicMin on (range bits << 32 | index)), and the blocks of its band.
// The point's statistics (valid, in a pixel, blocks it inserted) are added
// to `cnt`; the caller forms the totals.
__device__ __forceinline__ void points_item(const float *__restrict__ pts, const ScanConst &sc, const MapDev &md,
                                            const FrameDev &fd, long long i, long long (&cnt)[3]) {
    int valid = 0, inpix = 0, pix = -2;
    BandWalk w;
    w.live = false;
    if (i < sc.n) {
        const float x = pts[3 * i], y = pts[3 * i + 1], z = pts[3 * i + 2];
        if (isfinite(x) && isfinite(y) && isfinite(z)) {
            const float l = range_f32(x, y, z);
            if (l >= sc.r_min && l <= sc.r_max && l > 0.f) {
                valid = 1;
                const int p = point_pixel_poly(sc, x, y, z, l);
                pix = p;
                if (p >= 0) {
                    inpix = 1;
                    atomicMin(&fd.win[p], ((unsigned long long)__float_as_uint(l) << 32) | (unsigned)i);
                }
                band_begin(sc, x, y, z, l, w);
            }
        }
    }
    if (fd.dbg_point && i < sc.n) fd.dbg_point[i] = pix;
    cnt[0] += valid;
    cnt[1] += inpix;
    int n_new = 0;
    const int lane = threadIdx.x & 31;
    // Four band steps of every lane at a time.  Lanes holding the same block in
    // one step (neighbouring points of a beam) leave it to the lowest of them;
    // the owners' first hash probes, then their frame-stamp exchanges, are all
    // in flight together, and the blocks first touched in this frame are
    // appended to U_k with one counter update per warp.
    while (__any_sync(0xffffffffu, w.live)) {
        uint64_t key[4];
        bool own[4];
        int h[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int bx, by, bz;
            const bool got = band_next(w, bx, by, bz);
            key[q] = got ? pack_block(bx, by, bz) : EMPTY_KEY;
            const unsigned grp = __match_any_sync(0xffffffffu, key[q]);
            own[q] = got && __ffs(grp) - 1 == lane;
        }
        // the home slot's whole record: key, pool slot and frame stamp in one 16-byte load
        uint64_t probe[4];
        int pstamp[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            h[q] = (int)(fmix64(key[q]) & md.mask);
            pstamp[q] = -1;
            probe[q] = key[q];
            if (own[q]) {
                const HashSlot r = md.hs[h[q]];
                probe[q] = r.key;
                pstamp[q] = r.stamp;
            }
        }
        // Blocks not found at their home slot.  An empty home slot is claimed at once (its key
        // was just read): the winner of that compare-and-swap has a new block, and its frame
        // stamp exchange and pool slot allocation are issued together; a lost race to the
        // same key leaves an existing block, to another key the full find-or-insert.
        bool xchg[4], first[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            xchg[q] = false;
            first[q] = false;
            if (own[q] && probe[q] != key[q]) {
                int is_new = 0;
                pstamp[q] = -1;
                if (probe[q] == EMPTY_KEY) {
                    const uint64_t old = atomicCAS((unsigned long long *)&md.hs[h[q]].key,
                                                   (unsigned long long)EMPTY_KEY, (unsigned long long)key[q]);
                    if (old == EMPTY_KEY) {
                        ++n_new;
                        xchg[q] = true;
                        first[q] = atomicExch(&md.hs[h[q]].stamp, sc.frame) != sc.frame;
                        const unsigned long long s = atomicAdd(&md.st->pool_count, 1ull);
                        if (s < (unsigned long long)md.max_blocks) {
                            md.hs[h[q]].val = (int)s;
                            md.slot_key[s] = key[q];
                            md.slot_frame[s] = sc.frame;
                        } else {
                            md.hs[h[q]].val = -1;
                            atomicOr(&md.st->err, ERR_POOL_FULL);
                        }
                        continue;
                    }
                    if (old == key[q]) continue;   // inserted meanwhile by another lane or warp
                }
                h[q] = hash_insert(md, key[q], is_new);
                if (h[q] >= 0 && is_new) {
                    ++n_new;
                    const int sl = md.hs[h[q]].val;
                    if (sl >= 0) {
                        md.slot_key[sl] = key[q];
                        md.slot_frame[sl] = sc.frame;
                    }
                }
            }
        }
        // first touch in this scan: a stamp already at this frame was set by an exchange of this
        // scan (stamps change only by that exchange), so the exchange is needed only otherwise
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (!xchg[q])
                first[q] = own[q] && h[q] >= 0 && pstamp[q] != sc.frame &&
                           atomicExch(&md.hs[h[q]].stamp, sc.frame) != sc.frame;
        const int cnt = (int)first[0] + (int)first[1] + (int)first[2] + (int)first[3];
        int tot;
        int off = warp_exclusive_scan(cnt, tot);
        if (tot) {
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(&fd.ctr[CT_TOUCHED], (unsigned long long)tot);
            base = __shfl_sync(0xffffffffu, base, 0);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (first[q]) {
                    const unsigned long long idx = base + off++;
                    if (idx < (unsigned long long)md.max_blocks) fd.touched[idx] = h[q];
                    else atomicOr(&md.st->err, ERR_LIST_FULL);
                }
            }
        }
    }
    cnt[2] += n_new;
}

template <bool F16>
__device__ __forceinline__ float2 load_dw(const MapDev &md, long long vox) {
    if (F16) return __half22float2(md.dw16[vox]);
    return md.dw32[vox];
}
template <bool F16>
__device__ __forceinline__ void store_dw(const MapDev &md, long long vox, float D, float W) {
    if (F16) md.dw16[vox] = __floats2half2_rn(D, W);
    else md.dw32[vox] = make_float2(D, W);
}
template <bool F16>
__device__ __forceinline__ float load_lp(const MapDev &md, long long j) {
    if (F16) return __half2float(md.lp16[j]);
    return md.lp32[j];
}
template <bool F16>
__device__ __forceinline__ void store_lp(const MapDev &md, long long j, float v) {
    if (F16) md.lp16[j] = __float2half_rn(v);
    else md.lp32[j] = v;
}

// Projective TSDF update of every voxel of the touched blocks, one warp per
// block (16 voxels per lane, no block-wide barriers).  Voxels that also need
// the class update (|psi| <= tau, pixel with a likelihood) are appended to a
// compact list (voxel, pixel), warp-aggregated so that the list keeps voxel
// order within each warp.  Each block also queues itself and its lower
// neighbours for re-meshing, and a block allocated in this frame links
// itself with its neighbours.
// Offsets o (bit o, e_o = (o & 1, o >> 1 & 1, o >> 2)) whose lower neighbour
// b - e_o reads a voxel of b: those with e_o inside the set Z of axes on which
// the voxel sits at local coordinate 0.  Byte Z of the table is that set of o.
constexpr unsigned long long remesh_table() {
    unsigned long long t = 0;
    for (int z = 0; z < 8; ++z)
        for (int o = 0; o < 8; ++o)
            if ((o & ~z) == 0) t |= 1ull << (8 * z + o);
    return t;
}
constexpr unsigned long long REMESH_TABLE = remesh_table();
static_assert(REMESH_TABLE == 0xFF5533110F050301ull, "re-mesh offset table");

__device__ __forceinline__ unsigned remesh_offsets(int vi) {
    const int z = ((vi & 7) == 0 ? 1 : 0) | (((vi >> 3) & 7) == 0 ? 2 : 0) | ((vi >> 6) == 0 ? 4 : 0);
    return (unsigned)(REMESH_TABLE >> (8 * z)) & 0xffu;
}

// Direction of voxel vi of block (bx, by, bz) from the sensor, in the LiDAR
// frame and voxel units (exact integer offset minus the fraction's high part,
// rotated by R^T).  (Every rounding is explicit here and in the update bodies
// below, so that each kernel that inlines them computes the same bits.)
__device__ __forceinline__ void tsdf_dir(const ScanConst &sc, int bx, int by, int bz, int vi, float &x0, float &x1,
                                         float &x2) {
    const int lx = vi & 7, ly = (vi >> 3) & 7, lz = vi >> 6;
    const float s0 = __fsub_rn((float)(8 * bx + lx - sc.k[0]), sc.fhi[0]);
    const float s1 = __fsub_rn((float)(8 * by + ly - sc.k[1]), sc.fhi[1]);
    const float s2 = __fsub_rn((float)(8 * bz + lz - sc.k[2]), sc.fhi[2]);
    x0 = __fmaf_rn(sc.Rt[2], s2, __fmaf_rn(sc.Rt[1], s1, __fmul_rn(sc.Rt[0], s0)));
    x1 = __fmaf_rn(sc.Rt[5], s2, __fmaf_rn(sc.Rt[4], s1, __fmul_rn(sc.Rt[3], s0)));
    x2 = __fmaf_rn(sc.Rt[8], s2, __fmaf_rn(sc.Rt[7], s1, __fmul_rn(sc.Rt[6], s0)));
}

// Pixel of a voxel at LiDAR-frame direction (x0, x1, x2) (Sec. III-C.1), or -1
// outside the image; also returns |x_l|^2 (rr2) and its reciprocal square
// root (irr) in voxel units.
__device__ __forceinline__ int tsdf_pixel(const ScanConst &sc, float x0, float x1, float x2, float &rr2, float &irr) {
    rr2 = __fmaf_rn(x2, x2, __fmaf_rn(x1, x1, __fmul_rn(x0, x0)));
    irr = 0.f;
    if (!(rr2 > 0.f)) return -1;
    irr = rsqrtf(rr2);
    // (polynomial atan2 / acos: their errors, < 5e-7 rad, stay far below the
    // 1e-3-pixel margin within which FP32 and FP64 pixel choices may differ)
    const float uc = __fmul_rn(__fsub_rn(PI_F, atan2_poly(x1, x0)), sc.inv_dphi);
    const float vc = __fmul_rn(__fsub_rn(acos_poly(fminf(fmaxf(__fmul_rn(x2, irr), -1.f), 1.f)), sc.theta0),
                               sc.inv_dtheta);
    int u = (int)floorf(__fadd_rn(uc, 0.5f));
    const int v = (int)floorf(__fadd_rn(vc, 0.5f));
    if (u >= sc.W) u -= sc.W;
    if (u < 0) u += sc.W;
    return (v >= 0 && v < sc.H) ? v * sc.W + u : -1;
}

// ---------------------------------------------------------------------------
// non-projective distance (Sec. III-C.2, Eq. distance)
// ---------------------------------------------------------------------------
template <bool F16>
__device__ __forceinline__ float load_g(const MapDev &md, long long j) {
    if (F16) return __half2float(md.g16[j]);
    return md.g32[j];
}
template <bool F16>
__device__ __forceinline__ void store_g(const MapDev &md, long long j, float v) {
    if (F16) md.g16[j] = __float2half_rn(v);
    else md.g32[j] = v;
}

// Back-projection of pixel (v, u) at its winner's range: r (from the winner
// point, as a float pair) times the pixel's ray (float-pair tables), each
// coordinate a float pair, so that neighbour differences keep full precision.
__device__ __forceinline__ void backproject(const ScanConst &sc, unsigned long long win, int v, int u, float qh[3],
                                            float ql[3]) {
    const unsigned idx = (unsigned)(win & 0xffffffffu);
    const float x = sc.pts[3 * (long long)idx], y = sc.pts[3 * (long long)idx + 1], z = sc.pts[3 * (long long)idx + 2];
    float a, ae, b, be, c, ce, rh, rl;
    two_prod(x, x, a, ae);
    two_prod(y, y, b, be);
    two_prod(z, z, c, ce);
    df_add(a, ae, b, be, rh, rl);
    df_add(rh, rl, c, ce, rh, rl);
    df_sqrt(rh, rl, rh, rl);
    const float4 rd = sc.row_dir[v], cd = sc.col_dir[u];
    float dh, dl;
    df_mul(rd.x, rd.y, cd.x, cd.y, dh, dl);     // sin(theta) cos(phi)
    df_mul(rh, rl, dh, dl, qh[0], ql[0]);
    df_mul(rd.x, rd.y, cd.z, cd.w, dh, dl);     // sin(theta) sin(phi)
    df_mul(rh, rl, dh, dl, qh[1], ql[1]);
    df_mul(rh, rl, rd.z, rd.w, qh[2], ql[2]);   // cos(theta)
}

// Normal image N at pixel p (Sec. III-C.2): with p_j the pixel's back-projected
// point and p_j1, p_j2 those of pixels (u, v - 1) and (u - 1, v) (columns wrap),
// N = (p_j1 - p_j) x (p_j2 - p_j) / |...|, turned toward the sensor and rotated
// into the world frame.  No normal (w = 0) on the top row, next to a pixel
// without a return, or for a vanishing cross product.
__device__ __forceinline__ void normal_item(const ScanConst &sc, const unsigned long long *__restrict__ win, int p) {
    const int v = p / sc.W, u = p - v * sc.W;
    float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
    if (v > 0) {
        const int u2 = u == 0 ? sc.W - 1 : u - 1;
        const unsigned long long w0 = win[p], w1 = win[p - sc.W], w2 = win[v * sc.W + u2];
        if (w0 != ~0ull && w1 != ~0ull && w2 != ~0ull) {
            float qh[3], ql[3], ah[3], al[3], bh[3], bl[3], a[3], b[3];
            backproject(sc, w0, v, u, qh, ql);
            backproject(sc, w1, v - 1, u, ah, al);
            backproject(sc, w2, v, u2, bh, bl);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                float dh, dl;
                df_add(ah[k], al[k], -qh[k], -ql[k], dh, dl);
                a[k] = __fadd_rn(dh, dl);
                df_add(bh[k], bl[k], -qh[k], -ql[k], dh, dl);
                b[k] = __fadd_rn(dh, dl);
            }
            float c0 = diff_of_products(a[1], b[2], a[2], b[1]);
            float c1 = diff_of_products(a[2], b[0], a[0], b[2]);
            float c2 = diff_of_products(a[0], b[1], a[1], b[0]);
            const float l2 = c0 * c0 + c1 * c1 + c2 * c2;
            if (l2 > 0.f) {
                float il = rsqrtf(l2);
                if (c0 * qh[0] + c1 * qh[1] + c2 * qh[2] > 0.f) il = -il;   // face the sensor
                c0 *= il;
                c1 *= il;
                c2 *= il;
                // world frame: R N, R = (R^T)^T
                out.x = sc.Rt[0] * c0 + sc.Rt[3] * c1 + sc.Rt[6] * c2;
                out.y = sc.Rt[1] * c0 + sc.Rt[4] * c1 + sc.Rt[7] * c2;
                out.z = sc.Rt[2] * c0 + sc.Rt[5] * c1 + sc.Rt[8] * c2;
                out.w = 1.f;
            }
        }
    }
    sc.nrm[p] = out;
}

// d_i of Eq. (distance) for projective distance psi, unit ray u from the voxel
// toward the sensor, gradient g (all zero: none yet) and the pixel's normal N
// (N.w = 0: none): d = psi (|cos theta| - sin theta tan(alpha / 2)), theta the
// angle between the ray and g, alpha the signed angle between g and N
// (positive when g is turned from N toward the ray, a convex surface), so that
// the distance is exact for a circular surface through the ray's end point;
// the flat form |cos theta| psi without a normal or where cos alpha <= 0.
// sin theta = |g x u|; sin alpha is g's component along the unit tangent
// (u - (u.N) N) / |u - (u.N) N|; tan(alpha / 2) = sin alpha / (1 + cos alpha).
__device__ __forceinline__ float nonproj_distance(float psi, float u0, float u1, float u2, float g0, float g1,
                                                  float g2, float4 N) {
    if (g0 == 0.f && g1 == 0.f && g2 == 0.f) return psi;
    const float ct = fabsf(g0 * u0 + g1 * u1 + g2 * u2);
    if (!(N.w > 0.f)) return ct * psi;
    const float ca = g0 * N.x + g1 * N.y + g2 * N.z;
    if (!(ca > 0.f)) return ct * psi;
    const float c0 = g1 * u2 - g2 * u1, c1 = g2 * u0 - g0 * u2, c2 = g0 * u1 - g1 * u0;
    const float st = sqrtf(c0 * c0 + c1 * c1 + c2 * c2);
    const float un = u0 * N.x + u1 * N.y + u2 * N.z;
    const float p0 = u0 - un * N.x, p1 = u1 - un * N.y, p2 = u2 - un * N.z;
    const float l2 = p0 * p0 + p1 * p1 + p2 * p2;
    if (!(l2 > 0.f)) return ct * psi;
    const float sa = (g0 * p0 + g1 * p1 + g2 * p2) * rsqrtf(l2);
    return psi * (ct - st * sa / (1.f + ca));
}

// A voxel of the truncation band awaiting the float-pair psi (see below).
struct BandEntry {
    int vi;          // voxel index within the block (bits 0-8); non-projective mode: the pixel in bits 9-31
    unsigned idx;    // the pixel's winner point
    float r;         // its range
    float D, W;      // the voxel's stored {D, W}
};

// Per-warp shared state of the TSDF pass over one block.
struct TsdfWarpSmem {
    int2 wbuf[BV];           // class-update entries {voxel, winner point} of the block
    BandEntry band[64];      // band voxels queued for the float-pair psi
};

// Projective psi and the running-average update of one voxel whose pixel's
// range-image winner is `win` (range bits << 32 | point index, ~0 when the
// pixel has no return) (Sec. III-C.2), given the voxel's stored {D, W} (read
// ahead by the caller).  Plain FP32 psi is within ~1e-5 m of the exact value;
// away from +-tau it decides the update exactly: beyond +tau (+1 mm) sdf = tau
// and w = 1, below -tau (-1 mm) nothing.  Returns true for a voxel of the band
// in between, which needs the float-pair psi (tsdf_band).
template <bool F16, bool DIST>
__device__ __forceinline__ bool tsdf_fast(const ScanConst &sc, const MapDev &md, long long vox, int vi, int p,
                                          unsigned long long win, float2 dw, float rr2, float irr, long long &n_upd,
                                          unsigned &remesh, bool &upd) {
    upd = false;
    if (p < 0 || win == ~0ull) return false;
    const float tau = sc.tau;
    const float r = __uint_as_float((unsigned)(win >> 32));
    const float psi = __fmaf_rn(-sc.nu, __fmul_rn(rr2, irr), r);
    if (psi < __fsub_rn(-tau, 1e-3f)) return false;
    // non-projective: d_i may fall inside the band whatever psi, every update takes the long path
    if (DIST || psi <= __fadd_rn(tau, 1e-3f)) return true;
    const float Wn = __fadd_rn(dw.y, 1.f);
    store_dw<F16>(md, vox, __fdividef(__fmaf_rn(dw.y, dw.x, tau), Wn), Wn);
    ++n_upd;
    upd = true;
    remesh |= remesh_offsets(vi);
    return false;
}

// The band voxel e of block (bx, by, bz) at pool slot `slot`: psi formed as
// (r^2 - rho^2) / (r + rho) with r^2 (from the winner point) and rho^2 as
// unevaluated float pairs, the linear weight and the running average.
// Returns true when the voxel also takes the class update.
template <bool F16, bool DIST>
__device__ __forceinline__ bool tsdf_band(const ScanConst &sc, const MapDev &md, int slot, int bx, int by, int bz,
                                          const BandEntry &e, long long &n_upd, unsigned &remesh, bool &upd) {
    upd = false;
    const float tau = sc.tau;
    const int vi = e.vi & (BV - 1), lx = vi & 7, ly = (vi >> 3) & 7, lz = vi >> 6;
    const float m0 = (float)(8 * bx + lx - sc.k[0]), m1 = (float)(8 * by + ly - sc.k[1]),
                m2 = (float)(8 * bz + lz - sc.k[2]);
    const float x = sc.pts[3 * (long long)e.idx], y = sc.pts[3 * (long long)e.idx + 1],
                z = sc.pts[3 * (long long)e.idx + 2];
    float a, ae, b, be, c, ce, rh, rl;
    two_prod(x, x, a, ae);
    two_prod(y, y, b, be);
    two_prod(z, z, c, ce);
    df_add(a, ae, b, be, rh, rl);
    df_add(rh, rl, c, ce, rh, rl);
    float e0, e1, e2, t0, t1, t2;
    two_sum(m0, -sc.fhi[0], t0, e0);
    two_sum(m1, -sc.fhi[1], t1, e1);
    two_sum(m2, -sc.fhi[2], t2, e2);
    e0 = __fsub_rn(e0, sc.flo[0]);
    e1 = __fsub_rn(e1, sc.flo[1]);
    e2 = __fsub_rn(e2, sc.flo[2]);
    // rho^2 in voxel units, then metres^2, as float pairs; psi = (r^2 - rho^2) / (r + rho)
    float qh, ql, mh, ml, dh, dl;
    two_prod(t0, t0, a, ae);
    two_prod(t1, t1, b, be);
    two_prod(t2, t2, c, ce);
    ae = __fmaf_rn(2.f * t0, e0, ae);
    be = __fmaf_rn(2.f * t1, e1, be);
    ce = __fmaf_rn(2.f * t2, e2, ce);
    df_add(a, ae, b, be, qh, ql);
    df_add(qh, ql, c, ce, qh, ql);
    df_mul(qh, ql, sc.nu2hi, sc.nu2lo, mh, ml);
    df_add(rh, rl, -mh, -ml, dh, dl);
    const float psi = __fdividef(__fadd_rn(dh, dl), __fmaf_rn(mh, rsqrtf(mh), e.r));
    const float w = sc.weight_mode == 0 ? fminf(fmaxf(__fmul_rn(__fadd_rn(psi, tau), sc.inv_2tau), 0.f), 1.f) : 1.f;
    if (!(psi >= -tau && w > 0.f)) return false;
    float sdf = fminf(psi, tau);
    if (DIST) {
        // gradient g_i: the weight-averaged normal of the pixels seen, renormalised
        const long long gj = (long long)slot * 3 * BV + vi;
        float g0 = load_g<F16>(md, gj), g1 = load_g<F16>(md, gj + BV), g2 = load_g<F16>(md, gj + 2 * BV);
        const float4 N = sc.nrm[(unsigned)e.vi >> 9];
        if (N.w > 0.f) {
            const float s0 = __fmaf_rn(e.W, g0, w * N.x), s1 = __fmaf_rn(e.W, g1, w * N.y),
                        s2 = __fmaf_rn(e.W, g2, w * N.z);
            const float l2 = s0 * s0 + s1 * s1 + s2 * s2;
            if (l2 > 0.f) {
                const float il = rsqrtf(l2);
                g0 = s0 * il;
                g1 = s1 * il;
                g2 = s2 * il;
            }
            store_g<F16>(md, gj, g0);
            store_g<F16>(md, gj + BV, g1);
            store_g<F16>(md, gj + 2 * BV, g2);
        }
        // unit ray from the voxel toward the sensor (world frame)
        const float o0 = t0 + e0, o1 = t1 + e1, o2 = t2 + e2;
        const float io = -rsqrtf(o0 * o0 + o1 * o1 + o2 * o2);
        const float d = nonproj_distance(psi, o0 * io, o1 * io, o2 * io, g0, g1, g2, N);
        // truncation Gamma(d, tau), both sides
        sdf = d >= 0.f ? fminf(d, tau) : fmaxf(d, -tau);
    }
    const float Wn = __fadd_rn(e.W, w);
    store_dw<F16>(md, (long long)slot * BV + vi, __fdividef(__fmaf_rn(e.W, e.D, __fmul_rn(w, sdf)), Wn), Wn);
    ++n_upd;
    upd = true;
    remesh |= remesh_offsets(vi);
    if (fabsf(psi) > tau) return false;
    // the winner carries a class likelihood: a probability row, or a label in range
    if (sc.has_probs) return true;
    const int l = sc.labels[e.idx];
    return l >= 0 && l < sc.C;
}

// Class-update entries {voxel, winner point} collect in the warp's shared
// buffer (one global append per block).
__device__ __forceinline__ void tsdf_list(bool sem, int vox, int idx, int2 *wbuf, int &wcount) {
    const unsigned mk = __ballot_sync(0xffffffffu, sem);
    if (sem) wbuf[wcount + __popc(mk & ((1u << (threadIdx.x & 31)) - 1u))] = make_int2(vox, idx);
    wcount += __popc(mk);
}

// Voxels [v0, v1) of one touched block (hash slot h; v1 - v0 a multiple of
// 64), processed by one warp.  Voxels outside the truncation band are
// finished on the spot; band voxels are queued, and the queue is worked off
// 32 at a time with every lane busy (they take the long float-pair path,
// which would otherwise idle the rest of the warp).  Every part of a new
// block links it with its neighbours (the same writes), so that the part's
// own re-mesh queueing below reads links it has set itself.
// With DBG the warp also records each voxel's pixel, update and class-update
// decisions in fd.dbg_vox (parity instrumentation; needs H * W <= 2^23).
template <bool F16, bool DIST = false, bool DBG = false>
__device__ __forceinline__ void tsdf_block_warp(const ScanConst &sc, const MapDev &md, const FrameDev &fd, int h,
                                                TsdfWarpSmem &T, long long &n_upd, int v0 = 0, int v1 = BV) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const HashSlot hrec = md.hs[h];
    const int slot = hrec.val;
    if (slot < 0) return;
    const uint64_t key = hrec.key;
    int bx, by, bz;
    unpack_block(key, bx, by, bz);
    // a block allocated in this frame links itself with its neighbours
    if (lane >= 8 && lane < 15 && md.slot_frame[slot] == sc.frame) link_block(md, key, slot, lane - 7);
    unsigned remesh = 0;
    int wcount = 0, qn = 0;
    auto enqueue = [&](bool band, int vi, unsigned long long win, float2 dw, int pix) {
        const unsigned mb = __ballot_sync(0xffffffffu, band);
        if (band) {
            BandEntry &e = T.band[qn + __popc(mb & lt)];
            e.vi = (DIST || DBG) ? (int)((unsigned)vi | ((unsigned)pix << 9)) : vi;
            e.idx = (unsigned)(win & 0xffffffffu);
            e.r = __uint_as_float((unsigned)(win >> 32));
            e.D = dw.x;
            e.W = dw.y;
        }
        qn += __popc(mb);
    };
    // work off the first n (<= 32) queued voxels, one per lane, and move the rest up
    auto drain = [&](int n) {
        __syncwarp();
        bool sem = false;
        int vox = 0, idx = 0;
        if (lane < n) {
            const BandEntry e = T.band[lane];
            bool upd;
            sem = tsdf_band<F16, DIST>(sc, md, slot, bx, by, bz, e, n_upd, remesh, upd);
            vox = slot * BV + (e.vi & (BV - 1));
            idx = (int)e.idx;
            if (DBG)
                fd.dbg_vox[vox] = ((int)((unsigned)e.vi >> 9) + 1) | (upd ? 1 << 28 : 0) | (sem ? 1 << 29 : 0);
        }
        const bool keep = lane < qn - n;
        BandEntry rest;
        if (keep) rest = T.band[n + lane];
        __syncwarp();
        if (keep) T.band[lane] = rest;
        qn -= n;
        tsdf_list(sem, vox, idx, T.wbuf, wcount);
    };
    // the lane's voxels are (x, y, z), (x, y + 4, z) with z one higher each step: their
    // directions follow from the first by adding R^T's images of one z step and four y steps
    float da0, da1, da2;
    tsdf_dir(sc, bx, by, bz, v0 + lane, da0, da1, da2);
    const float ey0 = __fmul_rn(4.f, sc.Rt[1]), ey1 = __fmul_rn(4.f, sc.Rt[4]), ey2 = __fmul_rn(4.f, sc.Rt[7]);
    // voxels vi and vi + 32 per step: both {D, W} reads are issued before the
    // projections and both pixel reads before either update, so that their
    // latencies overlap
    for (int vi = v0 + lane; vi < v1; vi += 64) {
        const long long va = (long long)slot * BV + vi, vb = va + 32;
        const float2 dwa = load_dw<F16>(md, va), dwb = load_dw<F16>(md, vb);
        float ra, ia, rb, ib;
        const int pa = tsdf_pixel(sc, da0, da1, da2, ra, ia);
        const int pb = tsdf_pixel(sc, __fadd_rn(da0, ey0), __fadd_rn(da1, ey1), __fadd_rn(da2, ey2), rb, ib);
        da0 = __fadd_rn(da0, sc.Rt[2]);
        da1 = __fadd_rn(da1, sc.Rt[5]);
        da2 = __fadd_rn(da2, sc.Rt[8]);
        const unsigned long long wa = fd.win[pa < 0 ? 0 : pa], wb = fd.win[pb < 0 ? 0 : pb];
        bool ua, ub;
        const bool ba = tsdf_fast<F16, DIST>(sc, md, va, vi, pa, wa, dwa, ra, ia, n_upd, remesh, ua);
        const bool bb = tsdf_fast<F16, DIST>(sc, md, vb, vi + 32, pb, wb, dwb, rb, ib, n_upd, remesh, ub);
        if (DBG) {
            if (!ba) fd.dbg_vox[va] = (pa + 1) | (ua ? 1 << 28 : 0);
            if (!bb) fd.dbg_vox[vb] = (pb + 1) | (ub ? 1 << 28 : 0);
        }
        enqueue(ba, vi, wa, dwa, pa);
        if (qn >= 32) drain(32);
        enqueue(bb, vi + 32, wb, dwb, pb);
        if (qn >= 32) drain(32);
    }
    if (qn > 0) drain(qn);
    __syncwarp();
    int2 *wbuf = T.wbuf;
    // one append of the block's class-update entries
    if (wcount) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(&fd.ctr[CT_SEM], (unsigned long long)wcount);
        base = __shfl_sync(0xffffffffu, base, 0);
        for (int i = lane; i < wcount; i += 32) {
            if (base + i < (unsigned long long)fd.sem_cap) fd.sem_list[base + i] = wbuf[i];
            else atomicOr(&md.st->err, ERR_LIST_FULL);
        }
    }
    // queue for re-meshing this block (if any voxel changed) and each lower
    // neighbour b - e whose cubes read a changed voxel of b, once per frame each
    // (the block's own links: set before, or just above by this warp)
    remesh = __reduce_or_sync(0xffffffffu, remesh);
    bool q = false;
    int hs = -1;
    if (lane < 8 && ((remesh >> lane) & 1u)) {
        hs = lane == 0 ? slot : md.nbr[slot * 16 + 8 + lane];
        q = hs >= 0 && atomicExch(&md.dstamp_slot[hs], sc.frame) != sc.frame;
    }
    const unsigned mq = __ballot_sync(0xffffffffu, q);
    if (mq) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(&fd.ctr[CT_DIRTY], (unsigned long long)__popc(mq));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (q) {
            const unsigned long long idx = base + __popc(mq & ((1u << lane) - 1u));
            if (idx < (unsigned long long)md.max_blocks) fd.dirty[idx] = hs;
            else atomicOr(&md.st->err, ERR_LIST_FULL);
        }
    }
    __syncwarp();
}

// Recursive Bayesian class update (Eq. bayesian_filter) of the listed voxels,
// one voxel per thread: logP_c += log L_c, renormalise by logsumexp, floor,
// and refresh the voxel's argmax label.  A voxel's classes form one record of
// whole 16-byte chunks (FP32: 20 floats, FP16: 24 halves for 20 classes),
// read and written with vector accesses, padding included.  The logarithms
// and exponentials use the MUFU approximations (base 2 in class_update,
// __logf / __expf in the runtime-class-count path): their error, ~1e-6 per
// term, is two orders below the class log-probability tolerance of the
// oracle comparison (1e-4 sqrt(K) + 1e-5 after K scans).
template <bool F16, int NC>
__device__ __forceinline__ void load_record(const MapDev &md, long long vox, float *av) {
    if (F16) {
        const uint4 *q = reinterpret_cast<const uint4 *>(md.lp16 + lp_index(md, vox, 0));
#pragma unroll
        for (int j = 0; j < NC / 8; ++j) {
            const uint4 u = q[j];
            const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&u.x));
            const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&u.y));
            const float2 c = __half22float2(*reinterpret_cast<const __half2 *>(&u.z));
            const float2 d = __half22float2(*reinterpret_cast<const __half2 *>(&u.w));
            av[8 * j] = a.x; av[8 * j + 1] = a.y; av[8 * j + 2] = b.x; av[8 * j + 3] = b.y;
            av[8 * j + 4] = c.x; av[8 * j + 5] = c.y; av[8 * j + 6] = d.x; av[8 * j + 7] = d.y;
        }
#pragma unroll
        for (int cc = (NC / 8) * 8; cc < NC; ++cc) av[cc] = __half2float(md.lp16[lp_index(md, vox, cc)]);
    } else {
        const float4 *q = reinterpret_cast<const float4 *>(md.lp32 + lp_index(md, vox, 0));
#pragma unroll
        for (int j = 0; j < NC / 4; ++j) {
            const float4 v = q[j];
            av[4 * j] = v.x; av[4 * j + 1] = v.y; av[4 * j + 2] = v.z; av[4 * j + 3] = v.w;
        }
#pragma unroll
        for (int cc = (NC / 4) * 4; cc < NC; ++cc) av[cc] = md.lp32[lp_index(md, vox, cc)];
    }
}

// Store a full padded record (NCP elements, zeros beyond NC) so that every
// written sector is written whole.
template <bool F16, int NC, int NCP>
__device__ __forceinline__ void store_record(const MapDev &md, long long vox, const float *nv) {
    if (F16) {
        uint4 *q = reinterpret_cast<uint4 *>(md.lp16 + lp_index(md, vox, 0));
#pragma unroll
        for (int j = 0; j < NCP / 8; ++j) {
            float f[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) f[k] = (8 * j + k < NC) ? nv[8 * j + k] : 0.f;
            uint4 u;
            __half2 h0 = __floats2half2_rn(f[0], f[1]), h1 = __floats2half2_rn(f[2], f[3]);
            __half2 h2 = __floats2half2_rn(f[4], f[5]), h3 = __floats2half2_rn(f[6], f[7]);
            u.x = *reinterpret_cast<unsigned *>(&h0);
            u.y = *reinterpret_cast<unsigned *>(&h1);
            u.z = *reinterpret_cast<unsigned *>(&h2);
            u.w = *reinterpret_cast<unsigned *>(&h3);
            q[j] = u;
        }
    } else {
        float4 *q = reinterpret_cast<float4 *>(md.lp32 + lp_index(md, vox, 0));
#pragma unroll
        for (int j = 0; j < NCP / 4; ++j) {
            float f[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) f[k] = (4 * j + k < NC) ? nv[4 * j + k] : 0.f;
            q[j] = make_float4(f[0], f[1], f[2], f[3]);
        }
    }
}

// The Bayesian class update of one voxel (Eq. bayesian_filter) for a
// compile-time class count NC: av holds the voxel's stored log-probabilities
// (as floats) and receives the new ones (floored); q is the winner point's
// probability row (16-byte aligned when sc.probs_vec4), or null for the hard
// label l.  Returns the most probable class of the values as they will be
// stored (lowest class on ties).  Every path that updates classes (per-thread,
// bulk-staged, batched) runs this same body, so all compute the same bits.
// Base-2 logarithm and exponential by the MUFU approximations (PTX lg2.approx,
// ex2.approx): the class update works in natural-log units and converts with
// one multiply-add, ln x = ln 2 * log2 x and e^(a - m) = 2^(a log2 e - m log2 e).
__device__ __forceinline__ float lg2_mufu(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float ex2_mufu(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
constexpr float LN2_F = 0.6931471805599453f, LOG2E_F = 1.4426950408889634f;

template <bool F16, int NC, bool QLOG2 = false>
__device__ __forceinline__ int class_update(const ScanConst &sc, float *av, const float *q, int l) {
    if (QLOG2 && q) {
        // q already holds log2 max(q_c, lik_floor) (16-byte aligned)
#pragma unroll
        for (int cc = 0; cc < NC; cc += 4) {
            const float4 v = *reinterpret_cast<const float4 *>(q + cc);
            av[cc] = __fmaf_rn(v.x, LN2_F, av[cc]);
            av[cc + 1] = __fmaf_rn(v.y, LN2_F, av[cc + 1]);
            av[cc + 2] = __fmaf_rn(v.z, LN2_F, av[cc + 2]);
            av[cc + 3] = __fmaf_rn(v.w, LN2_F, av[cc + 3]);
        }
    } else if (q) {
        if (NC % 4 == 0 && sc.probs_vec4) {
#pragma unroll
            for (int cc = 0; cc < NC; cc += 4) {
                const float4 v = *reinterpret_cast<const float4 *>(q + cc);
                av[cc] = __fmaf_rn(lg2_mufu(fmaxf(v.x, sc.lik_floor)), LN2_F, av[cc]);
                av[cc + 1] = __fmaf_rn(lg2_mufu(fmaxf(v.y, sc.lik_floor)), LN2_F, av[cc + 1]);
                av[cc + 2] = __fmaf_rn(lg2_mufu(fmaxf(v.z, sc.lik_floor)), LN2_F, av[cc + 2]);
                av[cc + 3] = __fmaf_rn(lg2_mufu(fmaxf(v.w, sc.lik_floor)), LN2_F, av[cc + 3]);
            }
        } else {
#pragma unroll
            for (int cc = 0; cc < NC; ++cc) av[cc] = __fmaf_rn(lg2_mufu(fmaxf(q[cc], sc.lik_floor)), LN2_F, av[cc]);
        }
    } else {
#pragma unroll
        for (int cc = 0; cc < NC; ++cc) av[cc] = __fadd_rn(av[cc], cc == l ? sc.log_phit : sc.log_pmiss);
    }
    float m = -INFINITY;
#pragma unroll
    for (int cc = 0; cc < NC; ++cc) m = fmaxf(m, av[cc]);
    float ssum = 0.f;
    const float mb = __fmul_rn(m, LOG2E_F);
#pragma unroll
    for (int cc = 0; cc < NC; ++cc) ssum = __fadd_rn(ssum, ex2_mufu(__fmaf_rn(av[cc], LOG2E_F, -mb)));
    const float lse = __fmaf_rn(lg2_mufu(ssum), LN2_F, m);
    int best = 0;
    float bv = -INFINITY;
#pragma unroll
    for (int cc = 0; cc < NC; ++cc) {
        av[cc] = fmaxf(__fsub_rn(av[cc], lse), sc.logp_floor);
        const float stored = F16 ? __half2float(__float2half_rn(av[cc])) : av[cc];
        if (stored > bv) {
            bv = stored;
            best = cc;
        }
    }
    return best;
}

template <bool F16, int NC>
__device__ __forceinline__ void semantic_item(const ScanConst &sc, const MapDev &md, const FrameDev &fd,
                                              unsigned long long e) {
    constexpr int MAXC_RT = 64;
    // padded record length for the compile-time class count (16-byte chunks)
    constexpr int NCP = NC > 0 ? (F16 ? ((NC + 7) / 8) * 8 : ((NC + 3) / 4) * 4) : 1;
    const int C = NC > 0 ? NC : sc.C;
    const int2 ent = fd.sem_list[e];
    const long long vox = ent.x;
    const long long idx = ent.y;   // the pixel's winner point: log P(O = l | I_k) from its input
    if (NC > 0) {
        constexpr int N1 = NC > 0 ? NC : 1;
        float av[N1];
        load_record<F16, N1>(md, vox, av);
        const int best = class_update<F16, N1>(sc, av, sc.has_probs ? sc.probs + idx * C : nullptr,
                                               sc.has_probs ? 0 : sc.labels[idx]);
        store_record<F16, N1, NCP>(md, vox, av);
        md.label[vox] = (uint8_t)best;
    } else {
        float av[MAXC_RT];
        float m = -INFINITY;
        const float *q = sc.probs + idx * C;
        const int l = sc.has_probs ? -1 : sc.labels[idx];
        for (int cc = 0; cc < C; ++cc) {
            const float lik = sc.has_probs ? __logf(fmaxf(q[cc], sc.lik_floor)) : (cc == l ? sc.log_phit : sc.log_pmiss);
            av[cc] = __fadd_rn(load_lp<F16>(md, lp_index(md, vox, cc)), lik);
            m = fmaxf(m, av[cc]);
        }
        float ssum = 0.f;
        for (int cc = 0; cc < C; ++cc) ssum = __fadd_rn(ssum, __expf(__fsub_rn(av[cc], m)));
        const float lse = __fadd_rn(m, __logf(ssum));
        int best = 0;
        float bv = -INFINITY;
        for (int cc = 0; cc < C; ++cc) {
            const float nv = fmaxf(__fsub_rn(av[cc], lse), sc.logp_floor);
            store_lp<F16>(md, lp_index(md, vox, cc), nv);
            const float stored = F16 ? __half2float(__float2half_rn(nv)) : nv;
            if (stored > bv) {
                bv = stored;
                best = cc;
            }
        }
        md.label[vox] = (uint8_t)best;
    }
}

// --- the class update staged by a warp through shared memory ------------------
// A lane's own 80-byte (FP32) or 48-byte (FP16) class record, loaded with one
// 16-byte access per lane and instruction, touches a different cache line in
// every lane, and the L1's tag lookups then bound the update; here the warp's
// 32 lanes copy consecutive 16-byte chunks of the warp's 32 records (about five
// records per instruction) into shared memory, update them there (class_update,
// the same body as every other path) and write them back the same way.
constexpr int SEM_NC = 20;    // the class count of the staged path
template <bool F16>
struct SemStage {
    static constexpr int RC = F16 ? 3 : 5;    // 16-byte chunks per record (24 halves / 20 floats)
    static constexpr int RB = 16 * RC;
};
__device__ __forceinline__ void cp_async16(void *dst_smem, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst_smem)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// One warp updates the voxels of its active lanes (act): ent = {pool voxel,
// winner point} of the lane's list entry in map md (the lanes' maps may
// differ), R = 32 x RB bytes of the warp's shared memory, qrow = the lane's
// probability row (shared or global memory, 16-byte aligned), or null for a
// hard label.  Any cp.async copies the warp issued before are waited for too.
// With QLOG2 the warp's staged probability rows, qlog[0, nlog), are turned into
// log2 max(q, lik_floor) once the copies have landed (each row once, however
// many lanes share it), and qrow points at the lane's row there.
template <bool F16, bool QLOG2 = false>
__device__ __forceinline__ void class_update_warp(const ScanConst &sc, const MapDev &md, bool act, int2 ent,
                                                  unsigned char *R, const float *qrow, float *qlog = nullptr,
                                                  int nlog = 0) {
    using S = SemStage<F16>;
    const int lane = threadIdx.x & 31;
    unsigned char *mine = nullptr;
    if (act)
        mine = F16 ? reinterpret_cast<unsigned char *>(md.lp16 + lp_index(md, ent.x, 0))
                   : reinterpret_cast<unsigned char *>(md.lp32 + lp_index(md, ent.x, 0));
    const unsigned long long mp = reinterpret_cast<unsigned long long>(mine);
    // chunk k of the warp's records: record k / RC, 16-byte chunk k % RC
#pragma unroll
    for (int j = 0; j < S::RC; ++j) {
        const int k = 32 * j + lane, r = k / S::RC, c = k - r * S::RC;
        const unsigned long long src = __shfl_sync(0xffffffffu, mp, r);
        if (src) cp_async16(R + r * S::RB + 16 * c, reinterpret_cast<const unsigned char *>(src) + 16 * c);
    }
    cp_async_wait_all();
    __syncwarp();
    if (QLOG2 && nlog > 0) {
        for (int t = lane; t < nlog; t += 32) qlog[t] = lg2_mufu(fmaxf(qlog[t], sc.lik_floor));
        __syncwarp();
    }
    if (act) {
        float av[SEM_NC];
        unsigned char *rr = R + lane * S::RB;
        if (F16) {
            const uint4 *q = reinterpret_cast<const uint4 *>(rr);
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const uint4 u = q[j];
                const float2 f0 = __half22float2(*reinterpret_cast<const __half2 *>(&u.x));
                const float2 f1 = __half22float2(*reinterpret_cast<const __half2 *>(&u.y));
                const float2 f2 = __half22float2(*reinterpret_cast<const __half2 *>(&u.z));
                const float2 f3 = __half22float2(*reinterpret_cast<const __half2 *>(&u.w));
                const float g[8] = {f0.x, f0.y, f1.x, f1.y, f2.x, f2.y, f3.x, f3.y};
#pragma unroll
                for (int k = 0; k < 8; ++k)
                    if (8 * j + k < SEM_NC) av[8 * j + k] = g[k];
            }
        } else {
            const float4 *q = reinterpret_cast<const float4 *>(rr);
#pragma unroll
            for (int j = 0; j < SEM_NC / 4; ++j) {
                const float4 v = q[j];
                av[4 * j] = v.x;
                av[4 * j + 1] = v.y;
                av[4 * j + 2] = v.z;
                av[4 * j + 3] = v.w;
            }
        }
        const int best = class_update<F16, SEM_NC, QLOG2>(sc, av, qrow, qrow ? 0 : sc.labels[ent.y]);
        // the new record in place, padding zero
        if (F16) {
            uint4 *q = reinterpret_cast<uint4 *>(rr);
#pragma unroll
            for (int j = 0; j < S::RC; ++j) {
                float f[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) f[k] = (8 * j + k < SEM_NC) ? av[8 * j + k] : 0.f;
                __half2 h0 = __floats2half2_rn(f[0], f[1]), h1 = __floats2half2_rn(f[2], f[3]);
                __half2 h2 = __floats2half2_rn(f[4], f[5]), h3 = __floats2half2_rn(f[6], f[7]);
                uint4 u;
                u.x = *reinterpret_cast<unsigned *>(&h0);
                u.y = *reinterpret_cast<unsigned *>(&h1);
                u.z = *reinterpret_cast<unsigned *>(&h2);
                u.w = *reinterpret_cast<unsigned *>(&h3);
                q[j] = u;
            }
        } else {
            float4 *q = reinterpret_cast<float4 *>(rr);
#pragma unroll
            for (int j = 0; j < S::RC; ++j) {
                float f[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) f[k] = (4 * j + k < SEM_NC) ? av[4 * j + k] : 0.f;
                q[j] = make_float4(f[0], f[1], f[2], f[3]);
            }
        }
        md.label[ent.x] = (uint8_t)best;
    }
    __syncwarp();
    // the records back, chunk by chunk as they came
#pragma unroll
    for (int j = 0; j < S::RC; ++j) {
        const int k = 32 * j + lane, r = k / S::RC, c = k - r * S::RC;
        const unsigned long long dst = __shfl_sync(0xffffffffu, mp, r);
        if (dst)
            *reinterpret_cast<uint4 *>(reinterpret_cast<unsigned char *>(dst) + 16 * c) =
                *reinterpret_cast<const uint4 *>(R + r * S::RB + 16 * c);
    }
    __syncwarp();
}

constexpr int MESH_WARPS = 8;   // warps (blocks in flight) per CTA

// Per-warp staging of one block: the 9^3 region (block + upper faces) and
// the bit masks the extraction works on.  Voxel rows run along x and are
// indexed rw = y + 9 z; cube rows are indexed cy + 8 cz.
struct MeshWarpSmem {
    float D[729];
    uint32_t rowm[81];    // per voxel row: bits 0..8 observed (x = 0..8), bits 16..24 D < 0
    uint32_t ew[81];      // per voxel row: lattice edges that carry a vertex, from voxel (x, y, z):
                          // bits 0..7 +x edges (x = 0..7), 8..16 +y edges, 17..25 +z edges (x = 0..8)
    uint16_t woff[82];    // number of the first vertex of each row
    uint8_t okc[64];      // per cube row: cubes whose eight corners are observed (bit = ax)
    int nb[8];            // slots of this block (0) and its 7 upper neighbours, -1 if none
    union {
        uint4 F4[81];     // while staging: per voxel row, 16 bytes, byte x: bit 0 observed (W > 0), bit 1 D < 0
        uint16_t mc[512]; // then: the cubes that emit triangles (ax + 8 (ay + 8 az)), in order
    } u;
};

struct MeshCtaSmem {
    int8_t tri[256 * MC_MAXTRI * 3];
    uint8_t ntri[256];
    MeshWarpSmem w[MESH_WARPS];
};

// Bit position of the k-th (from 0) set bit of w; requires k < popc(w).
__device__ __forceinline__ int nth_set_bit(uint32_t w, int k) {
    int pos = 0, c = __popc(w & 0xffffu);
    if (k >= c) { k -= c; w >>= 16; pos += 16; }
    c = __popc(w & 0xffu);
    if (k >= c) { k -= c; w >>= 8; pos += 8; }
    c = __popc(w & 0xfu);
    if (k >= c) { k -= c; w >>= 4; pos += 4; }
    c = __popc(w & 0x3u);
    if (k >= c) { k -= c; w >>= 2; pos += 2; }
    return pos + (k >= (int)(w & 1u) ? 1 : 0);
}

// Case of cube a = ax + 8 (ay + 8 az): bit cx + 2 cy + 4 cz set when corner
// (ax + cx, ay + cy, az + cz) has D < 0.
__device__ __forceinline__ int cube_case(const uint32_t *rowm, int a) {
    const int ax = a & 7, r = ((a >> 3) & 7) + 9 * (a >> 6), sh = 16 + ax;
    return (int)(((rowm[r] >> sh) & 3u) | (((rowm[r + 1] >> sh) & 3u) << 2) | (((rowm[r + 9] >> sh) & 3u) << 4) |
                 (((rowm[r + 10] >> sh) & 3u) << 6));
}

// Cube edge ce (axis ce >> 2, offsets ce & 1 and (ce >> 1) & 1 along the next
// two axes, cyclically) lies on voxel row (ay + dy) + 9 (az + dz) of its cube
// and has bit b + ax of that row's edge mask: an x edge (dy, dz) = (o1, o2),
// b = 0; a y edge (0, o1), b = 8 + o2; a z edge (o2, 0), b = 17 + o1.  The
// 12 edges' (dy + 9 dz, b) in 9-bit fields, six to a word, so that a lookup
// is a shift and a mask rather than a branch on the axis (the lanes of a warp
// look up different edges).
constexpr unsigned long long cube_edge_table(int half) {
    unsigned long long t = 0;
    for (int k = 0; k < 6; ++k) {
        const int ce = 6 * half + k, axis = ce >> 2, o1 = ce & 1, o2 = (ce >> 1) & 1;
        const int dy = axis == 0 ? o1 : (axis == 2 ? o2 : 0);
        const int dz = axis == 0 ? o2 : (axis == 1 ? o1 : 0);
        const int b = axis == 0 ? 0 : (axis == 1 ? 8 + o2 : 17 + o1);
        t |= (unsigned long long)((dy + 9 * dz) | (b << 4)) << (9 * k);
    }
    return t;
}
constexpr unsigned long long CUBE_EDGE_LO = cube_edge_table(0), CUBE_EDGE_HI = cube_edge_table(1);
static_assert(CUBE_EDGE_LO == 0x11280050240200ull && CUBE_EDGE_HI == 0x24311904413290ull, "cube edge table");

// Vertex number of cube edge ce of the cube anchored at (ax, ay, az).
__device__ __forceinline__ int cube_edge_vertex(const MeshWarpSmem &W, int ce, int ax, int ay, int az) {
    const bool hi = ce >= 6;
    const int f = (int)(((hi ? CUBE_EDGE_HI : CUBE_EDGE_LO) >> (9 * (hi ? ce - 6 : ce))) & 0x1ffu);
    const int rw = ay + 9 * az + (f & 15), bit = ax + (f >> 4);
    return W.woff[rw] + __popc(W.ew[rw] & ((1u << bit) - 1u));
}

// One block to re-mesh (pool slot `slot`), processed by one warp with its
// staging area W; `part` selects the mesh-arena partition.
//
// A cube emits triangles when its eight corners are observed and not all on
// one side of the surface; a lattice edge carries a vertex when its two
// voxels are observed with opposite signs and one of its (up to four) cubes
// has all corners observed.  Both are evaluated for whole rows at once with
// bit operations on the row masks; vertices and emitting cubes are then
// numbered by prefix counts and emitted one per lane.
__device__ __forceinline__ void mesh_block_warp(const MapDev &md, const FrameDev &fd, const int8_t *__restrict__ tri,
                                                const uint8_t *__restrict__ ntri,
                                                MeshWarpSmem &W, int slot, int part, long long &n_v, long long &n_t) {
    const int lane = threadIdx.x & 31;
    const bool f32 = md.storage == 0;
    int bx, by, bz;
    unpack_block(md.slot_key[slot], bx, by, bz);
    // slots of the 7 upper neighbours, from the per-slot links
    if (lane < 8) W.nb[lane] = lane == 0 ? slot : md.nbr[slot * 16 + lane];
    int seen = 0;   // bit 0: an observed voxel with D < 0, bit 1: one with D >= 0
    uint8_t *F = reinterpret_cast<uint8_t *>(W.u.F4);
    // region voxel (x, y, z): D at x + 9 (y + 9 z), flags at x + 16 (y + 9 z)
    auto put = [&](int r, int fi, float2 dw) {
        const int f = (dw.y > 0.f ? 1 : 0) | (dw.x < 0.f ? 2 : 0);
        W.D[r] = dw.x;
        F[fi] = (uint8_t)f;
        if (f & 1) seen |= (f & 2) ? 1 : 2;
    };
    // The region's {D, W} in three rounds of reads, each round's reads issued
    // before any of its stores to shared memory (a read placed after such a
    // store would wait for it, one memory round trip per read): the block's
    // own 512 voxels in two rounds of four reads per lane (two neighbours
    // along x per read, 16 bytes FP32, 8 FP16), then the 217 voxels of the
    // upper neighbours' faces.
    const long long pair0 = (long long)slot * (BV / 2);
#pragma unroll
    for (int rnd = 0; rnd < 2; ++rnd) {
        uint4 q[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const long long pi = pair0 + lane + 32 * (4 * rnd + k);
            if (f32) {
                q[k] = reinterpret_cast<const uint4 *>(md.dw32)[pi];
            } else {
                const uint2 u = reinterpret_cast<const uint2 *>(md.dw16)[pi];
                q[k] = make_uint4(u.x, u.y, 0u, 0u);
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int v = 2 * (lane + 32 * (4 * rnd + k)), row = v >> 3, x = v & 7;   // row = y + 8 z
            const int yz9 = (row & 7) + 9 * (row >> 3);                                // y + 9 z
            float2 a, b;
            if (f32) {
                a = make_float2(__uint_as_float(q[k].x), __uint_as_float(q[k].y));
                b = make_float2(__uint_as_float(q[k].z), __uint_as_float(q[k].w));
            } else {
                a = __half22float2(*reinterpret_cast<const __half2 *>(&q[k].x));
                b = __half22float2(*reinterpret_cast<const __half2 *>(&q[k].y));
            }
            put(x + 9 * yz9, x + 16 * yz9, a);
            put(x + 1 + 9 * yz9, x + 1 + 16 * yz9, b);
        }
    }
    __syncwarp();
    auto nb_dw = [&](int s, int local) -> float2 {
        if (s < 0) return make_float2(0.f, 0.f);
        const long long vox = (long long)s * BV + local;
        return f32 ? md.dw32[vox] : __half22float2(md.dw16[vox]);
    };
    // faces: x = 8 (rows y + 9 z = j < 81: local x = 0 of the +x neighbours),
    // y = 8 (j = x + 8 z < 72: local y = 0 of the +y neighbours), z = 8
    // (j = x + 8 y < 64: local z = 0 of the +z neighbour)
    float2 fx[3], fy[3], fz[2];
#pragma unroll
    for (int t = 0; t < 3; ++t) {
        const int j = lane + 32 * t;
        fx[t] = fy[t] = make_float2(0.f, 0.f);
        if (j < 81) {
            const int y = j % 9, z = j / 9;
            fx[t] = nb_dw(W.nb[1 | ((y >> 3) << 1) | ((z >> 3) << 2)], 8 * (y & 7) + 64 * (z & 7));
        }
        if (j < 72) fy[t] = nb_dw(W.nb[2 | ((j >> 6) << 2)], (j & 7) + 64 * ((j >> 3) & 7));
        if (t < 2) fz[t] = nb_dw(W.nb[4], j);
    }
#pragma unroll
    for (int t = 0; t < 3; ++t) {
        const int j = lane + 32 * t;
        if (j < 81) put(8 + 9 * j, 8 + 16 * j, fx[t]);
        if (j < 72) {
            const int yz9 = 8 + 9 * (j >> 3);
            put((j & 7) + 9 * yz9, (j & 7) + 16 * yz9, fy[t]);
        }
        if (t < 2) {
            const int yz9 = (j >> 3) + 72;
            put((j & 7) + 9 * yz9, (j & 7) + 16 * yz9, fz[t]);
        }
    }
    const bool any_neg = __any_sync(0xffffffffu, seen & 1), any_pos = __any_sync(0xffffffffu, seen & 2);
    int tot_m = 0;
    if (any_neg && any_pos) {
        __syncwarp();
        // row masks of the 81 voxel rows
        // (bit 0, resp. 1, of four bytes gathered into 4 bits by one multiply: the
        // products b_i 2^(8i) 2^(24-7k) land on bit 24 + i for i = k, below bit 20
        // for i < k without overlapping, and beyond bit 31 for i > k)
        for (int rw = lane; rw < 81; rw += 32) {
            const uint4 q = W.u.F4[rw];
            const uint32_t ob = (((q.x & 0x01010101u) * 0x01020408u) >> 24) |
                                ((((q.y & 0x01010101u) * 0x01020408u) >> 24) << 4) | ((q.z & 1u) << 8);
            const uint32_t ng = ((((q.x >> 1) & 0x01010101u) * 0x01020408u) >> 24) |
                                (((((q.y >> 1) & 0x01010101u) * 0x01020408u) >> 24) << 4) | (((q.z >> 1) & 1u) << 8);
            W.rowm[rw] = ob | (ng << 16);
        }
        __syncwarp();
        // cube rows 2 lane and 2 lane + 1: observed cubes, and the emitting ones among them
        uint32_t mixl = 0;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int cr = 2 * lane + q, r = (cr & 7) + 9 * (cr >> 3);
            const uint32_t m00 = W.rowm[r], m10 = W.rowm[r + 1], m01 = W.rowm[r + 9], m11 = W.rowm[r + 10];
            const uint32_t o = m00 & m10 & m01 & m11;
            const uint32_t ok = o & (o >> 1) & 0xffu;
            const uint32_t na = o >> 16, nn = (m00 | m10 | m01 | m11) >> 16;
            W.okc[cr] = (uint8_t)ok;
            mixl |= (ok & (nn | (nn >> 1)) & ~(na & (na >> 1)) & 0xffu) << (8 * q);
        }
        const int moff = warp_exclusive_scan(__popc(mixl), tot_m);
        // the staging flags are dead: list the emitting cubes in their place (cube 16 lane + b)
        for (int o = moff; mixl; ++o) {
            const int b = __ffs(mixl) - 1;
            mixl &= mixl - 1u;
            W.u.mc[o] = (uint16_t)(16 * lane + b);
        }
    }
    if (tot_m == 0) {
        // no cube can emit: drop the old segment
        if (lane == 0) {
            const int4 old = md.seg[slot];
            if (old.y | old.w) md.seg[slot] = make_int4(0, 0, 0, 0);
        }
        __syncwarp();
        return;
    }
    __syncwarp();
    // lattice edges with a vertex, row by row
    for (int rw = lane; rw < 81; rw += 32) {
        const int y = rw % 9, z = rw / 9;
        const uint32_t m = W.rowm[rw];
        const uint32_t obs = m & 0x1ffu, neg = (m >> 16) & 0x1ffu;
        // observed cubes of the cube rows (y - 1 | y, z - 1 | z) around this voxel row
        const uint32_t c00 = (y > 0 && z > 0) ? W.okc[(y - 1) + 8 * (z - 1)] : 0u;
        const uint32_t c10 = (y < 8 && z > 0) ? W.okc[y + 8 * (z - 1)] : 0u;
        const uint32_t c01 = (y > 0 && z < 8) ? W.okc[(y - 1) + 8 * z] : 0u;
        const uint32_t c11 = (y < 8 && z < 8) ? W.okc[y + 8 * z] : 0u;
        uint32_t e = (neg ^ (neg >> 1)) & obs & (obs >> 1) & (c00 | c10 | c01 | c11) & 0xffu;
        if (y < 8) {
            const uint32_t m2 = W.rowm[rw + 1], c = c10 | c11;
            e |= ((neg ^ (m2 >> 16)) & obs & m2 & (c | (c << 1)) & 0x1ffu) << 8;
        }
        if (z < 8) {
            const uint32_t m3 = W.rowm[rw + 9], c = c01 | c11;
            e |= ((neg ^ (m3 >> 16)) & obs & m3 & (c | (c << 1)) & 0x1ffu) << 17;
        }
        W.ew[rw] = e;
    }
    __syncwarp();
    // vertex numbering: rows 3 lane .. 3 lane + 2
    int c0 = 0, c1 = 0, c2 = 0;
    if (lane < 27) {
        c0 = __popc(W.ew[3 * lane]);
        c1 = __popc(W.ew[3 * lane + 1]);
        c2 = __popc(W.ew[3 * lane + 2]);
    }
    int tot_v;
    const int voff = warp_exclusive_scan(c0 + c1 + c2, tot_v);
    if (lane < 27) {
        W.woff[3 * lane] = (uint16_t)voff;
        W.woff[3 * lane + 1] = (uint16_t)(voff + c0);
        W.woff[3 * lane + 2] = (uint16_t)(voff + c0 + c1);
    }
    // triangle count of the emitting cubes
    int cnt_t = 0;
    for (int i = lane; i < tot_m; i += 32) cnt_t += ntri[cube_case(W.rowm, W.u.mc[i])];
    const int tot_t = (int)__reduce_add_sync(0xffffffffu, (unsigned)cnt_t);
    // reserve arena space in this warp's partition (two lanes, two cursors)
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
        // vertices, one per lane
        for (int vid = lane; vid < tot_v; vid += 32) {
            int rw = 0;
#pragma unroll
            for (int st = 64; st > 0; st >>= 1)
                if (rw + st <= 80 && W.woff[rw + st] <= vid) rw += st;
            const int q = nth_set_bit(W.ew[rw], vid - W.woff[rw]);
            const int axis = q < 8 ? 0 : (q < 17 ? 1 : 2);
            const int x = q - (axis == 0 ? 0 : (axis == 1 ? 8 : 17)), y = rw % 9, z = rw / 9;
            const int r0 = x + 9 * rw;
            const int r1 = r0 + (axis == 0 ? 1 : (axis == 1 ? 9 : 81));
            const float D0 = W.D[r0], D1 = W.D[r1];
            const float t = D0 / (D0 - D1);
            const int gx = 8 * bx + x, gy = 8 * by + y, gz = 8 * bz + z;
            float px = md.nu * (float)gx, py = md.nu * (float)gy, pz = md.nu * (float)gz;
            if (axis == 0) px = md.nu * ((float)gx + t);
            else if (axis == 1) py = md.nu * ((float)gy + t);
            else pz = md.nu * ((float)gz + t);
            // the endpoint nearer the surface (lower endpoint on ties) gives the
            // vertex its class: its pool voxel index is stored, and the label
            // (and colour) are read when the mesh is extracted.  That is the label
            // after this scan's class update: a voxel's label changes only in a
            // scan that also re-meshes every block reading it.
            const int re = fabsf(D1) < fabsf(D0) ? r1 : r0;
            const int ex = re % 9, ey = (re / 9) % 9, ez = re / 81;
            const int es = W.nb[(ex >> 3) | ((ey >> 3) << 1) | ((ez >> 3) << 2)];
            const unsigned packed =
                es >= 0 ? (unsigned)es * BV + (ex & 7) + 8 * (ey & 7) + 64 * (ez & 7) : 0xffffffffu;
            md.av[vo + vid] = make_float4(px, py, pz, __uint_as_float(packed));
            md.ak[vo + vid] = edge_key(gx, gy, gz, axis);
        }
        // triangles: one emitting cube per lane, in list order
        long long tb = to;
        for (int i0 = 0; i0 < tot_m; i0 += 32) {
            const int i = i0 + lane;
            int a = 0, cs = 0, nt = 0;
            if (i < tot_m) {
                a = W.u.mc[i];
                cs = cube_case(W.rowm, a);
                nt = ntri[cs];
            }
            int round_t;
            const int off = warp_exclusive_scan(nt, round_t);
            const int ax = a & 7, ay = (a >> 3) & 7, az = a >> 6;
            for (int j = 0; j < nt; ++j) {
                const int8_t *tj = tri + (cs * MC_MAXTRI + j) * 3;
                const int v0 = cube_edge_vertex(W, tj[0], ax, ay, az);
                const int v1 = cube_edge_vertex(W, tj[1], ax, ay, az);
                const int v2 = cube_edge_vertex(W, tj[2], ax, ay, az);
                md.at[tb + off + j] = make_ushort4((unsigned short)v0, (unsigned short)v1, (unsigned short)v2,
                                                   (unsigned short)a);
            }
            tb += round_t;
        }
    }
    __syncwarp();
}

}  // namespace stsdf
