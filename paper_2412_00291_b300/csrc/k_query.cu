// Differentiable trilinear SDF queries and scan-to-map Gauss-Newton.
//
// D(x) interpolates the 8 voxel centres nu * v around x (v0 = floor(x / nu),
// f = x / nu - v0, weights prod_k (c_k f_k + (1 - c_k)(1 - f_k))); the query
// is valid only when all 8 voxels are allocated and observed (W > 0).
// dD/dx_k = (1/nu) sum_c (d weight / d f_k) D_c.  For a left perturbation
// T(xi) = Exp(xi) T of the pose, dx/dxi = [I | -[x]x], so the pose gradient
// of a loss L is (sum_i dL/dx_i, sum_i x_i x dL/dx_i).
#include "kernels.h"

namespace stsdf {

// g: position in voxel units relative to integer offset k (g_true = k + g).
// The 8 corners lie in at most 2 blocks per axis.  The slots of those blocks
// are found with every first hash probe in flight at once (a longer probe
// sequence only for a key not at its home slot), then all 8 voxels are read
// at once: three dependent memory steps per query.
__device__ __forceinline__ bool trilinear(const MapDev &md, const int k[3], const float g[3], float &D,
                                          float dg[3]) {
    int v0[3];
    float f[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float fl = floorf(g[a]);
        // outside the map's coordinate range (its keys would alias), or not a number: invalid
        const long long vl = (long long)fl + k[a];
        if (!(fabsf(g[a]) < 1e9f) || vl <= -MAX_VOXEL_COORD || vl >= MAX_VOXEL_COORD) return false;
        v0[a] = (int)vl;
        f[a] = g[a] - fl;
    }
    // block coordinates of the lower / upper corner along each axis
    const int b0[3] = {v0[0] >> 3, v0[1] >> 3, v0[2] >> 3};
    const int b1[3] = {(v0[0] + 1) >> 3, (v0[1] + 1) >> 3, (v0[2] + 1) >> 3};
    // block j = (jx, jy, jz) in {0,1}^3, needed only where the axis crosses
    uint64_t key[8];
    uint64_t hh[8];
    HashSlot first[8];
    bool need[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int jx = j & 1, jy = (j >> 1) & 1, jz = j >> 2;
        need[j] = (!jx || b1[0] != b0[0]) && (!jy || b1[1] != b0[1]) && (!jz || b1[2] != b0[2]);
        key[j] = pack_block(jx ? b1[0] : b0[0], jy ? b1[1] : b0[1], jz ? b1[2] : b0[2]);
        hh[j] = fmix64(key[j]) & md.mask;
        // the home slot's key and pool slot in one load
        if (need[j]) first[j] = md.hs[hh[j]];
        else first[j].key = key[j], first[j].val = 0;
    }
    int slot[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        slot[j] = 0;
        if (!need[j]) continue;
        if (first[j].key == key[j]) {
            slot[j] = first[j].val;
        } else {
            const int h = first[j].key == EMPTY_KEY ? -1 : hash_find(md.hs, md.mask, key[j]);
            slot[j] = h < 0 ? -1 : md.hs[h].val;
        }
    }
    float2 dw[8];
    bool ok = true;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int vx = v0[0] + (c & 1), vy = v0[1] + ((c >> 1) & 1), vz = v0[2] + (c >> 2);
        // block of this corner: index j with jx set only when the corner sits in the upper block
        const int j = ((vx >> 3) != b0[0] ? 1 : 0) | ((vy >> 3) != b0[1] ? 2 : 0) | ((vz >> 3) != b0[2] ? 4 : 0);
        const int sl = slot[j];
        ok = ok && sl >= 0;
        const long long vox = (long long)(sl < 0 ? 0 : sl) * BV + (vx & 7) + 8 * (vy & 7) + 64 * (vz & 7);
        dw[c] = sl < 0 ? make_float2(0.f, 0.f)
                       : (md.storage == 0 ? md.dw32[vox] : __half22float2(md.dw16[vox]));
    }
    if (!ok) return false;
    float Dc[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        if (!(dw[c].y > 0.f)) return false;
        Dc[c] = dw[c].x;
    }
    float s = 0.f, d0 = 0.f, d1 = 0.f, d2 = 0.f;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const float w0 = (c & 1) ? f[0] : 1.f - f[0];
        const float w1 = ((c >> 1) & 1) ? f[1] : 1.f - f[1];
        const float w2 = (c >> 2) ? f[2] : 1.f - f[2];
        const float s0 = (c & 1) ? 1.f : -1.f, s1 = ((c >> 1) & 1) ? 1.f : -1.f, s2 = (c >> 2) ? 1.f : -1.f;
        s += w0 * w1 * w2 * Dc[c];
        d0 += s0 * w1 * w2 * Dc[c];
        d1 += w0 * s1 * w2 * Dc[c];
        d2 += w0 * w1 * s2 * Dc[c];
    }
    D = s;
    dg[0] = d0;
    dg[1] = d1;
    dg[2] = d2;
    return true;
}

__device__ __forceinline__ void world_to_grid(const MapDev &md, const float *xyz, long long i, int k[3], float g[3]) {
    const float inv = 1.f / md.nu;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float q = xyz[3 * i + a] * inv;
        const float fl = floorf(q);
        k[a] = (int)fl;
        g[a] = q - fl;
    }
}

__global__ void __launch_bounds__(256) k_query(MapDev md, const float *__restrict__ xyz, long long m, float *sdf,
                                               uint8_t *valid) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    int k[3];
    float g[3], D, dg[3];
    world_to_grid(md, xyz, i, k, g);
    const bool ok = trilinear(md, k, g, D, dg);
    sdf[i] = ok ? D : __int_as_float(0x7fc00000);
    if (valid) valid[i] = ok ? 1 : 0;
}

// Backward of the query: grad_xyz = grad_sdf * dD/dx per point and, when
// `part` is non-null, this CTA's row of the pose-gradient sums
// (sum g, sum x x g) in part[8 b + 0..5], as float pairs (TwoProd / TwoSum)
// on the FP32 pipes and without atomics; k_pose_finish adds the rows.
constexpr int QB_MAX_CTAS = 148 * 8;

__global__ void __launch_bounds__(256) k_query_bwd(MapDev md, const float *__restrict__ xyz,
                                                   const float *__restrict__ gsdf, long long m, float *gxyz,
                                                   double *part) {
    __shared__ float s_h[8][6], s_l[8][6];
    float ah[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, al[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (long long)gridDim.x * blockDim.x) {
        int k[3];
        float g[3], D, dg[3];
        float gx[3] = {0.f, 0.f, 0.f};
        world_to_grid(md, xyz, i, k, g);
        if (trilinear(md, k, g, D, dg)) {
            const float s = gsdf[i] / md.nu;
#pragma unroll
            for (int a = 0; a < 3; ++a) gx[a] = s * dg[a];
        }
        float x[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            gxyz[3 * i + a] = gx[a];
            x[a] = xyz[3 * i + a];
        }
        if (part) {
#pragma unroll
            for (int a = 0; a < 3; ++a) df_add(ah[a], al[a], gx[a], 0.f, ah[a], al[a]);
            // x x g, each component a difference of two exact products
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const int b = (a + 1) % 3, c = (a + 2) % 3;
                float p1, e1, p2, e2, th, tl;
                two_prod(x[b], gx[c], p1, e1);
                two_prod(x[c], gx[b], p2, e2);
                df_add(p1, e1, -p2, -e2, th, tl);
                df_add(ah[3 + a], al[3 + a], th, tl, ah[3 + a], al[3 + a]);
            }
        }
    }
    if (!part) return;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float bh = __shfl_xor_sync(0xffffffffu, ah[j], o), bl = __shfl_xor_sync(0xffffffffu, al[j], o);
            df_add(ah[j], al[j], bh, bl, ah[j], al[j]);
        }
    }
    if (lane == 0) {
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            s_h[wid][j] = ah[j];
            s_l[wid][j] = al[j];
        }
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        float th = 0.f, tl = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) df_add(th, tl, s_h[w][threadIdx.x], s_l[w][threadIdx.x], th, tl);
        part[8 * blockIdx.x + threadIdx.x] = (double)th + (double)tl;
    }
}

// pose_grad[j] += sum over the CTA rows of part (fixed order).
__global__ void k_pose_finish(const double *part, int nparts, double *pose_grad) {
    const int j = threadIdx.x;
    if (j >= 6) return;
    double t = 0.0;
    for (int b = 0; b < nparts; ++b) t += part[8 * b + j];
    pose_grad[j] += t;
}

// Gauss-Newton terms for a left perturbation about the sensor position c = t
// of T (x' = Exp(xi)(x - c) + c, so J = grad D^T [I | -[R p]x]; about the
// world origin, far from a scan on a large map, a rotation needs a
// compensating translation as long as the lever arm, which the damping
// resists).  Accumulation: per CTA b, row b of float pairs (hi, lo) viewed as
// float2 row[32 b + j]: j = 0..20 upper triangle of H = sum J^T J, 21..26
// g = sum J^T D, 27 loss sum D^2, 28 valid count (plain stores, no atomics;
// k_gn_step sums the CTAs' rows in a fixed order).
constexpr int GN_ACC = 29;
constexpr int GN_MAX_CTAS = 148 * 8;

// Three CTAs per SM (at most 85 registers; 29 float-pair sums per thread then
// spill ~340 bytes to L1): 113,664 resident threads, so a scan's ~92,000
// valid points run in one wave instead of two at 128 registers.
__global__ void __launch_bounds__(256, 3) k_gn_terms(MapDev md, const float *__restrict__ pts, long long n,
                                                  const double *__restrict__ T, double *acc) {
    __shared__ float s_c[16];
    __shared__ int s_k[3];
    __shared__ float s_h[8][GN_ACC], s_l[8][GN_ACC];
    pdl_wait();      // the previous step's pose, and its reads of acc done
    pdl_trigger();   // the step kernel may be scheduled now
    if (threadIdx.x == 0) {
        // R / nu and the split t / nu = k + f (k integer)
        for (int r = 0; r < 3; ++r) {
            for (int c = 0; c < 3; ++c) s_c[3 * r + c] = (float)(T[4 * r + c] / (double)md.nu);
            const double tv = T[4 * r + 3] / (double)md.nu;
            const double fl = floor(tv);
            s_k[r] = (int)fl;
            s_c[9 + r] = (float)(tv - fl);
        }
    }
    __syncthreads();
    // sums as unevaluated float pairs (products exact by TwoProd, sums by TwoSum):
    // ~48-bit sums on the FP32 pipes (this GPU's FP64 rate is a small fraction)
    float ah[GN_ACC], al[GN_ACC];
#pragma unroll
    for (int j = 0; j < GN_ACC; ++j) ah[j] = al[j] = 0.f;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float p0 = pts[3 * i], p1 = pts[3 * i + 1], p2 = pts[3 * i + 2];
        if (!(isfinite(p0) && isfinite(p1) && isfinite(p2))) continue;
        float g[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) g[r] = s_c[3 * r] * p0 + s_c[3 * r + 1] * p1 + s_c[3 * r + 2] * p2 + s_c[9 + r];
        float D, dg[3];
        if (!trilinear(md, s_k, g, D, dg)) continue;
        const float inv = 1.f / md.nu;
        const float gr[3] = {dg[0] * inv, dg[1] * inv, dg[2] * inv};
        // rotation about the sensor position c = t: x - c = R p
        float rp[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) rp[r] = md.nu * (s_c[3 * r] * p0 + s_c[3 * r + 1] * p1 + s_c[3 * r + 2] * p2);
        const float J[6] = {gr[0], gr[1], gr[2], rp[1] * gr[2] - rp[2] * gr[1], rp[2] * gr[0] - rp[0] * gr[2],
                            rp[0] * gr[1] - rp[1] * gr[0]};
        float ph, pl;
        int q = 0;
#pragma unroll
        for (int r = 0; r < 6; ++r)
#pragma unroll
            for (int c = r; c < 6; ++c) {
                two_prod(J[r], J[c], ph, pl);
                df_add(ah[q], al[q], ph, pl, ah[q], al[q]);
                ++q;
            }
#pragma unroll
        for (int r = 0; r < 6; ++r) {
            two_prod(J[r], D, ph, pl);
            df_add(ah[21 + r], al[21 + r], ph, pl, ah[21 + r], al[21 + r]);
        }
        two_prod(D, D, ph, pl);
        df_add(ah[27], al[27], ph, pl, ah[27], al[27]);
        df_add(ah[28], al[28], 1.f, 0.f, ah[28], al[28]);
    }
    // warp sums, then the CTA's row of partial sums (as doubles)
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < GN_ACC; ++j) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float bh = __shfl_xor_sync(0xffffffffu, ah[j], o), bl = __shfl_xor_sync(0xffffffffu, al[j], o);
            df_add(ah[j], al[j], bh, bl, ah[j], al[j]);
        }
    }
    if (lane == 0) {
#pragma unroll
        for (int j = 0; j < GN_ACC; ++j) {
            s_h[wid][j] = ah[j];
            s_l[wid][j] = al[j];
        }
    }
    __syncthreads();
    if (threadIdx.x < GN_ACC) {
        float th = 0.f, tl = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) df_add(th, tl, s_h[w][threadIdx.x], s_l[w][threadIdx.x], th, tl);
        reinterpret_cast<float2 *>(acc)[32 * blockIdx.x + threadIdx.x] = make_float2(th, tl);
    }
}

// Rodrigues coefficients A = sin(t)/t, B = (1 - cos(t))/t^2, C = (t - sin(t))/t^3
// of the SE(3) exponential: their Taylor series in t^2 for t < 0.5 (terms to
// t^16, truncation below 1e-17), the closed forms otherwise.
__host__ __device__ constexpr double inv_factorial(int n) { return n <= 1 ? 1.0 : inv_factorial(n - 1) / (double)n; }
struct RodriguesSeries {
    double a[9], b[9], c[9];   // (-1)^k / (2k+1)!, (-1)^k / (2k+2)!, (-1)^k / (2k+3)!
};
__host__ __device__ constexpr RodriguesSeries rodrigues_series() {
    RodriguesSeries r{};
    for (int k = 0; k < 9; ++k) {
        const double sg = (k & 1) ? -1.0 : 1.0;
        r.a[k] = sg * inv_factorial(2 * k + 1);
        r.b[k] = sg * inv_factorial(2 * k + 2);
        r.c[k] = sg * inv_factorial(2 * k + 3);
    }
    return r;
}
__device__ __forceinline__ void rodrigues_coeffs(double th2, double &A1, double &B1, double &C1) {
    constexpr RodriguesSeries S = rodrigues_series();
    if (th2 < 0.25) {
        // Horner in t^2
        A1 = S.a[8];
        B1 = S.b[8];
        C1 = S.c[8];
#pragma unroll
        for (int k = 7; k >= 0; --k) {
            A1 = fma(A1, th2, S.a[k]);
            B1 = fma(B1, th2, S.b[k]);
            C1 = fma(C1, th2, S.c[k]);
        }
    } else {
        const double th = sqrt(th2);
        double sn, cs;
        sincos(th, &sn, &cs);
        A1 = sn / th;
        B1 = (1.0 - cs) / th2;
        C1 = (th - sn) / (th2 * th);
    }
}

// One CTA: sum the per-CTA rows (fixed order), then one thread solves
// (H + mu I) d = -g (Cholesky; H is a sum of outer products plus mu I), and
// twelve threads apply the step about the sensor position (see k_gn_terms).
__global__ void __launch_bounds__(256) k_gn_step(double *T, const double *acc, int nparts) {
    __shared__ float s_ph[8][32], s_pl[8][32];
    __shared__ double s_a[32];
    pdl_wait();      // the terms kernel's rows
    pdl_trigger();   // the next iteration's terms kernel may be scheduled now
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const float2 *rows = reinterpret_cast<const float2 *>(acc);
    if (lane < GN_ACC) {
        // rows wid, wid + 8, ... in order (float pairs, TwoSum on the FP32 pipes);
        // eight loads in flight per step
        float th = 0.f, tl = 0.f;
        for (int b0 = wid; b0 < nparts; b0 += 64) {
            float2 v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u)
                v[u] = b0 + 8 * u < nparts ? rows[32 * (b0 + 8 * u) + lane] : make_float2(0.f, 0.f);
#pragma unroll
            for (int u = 0; u < 8; ++u) df_add(th, tl, v[u].x, v[u].y, th, tl);
        }
        s_ph[wid][lane] = th;
        s_pl[wid][lane] = tl;
    }
    __syncthreads();
    if (threadIdx.x < GN_ACC) {
        float th = 0.f, tl = 0.f;
        for (int w = 0; w < 8; ++w) df_add(th, tl, s_ph[w][threadIdx.x], s_pl[w][threadIdx.x], th, tl);
        s_a[threadIdx.x] = (double)th + (double)tl;
    }
    __syncthreads();
    // the 6x6 solve and the step in FP32 (one thread; this GPU's FP64 latency
    // is long): H is well conditioned with the sensor-centred perturbation, and
    // the iteration's fixed point is set by g, which the float-pair sums carry
    // exactly; only the pose composition below is FP64 (12 threads)
    __shared__ float s_step[21];   // dR (row-major) and V rho
    if (threadIdx.x == 0) {
        const double *a = s_a;
        float Hm[6][6];
        {
            int q = 0;
#pragma unroll
            for (int r = 0; r < 6; ++r)
#pragma unroll
                for (int c = r; c < 6; ++c) {
                    Hm[r][c] = (float)a[q];
                    Hm[c][r] = (float)a[q];
                    ++q;
                }
        }
        float tr = 0.f;
#pragma unroll
        for (int r = 0; r < 6; ++r) tr += Hm[r][r];
        const float mu = 1e-6f * (tr / 6.f + 1e-12f);
        float Lc[6][6], inv_diag[6];
        bool ok = true;
#pragma unroll
        for (int i = 0; i < 6; ++i) {
#pragma unroll
            for (int j = 0; j <= i; ++j) {
                float sum = Hm[i][j] + (i == j ? mu : 0.f);
#pragma unroll
                for (int k = 0; k < j; ++k) sum -= Lc[i][k] * Lc[j][k];
                if (i == j) {
                    ok = ok && sum > 0.f;
                    Lc[i][i] = sqrtf(sum > 0.f ? sum : 1.f);
                    inv_diag[i] = 1.f / Lc[i][i];
                } else {
                    Lc[i][j] = sum * inv_diag[j];
                }
            }
        }
        float d[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (ok) {
            float y[6];
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                float sum = -(float)a[21 + i];
#pragma unroll
                for (int k = 0; k < i; ++k) sum -= Lc[i][k] * y[k];
                y[i] = sum * inv_diag[i];
            }
#pragma unroll
            for (int i = 5; i >= 0; --i) {
                float sum = y[i];
#pragma unroll
                for (int k = i + 1; k < 6; ++k) sum -= Lc[k][i] * d[k];
                d[i] = sum * inv_diag[i];
            }
        }
        // Exp(rho, phi): Rodrigues rotation dR, translation V(phi) rho
        const float *rho = d, *phi = d + 3;
        const double th2 = (double)phi[0] * phi[0] + (double)phi[1] * phi[1] + (double)phi[2] * phi[2];
        double A1d, B1d, C1d;
        rodrigues_coeffs(th2, A1d, B1d, C1d);
        const float A1 = (float)A1d, B1 = (float)B1d, C1 = (float)C1d;
        const float K[3][3] = {{0.f, -phi[2], phi[1]}, {phi[2], 0.f, -phi[0]}, {-phi[1], phi[0], 0.f}};
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            float vr = 0.f;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                float k2 = 0.f;
#pragma unroll
                for (int k = 0; k < 3; ++k) k2 += K[i][k] * K[k][j];
                const float I = i == j ? 1.f : 0.f;
                s_step[3 * i + j] = I + A1 * K[i][j] + B1 * k2;
                vr += (I + B1 * K[i][j] + C1 * k2) * rho[j];
            }
            s_step[9 + i] = vr;
        }
    }
    __syncthreads();
    // T <- Tr(c) Exp(d) Tr(-c) T about the sensor position c = t: R <- dR R, t <- t + V rho
    double v = 0.0;
    const int e = threadIdx.x;
    if (e < 9) {
        const int r = e / 3, c = e % 3;
        v = (double)s_step[3 * r] * T[c] + (double)s_step[3 * r + 1] * T[4 + c] + (double)s_step[3 * r + 2] * T[8 + c];
    } else if (e < 12) {
        v = T[4 * (e - 9) + 3] + (double)s_step[9 + (e - 9)];
    }
    __syncthreads();   // every thread has read T
    if (e < 9) T[4 * (e / 3) + (e % 3)] = v;
    else if (e < 12) T[4 * (e - 9) + 3] = v;
}

void launch_query(const MapDev &md, const float *xyz, long long m, float *sdf, uint8_t *valid, cudaStream_t s) {
    if (m > 0) k_query<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(md, xyz, m, sdf, valid);
}
void launch_query_bwd(const MapDev &md, const float *xyz, const float *gsdf, long long m, float *gxyz,
                      double *pose_grad, double *part, cudaStream_t s) {
    if (m <= 0) return;
    long long grid = (m + 255) / 256;
    if (grid > QB_MAX_CTAS) grid = QB_MAX_CTAS;
    k_query_bwd<<<(unsigned)grid, 256, 0, s>>>(md, xyz, gsdf, m, gxyz, pose_grad ? part : nullptr);
    if (pose_grad) k_pose_finish<<<1, 32, 0, s>>>(part, (int)grid, pose_grad);
}
int gn_terms_grid(long long n) {
    long long grid = (n + 255) / 256;
    if (grid > GN_MAX_CTAS) grid = GN_MAX_CTAS;
    if (grid < 1) grid = 1;
    return (int)grid;
}
void launch_gn_terms(const MapDev &md, const float *pts, long long n, const double *T_dev, double *acc,
                     cudaStream_t s) {
    // both Gauss-Newton kernels are launched as programmatic dependents of the one before
    launch_pdl(k_gn_terms, dim3(gn_terms_grid(n)), dim3(256), 0, s, md, pts, n, T_dev, acc);
}
void launch_gn_step(double *T_dev, const double *acc, int nparts, cudaStream_t s) {
    launch_pdl(k_gn_step, dim3(1), dim3(256), 0, s, T_dev, acc, nparts);
}

}  // namespace stsdf
