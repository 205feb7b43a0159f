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
__device__ __forceinline__ bool trilinear(const MapDev &md, const int k[3], const float g[3], float &D,
                                          float dg[3]) {
    int v0[3];
    float f[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float fl = floorf(g[a]);
        v0[a] = (int)fl + k[a];
        f[a] = g[a] - fl;
    }
    uint64_t ck[8];
    int cs[8];
    int nc = 0;
    float Dc[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int vx = v0[0] + (c & 1), vy = v0[1] + ((c >> 1) & 1), vz = v0[2] + (c >> 2);
        const uint64_t key = pack_block(vx >> 3, vy >> 3, vz >> 3);
        int slot = -2;
        for (int j = 0; j < nc; ++j)
            if (ck[j] == key) slot = cs[j];
        if (slot == -2) {
            const int h = hash_find(md.keys, md.mask, key);
            slot = h < 0 ? -1 : md.vals[h];
            ck[nc] = key;
            cs[nc] = slot;
            ++nc;
        }
        if (slot < 0) return false;
        const long long vox = (long long)slot * BV + (vx & 7) + 8 * (vy & 7) + 64 * (vz & 7);
        const float2 dw = md.storage == 0 ? md.dw32[vox] : __half22float2(md.dw16[vox]);
        if (!(dw.y > 0.f)) return false;
        Dc[c] = dw.x;
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

__device__ __forceinline__ double block_sum_d(double v, double *s_tmp) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) s_tmp[wid] = v;
    __syncthreads();
    double t = 0.0;
    for (int j = 0; j < nw; ++j) t += s_tmp[j];
    __syncthreads();
    return t;
}

__global__ void __launch_bounds__(256) k_query_bwd(MapDev md, const float *__restrict__ xyz,
                                                   const float *__restrict__ gsdf, long long m, float *gxyz,
                                                   double *pose_grad) {
    __shared__ double s_tmp[8];
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    float gx[3] = {0.f, 0.f, 0.f};
    float x[3] = {0.f, 0.f, 0.f};
    if (i < m) {
        int k[3];
        float g[3], D, dg[3];
        world_to_grid(md, xyz, i, k, g);
        if (trilinear(md, k, g, D, dg)) {
            const float s = gsdf[i] / md.nu;
#pragma unroll
            for (int a = 0; a < 3; ++a) gx[a] = s * dg[a];
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            gxyz[3 * i + a] = gx[a];
            x[a] = xyz[3 * i + a];
        }
    }
    if (pose_grad) {
        const double v[6] = {gx[0], gx[1], gx[2], (double)x[1] * gx[2] - (double)x[2] * gx[1],
                             (double)x[2] * gx[0] - (double)x[0] * gx[2], (double)x[0] * gx[1] - (double)x[1] * gx[0]};
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            const double t = block_sum_d(v[j], s_tmp);
            if (threadIdx.x == 0 && t != 0.0) atomicAdd(&pose_grad[j], t);
        }
    }
}

// Gauss-Newton accumulation: acc[0..20] upper triangle of H = sum J^T J,
// acc[21..26] g = sum J^T D, acc[27] loss sum D^2, acc[28] valid count.
constexpr int GN_ACC = 29;

__global__ void __launch_bounds__(256) k_gn_terms(MapDev md, const float *__restrict__ pts, long long n,
                                                  const double *__restrict__ T, double *acc) {
    __shared__ float s_c[16];
    __shared__ int s_k[3];
    __shared__ double s_tmp[8];
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
    double a[GN_ACC];
#pragma unroll
    for (int j = 0; j < GN_ACC; ++j) a[j] = 0.0;
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
        float x[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) x[r] = md.nu * ((float)s_k[r] + g[r]);
        const float J[6] = {gr[0], gr[1], gr[2], x[1] * gr[2] - x[2] * gr[1], x[2] * gr[0] - x[0] * gr[2],
                            x[0] * gr[1] - x[1] * gr[0]};
        int q = 0;
#pragma unroll
        for (int r = 0; r < 6; ++r)
#pragma unroll
            for (int c = r; c < 6; ++c) a[q++] += (double)J[r] * (double)J[c];
#pragma unroll
        for (int r = 0; r < 6; ++r) a[21 + r] += (double)J[r] * (double)D;
        a[27] += (double)D * (double)D;
        a[28] += 1.0;
    }
#pragma unroll
    for (int j = 0; j < GN_ACC; ++j) {
        const double t = block_sum_d(a[j], s_tmp);
        if (threadIdx.x == 0 && t != 0.0) atomicAdd(&acc[j], t);
    }
}

// One thread: solve (H + mu I) d = -g, T <- Exp(d) T, clear the accumulators.
__global__ void k_gn_step(double *T, double *acc) {
    double H[6][6], A[6][7];
    int q = 0;
    for (int r = 0; r < 6; ++r)
        for (int c = r; c < 6; ++c) {
            H[r][c] = acc[q];
            H[c][r] = acc[q];
            ++q;
        }
    double tr = 0.0;
    for (int r = 0; r < 6; ++r) tr += H[r][r];
    const double mu = 1e-6 * (tr / 6.0 + 1e-12);
    for (int r = 0; r < 6; ++r) {
        for (int c = 0; c < 6; ++c) A[r][c] = H[r][c] + (r == c ? mu : 0.0);
        A[r][6] = -acc[21 + r];
    }
    bool ok = true;
    for (int c = 0; c < 6 && ok; ++c) {
        int piv = c;
        for (int r = c + 1; r < 6; ++r)
            if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
        for (int k = 0; k < 7; ++k) {
            const double t = A[c][k];
            A[c][k] = A[piv][k];
            A[piv][k] = t;
        }
        if (A[c][c] == 0.0) {
            ok = false;
            break;
        }
        for (int r = c + 1; r < 6; ++r) {
            const double f = A[r][c] / A[c][c];
            for (int k = c; k < 7; ++k) A[r][k] -= f * A[c][k];
        }
    }
    double d[6] = {0, 0, 0, 0, 0, 0};
    if (ok) {
        for (int c = 5; c >= 0; --c) {
            double s = A[c][6];
            for (int k = c + 1; k < 6; ++k) s -= A[c][k] * d[k];
            d[c] = s / A[c][c];
        }
    }
    // Exp(rho, phi): Rodrigues rotation, translation V(phi) rho
    const double *rho = d, *phi = d + 3;
    const double th2 = phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2];
    const double th = sqrt(th2);
    double A1, B1, C1;
    if (th < 1e-8) {
        A1 = 1.0 - th2 / 6.0;
        B1 = 0.5 - th2 / 24.0;
        C1 = 1.0 / 6.0 - th2 / 120.0;
    } else {
        A1 = sin(th) / th;
        B1 = (1.0 - cos(th)) / th2;
        C1 = (th - sin(th)) / (th2 * th);
    }
    const double K[3][3] = {{0, -phi[2], phi[1]}, {phi[2], 0, -phi[0]}, {-phi[1], phi[0], 0}};
    double K2[3][3], R[3][3], V[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += K[i][k] * K[k][j];
            K2[i][j] = s;
        }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            const double I = i == j ? 1.0 : 0.0;
            R[i][j] = I + A1 * K[i][j] + B1 * K2[i][j];
            V[i][j] = I + B1 * K[i][j] + C1 * K2[i][j];
        }
    double Tn[16];
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) Tn[4 * r + c] = R[r][0] * T[c] + R[r][1] * T[4 + c] + R[r][2] * T[8 + c];
        Tn[4 * r + 3] = R[r][0] * T[3] + R[r][1] * T[7] + R[r][2] * T[11] + V[r][0] * rho[0] + V[r][1] * rho[1] +
                        V[r][2] * rho[2];
    }
    for (int r = 0; r < 12; ++r) T[r] = Tn[r];
    for (int j = 0; j < GN_ACC; ++j) acc[j] = 0.0;
}

void launch_query(const MapDev &md, const float *xyz, long long m, float *sdf, uint8_t *valid, cudaStream_t s) {
    if (m > 0) k_query<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(md, xyz, m, sdf, valid);
}
void launch_query_bwd(const MapDev &md, const float *xyz, const float *gsdf, long long m, float *gxyz,
                      double *pose_grad, cudaStream_t s) {
    if (m > 0) k_query_bwd<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(md, xyz, gsdf, m, gxyz, pose_grad);
}
void launch_gn_terms(const MapDev &md, const float *pts, long long n, const double *T_dev, double *acc,
                     cudaStream_t s) {
    long long grid = (n + 255) / 256;
    if (grid > 148 * 8) grid = 148 * 8;
    if (grid < 1) grid = 1;
    k_gn_terms<<<(unsigned)grid, 256, 0, s>>>(md, pts, n, T_dev, acc);
}
void launch_gn_step(double *T_dev, double *acc, cudaStream_t s) { k_gn_step<<<1, 1, 0, s>>>(T_dev, acc); }

}  // namespace stsdf
