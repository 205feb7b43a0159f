/*
 * FP64 CPU oracle for the per-frame metric-semantic mapping path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the package smoke check and the
 * benchmark's CPU-baseline leg may.  It shares no code, header, table or
 * constant generator with the CUDA path.
 *
 * What it follows (Liu et al., "Real-Time Metric-Semantic Mapping for
 * Autonomous Navigation in Outdoor Environments", 2024):
 *   - Sec. III-C.1, range-image equation: u = (pi - atan2(y, x)) / dphi,
 *     v = (acos(z / r) - theta0) / dtheta.
 *   - Sec. III-C.2: voxel centre x_i = nu * v_i; two-level storage, a hash of
 *     8x8x8-voxel blocks; projective distance psi along the ray, negative
 *     behind the surface; linear weight W_i = (psi + tau) / (2 tau); the
 *     running-average update of D and W with truncation Gamma(d, tau).
 *   - Sec. III-C.3, Eq. (bayesian_filter): uniform prior per new voxel and
 *     the recursive Bayesian product with the per-pixel class likelihood,
 *     normalised by Z; mesh by marching cubes with each vertex labelled by
 *     its most probable class.
 *
 * Readings where the paper is silent (each is also listed in the design
 * notes): nearest point wins a pixel; blocks are allocated along
 * [p - tau d, p + tau d] of every valid point; voxels of the touched
 * blocks only are updated; psi < -tau is skipped; the linear weight is
 * clamped to [0, 1]; the semantic update is gated to |psi| <= tau; the
 * hard-label likelihood is p_hit / (1 - p_hit)/(C - 1); log-probabilities
 * are floored; marching-cubes faces with four crossings separate the inside
 * corners; a cube needs all 8 corners observed (W > 0).
 *
 * Non-projective distance (Sec. III-C.2, Eq. distance), optional per map:
 * the normal image from each pixel's back-projected point and its (u, v-1)
 * and (u-1, v) neighbours, turned to face the sensor; the voxel gradient
 * g_i as the weight-averaged, renormalised normal of the pixels the voxel
 * projected to; d_i = psi (|cos theta| - sin theta tan(alpha / 2)) with a
 * signed alpha (positive when g_i turns from the normal toward the ray,
 * a convex surface), which is the printed curved-surface case derived from
 * the figure's circle (the print lacks the factor psi on that term and
 * drops the sign) and equals the printed flat case at alpha = 0; the flat
 * case also where cos alpha <= 0, where the pixel has no normal (g_i kept)
 * or the voxel has no gradient yet (then d_i = psi).  The weight and the
 * skip below -tau stay on psi; Gamma(d_i, tau) is the fused value.
 *
 * The fusion of probability vectors has no worked example in the paper; it
 * is pinned by closed forms and invariants: the normalised product of the
 * scans' vectors, the normalisation invariant, independence of the scan
 * order, a uniform likelihood leaving the posterior unchanged, and the two
 * floors (an entry below lik_floor counts as lik_floor; a class held there
 * reaches logp_floor exactly while the others keep their product's closed
 * form).
 *
 * Precision: every value and every decision is FP64: point validity and
 * pixel, the nearest-point winner of each pixel, the blocks met by each
 * point's band (an exact segment-box clearance test, band_blocks below), each
 * voxel's pixel and its update and class-update gates.  Each decision also
 * has an ambiguity band in which a single-precision implementation may
 * legitimately decide otherwise: a projection within delta_px of a pixel
 * boundary, a range within 2^-20 (relative) of r_min, r_max or of the
 * pixel's nearest range, a block whose clearance is within band_margin of
 * zero, psi within eps_psi of +-tau.  Given such an implementation's
 * recorded choices (struct Decisions), the oracle follows them inside those
 * bands when they are FP64 candidates, and counts every choice outside them
 * that differs from its own (orc_check); without a record it takes its own
 * choices and marks ambiguous voxels "tainted" (sticky).
 */
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <unordered_map>
#include <unordered_set>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

constexpr int BS = 8;            // voxels per block side (Sec. III-C.2)
constexpr int BV = BS * BS * BS;
constexpr double PI = 3.14159265358979323846;

// ---------------------------------------------------------------------------
// integer helpers
// ---------------------------------------------------------------------------
inline int64_t floordiv(int64_t a, int64_t b) {
    int64_t q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) --q;
    return q;
}

struct I3 {
    int64_t x, y, z;
    bool operator==(const I3 &o) const { return x == o.x && y == o.y && z == o.z; }
    bool operator<(const I3 &o) const {
        if (x != o.x) return x < o.x;
        if (y != o.y) return y < o.y;
        return z < o.z;
    }
};
struct I3Hash {
    size_t operator()(const I3 &k) const {
        uint64_t h = (uint64_t)k.x * 0x9E3779B97F4A7C15ULL;
        h ^= (uint64_t)k.y * 0xC2B2AE3D27D4EB4FULL + (h << 6) + (h >> 2);
        h ^= (uint64_t)k.z * 0x165667B19E3779F9ULL + (h << 6) + (h >> 2);
        return (size_t)h;
    }
};

// Global key of a lattice edge: its lower end voxel and its axis.  The
// order of keys is lexicographic in (z, y, x, axis); this order decides
// which loop vertex starts a triangle fan.
inline int64_t edge_key(int64_t x, int64_t y, int64_t z, int axis) {
    const int64_t bias = (int64_t)1 << 19;
    return ((((z + bias) << 20 | (y + bias)) << 20 | (x + bias)) << 2) | axis;
}

// ---------------------------------------------------------------------------
// map state
// ---------------------------------------------------------------------------
struct Block {
    std::vector<double> D, W, logP;  // D[512], W[512], logP[C][512] (class-major)
    std::vector<uint8_t> taint;      // bit 0: distance/weight, bit 1: semantics
    std::vector<int32_t> nupd, nsem; // per voxel: distance updates and class updates so far
    std::vector<double> G;           // non-projective mode: gradient g_i, G[k][512] (k = x, y, z)
};

struct Lidar {
    int H, W;
    double fov_up, fov_down, r_min, r_max;
    double dphi, dtheta, theta0;
};

struct Stats {
    int64_t valid_points = 0, pixel_points = 0, ambiguous_points = 0;
    int64_t touched_blocks = 0, new_blocks = 0;
    int64_t voxels_updated = 0, voxels_semantic = 0, voxels_seen = 0;
    int64_t taint_events = 0;
    int64_t sure_blocks = 0, ambiguous_blocks = 0;   // band blocks: sure, and within the margin only
};

/*
 * The choices a single-precision implementation made for one scan, offered
 * for candidate acceptance.  Where the FP64 computation finds a decision
 * within its ambiguity band (a point or voxel projecting within delta_px of
 * a pixel boundary, a range within 2^-20 of r_min, r_max or of the pixel's
 * nearest range, a block within the band margin, a psi within eps_psi of
 * +-tau), the recorded choice is accepted if it is one of the FP64
 * candidates and then used, so that both maps stay in step; everywhere else
 * the recorded choice must equal the FP64 one.  Either way every mismatch
 * is counted (Check) and the FP64 choice is kept.
 */
struct Decisions {
    const int32_t *point_pix = nullptr;   // [n] pixel of each point, -1 valid without a pixel, -2 invalid
    const uint64_t *winner = nullptr;     // [H*W] (range bits << 32) | winning point, ~0 for none
    const int32_t *touched = nullptr;     // [n_touched][3] blocks of U_k
    int64_t n_touched = 0;
    const int32_t *vox = nullptr;         // [n_touched][512] per voxel: pixel + 1 (0: none) | upd << 28 | sem << 29
};

enum {
    CK_POINTS = 0, CK_POINTS_AMB, CK_POINTS_BAD,
    CK_PIXELS, CK_WINNERS_AMB, CK_WINNERS_BAD,
    CK_BLOCKS_SURE, CK_BLOCKS_AMB, CK_BLOCKS_AMB_TAKEN, CK_BLOCKS_MISSING, CK_BLOCKS_EXTRA,
    CK_VOXELS, CK_VOX_PIX_AMB, CK_VOX_PIX_BAD, CK_VOX_UPD_AMB, CK_VOX_UPD_BAD, CK_VOX_SEM_AMB, CK_VOX_SEM_BAD,
    CK_VOX_NO_RECORD,
    CK_COUNT = 24
};

struct Map {
    double nu, tau;
    int C;
    int weight_mode;                 // 0: linear weight (Sec. III-C.2), 1: constant 1
    int dist_mode = 0;               // 0: projective psi, 1: non-projective d_i (Eq. distance)
    double p_hit, logp_floor, lik_floor;
    double delta_px = 1e-3;          // pixel-boundary ambiguity band, in pixels
    double eps_psi;                  // psi ambiguity band around +-tau, metres
    std::unordered_map<I3, Block, I3Hash> blocks;
    bool track = false;              // keep voxel data only for track_keys
    std::unordered_set<I3, I3Hash> track_keys;
    std::unordered_set<I3, I3Hash> alloc;   // every allocated block (keys)
    std::vector<I3> touched;                // U_k of the last frame
    std::vector<double> normals;            // non-projective mode: last normal image, world frame [H*W][3]
    std::vector<uint8_t> normal_flag;       // bit 0: normal valid, bit 1: orientation nearly ambiguous
    Stats st;
    int64_t check[CK_COUNT] = {};           // candidate-acceptance counts of the last scan
    int64_t frame = 0;
};

Block new_block(int C, int dist_mode) {
    Block b;
    b.D.assign(BV, 0.0);
    b.W.assign(BV, 0.0);
    // uniform prior over the classes for every new voxel (Sec. III-C.3)
    b.logP.assign((size_t)C * BV, -std::log((double)C));
    b.taint.assign(BV, 0);
    b.nupd.assign(BV, 0);
    b.nsem.assign(BV, 0);
    if (dist_mode == 1) b.G.assign(3 * BV, 0.0);   // no gradient until a normal is seen
    return b;
}

inline int vidx(int lx, int ly, int lz) { return lx + BS * (ly + BS * lz); }

// ---------------------------------------------------------------------------
// band allocation in FP64 (Sec. III-C.2: the voxel blocks around each
// measurement are found along its ray and inserted in the block hash)
// ---------------------------------------------------------------------------
/*
 * Band endpoints of one point x (LiDAR frame) in voxel units plus one half,
 * so that voxel v occupies [v, v + 1) and block b occupies [8 b, 8 b + 8) on
 * every axis:  s = R x (the ray from the sensor to the world point
 * p = s + t), l = |x|, q = tau / l,
 *   e0 = (t + max(0, 1 - q) s) / nu + 1/2,   e1 = (t + (1 + q) s) / nu + 1/2,
 * i.e. the symmetric band [p - tau d, p + tau d], d = s / l, started at the
 * sensor when l < tau.
 */
void band_endpoints(const Map &m, const double R[9], const double t[3], const float x[3], double e0[3],
                    double e1[3], double *len) {
    const double X = x[0], Y = x[1], Z = x[2];
    const double l = std::sqrt(X * X + Y * Y + Z * Z);
    const double q = m.tau / l;
    const double f0 = std::max(0.0, 1.0 - q), f1 = 1.0 + q;
    for (int k = 0; k < 3; ++k) {
        const double sk = (R[3 * k] * X + R[3 * k + 1] * Y) + R[3 * k + 2] * Z;
        e0[k] = (t[k] + f0 * sk) / m.nu + 0.5;
        e1[k] = (t[k] + f1 * sk) / m.nu + 0.5;
    }
    if (len) *len = l;
}

/*
 * Clearance of block b from the segment e(u) = e0 + u (e1 - e0), u in [0, 1]:
 * the largest, over the segment's points, of the distance from the point to
 * the nearest face of b's box [8b, 8b + 8)^3, counted negative outside the
 * box (an L-infinity depth).  It is the maximum over u of the minimum of six
 * linear functions, a concave piecewise-linear function, so its maximum lies
 * at u = 0, u = 1 or where two of the six lines cross: all are evaluated.
 * Positive: the segment runs through the block's interior; negative: it
 * misses the block; zero: it touches the boundary.
 */
double block_clearance(const double e0[3], const double e1[3], const I3 &b) {
    double a[6], sl[6];
    const int64_t bb[3] = {b.x, b.y, b.z};
    for (int k = 0; k < 3; ++k) {
        const double lo = 8.0 * (double)bb[k], hi = lo + 8.0, d = e1[k] - e0[k];
        a[2 * k] = e0[k] - lo;          // distance above the lower face
        sl[2 * k] = d;
        a[2 * k + 1] = hi - e0[k];      // distance below the upper face
        sl[2 * k + 1] = -d;
    }
    auto depth = [&](double u) {
        double v = INFINITY;
        for (int j = 0; j < 6; ++j) v = std::min(v, a[j] + sl[j] * u);
        return v;
    };
    double best = std::max(depth(0.0), depth(1.0));
    for (int i = 0; i < 6; ++i)
        for (int j = i + 1; j < 6; ++j) {
            if (sl[i] == sl[j]) continue;
            const double u = (a[j] - a[i]) / (sl[i] - sl[j]);
            if (u > 0.0 && u < 1.0) best = std::max(best, depth(u));
        }
    return best;
}

/*
 * Half-width (voxel units) of the band of clearances within which an IEEE
 * single-precision evaluation of the endpoints (R / nu and t / nu + 1/2
 * rounded to FP32, a few roundings of magnitude |t / nu| + |s| / nu) may
 * place the segment on the other side of a block face: 2^-20 (16 units of
 * single-precision roundoff) times the magnitudes involved.
 */
double band_margin(const Map &m, const double t[3], double len) {
    const double T = std::max(std::fabs(t[0]), std::max(std::fabs(t[1]), std::fabs(t[2]))) / m.nu + 0.5;
    const double S = (len + m.tau) / m.nu;
    return std::ldexp(T + 2.0 * S + 16.0, -20);
}

/*
 * Blocks met by the band of one point: `sure` those whose clearance exceeds
 * the margin (every faithful evaluation allocates them), `amb` those within
 * the margin of zero (an FP32 evaluation may take them or not).  Candidates
 * are the blocks overlapping the segment's bounding box widened by the
 * margin.
 */
void band_blocks(const double e0[3], const double e1[3], double margin, std::vector<I3> &sure,
                 std::vector<I3> &amb) {
    int64_t lo[3], hi[3];
    for (int k = 0; k < 3; ++k) {
        lo[k] = (int64_t)std::floor((std::min(e0[k], e1[k]) - margin) / 8.0);
        hi[k] = (int64_t)std::floor((std::max(e0[k], e1[k]) + margin) / 8.0);
    }
    for (int64_t x = lo[0]; x <= hi[0]; ++x)
        for (int64_t y = lo[1]; y <= hi[1]; ++y)
            for (int64_t z = lo[2]; z <= hi[2]; ++z) {
                const I3 b{x, y, z};
                const double c = block_clearance(e0, e1, b);
                if (c > margin) sure.push_back(b);
                else if (c >= -margin) amb.push_back(b);
            }
}

inline double dist_to_int(double a) { return std::fabs(a - std::floor(a + 0.5)); }

inline double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

// ---------------------------------------------------------------------------
// non-projective distance (Sec. III-C.2, Eq. distance)
// ---------------------------------------------------------------------------
// Unit ray of pixel (v, u): polar angle theta0 + v dtheta, azimuth pi - u dphi
// (the range-image model of Sec. III-C.1 read backwards).
inline void pixel_ray(const Lidar &L, int64_t v, int64_t u, double dir[3]) {
    const double th = L.theta0 + (double)v * L.dtheta, ph = PI - (double)u * L.dphi;
    dir[0] = std::sin(th) * std::cos(ph);
    dir[1] = std::sin(th) * std::sin(ph);
    dir[2] = std::cos(th);
}

/*
 * Normal image N (Sec. III-C.2): p_j is the pixel's range r(u, v) along its
 * ray, p_j1 the same for pixel (u, v - 1), p_j2 for (u - 1, v) (columns wrap
 * around the scan); N(u, v) = (p_j1 - p_j) x (p_j2 - p_j) / |...|, turned to
 * face the sensor (N . p_j <= 0), rotated into the world frame by R.  No
 * normal on the top row, next to a pixel without a return, or where the
 * cross product vanishes.  flag bit 0: valid; bit 1: |N . p_j| / |p_j| below
 * 1e-5 (an FP32 evaluation may turn the normal the other way).
 */
void normal_image(const Lidar &L, const std::vector<double> &range, const double R[9], std::vector<double> &N,
                  std::vector<uint8_t> &flag) {
    const int64_t NP = (int64_t)L.H * L.W;
    N.assign((size_t)NP * 3, 0.0);
    flag.assign(NP, 0);
    for (int64_t v = 1; v < L.H; ++v)
        for (int64_t u = 0; u < L.W; ++u) {
            const int64_t p = v * L.W + u, p1 = (v - 1) * L.W + u, p2 = v * L.W + (u + L.W - 1) % L.W;
            if (range[p] < 0.0 || range[p1] < 0.0 || range[p2] < 0.0) continue;
            double d0[3], d1[3], d2[3], q[3], q1[3], q2[3];
            pixel_ray(L, v, u, d0);
            pixel_ray(L, v - 1, u, d1);
            pixel_ray(L, v, (u + L.W - 1) % L.W, d2);
            for (int k = 0; k < 3; ++k) {
                q[k] = range[p] * d0[k];
                q1[k] = range[p1] * d1[k];
                q2[k] = range[p2] * d2[k];
            }
            const double a[3] = {q1[0] - q[0], q1[1] - q[1], q1[2] - q[2]};
            const double b[3] = {q2[0] - q[0], q2[1] - q[1], q2[2] - q[2]};
            double c[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
            const double len = std::sqrt(dot3(c, c));
            if (!(len > 0.0)) continue;
            for (int k = 0; k < 3; ++k) c[k] /= len;
            const double facing = dot3(c, q);
            if (facing > 0.0)
                for (int k = 0; k < 3; ++k) c[k] = -c[k];
            uint8_t f = 1;
            if (std::fabs(facing) < 1e-5 * range[p]) f |= 2;
            for (int k = 0; k < 3; ++k) N[3 * p + k] = R[3 * k] * c[0] + R[3 * k + 1] * c[1] + R[3 * k + 2] * c[2];
            flag[p] = f;
        }
}

/*
 * d_i of Eq. (distance) for a voxel at projective distance psi, with u the
 * unit ray from the voxel toward the sensor, g its gradient (zero: none yet)
 * and N the normal of its pixel (null: none).  theta is the angle between
 * the ray and g, alpha the angle between g and N.  For a circle through the
 * ray's surface point p_j with normal N whose point nearest the voxel has
 * normal g (the figure's curved surface), the law of sines in the triangle
 * (centre, p_j, voxel) gives the exact distance
 *   d = psi (cos theta + sin theta (cos alpha - 1) / sin alpha)
 *     = psi (cos theta - sin theta tan(alpha / 2)),
 * alpha > 0 when g is turned from N toward the ray (convex) and < 0 away
 * from it (concave).  The signed sin alpha is g's component along the unit
 * tangent t = (u - (u.N) N) / |u - (u.N) N| and tan(alpha / 2) =
 * sin alpha / (1 + cos alpha).  taint receives 1 where an FP32 evaluation
 * may take another branch or lose the tangent's direction.
 */
double nonprojective_distance(double psi, const double u[3], const double g[3], const double *N, uint8_t *taint) {
    if (!(dot3(g, g) > 0.0)) return psi;
    const double ct = std::fabs(dot3(g, u));
    if (!N) return ct * psi;
    const double ca = dot3(g, N);
    if (std::fabs(ca) < 1e-6 && taint) *taint |= 1;
    if (!(ca > 0.0)) return ct * psi;
    const double un = dot3(u, N);
    const double up[3] = {u[0] - un * N[0], u[1] - un * N[1], u[2] - un * N[2]};
    const double len = std::sqrt(dot3(up, up));
    if (len < 1e-3 && taint) *taint |= 1;
    if (!(len > 0.0)) return ct * psi;
    const double sa = dot3(g, up) / len;
    const double st = std::sqrt(std::max(0.0, 1.0 - ct * ct));
    return psi * (ct - st * sa / (1.0 + ca));
}

// ---------------------------------------------------------------------------
// one frame
// ---------------------------------------------------------------------------
// Candidate pixels of a projection (u_c, v_c) (Sec. III-C.1, rounding half
// up): the FP64 pixel first and, within delta_px of a rounding boundary, the
// pixel on the other side of it too (-1 for a row outside [0, H)).  Returns
// the number written.
int pixel_candidates(const Lidar &L, double uc, double vc, double delta, int64_t out[4], bool *amb) {
    int64_t us[2], vs[2];
    int nu_ = 1, nv_ = 1;
    us[0] = (int64_t)std::floor(uc + 0.5);
    vs[0] = (int64_t)std::floor(vc + 0.5);
    const double bu = std::floor(uc + 0.5 + 0.5), bv = std::floor(vc + 0.5 + 0.5);   // nearest boundaries
    if (std::fabs(uc + 0.5 - bu) < delta) {
        us[1] = us[0] == (int64_t)bu ? (int64_t)bu - 1 : (int64_t)bu;
        nu_ = 2;
    }
    if (std::fabs(vc + 0.5 - bv) < delta) {
        vs[1] = vs[0] == (int64_t)bv ? (int64_t)bv - 1 : (int64_t)bv;
        nv_ = 2;
    }
    *amb = nu_ > 1 || nv_ > 1;
    int n = 0;
    for (int j = 0; j < nv_; ++j)
        for (int i = 0; i < nu_; ++i) {
            const int64_t u = ((us[i] % L.W) + L.W) % L.W, v = vs[j];
            out[n++] = (v < 0 || v >= L.H) ? -1 : v * L.W + u;
        }
    return n;
}

int integrate(Map &m, const Lidar &L, const float *pts, const int32_t *labels, const float *probs,
              int64_t n, const double T[16], int nthreads, const Decisions *dec) {
    m.st = Stats();
    std::memset(m.check, 0, sizeof(m.check));
    int64_t *ck = m.check;
    const int C = m.C;
    double R[9], t[3];
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) R[3 * r + c] = T[4 * r + c];
        t[r] = T[4 * r + 3];
    }
    const int64_t NP = (int64_t)L.H * L.W;
    const double eps_r = std::ldexp(1.0, -20);   // relative range band of FP32 range decisions

    // --- measurement preprocessing: range image (Sec. III-C.1) -------------
    // validity (finite, r_min <= r <= r_max) and pixel of each point, FP64
    std::vector<int64_t> ppix(n, -2);            // pixel, -1 valid without one, -2 invalid
    for (int64_t i = 0; i < n; ++i) {
        const float x = pts[3 * i], y = pts[3 * i + 1], z = pts[3 * i + 2];
        if (!(std::isfinite(x) && std::isfinite(y) && std::isfinite(z))) {
            if (dec && dec->point_pix) {
                ck[CK_POINTS]++;
                if (dec->point_pix[i] != -2) ck[CK_POINTS_BAD]++;
            }
            continue;
        }
        const double X = x, Y = y, Z = z;
        const double r = std::sqrt(X * X + Y * Y + Z * Z);
        bool valid = r >= L.r_min && r <= L.r_max && r > 0.0;
        const bool amb_valid = std::fabs(r - L.r_min) <= eps_r * r || std::fabs(r - L.r_max) <= eps_r * r;
        int64_t cand[4] = {-1, -1, -1, -1};
        int nc = 0;
        bool amb_pix = false;
        if (r > 0.0) {
            const double uc = (PI - std::atan2(Y, X)) / L.dphi;
            const double vc = (std::acos(Z / r) - L.theta0) / L.dtheta;
            nc = pixel_candidates(L, uc, vc, m.delta_px, cand, &amb_pix);
        }
        int64_t pix = valid ? cand[0] : -2;
        if (amb_valid || (valid && amb_pix)) m.st.ambiguous_points++;
        if (dec && dec->point_pix) {
            const int64_t g = dec->point_pix[i];
            ck[CK_POINTS]++;
            bool ok;
            if (g == -2) ok = !valid || amb_valid;
            else {
                ok = (valid || amb_valid) && r > 0.0;
                bool in = false;
                for (int j = 0; j < nc; ++j) in = in || cand[j] == g;
                ok = ok && in && (g == pix || amb_pix || !valid);
            }
            if (!ok) ck[CK_POINTS_BAD]++;
            else {
                if (amb_valid || amb_pix) ck[CK_POINTS_AMB]++;
                pix = g;
            }
        }
        ppix[i] = pix;
        if (pix == -2) continue;
        m.st.valid_points++;
        if (pix >= 0) m.st.pixel_points++;
    }
    // nearest point wins the pixel (equal ranges: the lower index); FP64 ranges
    std::vector<int64_t> win(NP, -1);
    std::vector<double> win_r(NP, INFINITY);
    std::vector<double> rng(n, 0.0);
    for (int64_t i = 0; i < n; ++i) {
        if (ppix[i] == -2) continue;
        const double X = pts[3 * i], Y = pts[3 * i + 1], Z = pts[3 * i + 2];
        rng[i] = std::sqrt(X * X + Y * Y + Z * Z);
        const int64_t p = ppix[i];
        if (p < 0) continue;
        if (rng[i] < win_r[p] || (rng[i] == win_r[p] && i < win[p])) {
            win[p] = i;
            win_r[p] = rng[i];
        }
    }
    if (dec && dec->winner) {
        // candidates: the pixel's points within the FP32 range band of its nearest range
        std::vector<uint8_t> cand(n, 0);
        std::vector<int32_t> ncand(NP, 0);
        for (int64_t i = 0; i < n; ++i)
            if (ppix[i] >= 0 && rng[i] <= win_r[ppix[i]] * (1.0 + eps_r)) {
                cand[i] = 1;
                ncand[ppix[i]]++;
            }
        for (int64_t p = 0; p < NP; ++p) {
            const uint64_t g = dec->winner[p];
            const int64_t gi = g == ~0ull ? -1 : (int64_t)(g & 0xffffffffull);
            ck[CK_PIXELS]++;
            const bool ok = gi == win[p] || (gi >= 0 && win[p] >= 0 && gi < n && ppix[gi] == p && cand[gi]);
            if (!ok) ck[CK_WINNERS_BAD]++;
            else {
                if (ncand[p] > 1) ck[CK_WINNERS_AMB]++;
                win[p] = gi;
                win_r[p] = gi >= 0 ? rng[gi] : INFINITY;
            }
        }
    }
    // per-pixel log-likelihood of each class (Eq. bayesian_filter's P(O = l | I_k))
    std::vector<double> logL;
    std::vector<uint8_t> has_sem(NP, 0);
    logL.assign((size_t)NP * C, 0.0);
    for (int64_t p = 0; p < NP; ++p) {
        int64_t i = win[p];
        if (i < 0) continue;
        double *row = &logL[(size_t)p * C];
        if (probs) {
            for (int c = 0; c < C; ++c) row[c] = std::log(std::max((double)probs[(size_t)i * C + c], m.lik_floor));
            has_sem[p] = 1;
        } else if (labels && labels[i] >= 0 && labels[i] < C) {
            double lo = std::log((1.0 - m.p_hit) / (C - 1)), hi = std::log(m.p_hit);
            for (int c = 0; c < C; ++c) row[c] = (c == labels[i]) ? hi : lo;
            has_sem[p] = 1;
        }
    }

    // --- normal image (non-projective mode, Sec. III-C.2) ---------------------
    if (m.dist_mode == 1) {
        std::vector<double> range(NP, -1.0);
        for (int64_t p = 0; p < NP; ++p) {
            const int64_t i = win[p];
            if (i < 0) continue;
            const double X = pts[3 * i], Y = pts[3 * i + 1], Z = pts[3 * i + 2];
            range[p] = std::sqrt(X * X + Y * Y + Z * Z);
        }
        normal_image(L, range, R, m.normals, m.normal_flag);
    }

    // --- block allocation along each point's truncation band (FP64) ----------
    std::unordered_set<I3, I3Hash> sure, amb;
    {
        std::vector<I3> vs, va;
        for (int64_t i = 0; i < n; ++i) {
            if (ppix[i] == -2) continue;
            double e0[3], e1[3], len;
            band_endpoints(m, R, t, &pts[3 * i], e0, e1, &len);
            vs.clear();
            va.clear();
            band_blocks(e0, e1, band_margin(m, t, len), vs, va);
            for (const I3 &b : vs) sure.insert(b);
            for (const I3 &b : va) amb.insert(b);
        }
        for (const I3 &b : sure) amb.erase(b);
    }
    m.st.sure_blocks = (int64_t)sure.size();
    m.st.ambiguous_blocks = (int64_t)amb.size();
    std::unordered_set<I3, I3Hash> touched;
    if (dec && dec->touched) {
        // accept the recorded set when sure <= it <= sure + ambiguous
        ck[CK_BLOCKS_SURE] = (int64_t)sure.size();
        ck[CK_BLOCKS_AMB] = (int64_t)amb.size();
        for (int64_t j = 0; j < dec->n_touched; ++j) {
            const I3 b{dec->touched[3 * j], dec->touched[3 * j + 1], dec->touched[3 * j + 2]};
            if (sure.count(b)) touched.insert(b);
            else if (amb.count(b)) {
                touched.insert(b);
                ck[CK_BLOCKS_AMB_TAKEN]++;
            } else {
                ck[CK_BLOCKS_EXTRA]++;
            }
        }
        for (const I3 &b : sure)
            if (!touched.count(b)) {
                ck[CK_BLOCKS_MISSING]++;
                touched.insert(b);
            }
    } else {
        // alone: the sure blocks and the ambiguous ones the exact segment touches
        touched = sure;
        for (const I3 &b : amb) touched.insert(b);
    }
    m.touched.assign(touched.begin(), touched.end());
    std::sort(m.touched.begin(), m.touched.end());
    m.st.touched_blocks = (int64_t)m.touched.size();
    std::vector<Block *> work;
    std::vector<I3> work_key;
    std::vector<const int32_t *> work_rec;
    std::unordered_map<I3, const int32_t *, I3Hash> recs;
    if (dec && dec->vox)
        for (int64_t j = 0; j < dec->n_touched; ++j)
            recs[{dec->touched[3 * j], dec->touched[3 * j + 1], dec->touched[3 * j + 2]}] = dec->vox + j * BV;
    for (const I3 &b : m.touched) {
        if (m.alloc.insert(b).second) m.st.new_blocks++;
        if (m.track && !m.track_keys.count(b)) continue;
        auto it = m.blocks.find(b);
        if (it == m.blocks.end()) it = m.blocks.emplace(b, new_block(C, m.dist_mode)).first;
        work.push_back(&it->second);
        work_key.push_back(b);
        const int32_t *rec = nullptr;
        if (dec && dec->vox) {
            auto r = recs.find(b);
            if (r == recs.end()) ck[CK_VOX_NO_RECORD]++;
            else rec = r->second;
        }
        work_rec.push_back(rec);
    }

    // --- projective TSDF + Bayesian semantic update, per voxel ----------------
    const double nu = m.nu, tau = m.tau;
    const bool follow = dec && dec->vox;
    int64_t n_upd = 0, n_sem = 0, n_seen = 0, n_taint = 0;
    int64_t c_vox = 0, c_pa = 0, c_pb = 0, c_ua = 0, c_ub = 0, c_sa = 0, c_sb = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4) \
    reduction(+ : n_upd, n_sem, n_seen, n_taint, c_vox, c_pa, c_pb, c_ua, c_ub, c_sa, c_sb)
#endif
    for (int64_t wi = 0; wi < (int64_t)work.size(); ++wi) {
        Block &blk = *work[wi];
        const I3 bk = work_key[wi];
        const int32_t *rec = work_rec[wi];
        std::vector<double> a(C);
        for (int lz = 0; lz < BS; ++lz)
            for (int ly = 0; ly < BS; ++ly)
                for (int lx = 0; lx < BS; ++lx) {
                    const int vi = vidx(lx, ly, lz);
                    // the recorded choices of this voxel: pixel, updated, class update
                    const int64_t gpix = rec ? (int64_t)(rec[vi] & 0x0fffffff) - 1 : -2;
                    const bool gupd = rec && ((rec[vi] >> 28) & 1), gsem = rec && ((rec[vi] >> 29) & 1);
                    if (rec) c_vox++;
                    // voxel centre x_i = nu * v_i (Sec. III-C.2)
                    double xw[3] = {nu * (double)(BS * bk.x + lx), nu * (double)(BS * bk.y + ly),
                                    nu * (double)(BS * bk.z + lz)};
                    double d[3] = {xw[0] - t[0], xw[1] - t[1], xw[2] - t[2]};
                    double xl[3];
                    for (int k = 0; k < 3; ++k) xl[k] = R[k] * d[0] + R[3 + k] * d[1] + R[6 + k] * d[2];
                    double rho = std::sqrt(xl[0] * xl[0] + xl[1] * xl[1] + xl[2] * xl[2]);
                    if (!(rho > 0.0)) {
                        if (rec && (gpix != -1 || gupd || gsem)) c_pb++;
                        continue;
                    }
                    n_seen++;
                    const double uc = (PI - std::atan2(xl[1], xl[0])) / L.dphi;
                    const double vc = (std::acos(xl[2] / rho) - L.theta0) / L.dtheta;
                    int64_t cand[4];
                    bool amb_pix = false;
                    const int nc = pixel_candidates(L, uc, vc, m.delta_px, cand, &amb_pix);
                    int64_t p = cand[0];
                    if (follow && rec) {
                        bool in = false;
                        for (int j = 0; j < nc; ++j) in = in || cand[j] == gpix;
                        if (!in) c_pb++;
                        else {
                            if (amb_pix) c_pa++;
                            p = gpix;
                        }
                    } else if (amb_pix) {
                        blk.taint[vi] |= 3;
                        n_taint++;
                    }
                    const bool amb_psi_lo_rec = follow && rec;
                    auto no_update = [&]() {
                        if (rec && (gupd || gsem)) c_ub++;
                    };
                    if (p < 0) {
                        no_update();
                        continue;
                    }
                    int64_t wpt = win[p];
                    if (wpt < 0) {
                        no_update();
                        continue;
                    }
                    double P0 = pts[3 * wpt], P1 = pts[3 * wpt + 1], P2 = pts[3 * wpt + 2];
                    double r = std::sqrt(P0 * P0 + P1 * P1 + P2 * P2);
                    // projective signed distance along the ray: > 0 in front of the surface
                    double psi = r - rho;
                    // update iff psi > -tau (psi >= -tau and a positive weight)
                    bool upd = psi >= -tau && (m.weight_mode != 0 || psi + tau > 0.0);
                    if (std::fabs(psi + tau) < m.eps_psi) {
                        if (amb_psi_lo_rec) {
                            c_ua++;
                            upd = gupd;
                        } else {
                            blk.taint[vi] |= 3;
                            n_taint++;
                        }
                    } else if (rec && gupd != upd) {
                        c_ub++;
                    }
                    if (!upd) continue;
                    double w;
                    if (m.weight_mode == 0) {
                        // linear weight (psi + tau) / (2 tau), clamped to [0, 1]
                        w = (psi + tau) / (2.0 * tau);
                        if (w > 1.0) w = 1.0;
                        if (w < 0.0) w = 0.0;
                    } else {
                        w = 1.0;
                    }
                    double Wo = blk.W[vi];
                    double dist = psi;
                    if (m.dist_mode == 1) {
                        // gradient g_i: weight-averaged normal of the pixels seen, renormalised
                        const double *Nw = (m.normal_flag[p] & 1) ? &m.normals[3 * p] : nullptr;
                        if (m.normal_flag[p] & 2) { blk.taint[vi] |= 3; n_taint++; }
                        double g[3] = {blk.G[vi], blk.G[BV + vi], blk.G[2 * BV + vi]};
                        if (Nw) {
                            double gs[3];
                            for (int k = 0; k < 3; ++k) gs[k] = Wo * g[k] + w * Nw[k];
                            const double gl = std::sqrt(dot3(gs, gs));
                            if (gl < 1e-6 * (Wo + w)) { blk.taint[vi] |= 3; n_taint++; }
                            if (gl > 0.0)
                                for (int k = 0; k < 3; ++k) g[k] = gs[k] / gl;
                            for (int k = 0; k < 3; ++k) blk.G[k * BV + vi] = g[k];
                        }
                        // unit ray from the voxel toward the sensor (world frame)
                        const double uw[3] = {-d[0] / rho, -d[1] / rho, -d[2] / rho};
                        uint8_t tf = 0;
                        dist = nonprojective_distance(psi, uw, g, Nw, &tf);
                        if (tf) { blk.taint[vi] |= 3; n_taint++; }
                    }
                    // truncation Gamma(d, tau): min(d, tau) for d >= 0, max(d, -tau) otherwise
                    double sdf = dist >= 0.0 ? std::min(dist, tau) : std::max(dist, -tau);
                    blk.D[vi] = (Wo * blk.D[vi] + w * sdf) / (Wo + w);
                    blk.W[vi] = Wo + w;
                    n_upd++;
                    blk.nupd[vi]++;
                    // class update: the surface band |psi| <= tau, a pixel with a likelihood
                    bool sem = std::fabs(psi) <= tau && has_sem[p];
                    if (std::fabs(psi - tau) < m.eps_psi && has_sem[p]) {
                        if (follow && rec) {
                            c_sa++;
                            sem = gsem;
                        } else {
                            blk.taint[vi] |= 2;
                            n_taint++;
                        }
                    } else if (rec && gsem != sem) {
                        c_sb++;
                    }
                    if (sem) {
                        // recursive Bayesian update in log space, normalised by Z
                        const double *lrow = &logL[(size_t)p * C];
                        double mx = -INFINITY;
                        for (int c = 0; c < C; ++c) {
                            a[c] = blk.logP[(size_t)c * BV + vi] + lrow[c];
                            mx = std::max(mx, a[c]);
                        }
                        double s = 0.0;
                        for (int c = 0; c < C; ++c) s += std::exp(a[c] - mx);
                        double lse = mx + std::log(s);
                        for (int c = 0; c < C; ++c)
                            blk.logP[(size_t)c * BV + vi] = std::max(a[c] - lse, m.logp_floor);
                        n_sem++;
                        blk.nsem[vi]++;
                    }
                }
    }
    m.st.voxels_updated = n_upd;
    m.st.voxels_semantic = n_sem;
    m.st.voxels_seen = n_seen;
    ck[CK_VOXELS] = c_vox;
    ck[CK_VOX_PIX_AMB] = c_pa;
    ck[CK_VOX_PIX_BAD] = c_pb;
    ck[CK_VOX_UPD_AMB] = c_ua;
    ck[CK_VOX_UPD_BAD] = c_ub;
    ck[CK_VOX_SEM_AMB] = c_sa;
    ck[CK_VOX_SEM_BAD] = c_sb;
    m.st.taint_events = n_taint;
    m.frame++;
    return 0;
}

// ---------------------------------------------------------------------------
// voxel access
// ---------------------------------------------------------------------------
struct VoxRef {
    const Block *b = nullptr;
    int vi = 0;
};

VoxRef voxel(const Map &m, int64_t x, int64_t y, int64_t z) {
    VoxRef r;
    I3 k{floordiv(x, BS), floordiv(y, BS), floordiv(z, BS)};
    auto it = m.blocks.find(k);
    if (it == m.blocks.end()) return r;
    r.b = &it->second;
    r.vi = vidx((int)(x - BS * k.x), (int)(y - BS * k.y), (int)(z - BS * k.z));
    return r;
}

// most probable class, lowest index on exact ties; gap to the runner-up
int argmax_label(const Map &m, const Block &b, int vi, double *gap) {
    int best = 0;
    double bv = b.logP[vi], second = -INFINITY;
    for (int c = 1; c < m.C; ++c) {
        double v = b.logP[(size_t)c * BV + vi];
        if (v > bv) { second = bv; bv = v; best = c; }
        else if (v > second) second = v;
    }
    if (gap) *gap = m.C > 1 ? bv - second : INFINITY;
    return best;
}

// ---------------------------------------------------------------------------
// marching cubes by face walk (no case table)
// ---------------------------------------------------------------------------
struct MeshVertex {
    double pos[3];
    int label;
    double gap;
    uint8_t taint;
};
struct MeshTri {
    int64_t k[3];
    I3 anchor;      // voxel anchoring the cube (its lowest corner)
    uint8_t taint;
};
struct Mesh {
    std::map<int64_t, MeshVertex> verts;
    std::vector<MeshTri> tris;
};

struct Face { int c[4]; };   // corners counter-clockwise about the outward normal

// Derive the six faces of the unit cube with corners id = dx + 2 dy + 4 dz.
std::vector<Face> cube_faces() {
    std::vector<Face> faces;
    for (int axis = 0; axis < 3; ++axis)
        for (int side = 0; side < 2; ++side) {
            int a1 = (axis + 1) % 3, a2 = (axis + 2) % 3;
            // square (0,0),(1,0),(1,1),(0,1) in the (a1, a2) plane; a1 x a2 = +axis
            int uv[4][2] = {{0, 0}, {1, 0}, {1, 1}, {0, 1}};
            Face f;
            for (int j = 0; j < 4; ++j) {
                int off[3] = {0, 0, 0};
                off[axis] = side;
                off[a1] = uv[j][0];
                off[a2] = uv[j][1];
                f.c[j] = off[0] + 2 * off[1] + 4 * off[2];
            }
            if (side == 0) std::swap(f.c[1], f.c[3]);   // outward normal is -axis: reverse
            faces.push_back(f);
        }
    return faces;
}

// Mesh the cubes anchored in block bk; vertices are keyed globally.
void mesh_block(const Map &m, const I3 &bk, Mesh &out) {
    static const std::vector<Face> faces = cube_faces();
    if (m.blocks.find(bk) == m.blocks.end()) return;
    for (int lz = 0; lz < BS; ++lz)
        for (int ly = 0; ly < BS; ++ly)
            for (int lx = 0; lx < BS; ++lx) {
                int64_t ax = BS * bk.x + lx, ay = BS * bk.y + ly, az = BS * bk.z + lz;
                double Dc[8];
                bool in[8];
                VoxRef vr[8];
                bool ok = true;
                uint8_t ctaint = 0;
                for (int c = 0; c < 8 && ok; ++c) {
                    vr[c] = voxel(m, ax + (c & 1), ay + ((c >> 1) & 1), az + ((c >> 2) & 1));
                    if (!vr[c].b || !(vr[c].b->W[vr[c].vi] > 0.0)) { ok = false; break; }
                    Dc[c] = vr[c].b->D[vr[c].vi];
                    in[c] = Dc[c] < 0.0;
                    if (std::fabs(Dc[c]) < 1e-6) ctaint |= 1;
                    ctaint |= vr[c].b->taint[vr[c].vi] & 1;
                }
                // also taint when any corner might be observed on one side only
                if (!ok) continue;
                int nin = 0;
                for (int c = 0; c < 8; ++c) nin += in[c];
                if (nin == 0 || nin == 8) continue;
                // vertex of the crossing edge between corners ca, cb (differ in one axis)
                auto vkey = [&](int ca, int cb) -> int64_t {
                    int lo = std::min(ca, cb), hi = std::max(ca, cb);
                    int axis = (hi - lo) == 1 ? 0 : ((hi - lo) == 2 ? 1 : 2);
                    int64_t k = edge_key(ax + (lo & 1), ay + ((lo >> 1) & 1), az + ((lo >> 2) & 1), axis);
                    if (!out.verts.count(k)) {
                        double Da = Dc[lo], Db = Dc[hi];
                        double tt = Da / (Da - Db);
                        double base[3] = {(double)(ax + (lo & 1)), (double)(ay + ((lo >> 1) & 1)),
                                          (double)(az + ((lo >> 2) & 1))};
                        MeshVertex mv;
                        for (int q = 0; q < 3; ++q) mv.pos[q] = m.nu * base[q];
                        mv.pos[axis] = m.nu * (base[axis] + tt);
                        // label from the endpoint nearer the surface (lower end on ties)
                        int pick = std::fabs(Db) < std::fabs(Da) ? hi : lo;
                        mv.label = argmax_label(m, *vr[pick].b, vr[pick].vi, &mv.gap);
                        mv.taint = (uint8_t)(vr[pick].b->taint[vr[pick].vi] | vr[lo].b->taint[vr[lo].vi] |
                                             vr[hi].b->taint[vr[hi].vi]);
                        out.verts.emplace(k, mv);
                    }
                    return k;
                };
                // directed segments: on each face, each entering edge (out -> in,
                // counter-clockwise) joins the next leaving edge (in -> out)
                std::map<int64_t, int64_t> next;
                for (const Face &f : faces) {
                    for (int j = 0; j < 4; ++j) {
                        int ca = f.c[j], cb = f.c[(j + 1) % 4];
                        if (!(!in[ca] && in[cb])) continue;
                        for (int s = 1; s < 4; ++s) {
                            int cc = f.c[(j + s) % 4], cd = f.c[(j + s + 1) % 4];
                            if (in[cc] && !in[cd]) {
                                next[vkey(ca, cb)] = vkey(cc, cd);
                                break;
                            }
                        }
                    }
                }
                // loops, each fanned from its lowest key
                std::unordered_set<int64_t> seen;
                for (auto &kv : next) {
                    if (seen.count(kv.first)) continue;
                    std::vector<int64_t> loop;
                    int64_t cur = kv.first;
                    while (!seen.count(cur)) {
                        seen.insert(cur);
                        loop.push_back(cur);
                        cur = next.at(cur);
                    }
                    auto mn = std::min_element(loop.begin(), loop.end());
                    std::rotate(loop.begin(), mn, loop.end());
                    for (size_t q = 1; q + 1 < loop.size(); ++q) {
                        MeshTri tr;
                        tr.k[0] = loop[0];
                        tr.k[1] = loop[q];
                        tr.k[2] = loop[q + 1];
                        tr.anchor = {ax, ay, az};
                        tr.taint = ctaint;
                        out.tris.push_back(tr);
                    }
                }
            }
}

// ---------------------------------------------------------------------------
// trilinear SDF query and its gradients
// ---------------------------------------------------------------------------
bool query(const Map &m, const double x[3], double *sdf, double grad[3]) {
    double g[3], f[3];
    int64_t v0[3];
    for (int k = 0; k < 3; ++k) {
        g[k] = x[k] / m.nu;
        v0[k] = (int64_t)std::floor(g[k]);
        f[k] = g[k] - (double)v0[k];
    }
    double Dc[8];
    for (int c = 0; c < 8; ++c) {
        VoxRef r = voxel(m, v0[0] + (c & 1), v0[1] + ((c >> 1) & 1), v0[2] + ((c >> 2) & 1));
        if (!r.b || !(r.b->W[r.vi] > 0.0)) {
            *sdf = NAN;
            if (grad) grad[0] = grad[1] = grad[2] = 0.0;
            return false;
        }
        Dc[c] = r.b->D[r.vi];
    }
    double s = 0.0, dg[3] = {0.0, 0.0, 0.0};
    for (int c = 0; c < 8; ++c) {
        int b[3] = {c & 1, (c >> 1) & 1, (c >> 2) & 1};
        double wk[3], dk[3];
        for (int k = 0; k < 3; ++k) {
            wk[k] = b[k] ? f[k] : 1.0 - f[k];
            dk[k] = b[k] ? 1.0 : -1.0;
        }
        s += wk[0] * wk[1] * wk[2] * Dc[c];
        dg[0] += dk[0] * wk[1] * wk[2] * Dc[c];
        dg[1] += wk[0] * dk[1] * wk[2] * Dc[c];
        dg[2] += wk[0] * wk[1] * dk[2] * Dc[c];
    }
    *sdf = s;
    if (grad)
        for (int k = 0; k < 3; ++k) grad[k] = dg[k] / m.nu;
    return true;
}

// SE(3) exponential of (rho, phi): rotation by Rodrigues' formula, translation V(phi) rho.
void se3_exp(const double xi[6], double R[9], double t[3]) {
    const double *rho = xi, *phi = xi + 3;
    double th = std::sqrt(phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2]);
    double K[9] = {0, -phi[2], phi[1], phi[2], 0, -phi[0], -phi[1], phi[0], 0};
    double K2[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0;
            for (int k = 0; k < 3; ++k) s += K[3 * i + k] * K[3 * k + j];
            K2[3 * i + j] = s;
        }
    double A, Bc, Cc;
    if (th < 1e-8) {
        A = 1.0 - th * th / 6.0;
        Bc = 0.5 - th * th / 24.0;
        Cc = 1.0 / 6.0 - th * th / 120.0;
    } else {
        A = std::sin(th) / th;
        Bc = (1.0 - std::cos(th)) / (th * th);
        Cc = (th - std::sin(th)) / (th * th * th);
    }
    double V[9];
    for (int i = 0; i < 9; ++i) {
        double I = (i % 4 == 0) ? 1.0 : 0.0;
        R[i] = I + A * K[i] + Bc * K2[i];
        V[i] = I + Bc * K[i] + Cc * K2[i];
    }
    for (int i = 0; i < 3; ++i) t[i] = V[3 * i] * rho[0] + V[3 * i + 1] * rho[1] + V[3 * i + 2] * rho[2];
}

}  // namespace

// ===========================================================================
// C interface (ctypes)
// ===========================================================================
extern "C" {

void *orc_new(double voxel_size, double truncation, int n_classes, int weight_mode, double p_hit,
              double logp_floor, double lik_floor) {
    Map *m = new Map();
    m->nu = voxel_size;
    m->tau = truncation;
    m->C = n_classes;
    m->weight_mode = weight_mode;
    m->p_hit = p_hit;
    m->logp_floor = logp_floor;
    m->lik_floor = lik_floor;
    m->eps_psi = 1e-5 * voxel_size;
    return m;
}

void orc_free(void *h) { delete (Map *)h; }

// 0: projective psi, 1: non-projective d_i (Eq. distance); set before the first scan
void orc_set_distance_mode(void *h, int mode) { ((Map *)h)->dist_mode = mode; }

// the last scan's normal image (world frame) and flags; returns H * W (0 in projective mode)
int64_t orc_get_normals(void *h, double *N, uint8_t *flag, int64_t cap) {
    Map *m = (Map *)h;
    const int64_t np = (int64_t)m->normal_flag.size();
    const int64_t k = std::min(cap, np);
    if (N && k > 0) std::memcpy(N, m->normals.data(), sizeof(double) * 3 * k);
    if (flag && k > 0) std::memcpy(flag, m->normal_flag.data(), k);
    return np;
}

// one block's gradients G[3][512]; 0 when the block holds them, -1 otherwise
int orc_read_grad(void *h, const int32_t *coord, double *G) {
    Map *m = (Map *)h;
    auto it = m->blocks.find({coord[0], coord[1], coord[2]});
    if (it == m->blocks.end() || it->second.G.empty()) return -1;
    std::memcpy(G, it->second.G.data(), sizeof(double) * 3 * BV);
    return 0;
}

// d_i of Eq. (distance) for given psi, ray u, gradient g and normal N (has_n = 0: no normal)
double orc_nonproj_distance(double psi, const double *u, const double *g, const double *N, int has_n) {
    return nonprojective_distance(psi, u, g, has_n ? N : nullptr, nullptr);
}

void orc_set_bands(void *h, double delta_px, double eps_psi) {
    Map *m = (Map *)h;
    m->delta_px = delta_px;
    m->eps_psi = eps_psi;
}

// Keep voxel data only for the listed blocks; allocation is still tracked for all.
void orc_set_track(void *h, const int32_t *coords, int64_t n) {
    Map *m = (Map *)h;
    m->track = true;
    m->track_keys.clear();
    for (int64_t i = 0; i < n; ++i) m->track_keys.insert({coords[3 * i], coords[3 * i + 1], coords[3 * i + 2]});
}

// lidar6 = {H, W, fov_up, fov_down, r_min, r_max} (angles in radians).  The
// decision arguments (all may be null) are a single-precision implementation's
// choices for this scan, for candidate acceptance (struct Decisions).
int orc_integrate(void *h, const double *lidar6, const float *pts, const int32_t *labels, const float *probs,
                  int64_t n, const double *T16, int nthreads, const int32_t *point_pix, const uint64_t *winner,
                  const int32_t *touched, int64_t n_touched, const int32_t *vox_rec) {
    Map *m = (Map *)h;
    Lidar L;
    L.H = (int)lidar6[0];
    L.W = (int)lidar6[1];
    L.fov_up = lidar6[2];
    L.fov_down = lidar6[3];
    L.r_min = lidar6[4];
    L.r_max = lidar6[5];
    L.dphi = 2.0 * PI / L.W;
    L.dtheta = (L.fov_up - L.fov_down) / (L.H - 1);
    L.theta0 = PI / 2.0 - L.fov_up;
    Decisions d;
    d.point_pix = point_pix;
    d.winner = winner;
    d.touched = touched;
    d.n_touched = n_touched;
    d.vox = touched ? vox_rec : nullptr;
    const bool any = point_pix || winner || touched;
    return integrate(*m, L, pts, labels, probs, n, T16, nthreads, any ? &d : nullptr);
}

// candidate-acceptance counts of the last scan (CK_* order, CK_COUNT entries)
void orc_check(void *h, int64_t *out) { std::memcpy(out, ((Map *)h)->check, sizeof(int64_t) * CK_COUNT); }

// valid, in-pixel, ambiguous points; touched, new blocks; updated, semantic, seen voxels; taint events
void orc_stats(void *h, int64_t *out) {
    Map *m = (Map *)h;
    const Stats &s = m->st;
    int64_t v[11] = {s.valid_points, s.pixel_points, s.ambiguous_points, s.touched_blocks, s.new_blocks,
                     s.voxels_updated, s.voxels_semantic, s.voxels_seen, s.taint_events, s.sure_blocks,
                     s.ambiguous_blocks};
    std::memcpy(out, v, sizeof(v));
}

int64_t orc_num_alloc(void *h) { return (int64_t)((Map *)h)->alloc.size(); }

// all allocated blocks, sorted (x, y, z)
int64_t orc_get_alloc(void *h, int32_t *coords, int64_t cap) {
    Map *m = (Map *)h;
    std::vector<I3> v(m->alloc.begin(), m->alloc.end());
    std::sort(v.begin(), v.end());
    int64_t n = std::min<int64_t>(cap, (int64_t)v.size());
    for (int64_t i = 0; i < n; ++i) {
        coords[3 * i] = (int32_t)v[i].x;
        coords[3 * i + 1] = (int32_t)v[i].y;
        coords[3 * i + 2] = (int32_t)v[i].z;
    }
    return (int64_t)v.size();
}

// blocks touched by the last frame, sorted
int64_t orc_get_touched(void *h, int32_t *coords, int64_t cap) {
    Map *m = (Map *)h;
    int64_t n = std::min<int64_t>(cap, (int64_t)m->touched.size());
    for (int64_t i = 0; i < n; ++i) {
        coords[3 * i] = (int32_t)m->touched[i].x;
        coords[3 * i + 1] = (int32_t)m->touched[i].y;
        coords[3 * i + 2] = (int32_t)m->touched[i].z;
    }
    return (int64_t)m->touched.size();
}

// Copy one block's voxels; returns 0 when the block holds data, -1 otherwise.
int orc_read_block(void *h, const int32_t *coord, double *D, double *W, double *logP, uint8_t *taint,
                   int32_t *label, double *gap, int32_t *nupd, int32_t *nsem) {
    Map *m = (Map *)h;
    auto it = m->blocks.find({coord[0], coord[1], coord[2]});
    if (it == m->blocks.end()) return -1;
    const Block &b = it->second;
    if (D) std::memcpy(D, b.D.data(), sizeof(double) * BV);
    if (W) std::memcpy(W, b.W.data(), sizeof(double) * BV);
    if (logP) std::memcpy(logP, b.logP.data(), sizeof(double) * BV * m->C);
    if (taint) std::memcpy(taint, b.taint.data(), BV);
    if (nupd) std::memcpy(nupd, b.nupd.data(), sizeof(int32_t) * BV);
    if (nsem) std::memcpy(nsem, b.nsem.data(), sizeof(int32_t) * BV);
    if (label)
        for (int vi = 0; vi < BV; ++vi) label[vi] = argmax_label(*m, b, vi, gap ? gap + vi : nullptr);
    return 0;
}

// Overwrite (creating if needed) one block's voxels: test fixtures for meshing and queries.
int orc_write_block(void *h, const int32_t *coord, const double *D, const double *W, const double *logP) {
    Map *m = (Map *)h;
    I3 k{coord[0], coord[1], coord[2]};
    auto it = m->blocks.find(k);
    if (it == m->blocks.end()) it = m->blocks.emplace(k, new_block(m->C, m->dist_mode)).first;
    m->alloc.insert(k);
    Block &b = it->second;
    if (D) std::memcpy(b.D.data(), D, sizeof(double) * BV);
    if (W) std::memcpy(b.W.data(), W, sizeof(double) * BV);
    if (logP) std::memcpy(b.logP.data(), logP, sizeof(double) * BV * m->C);
    return 0;
}

// --- meshing: build into a handle, then fetch ------------------------------
// scope 0: all blocks holding data; 1: the listed blocks only.
void *orc_mesh_build(void *h, int scope, const int32_t *coords, int64_t n, int64_t *counts) {
    Map *m = (Map *)h;
    Mesh *mesh = new Mesh();
    std::vector<I3> keys;
    if (scope == 0) {
        for (auto &kv : m->blocks) keys.push_back(kv.first);
        std::sort(keys.begin(), keys.end());
    } else {
        for (int64_t i = 0; i < n; ++i) keys.push_back({coords[3 * i], coords[3 * i + 1], coords[3 * i + 2]});
    }
    for (const I3 &k : keys) mesh_block(*m, k, *mesh);
    counts[0] = (int64_t)mesh->verts.size();
    counts[1] = (int64_t)mesh->tris.size();
    return mesh;
}

// vertices sorted by key: key, position (m), label, gap to runner-up class, taint bits
// triangles: three keys, cube anchor voxel, taint (corner |D| < 1e-6 or distance-tainted corner)
void orc_mesh_fetch(void *hm, int64_t *vkey, double *vpos, int32_t *vlab, double *vgap, uint8_t *vtaint,
                    int64_t *tkeys, int32_t *tanchor, uint8_t *ttaint) {
    Mesh *mesh = (Mesh *)hm;
    int64_t i = 0;
    for (auto &kv : mesh->verts) {
        vkey[i] = kv.first;
        for (int q = 0; q < 3; ++q) vpos[3 * i + q] = kv.second.pos[q];
        vlab[i] = kv.second.label;
        vgap[i] = kv.second.gap;
        vtaint[i] = kv.second.taint;
        ++i;
    }
    for (size_t j = 0; j < mesh->tris.size(); ++j) {
        const MeshTri &t = mesh->tris[j];
        for (int q = 0; q < 3; ++q) tkeys[3 * j + q] = t.k[q];
        tanchor[3 * j] = (int32_t)t.anchor.x;
        tanchor[3 * j + 1] = (int32_t)t.anchor.y;
        tanchor[3 * j + 2] = (int32_t)t.anchor.z;
        ttaint[j] = t.taint;
    }
}

void orc_mesh_free(void *hm) { delete (Mesh *)hm; }

int64_t orc_edge_key(int64_t x, int64_t y, int64_t z, int axis) { return edge_key(x, y, z, axis); }

// --- queries ----------------------------------------------------------------
void orc_query(void *h, const double *xyz, int64_t n, double *sdf, uint8_t *valid, double *grad) {
    Map *m = (Map *)h;
    for (int64_t i = 0; i < n; ++i) {
        double s, g[3];
        bool ok = query(*m, xyz + 3 * i, &s, g);
        sdf[i] = s;
        valid[i] = ok ? 1 : 0;
        if (grad)
            for (int k = 0; k < 3; ++k) grad[3 * i + k] = g[k];
    }
}

/*
 * Loss L = sum_i D(T p_i)^2 over valid queries, its gradient with respect
 * to the left se(3) perturbation xi = (rho, phi) of T (dx/dxi = [I | -[x]x]),
 * and the Gauss-Newton system H = sum J^T J, g = sum J^T D with
 * J_i = grad D(x_i)^T [I | -[x_i]x].  Returns the number of valid points.
 */
int64_t orc_pose_terms(void *h, const float *pts, int64_t n, const double *T16, double *loss, double *dL,
                       double *Hm, double *gv) {
    Map *m = (Map *)h;
    double L = 0.0, G[6] = {0}, H[36] = {0}, g6[6] = {0};
    int64_t nv = 0;
    for (int64_t i = 0; i < n; ++i) {
        double p[3] = {pts[3 * i], pts[3 * i + 1], pts[3 * i + 2]};
        if (!(std::isfinite(p[0]) && std::isfinite(p[1]) && std::isfinite(p[2]))) continue;
        double x[3];
        for (int r = 0; r < 3; ++r) x[r] = T16[4 * r] * p[0] + T16[4 * r + 1] * p[1] + T16[4 * r + 2] * p[2] + T16[4 * r + 3];
        double s, gr[3];
        if (!query(*m, x, &s, gr)) continue;
        ++nv;
        double J[6] = {gr[0], gr[1], gr[2], x[1] * gr[2] - x[2] * gr[1], x[2] * gr[0] - x[0] * gr[2],
                       x[0] * gr[1] - x[1] * gr[0]};
        L += s * s;
        for (int a = 0; a < 6; ++a) {
            G[a] += 2.0 * s * J[a];
            g6[a] += J[a] * s;
            for (int b = 0; b < 6; ++b) H[6 * a + b] += J[a] * J[b];
        }
    }
    if (loss) *loss = L;
    if (dL) std::memcpy(dL, G, sizeof(G));
    if (Hm) std::memcpy(Hm, H, sizeof(H));
    if (gv) std::memcpy(gv, g6, sizeof(g6));
    return nv;
}

/*
 * Gauss-Newton system for a left perturbation about the sensor position c = t
 * of T: x' = Exp(xi) applied to x - c, plus c, so dx/dxi = [I | -[x - c]x] and
 * J_i = grad D(x_i)^T [I | -[R p_i]x] (x_i - c = R p_i).  Returns the number of
 * valid points.
 */
static int64_t pose_terms_at_sensor(Map &m, const float *pts, int64_t n, const double *T16, double *H, double *g6) {
    int64_t nv = 0;
    for (int a = 0; a < 36; ++a) H[a] = 0.0;
    for (int a = 0; a < 6; ++a) g6[a] = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double p[3] = {pts[3 * i], pts[3 * i + 1], pts[3 * i + 2]};
        if (!(std::isfinite(p[0]) && std::isfinite(p[1]) && std::isfinite(p[2]))) continue;
        double q[3], x[3];
        for (int r = 0; r < 3; ++r) {
            q[r] = T16[4 * r] * p[0] + T16[4 * r + 1] * p[1] + T16[4 * r + 2] * p[2];
            x[r] = q[r] + T16[4 * r + 3];
        }
        double s, gr[3];
        if (!query(m, x, &s, gr)) continue;
        ++nv;
        const double J[6] = {gr[0], gr[1], gr[2], q[1] * gr[2] - q[2] * gr[1], q[2] * gr[0] - q[0] * gr[2],
                             q[0] * gr[1] - q[1] * gr[0]};
        for (int a = 0; a < 6; ++a) {
            g6[a] += J[a] * s;
            for (int b = 0; b < 6; ++b) H[6 * a + b] += J[a] * J[b];
        }
    }
    return nv;
}

/*
 * Gauss-Newton scan-to-map alignment: iters steps of
 * (H + mu I) delta = -g with mu = 1e-6 (trace(H)/6 + 1e-12), then
 * T <- Tr(c) Exp(delta) Tr(-c) T with c the current sensor position, i.e.
 * R <- dR R, t <- t + dt for (dR, dt) = Exp(delta).  (About the world origin,
 * far from a scan on a large map, the rotation needs a compensating
 * translation of the lever arm's size, which the damping resists.)
 */
int orc_align(void *h, const float *pts, int64_t n, const double *T0, int iters, double *T_out) {
    double T[16];
    std::memcpy(T, T0, sizeof(T));
    for (int it = 0; it < iters; ++it) {
        double H[36], g[6];
        pose_terms_at_sensor(*(Map *)h, pts, n, T, H, g);
        double tr = 0.0;
        for (int a = 0; a < 6; ++a) tr += H[7 * a];
        double mu = 1e-6 * (tr / 6.0 + 1e-12);
        // solve (H + mu I) x = -g by Gaussian elimination with partial pivoting
        double A[6][7];
        for (int a = 0; a < 6; ++a) {
            for (int b = 0; b < 6; ++b) A[a][b] = H[6 * a + b] + (a == b ? mu : 0.0);
            A[a][6] = -g[a];
        }
        for (int c = 0; c < 6; ++c) {
            int piv = c;
            for (int r = c + 1; r < 6; ++r)
                if (std::fabs(A[r][c]) > std::fabs(A[piv][c])) piv = r;
            for (int k = 0; k < 7; ++k) std::swap(A[c][k], A[piv][k]);
            if (A[c][c] == 0.0) return -1;
            for (int r = c + 1; r < 6; ++r) {
                double f = A[r][c] / A[c][c];
                for (int k = c; k < 7; ++k) A[r][k] -= f * A[c][k];
            }
        }
        double d[6];
        for (int c = 5; c >= 0; --c) {
            double s = A[c][6];
            for (int k = c + 1; k < 6; ++k) s -= A[c][k] * d[k];
            d[c] = s / A[c][c];
        }
        double dR[9], dt[3];
        se3_exp(d, dR, dt);
        double Tn[16];
        std::memcpy(Tn, T, sizeof(T));
        for (int r = 0; r < 3; ++r) {
            for (int c = 0; c < 3; ++c)
                Tn[4 * r + c] = dR[3 * r] * T[c] + dR[3 * r + 1] * T[4 + c] + dR[3 * r + 2] * T[8 + c];
            Tn[4 * r + 3] = T[4 * r + 3] + dt[r];
        }
        std::memcpy(T, Tn, sizeof(T));
    }
    std::memcpy(T_out, T, sizeof(T));
    return 0;
}

void orc_se3_exp(const double *xi, double *R9, double *t3) { se3_exp(xi, R9, t3); }

// HSV palette with hue l / C of a full turn, full saturation and value
void orc_palette(int C, uint8_t *rgb) {
    for (int l = 0; l < C; ++l) {
        double h = 6.0 * (double)l / (double)C;
        int sector = (int)std::floor(h);
        double f = h - sector;
        double v = 1.0, p = 0.0, q = 1.0 - f, t = f;
        double r, g, b;
        switch (sector % 6) {
            case 0: r = v; g = t; b = p; break;
            case 1: r = q; g = v; b = p; break;
            case 2: r = p; g = v; b = t; break;
            case 3: r = p; g = q; b = v; break;
            case 4: r = t; g = p; b = v; break;
            default: r = v; g = p; b = q; break;
        }
        rgb[3 * l] = (uint8_t)std::lround(255.0 * r);
        rgb[3 * l + 1] = (uint8_t)std::lround(255.0 * g);
        rgb[3 * l + 2] = (uint8_t)std::lround(255.0 * b);
    }
}

// Band blocks of one point (test hook for the allocation pins): the sure
// blocks, then the ambiguous ones; cls[i] = 1 for sure, 0 for ambiguous.
int64_t orc_point_blocks(void *h, const float *pt, const double *T16, int32_t *out, int8_t *cls, int64_t cap) {
    Map *m = (Map *)h;
    double R[9], t[3];
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) R[3 * r + c] = T16[4 * r + c];
        t[r] = T16[4 * r + 3];
    }
    double e0[3], e1[3], len;
    band_endpoints(*m, R, t, pt, e0, e1, &len);
    std::vector<I3> vs, va;
    band_blocks(e0, e1, band_margin(*m, t, len), vs, va);
    int64_t k = 0;
    for (int pass = 0; pass < 2; ++pass)
        for (const I3 &b : pass == 0 ? vs : va) {
            if (k < cap) {
                out[3 * k] = (int32_t)b.x;
                out[3 * k + 1] = (int32_t)b.y;
                out[3 * k + 2] = (int32_t)b.z;
                cls[k] = pass == 0 ? 1 : 0;
            }
            ++k;
        }
    return k;
}

// FP64 band endpoints of one point (voxel units + 1/2) and the ambiguity margin (test hook)
double orc_point_band(void *h, const float *pt, const double *T16, double *e0, double *e1) {
    Map *m = (Map *)h;
    double R[9], t[3];
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) R[3 * r + c] = T16[4 * r + c];
        t[r] = T16[4 * r + 3];
    }
    double len;
    band_endpoints(*m, R, t, pt, e0, e1, &len);
    return band_margin(*m, t, len);
}

// clearance of block b from the segment e0 -> e1 (voxel units + 1/2; test hook)
double orc_block_clearance(const double *e0, const double *e1, const int32_t *b) {
    return block_clearance(e0, e1, I3{b[0], b[1], b[2]});
}

}  // extern "C"
