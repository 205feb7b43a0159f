/*
 * Analytic LiDAR ray caster for the seeded synthetic scenes.
 *
 * Test and benchmark input generation only: this file computes where a
 * ray first meets the scene (ground plane, axis-aligned boxes, vertical
 * cylinders and sloped planar patches) and nothing of the mapping method
 * itself.  It is shared by the FP64 oracle tests and the CUDA path tests
 * through the Python module next to it.
 *
 * Acceleration: a uniform 2-D grid over the xy footprint of all
 * primitives, walked with the Amanatides-Woo digital differential
 * analyser; every ray is independent, so the OpenMP loop is deterministic.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define SY_EPS 1e-9

typedef struct {
    int kind;   /* 0 box, 1 cylinder, 2 ramp */
    int idx;
} prim_ref;

typedef struct {
    const double *boxes; int nbox;     /* [nbox][6]: lo xyz, hi xyz            */
    const double *cyls; int ncyl;      /* [ncyl][4]: cx, cy, r, h              */
    const double *ramps; int nramp;    /* [nramp][7]: cx, cy, hx, hy, z0, gx, gy */
    double x0, y0, cs;                 /* grid origin and cell size            */
    int nx, ny;
    int *cell_start;                   /* CSR over cells                       */
    prim_ref *refs;
    double z_top;
} scene_t;

static double hit_box(const double *b, const double o[3], const double d[3]) {
    double tn = -INFINITY, tf = INFINITY;
    for (int k = 0; k < 3; ++k) {
        if (fabs(d[k]) < 1e-300) {
            if (o[k] < b[k] || o[k] > b[3 + k]) return INFINITY;
        } else {
            double t1 = (b[k] - o[k]) / d[k], t2 = (b[3 + k] - o[k]) / d[k];
            if (t1 > t2) { double s = t1; t1 = t2; t2 = s; }
            if (t1 > tn) tn = t1;
            if (t2 < tf) tf = t2;
        }
    }
    if (tn > tf || tn <= SY_EPS) return INFINITY;
    return tn;
}

static double hit_cyl(const double *c, const double o[3], const double d[3]) {
    double best = INFINITY;
    double ox = o[0] - c[0], oy = o[1] - c[1], r = c[2], h = c[3];
    double a = d[0] * d[0] + d[1] * d[1];
    if (a > 1e-300) {
        double b = 2.0 * (d[0] * ox + d[1] * oy);
        double cc = ox * ox + oy * oy - r * r;
        double disc = b * b - 4.0 * a * cc;
        if (disc >= 0.0) {
            double t1 = (-b - sqrt(disc)) / (2.0 * a);
            if (t1 > SY_EPS) {
                double z = o[2] + t1 * d[2];
                if (z >= 0.0 && z <= h) best = t1;
            }
        }
    }
    if (fabs(d[2]) > 1e-300) {
        double t = (h - o[2]) / d[2];
        if (t > SY_EPS && t < best) {
            double x = ox + t * d[0], y = oy + t * d[1];
            if (x * x + y * y <= r * r) best = t;
        }
    }
    return best;
}

static double hit_ramp(const double *p, const double o[3], const double d[3]) {
    /* surface z = z0 + gx (x - cx) + gy (y - cy) over |x-cx|<=hx, |y-cy|<=hy, z >= 0 */
    double den = d[2] - p[5] * d[0] - p[6] * d[1];
    if (fabs(den) < 1e-12) return INFINITY;
    double t = (p[4] + p[5] * (o[0] - p[0]) + p[6] * (o[1] - p[1]) - o[2]) / den;
    if (t <= SY_EPS) return INFINITY;
    double x = o[0] + t * d[0], y = o[1] + t * d[1], z = o[2] + t * d[2];
    if (fabs(x - p[0]) > p[2] || fabs(y - p[1]) > p[3] || z < 0.0) return INFINITY;
    return t;
}

static void prim_aabb(const scene_t *s, prim_ref r, double lo[2], double hi[2], double *ztop) {
    if (r.kind == 0) {
        const double *b = s->boxes + 6 * r.idx;
        lo[0] = b[0]; lo[1] = b[1]; hi[0] = b[3]; hi[1] = b[4]; *ztop = b[5];
    } else if (r.kind == 1) {
        const double *c = s->cyls + 4 * r.idx;
        lo[0] = c[0] - c[2]; lo[1] = c[1] - c[2]; hi[0] = c[0] + c[2]; hi[1] = c[1] + c[2]; *ztop = c[3];
    } else {
        const double *p = s->ramps + 7 * r.idx;
        lo[0] = p[0] - p[2]; lo[1] = p[1] - p[3]; hi[0] = p[0] + p[2]; hi[1] = p[1] + p[3];
        *ztop = p[4] + fabs(p[5]) * p[2] + fabs(p[6]) * p[3];
    }
}

static int build_grid(scene_t *s, double cs) {
    int n = s->nbox + s->ncyl + s->nramp;
    s->cs = cs; s->z_top = 0.0;
    s->cell_start = NULL; s->refs = NULL; s->nx = s->ny = 0;
    if (n == 0) return 0;
    prim_ref *all = (prim_ref *)malloc(sizeof(prim_ref) * (size_t)n);
    int k = 0;
    for (int i = 0; i < s->nbox; ++i) { all[k].kind = 0; all[k].idx = i; ++k; }
    for (int i = 0; i < s->ncyl; ++i) { all[k].kind = 1; all[k].idx = i; ++k; }
    for (int i = 0; i < s->nramp; ++i) { all[k].kind = 2; all[k].idx = i; ++k; }
    double xlo = INFINITY, ylo = INFINITY, xhi = -INFINITY, yhi = -INFINITY;
    for (int i = 0; i < n; ++i) {
        double lo[2], hi[2], zt;
        prim_aabb(s, all[i], lo, hi, &zt);
        if (lo[0] < xlo) xlo = lo[0];
        if (lo[1] < ylo) ylo = lo[1];
        if (hi[0] > xhi) xhi = hi[0];
        if (hi[1] > yhi) yhi = hi[1];
        if (zt > s->z_top) s->z_top = zt;
    }
    s->x0 = xlo - cs; s->y0 = ylo - cs;
    s->nx = (int)ceil((xhi - s->x0) / cs) + 1;
    s->ny = (int)ceil((yhi - s->y0) / cs) + 1;
    size_t ncell = (size_t)s->nx * s->ny;
    int *cnt = (int *)calloc(ncell + 1, sizeof(int));
    for (int pass = 0; pass < 2; ++pass) {
        if (pass == 1) {
            int acc = 0;
            for (size_t c = 0; c < ncell; ++c) { int t = cnt[c]; cnt[c] = acc; acc += t; }
            cnt[ncell] = acc;
            s->cell_start = (int *)malloc(sizeof(int) * (ncell + 1));
            memcpy(s->cell_start, cnt, sizeof(int) * (ncell + 1));
            s->refs = (prim_ref *)malloc(sizeof(prim_ref) * (size_t)(acc > 0 ? acc : 1));
        }
        for (int i = 0; i < n; ++i) {
            double lo[2], hi[2], zt;
            prim_aabb(s, all[i], lo, hi, &zt);
            int ix0 = (int)floor((lo[0] - s->x0) / cs), ix1 = (int)floor((hi[0] - s->x0) / cs);
            int iy0 = (int)floor((lo[1] - s->y0) / cs), iy1 = (int)floor((hi[1] - s->y0) / cs);
            for (int iy = iy0; iy <= iy1; ++iy)
                for (int ix = ix0; ix <= ix1; ++ix) {
                    size_t c = (size_t)iy * s->nx + ix;
                    if (pass == 0) cnt[c]++;
                    else s->refs[cnt[c]++] = all[i];
                }
        }
    }
    free(cnt);
    free(all);
    return 0;
}

static double hit_prim(const scene_t *s, prim_ref r, const double o[3], const double d[3]) {
    if (r.kind == 0) return hit_box(s->boxes + 6 * r.idx, o, d);
    if (r.kind == 1) return hit_cyl(s->cyls + 4 * r.idx, o, d);
    return hit_ramp(s->ramps + 7 * r.idx, o, d);
}

/* Nearest hit with t in (0, t_end]; returns t or INFINITY and the primitive. */
static double trace(const scene_t *s, const double o[3], const double d[3], double t_end, prim_ref *hit) {
    double best = INFINITY;
    if (s->nx == 0) return best;
    /* clip [0, t_end] to the grid's xy rectangle */
    double xmin = s->x0, xmax = s->x0 + s->nx * s->cs, ymin = s->y0, ymax = s->y0 + s->ny * s->cs;
    double t0 = 0.0, t1 = t_end;
    const double lo[2] = {xmin, ymin}, hi[2] = {xmax, ymax};
    for (int k = 0; k < 2; ++k) {
        if (fabs(d[k]) < 1e-300) {
            if (o[k] < lo[k] || o[k] >= hi[k]) return best;
        } else {
            double a = (lo[k] - o[k]) / d[k], b = (hi[k] - o[k]) / d[k];
            if (a > b) { double t = a; a = b; b = t; }
            if (a > t0) t0 = a;
            if (b < t1) t1 = b;
        }
    }
    if (t0 > t1) return best;
    double px = o[0] + t0 * d[0], py = o[1] + t0 * d[1];
    int ix = (int)floor((px - s->x0) / s->cs), iy = (int)floor((py - s->y0) / s->cs);
    if (ix < 0) ix = 0;
    if (ix >= s->nx) ix = s->nx - 1;
    if (iy < 0) iy = 0;
    if (iy >= s->ny) iy = s->ny - 1;
    int stx = d[0] > 0 ? 1 : (d[0] < 0 ? -1 : 0), sty = d[1] > 0 ? 1 : (d[1] < 0 ? -1 : 0);
    double tmx = INFINITY, tmy = INFINITY, tdx = INFINITY, tdy = INFINITY;
    if (stx != 0) {
        double bx = s->x0 + (ix + (stx > 0 ? 1 : 0)) * s->cs;
        tmx = (bx - o[0]) / d[0];
        tdx = s->cs / fabs(d[0]);
    }
    if (sty != 0) {
        double by = s->y0 + (iy + (sty > 0 ? 1 : 0)) * s->cs;
        tmy = (by - o[1]) / d[1];
        tdy = s->cs / fabs(d[1]);
    }
    for (;;) {
        size_t c = (size_t)iy * s->nx + ix;
        for (int j = s->cell_start[c]; j < s->cell_start[c + 1]; ++j) {
            double t = hit_prim(s, s->refs[j], o, d);
            if (t < best && t <= t_end) { best = t; *hit = s->refs[j]; }
        }
        double t_exit = tmx < tmy ? tmx : tmy;
        if (best <= t_exit || t_exit > t1) break;
        if (tmx < tmy) { ix += stx; tmx += tdx; if (ix < 0 || ix >= s->nx) break; }
        else { iy += sty; tmy += tdy; if (iy < 0 || iy >= s->ny) break; }
    }
    return best;
}

/* Hit distance along one world ray; INFINITY when nothing lies within t_max. */
static double cast_one(const scene_t *s, int ground_cls, const double o[3], const double d[3],
                       double t_max, int *cls_out, const int *box_cls, const int *cyl_cls,
                       const int *ramp_cls) {
    double t_end = t_max;
    int cls = -1;
    double tg = INFINITY;
    if (ground_cls >= 0 && d[2] < 0.0 && o[2] > 0.0) tg = -o[2] / d[2];
    if (tg < t_end) t_end = tg;
    if (d[2] > 0.0) {
        double tt = (s->z_top - o[2]) / d[2];
        if (tt < t_end) t_end = tt < 0.0 ? 0.0 : tt;
    }
    prim_ref hit = {-1, -1};
    double t = trace(s, o, d, t_end, &hit);
    if (t < INFINITY) {
        cls = hit.kind == 0 ? box_cls[hit.idx] : (hit.kind == 1 ? cyl_cls[hit.idx] : ramp_cls[hit.idx]);
    } else if (tg <= t_max) {
        t = tg;
        cls = ground_cls;
    }
    if (t > t_max) { t = INFINITY; cls = -1; }
    *cls_out = cls;
    return t;
}

/*
 * Cast n rays from one origin.  dirs: [n][3] world-frame unit vectors.
 * Outputs the hit distance (INFINITY when nothing is hit within t_max) and
 * the class of the primitive hit (-1 when nothing is hit).  Ground z = 0
 * carries ground_cls (pass a negative value for a scene without ground).
 */
int synth_raycast(const double *boxes, const int *box_cls, int nbox,
                  const double *cyls, const int *cyl_cls, int ncyl,
                  const double *ramps, const int *ramp_cls, int nramp,
                  int ground_cls, const double *origin, const double *dirs, long n,
                  double t_max, double cell_size, double *t_out, int *cls_out, int nthreads) {
    scene_t s;
    s.boxes = boxes; s.nbox = nbox; s.cyls = cyls; s.ncyl = ncyl; s.ramps = ramps; s.nramp = nramp;
    build_grid(&s, cell_size);
    const double o[3] = {origin[0], origin[1], origin[2]};
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1024)
#endif
    for (long i = 0; i < n; ++i) {
        const double d[3] = {dirs[3 * i], dirs[3 * i + 1], dirs[3 * i + 2]};
        t_out[i] = cast_one(&s, ground_cls, o, d, t_max, &cls_out[i], box_cls, cyl_cls, ramp_cls);
    }
    free(s.cell_start);
    free(s.refs);
    return 0;
}

/* ---- counter-based random numbers: SplitMix64 (Steele, Lea, Flood 2014) ---- */
static uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}
typedef struct { uint64_t state; } rng_t;
static rng_t rng_at(uint64_t seed, uint64_t frame, uint64_t pixel) {
    rng_t r;
    r.state = mix64(mix64(seed * 0x9e3779b97f4a7c15ULL + 0x632be59bd9b4e019ULL) ^ (frame * 0xd1b54a32d192ed03ULL))
              ^ mix64(pixel + 0x8cb92ba72f3d8dd7ULL);
    return r;
}
static uint64_t rng_u64(rng_t *r) {
    r->state += 0x9e3779b97f4a7c15ULL;
    return mix64(r->state);
}
static double rng_unit(rng_t *r) {          /* uniform in (0, 1) */
    return ((double)(rng_u64(r) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}
static double rng_normal(rng_t *r) {        /* Box-Muller, cosine branch */
    double u1 = rng_unit(r), u2 = rng_unit(r);
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

/*
 * One synthetic scan.  Pixel (v, u) (row-major index v*W + u) looks along
 * polar angle theta0 + v*dtheta and azimuth pi - u*dphi in the LiDAR frame;
 * R (row-major 3x3) and t map that frame to the world.  The returned point
 * is (true range + N(0, sigma)) along the same ray, as float32, or NaN when
 * nothing is hit within r_max.
 *
 * label_mode 0: labels[i] = hit class, replaced with probability p_flip by a
 *               class drawn uniformly from the other n_classes - 1.
 * label_mode 1: probs[i][c] = 0.6 * onehot(class) + 0.4 * Dirichlet(1/2,...),
 *               the Dirichlet drawn as normalised Z^2/2 (Z standard normal);
 *               labels[i] = hit class.
 * Rows with no hit get label -1 and an all-zero probability row.
 * true_range / true_cls (optional) receive the analytic hit.
 * jitter_px > 0: the ray of pixel (v, u) is turned by independent normal
 * offsets of jitter_px * dtheta in polar angle and jitter_px * dphi in
 * azimuth (a real scanner's firing-time and beam-angle spread), drawn from a
 * stream of their own, so that points no longer lie on their pixel's centre
 * ray; the point is (true range + noise) along the turned ray.
 */
int synth_scan(const double *boxes, const int *box_cls, int nbox,
               const double *cyls, const int *cyl_cls, int ncyl,
               const double *ramps, const int *ramp_cls, int nramp, int ground_cls,
               const double *R, const double *t, int H, int W, double theta0, double dtheta,
               double dphi, double r_max, double sigma, int n_classes, int label_mode,
               double p_flip, uint64_t seed, uint64_t frame, float *points, int *labels,
               float *probs, double *true_range, int *true_cls, int nthreads, double jitter_px) {
    scene_t s;
    s.boxes = boxes; s.nbox = nbox; s.cyls = cyls; s.ncyl = ncyl; s.ramps = ramps; s.nramp = nramp;
    build_grid(&s, 4.0);
    const double o[3] = {t[0], t[1], t[2]};
    long n = (long)H * W;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1024)
#endif
    for (long i = 0; i < n; ++i) {
        int v = (int)(i / W), u = (int)(i % W);
        double th = theta0 + v * dtheta, ph = 3.141592653589793 - u * dphi;
        if (jitter_px > 0.0) {
            rng_t rj = rng_at(seed, frame, (uint64_t)i + (1ULL << 40));
            th += jitter_px * dtheta * rng_normal(&rj);
            ph += jitter_px * dphi * rng_normal(&rj);
        }
        double dl[3] = {sin(th) * cos(ph), sin(th) * sin(ph), cos(th)};
        double dw[3];
        for (int k = 0; k < 3; ++k) dw[k] = R[3 * k] * dl[0] + R[3 * k + 1] * dl[1] + R[3 * k + 2] * dl[2];
        int cls;
        double th_hit = cast_one(&s, ground_cls, o, dw, r_max, &cls, box_cls, cyl_cls, ramp_cls);
        rng_t rg = rng_at(seed, frame, (uint64_t)i);
        double noise = sigma * rng_normal(&rg);
        if (true_range) true_range[i] = th_hit;
        if (true_cls) true_cls[i] = cls;
        if (th_hit < INFINITY) {
            double r = th_hit + noise;
            for (int k = 0; k < 3; ++k) points[3 * i + k] = (float)(dl[k] * r);
        } else {
            for (int k = 0; k < 3; ++k) points[3 * i + k] = NAN;
        }
        int lab = th_hit < INFINITY ? cls : -1;
        if (label_mode == 0) {
            double uflip = rng_unit(&rg);
            uint64_t pick = rng_u64(&rg) % (uint64_t)(n_classes - 1);
            if (lab >= 0 && uflip < p_flip) lab = (int)((lab + 1 + (int)pick) % n_classes);
            labels[i] = lab;
        } else {
            labels[i] = lab;
            float *q = probs + (size_t)i * n_classes;
            if (lab < 0) {
                for (int c = 0; c < n_classes; ++c) q[c] = 0.0f;
            } else {
                double g[256], sum = 0.0;
                for (int c = 0; c < n_classes; ++c) {
                    double z = rng_normal(&rg);
                    g[c] = 0.5 * z * z;
                    sum += g[c];
                }
                for (int c = 0; c < n_classes; ++c)
                    q[c] = (float)(0.4 * g[c] / sum + (c == lab ? 0.6 : 0.0));
            }
        }
    }
    free(s.cell_start);
    free(s.refs);
    return 0;
}
