// Launchers of the CUDA kernels (host side), one per kernel file.
#pragma once

#include "common.cuh"

namespace stsdf {

// The kernels of a scan all prefer the largest shared-memory carveout: an SM
// changes its L1 / shared split only when idle, so kernels with different
// splits could not share an SM as one scan's grids hand over to the next.
void alloc_kernel_attributes();
void integrate_kernel_attributes();
void mesh_kernel_attributes();

// k_alloc.cu: per-point range-image winners and band allocation (touched list)
void launch_points(const float *pts, const ScanConst &sc, const MapDev &md, const FrameDev &fd, cudaStream_t s);
void launch_snapshot(const unsigned long long *ctr, const DevState *st, unsigned char *rec, cudaStream_t s);
void launch_list_all(const MapDev &md, const FrameDev &fd, int frame, cudaStream_t s);
void launch_init_pool(const MapDev &md, cudaStream_t s);
void launch_link_all(const MapDev &md, cudaStream_t s);
void launch_write_block(const MapDev &md, uint64_t key, const float *D, const float *W, const float *logP,
                        cudaStream_t s);
// G (may be null): gradient planes [n][3][512] of the non-projective mode
void launch_read_blocks(const MapDev &md, const uint64_t *keys, int n, float *D, float *W, float *logP,
                        uint8_t *label, uint8_t *found, float *G, cudaStream_t s);
void launch_collect_blocks(const MapDev &md, int32_t *coords, unsigned long long *count, cudaStream_t s);
// parity instrumentation: coordinates [nt][3] and voxel decision records [nt][512] of the touched list
void launch_dbg_gather(const MapDev &md, const int *touched, long long nt, const int *vrec, int32_t *coords,
                       int32_t *out, cudaStream_t s);

// k_integrate.cu: projective TSDF + Bayesian semantic fusion (Sec. III-C.2, III-C.3)
void launch_integrate(const ScanConst &sc, const MapDev &md, const FrameDev &fd, int grid, cudaStream_t s);
void launch_semantic(const ScanConst &sc, const MapDev &md, const FrameDev &fd, int grid, cudaStream_t s);
// non-projective mode: the scan's normal image (after launch_points, before launch_integrate)
void launch_normals(const ScanConst &sc, const FrameDev &fd, cudaStream_t s);
int integrate_blocks_per_sm(int storage, int C, int dist_mode);
int semantic_blocks_per_sm(int storage, int C);

// k_mesh.cu: incremental marching cubes and mesh gathering
int mesh_upload_tables(const int8_t *tri, const uint8_t *ntri);
void launch_mesh(const MapDev &md, const FrameDev &fd, int grid, cudaStream_t s);
int mesh_blocks_per_sm();
struct GatherBufs {
    long long *voff, *toff;          // [max_blocks] per-slot exclusive offsets within a chunk
    long long *bsum_v, *bsum_t;      // [chunks]
    long long *totals;               // [2]
};
void launch_seg_scan(const MapDev &md, const GatherBufs &g, int max_blocks, cudaStream_t s);
// mode 0: compact into (av2, ak2, at2) and rewrite seg; mode 1: write the user mesh arrays
void launch_seg_gather(const MapDev &md, const GatherBufs &g, int max_blocks, int mode, float4 *av2,
                       int64_t *ak2, ushort4 *at2, float *pos, uint8_t *col, int64_t *keys, int32_t *tri,
                       int32_t *anchors, cudaStream_t s);
void launch_set_cursors(const MapDev &md, const GatherBufs &g, cudaStream_t s);

// k_query.cu: trilinear queries, gradients, Gauss-Newton
void launch_query(const MapDev &md, const float *xyz, long long m, float *sdf, uint8_t *valid, cudaStream_t s);
constexpr int QB_PART_DOUBLES = 148 * 8 * 8;   // per-CTA rows of pose-gradient partial sums
void launch_query_bwd(const MapDev &md, const float *xyz, const float *gsdf, long long m, float *gxyz,
                      double *pose_grad, double *part, cudaStream_t s);
void launch_gn_terms(const MapDev &md, const float *pts, long long n, const double *T_dev, double *acc,
                     cudaStream_t s);
constexpr int GN_ACC_STRIDE = 32;             // doubles per CTA row of Gauss-Newton partial sums
constexpr int GN_ACC_ROWS = 148 * 8;          // most CTAs of k_gn_terms
int gn_terms_grid(long long n);
void launch_gn_step(double *T_dev, const double *acc, int nparts, cudaStream_t s);

// k_trav.cu: mesh traversability (Sec. III-D) over an extracted mesh
struct TravDev {
    uint64_t *vkeys;              // [vmask + 1] vertex-key hash
    int *vfirst;                  // [vmask + 1] lowest vertex index of each key
    uint64_t vmask;
    int *rep;                     // [nv] representative (welded) vertex
    float4 *nacc;                 // [nv] normal sums, then unit normals (w = 1 valid)
    int *vcell;                   // [nv] cell slot of a representative, -1 otherwise
    uint64_t *ckeys;              // [cmask + 1] cell hash
    int *ccount, *cstart, *cfill; // [cmask + 1] per cell: vertices, first sorted index, fill cursor
    uint64_t cmask;
    float4 *spos, *snrm;          // [nv] cell-sorted representatives: {x, y, z, label bits}, normal
    unsigned long long *cursor;   // sorted-array allocation cursor
    unsigned *err;                // bit 1 (ERR_HASH_PROBES) when a hash overflows its probe bound
    float inv_cell;               // 1 / cell edge (the radius, enlarged by 1e-5)
};
struct TravParamsDev {
    float r2, t_hd, t_s, t_r;     // radius^2 (m^2), height (m), steepness and roughness (rad)
    unsigned long long class_mask;
};
void launch_traversability(const TravDev &b, const TravParamsDev &p, const float *pos, const uint8_t *col,
                           const int64_t *vkey, const int32_t *tri, long long nv, long long nt, float4 *props,
                           uint8_t *trav, cudaStream_t s);
// welding only: rep[i] = lowest index with vertex i's key (the b.vkeys / b.vfirst tables reset before)
void launch_weld(const TravDev &b, const int64_t *vkey, long long nv, cudaStream_t s);

// k_camera.cu: class update from a camera label image (Sec. III-C.3)
struct CamConst {
    int W, H, max_steps;          // image size; traversal step bound
    float fx, fy, cx, cy, inv_fx, inv_fy;
    float R[9];                   // world-from-camera rotation, row-major (x right, y down, z forward)
    float c[3];                   // camera centre, world
    float nu, inv_nu, r_max;
};
// range [H*W]: hit range per pixel (NaN: none); sc carries tau, C, the likelihood model and the
// label image (labels or probs, per pixel) for the class update
// bounds: int[6] scratch, set to {+big x3, -big x3} before the call
void launch_camera(const CamConst &cc, const ScanConst &sc, const MapDev &md, const FrameDev &fd, float *range,
                   int *bounds, int grid_semantic, cudaStream_t s);

// k_quality.cu: map quality against a ground-truth cloud (Sec. IV-B.1)
struct GridDev {                  // points of one cloud sorted by cell of edge ~truncation
    uint64_t *ckeys;              // [cmask + 1] cell hash
    int *ccount, *cstart, *cfill; // [cmask + 1]
    uint64_t cmask;
    float4 *spts;                 // [n] sorted {x, y, z, class bits}
    int *slot;                    // [n] cell slot of each point (-1: not in the cloud)
    unsigned long long *cursor;
    unsigned *err;
    float inv_cell;
};
struct QualityAcc {               // device accumulators, reset before a run
    double sum_d_map, sum_d2_map, sum_d_gt;
    unsigned long long n_map, n_gt, n_gt_covered, n_labeled;
};
// cloud 0 = welded mesh vertices (rep[i] == i), cloud 1 = ground truth
void launch_quality(const GridDev &gmap, const GridDev &ggt, const int *rep, const float *mpos, const uint8_t *mcol,
                    long long nv, const float *gpos, const int32_t *glab, long long ng, float trunc, int C,
                    QualityAcc *acc, unsigned long long *conf, cudaStream_t s);

}  // namespace stsdf
