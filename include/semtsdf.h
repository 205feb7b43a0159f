/*
 * semtsdf: per-frame metric-semantic TSDF mapping on one B300 (sm_103a).
 *
 * C ABI of the product library (libsemtsdf.so).  Plain pointers and sizes;
 * no C++ or PyTorch types.  Streams are passed as `void *` holding a
 * `cudaStream_t` (NULL = the legacy default stream).
 *
 * Method (Liu et al. 2024, "Real-Time Metric-Semantic Mapping for
 * Autonomous Navigation in Outdoor Environments"):
 *   - Sec. III-C.1: each scan is projected into a range image with
 *     u = (pi - atan2(y, x)) / dphi, v = (acos(z / r) - theta0) / dtheta.
 *   - Sec. III-C.2: voxels x_i = nu * v_i stored in 8x8x8 blocks behind a
 *     hash table; projective distance psi along the ray; linear weight
 *     (psi + tau) / (2 tau); running-average update of D and W with the
 *     truncation Gamma(d, tau).
 *   - Sec. III-C.3, Eq. (bayesian_filter): per-voxel class distribution,
 *     uniform at allocation, multiplied by each scan's class likelihood and
 *     renormalised; marching-cubes mesh whose vertices take the most
 *     probable class.
 *
 * Conventions shared by every call:
 *   - Errors are returned as map_status; nothing aborts, traps or exits.
 *     Errors found on the device (pool, hash or mesh arena exhausted, a
 *     bounded wait that gave up) are latched in a device word and reported
 *     by the next call that synchronises (map_sync, map_get_frame_stats,
 *     the parity helpers) as MAP_ERR_CAPACITY or MAP_ERR_TIMEOUT.
 *   - Device input pointers stay owned by the caller, are only read, and
 *     must stay valid until the stream has executed the call.
 *   - The map owns all map storage, scratch buffers and mesh buffers.
 *   - Only the calls documented as synchronising block the host.
 *   - One map is used from one host thread at a time.
 */
#ifndef SEMTSDF_H
#define SEMTSDF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct map_t map_t;

typedef enum {
    MAP_OK = 0,
    MAP_ERR_ARG = 1,        /* a null pointer, a bad size or an inconsistent config  */
    MAP_ERR_CUDA = 2,       /* a CUDA runtime call failed (see map_last_error)       */
    MAP_ERR_CAPACITY = 3,   /* block pool, hash table, work list or mesh arena full   */
    MAP_ERR_BAD_POSE = 4,   /* T_world_lidar is not a rigid transform                 */
    MAP_ERR_TIMEOUT = 5,    /* a bounded device-side wait gave up                     */
    MAP_ERR_STATE = 6,      /* call not valid in the map's current state              */
    MAP_ERR_NOMEM = 7       /* device or pinned host allocation failed                */
} map_status;

/* Spinning multi-beam LiDAR (Sec. III-C.1).  Beam v (0 = top) has polar
 * angle theta0 + v * dtheta, theta0 = pi/2 - fov_up,
 * dtheta = (fov_up - fov_down) / (H - 1); column u has azimuth
 * pi - u * 2 pi / W.  Angles in radians.  Points with range outside
 * [r_min, r_max] or any non-finite coordinate are ignored. */
typedef struct {
    int32_t H, W;
    double fov_up, fov_down;
    double r_min, r_max;
} lidar_intrinsics;

/* Map parameters.  Fill with map_config_default() and override. */
typedef struct {
    double voxel_size;        /* nu, metres (Sec. III-C.2)                               */
    double truncation;        /* tau, metres; the band [p - tau d, p + tau d] is allocated */
    int32_t n_classes;        /* C >= 2 (Eq. bayesian_filter)                            */
    int32_t weight_mode;      /* 0: linear (psi + tau)/(2 tau) clamped to [0, 1]; 1: 1   */
    double p_hit;             /* hard-label likelihood of the given class (default 0.9)  */
    double logp_floor;        /* lower bound of stored log-probabilities (default -30)   */
    double lik_floor;         /* lower bound of probability-vector entries (1e-6)        */
    int32_t storage;          /* 0: FP32 {D, W} and log-probabilities; 1: FP16 storage   */
    int32_t distance_mode;    /* 0: projective psi; 1: non-projective d_i (see below)    */
    int64_t max_blocks;       /* block pool size (8^3 voxels each), at most 2^22             */
    int64_t hash_capacity;    /* hash slots, rounded up to a power of two                 */
    int64_t max_points;       /* largest scan accepted by integrate_scan                  */
    int64_t max_pixels;       /* largest H * W accepted                                    */
    int64_t mesh_vertex_capacity;    /* mesh arena sizes (vertices / triangles)          */
    int64_t mesh_triangle_capacity;
} map_config;

/* Non-projective distance (Sec. III-C.2, Eq. distance), distance_mode = 1:
 * each scan's normal image N is built from the range image (pixel (u, v)
 * back-projected along its ray at its range, with its (u, v - 1) and
 * (u - 1, v) neighbours: N = (p1 - p) x (p2 - p) normalised, turned toward
 * the sensor; none on the top row or next to a pixel without a return);
 * every voxel keeps a unit gradient g_i, the weight-averaged normal of the
 * pixels it projected to (12 B per voxel in FP32 storage, 6 B in FP16); the
 * fused value is Gamma(d_i, tau) with
 *   d_i = psi (|cos theta| - sin theta tan(alpha / 2)),
 * theta the angle between the ray and g_i, alpha the signed angle between
 * g_i and the pixel's normal (positive for a convex surface), which is the
 * exact distance for a circular surface through the ray's end point and
 * |cos theta| psi for a plane; the flat form where the pixel has no normal
 * or cos alpha <= 0, and psi before the voxel's first normal.  The weight,
 * the skip below -tau and the class-update gate stay on psi.  Needs
 * max_pixels <= 2^23; not available to map_batch_* (MAP_ERR_ARG). */

/* Device view of an extracted mesh (owned by the map; valid until the next
 * extract_mesh, integrate_scan or map_destroy on that map).
 * positions[n_vertices][3] float32 (metres, world frame);
 * colors[n_vertices][4] uint8 = {r, g, b, label}: label is the most probable
 *   class of the edge endpoint nearer the surface, rgb its palette colour;
 * vertex_keys[n_vertices]: lattice edge of the vertex, bits [0,2) axis,
 *   [2,22) x + 2^19, [22,42) y + 2^19, [42,62) z + 2^19 of its lower voxel;
 *   vertices on block seams appear once per block that uses them, so equal
 *   keys mark one welded vertex;
 * triangles[n_triangles][3] int32 indices into the vertex arrays, wound so
 *   the normal points to positive distance (free space);
 * triangle_anchors[n_triangles][3] int32 voxel anchoring the triangle's cube. */
typedef struct {
    int64_t n_vertices, n_triangles;
    float *positions;
    uint8_t *colors;
    int64_t *vertex_keys;
    int32_t *triangles;
    int32_t *triangle_anchors;
} mesh_view;

/* Per-frame counters (map_get_frame_stats), all counts of the last frame. */
enum {
    MAP_STAT_VALID_POINTS = 0,   /* finite points with r_min <= r <= r_max      */
    MAP_STAT_PIXEL_POINTS = 1,   /* valid points that fall on a beam row        */
    MAP_STAT_TOUCHED_BLOCKS = 2, /* blocks met by a truncation band (U_k)       */
    MAP_STAT_NEW_BLOCKS = 3,     /* of those, allocated this frame              */
    MAP_STAT_VOXELS_UPDATED = 4, /* voxels whose D, W were updated              */
    MAP_STAT_VOXELS_SEMANTIC = 5,/* voxels whose class distribution was updated */
    MAP_STAT_DIRTY_BLOCKS = 6,   /* blocks re-meshed (touched + -x/-y/-z nbrs)  */
    MAP_STAT_MESH_VERTICES = 7,  /* vertices emitted by this frame's re-mesh    */
    MAP_STAT_MESH_TRIANGLES = 8, /* triangles emitted by this frame's re-mesh   */
    MAP_STAT_TOTAL_BLOCKS = 9,   /* blocks allocated in the map so far          */
    MAP_STAT_ERROR_BITS = 10,    /* latched device error bits                   */
    MAP_STAT_KERNEL_LAUNCHES = 11, /* kernels this map has launched so far      */
    MAP_STAT_COUNT = 16
};

/* Defaults: weight_mode 0, p_hit 0.9, logp_floor -30, lik_floor 1e-6,
 * FP32 storage, capacities for a 64 x 2048 scanner at 0.1 m. */
map_status map_config_default(map_config *cfg);

/* Create an empty map (Sec. III-C.2: voxels of size nu = voxel_size at
 * centres nu * v_i, stored in 8x8x8-voxel blocks found through a hash table;
 * truncation tau bounds the fused distance and sets the allocated band;
 * n_classes is the size of the per-voxel class distribution of Sec. III-C.3).
 * Allocates and initialises all device storage (every pool voxel starts at
 * D = 0, W = 0 and the uniform class distribution).  Voxel coordinates are
 * limited to |v| < 2^19 - 16 on every axis (the range of the block and mesh
 * vertex keys): 52 km at 0.1 m voxels. */
map_status map_create(const map_config *cfg, map_t **out);

/* The pose checks integrate_scan applies, without a map: MAP_ERR_BAD_POSE
 * when T_world_lidar is not a rigid transform (rotation orthonormal to 1e-6,
 * det +1, last row 0 0 0 1) or when a voxel the scan can reach (any point up
 * to lidar->r_max, plus the band's truncation) lies outside the coordinate
 * range above on some axis: (|t_k| + r_max + tau) / voxel_size + 1 must stay
 * below 2^19 - 16.  MAP_ERR_ARG for a null pointer or inconsistent
 * intrinsics.  Host only; touches no device. */
map_status map_check_scan_pose(const map_config *cfg, const lidar_intrinsics *lidar, const double T_world_lidar[16]);
map_status map_destroy(map_t *map);

/* Fuse one posed scan (Sec. III-C): range image, band allocation, projective
 * TSDF + Bayesian label update of every voxel of the touched blocks, then
 * incremental marching cubes over the touched blocks and their -x/-y/-z
 * neighbours.  Asynchronous on `stream`.
 *   points_dev   [n][3] float32, LiDAR frame (NaN = no return);
 *   labels_dev   [n] int32 class per point (< 0 or >= C: no label), or NULL;
 *   probs_dev    [n][C] float32 class probabilities per point, or NULL;
 *                exactly one of labels_dev / probs_dev is non-NULL (n > 0);
 *   T_world_lidar  host double[16], row-major 4x4 world-from-LiDAR pose.
 * Returns MAP_ERR_ARG for n > max_points or H*W > max_pixels,
 * MAP_ERR_BAD_POSE when the rotation part is not orthonormal to 1e-6. */
map_status integrate_scan(map_t *map, const lidar_intrinsics *lidar, const float *points_dev,
                          const int32_t *labels_dev, const float *probs_dev, int64_t n,
                          const double T_world_lidar[16], void *stream);

/* Same as integrate_scan, for HOST buffers (pinned for best speed).  The
 * map uploads them into one of two device staging sets on an internal copy
 * stream; the scan's kernels on `stream` wait for the upload, and the upload
 * waits only for the scan that last used the same set, so consecutive calls
 * overlap a scan's upload with the previous scan's kernels.  Asynchronous:
 * the host buffers must stay unchanged until this scan's counters are
 * available (map_frame_stats for its frame index, map_sync, or any
 * synchronising call). */
map_status integrate_scan_host(map_t *map, const lidar_intrinsics *lidar, const float *points_host,
                               const int32_t *labels_host, const float *probs_host, int64_t n,
                               const double T_world_lidar[16], void *stream);

/* Number of scans integrated so far; scan k (from 0) has frame index k. */
int64_t map_frame_count(map_t *map);

/* Counters (MAP_STAT_*) of frame `frame`, one of the last 8 integrated
 * scans: waits for that scan only (not for later ones), then reads the copy
 * taken at its end.  MAP_ERR_ARG for an older or future frame; the device
 * error bits of that scan are reported as by map_sync. */
map_status map_frame_stats(map_t *map, int64_t frame, int64_t *out);

/* Gather every block's current mesh segment into one indexed mesh (device
 * arrays owned by the map).  The segments come from marching cubes over the
 * TSDF (Sec. III-C.3: the mesh of the zero level set, each vertex labelled
 * with its most probable class), re-run for the touched blocks by every
 * integrate_scan or for all blocks by map_remesh_all.  Synchronises `stream`
 * to learn the sizes. */
map_status extract_mesh(map_t *map, mesh_view *out, void *stream);

/* extract_mesh for callers that cannot allocate device memory (a real-time
 * loop that must not block on cudaMalloc, or a host framework that gives the
 * library only memory it reserved up front).  The paper has no counterpart;
 * this is an integration aid.  Same result as extract_mesh, written into the
 * caller's device buffers:
 *   positions[vertex_capacity][3] float32, colors[vertex_capacity][4] uint8,
 *   vertex_keys[vertex_capacity] int64, triangles[triangle_capacity][3] int32
 *   (indices into these vertex arrays), triangle_anchors[triangle_capacity][3].
 * *n_vertices / *n_triangles receive the mesh size; when it exceeds either
 * capacity nothing is written and MAP_ERR_CAPACITY is returned (call again
 * with larger buffers).  Allocates nothing: its scan scratch is one static
 * device array of 2^19 block slots (8.4 MB); maps whose pool exceeds 2^19
 * blocks get MAP_ERR_ARG.  The CUDA runtime places that array in a device's
 * memory when it is first used there (lazy module loading): map_create does
 * that on the map's device, so create the maps before reserving the rest of
 * the GPU's memory or capturing a stream; the array then stays until the
 * process exits.  The map and all five buffers must be device memory of the
 * current device (MAP_ERR_ARG otherwise); the three vertex buffers each hold
 * vertex_capacity entries and the two triangle buffers triangle_capacity.
 * All calls share the array: calls whose work overlaps on the GPU (different
 * streams or threads) race.  Synchronises `stream` to learn the mesh size. */
map_status extract_mesh_noalloc(map_t *map, float *positions, uint8_t *colors, int64_t *vertex_keys,
                                int32_t *triangles, int32_t *triangle_anchors, int64_t vertex_capacity,
                                int64_t triangle_capacity, int64_t *n_vertices, int64_t *n_triangles, void *stream);

/* ---- parity instrumentation (tests; not on the product path) ----
 * These two calls make a map record the integer decisions its single-
 * precision kernels take in each scan, so that a test can check them one by
 * one against an FP64 reference that takes the same decisions in double
 * precision and follows the recorded choice only where its own computation
 * lies within an ambiguity band (a projection within 1e-3 pixel of a pixel
 * boundary, a range within 2^-20 of r_min / r_max or of the pixel's nearest
 * range, a block whose distance from the band segment is within rounding of
 * zero, psi within rounding of +-tau).  The paper has no counterpart: this is
 * verification machinery for Sec. III-C.1's range image, Sec. III-C.2's
 * block allocation and voxel projection, and the class-update gate.
 *
 * map_set_decision_record(map, 1) allocates the record buffers (max_points
 * ints and max_blocks * 512 ints; max_pixels must be <= 2^23) and makes every
 * following integrate_scan / integrate_scan_host write:
 *   per point i: the pixel v * W + u it was put in, -1 when valid (finite,
 *     r_min <= r <= r_max) without a beam row, -2 when invalid;
 *   per voxel of every touched block: (pixel + 1) | updated << 28 |
 *     class-updated << 29 (pixel + 1 = 0: the voxel has no pixel).
 * The scans compute the same values as without the record (the kernels only
 * add the stores).  map_set_decision_record(map, 0) frees the buffers.
 * Both synchronise the device.  map_batch_integrate records nothing.
 *
 * map_read_decision_record reads the record of the LAST scan (MAP_ERR_STATE
 * when the last call on the map was not a recorded scan, or another call
 * has used the map's frame buffers since): point_pix[n_points] (n_points =
 * the scan's n), winner[n_pixels] (n_pixels = H * W: the range-image
 * winner of each pixel, (float bits of its range << 32) | point index, or
 * ~0 for none), the touched blocks' coordinates touched[touched_cap][3]
 * with their count in *n_touched, and voxel_rec[touched_cap][512] in the
 * same block order.  Any output may be NULL.  Synchronises the device;
 * allocates two temporary device buffers. */
map_status map_set_decision_record(map_t *map, int32_t enable);
map_status map_read_decision_record(map_t *map, int32_t *point_pix, int64_t n_points, uint64_t *winner,
                                    int64_t n_pixels, int32_t *touched, int64_t touched_cap, int64_t *n_touched,
                                    int32_t *voxel_rec);

/* Re-mesh every allocated block from scratch, replacing all mesh segments
 * (the arena is emptied first, nothing is compacted).  Asynchronous.  With
 * per-frame meshing switched off this is the paper's regime: a global
 * marching-cubes pass at a fixed rate (Sec. III-C.3, Table IV); it also
 * checks that incremental meshing equals a full pass.  Afterwards
 * map_get_frame_stats reports this pass: MAP_STAT_DIRTY_BLOCKS = blocks
 * meshed, MAP_STAT_MESH_VERTICES / _TRIANGLES = the whole mesh. */
map_status map_remesh_all(map_t *map, void *stream);

/* Per-frame incremental meshing in integrate_scan: 1 (default) re-meshes
 * the touched blocks and their -x/-y/-z neighbours every scan; 0 leaves
 * the mesh as it is until map_remesh_all (the scan's kernels minus k_mesh).
 * MAP_ERR_ARG for other values.  Applies to the following integrate_scan /
 * integrate_scan_host calls; map_batch_integrate always re-meshes. */
map_status map_set_incremental_mesh(map_t *map, int32_t enabled);

/* ---- class update from camera label images (Sec. III-C.3) ---- */

/* Pinhole camera: x right, y down, z forward; pixel (u, v) looks along
 * ((u - cx) / fx, (v - cy) / fy, 1); surfaces are searched up to r_max. */
typedef struct {
    int32_t width, height;
    double fx, fy, cx, cy;
    double r_max;
} camera_intrinsics;

/* Fuse one label image: only visible, observed voxels (W > 0) in the camera
 * frustum take its class likelihood (Sec. III-C.3, Eq. bayesian_filter).
 * Visibility by ray casting the TSDF: each pixel's ray visits the voxels it
 * passes through in order (exact cell traversal from the camera centre up
 * to r_max); the first pair of consecutive observed voxels with D >= 0 then
 * D < 0 is the visible surface, its range interpolated between the two
 * voxel centres' ranges along the ray.  Every observed voxel that projects
 * to a pixel with a surface and lies within the truncation of it
 * (|range - distance from the camera| <= tau) takes the pixel's likelihood,
 * exactly as a scan point's (hard label: p_hit model; probabilities:
 * floored).  The metric map (D, W) and the mesh are unchanged; vertex
 * classes follow at the next extract_mesh.
 *   labels_dev [height][width] int32 (< 0 or >= C: no label) or NULL;
 *   probs_dev [height][width][C] float32 or NULL (exactly one non-NULL);
 *   T_world_cam host double[16] row-major pose of the camera;
 *   range_dev [height][width] float32 (may be NULL): receives each pixel's
 *   surface range (NaN where none).
 * Asynchronous.  map_get_frame_stats then reports MAP_STAT_VOXELS_SEMANTIC
 * for this image. */
map_status integrate_labels_camera(map_t *map, const camera_intrinsics *cam, const int32_t *labels_dev,
                                   const float *probs_dev, const double T_world_cam[16], float *range_dev,
                                   void *stream);

/* ---- mesh traversability (Sec. III-D, Table II) ---- */

/* Thresholds of the traversability test.  Defaults (map_trav_params_default)
 * are Table II's: radius 0.25 m, height difference 0.6 m, steepness 20 deg,
 * roughness 30 deg; every class allowed.  With radius r the height
 * difference within the ball cannot exceed 2 r, so at the defaults the 0.6 m
 * threshold never rejects a vertex. */
typedef struct {
    double radius;            /* r, metres: the ball around each vertex                  */
    double max_height_diff;   /* t_hd, metres                                            */
    double max_steepness;     /* t_s, radians                                            */
    double max_roughness;     /* t_r, radians                                            */
    uint64_t class_mask;      /* bit c set: class c may be driven on (classes >= 64: no) */
} trav_params;

map_status map_trav_params_default(trav_params *params);

/* Traversability of every vertex of the mesh the last extract_mesh returned
 * (Sec. III-D): vertices are welded by vertex_keys (seam copies are one
 * vertex), a vertex normal is the area-weighted sum of its triangles'
 * normals, and within the ball B of radius r around the vertex
 *   v_hd = max z - min z over B          (height difference, metres),
 *   v_s  = angle of the normal from +z    (steepness, radians),
 *   v_r  = angle between the normal and the mean normal of B (roughness);
 * the vertex is traversable when v_hd < t_hd, v_s < t_s, v_r < t_r and its
 * class (colors[v][3]) is in class_mask.  The printed formulas are garbled:
 * the height difference is read as the elevation range, steepness and
 * roughness as the angles above, and the printed "all larger than the
 * thresholds" as all smaller (traversable).  Output per extracted vertex
 * (copies get their welded vertex's values): props_dev[nv][4] float32 =
 * {v_hd, v_s, v_r, |B|}, traversable_dev[nv] uint8.  Asynchronous;
 * MAP_ERR_STATE before any extract_mesh.  Scratch (~80 B per vertex) is
 * kept by the map and grown when a larger mesh comes (that growth
 * synchronises `stream`). */
map_status map_traversability(map_t *map, const trav_params *params, float *props_dev, uint8_t *traversable_dev,
                              void *stream);

/* ---- map quality against a ground-truth point cloud (Sec. IV-B.1) ---- */

typedef struct {
    double re;        /* Reconstruction Error: sqrt(mean over M of d(p, G)^2), metres   */
    double cd;        /* Chamfer-L1: mean_M d(p, G) / 2 + mean_G d(q, M) / 2, metres   */
    double rc;        /* Reconstruction Coverage: fraction of G within trunc of M    */
    double miou;      /* mean IoU over the classes that occur                          */
    double acc;       /* fraction of correctly classed vertices                        */
    int64_t n_map, n_gt, n_labeled, n_correct;
} quality_report;

/* Compare the mesh the last extract_mesh returned with a ground-truth cloud:
 * M = its welded vertices (one per vertex key), G = gt_points_dev [n_gt][3]
 * float32 (world frame) with classes gt_labels_dev [n_gt] int32;
 * d(p, X) = min(trunc, distance to the nearest point of X) (the paper uses
 * trunc = 2 nu).  mIoU and Acc count the vertices with a ground-truth point
 * within trunc: the class of that nearest point against the vertex's class;
 * IoU_c = TP / (TP + FP + FN) over the classes with TP + FP + FN > 0.
 * confusion (may be NULL): host int64 [C][C], rows ground-truth class,
 * columns vertex class.  Synchronises `stream`; MAP_ERR_STATE before any
 * extract_mesh or for an empty mesh, MAP_ERR_ARG for n_gt < 1. */
map_status map_quality(map_t *map, const float *gt_points_dev, const int32_t *gt_labels_dev, int64_t n_gt,
                       double trunc, quality_report *out, int64_t *confusion, void *stream);

/* Trilinear interpolation of D at m world points (from the 8 voxel centres
 * nu * v around x).  Not in the paper: a query interface for using the map
 * (differentiable reads, scan-to-map alignment).  sdf_dev[m] float32 (NaN
 * when any of the 8 voxels is unallocated or unobserved, W = 0, and for
 * non-finite points or points outside the map's coordinate range),
 * valid_dev[m] uint8 (1 = valid), may be NULL.  Asynchronous. */
map_status query_sdf(map_t *map, const float *xyz_dev, int64_t m, float *sdf_dev, uint8_t *valid_dev,
                     void *stream);

/* Backward of query_sdf: grad_xyz_dev[m][3] = grad_sdf_dev[m] * dD/dx at
 * each point (0 where invalid).  If pose_grad_dev (double[6]) is non-NULL
 * the left-perturbation pose gradient sum_i grad_xyz_i^T [I | -[x_i]x] is
 * ADDED to it (rho first, then phi).  Asynchronous. */
map_status query_sdf_backward(map_t *map, const float *xyz_dev, const float *grad_sdf_dev, int64_t m,
                              float *grad_xyz_dev, double *pose_grad_dev, void *stream);

/* Scan-to-map alignment: `iters` Gauss-Newton steps on sum_i D(T p_i)^2,
 * (H + mu I) delta = -g with mu = 1e-6 (trace(H)/6 + 1e-12), the left
 * perturbation taken about the current sensor position t:
 * T <- Tr(t) Exp(delta) Tr(-t) T, all on the device.  points_dev [n][3]
 * float32 LiDAR frame.  T0 and T_out are host double[16].  Synchronises
 * `stream`. */
map_status map_align_scan(map_t *map, const float *points_dev, int64_t n, const double T0[16], int32_t iters,
                          double T_out[16], void *stream);

/* ---- batched persistent integration (many maps, one launch) ---- */

/* One map's scan in a batch step (same meaning as the integrate_scan arguments). */
typedef struct {
    map_t *map;
    lidar_intrinsics lidar;
    const float *points_dev;
    const int32_t *labels_dev;
    const float *probs_dev;
    int64_t n;
    double T_world_lidar[16];
} scan_desc;

typedef struct map_batch_t map_batch_t;

enum {
    MAP_BATCH_GRAPH = 1,     /* replay the launch from a CUDA graph (one per launch configuration) */
    MAP_BATCH_AUTOTUNE = 2,  /* time each launch configuration on the first steps, keep the fastest */
    MAP_BATCH_STREAMS = 4    /* instead of the cooperative kernel: each map's integrate_scan kernels on
                                a stream of the batch's own, all maps concurrently, forked from and
                                joined to the caller's stream (AUTOTUNE then does nothing; with GRAPH
                                the step is captured on a private stream, an executable graph updated
                                in place from the capture, or instantiated again when the step's shape
                                changes, and launched once on the caller's stream) */
};

/* Group 1..48 maps (each used by this batch only while it exists).  The batch
 * kernel needs cooperative launch support (MAP_ERR_STATE otherwise) and maps
 * in the projective distance mode (MAP_ERR_ARG otherwise, unless the batch
 * is created with MAP_BATCH_STREAMS). */
map_status map_batch_create(map_t *const *maps, int32_t n_maps, int32_t flags, map_batch_t **out);
map_status map_batch_destroy(map_batch_t *batch);

/* Fuse scans[i] into the batch's i-th map for every i, in ONE cooperative
 * persistent kernel launch (Sec. III-C per map: range image, band
 * allocation, projective TSDF, Bayesian class fusion, incremental marching
 * cubes), with grid-wide barriers between the phases instead of host round
 * trips.  Results are identical to n_maps integrate_scan calls.  With
 * MAP_BATCH_AUTOTUNE the first 3 x 6 steps rotate through six launch
 * configurations (threads per block 128/256 x items per thread 1/2/4) and the
 * fastest median is kept.  Waits for the previous batch step (at most one in
 * flight); errors of the previous step (MAP_ERR_TIMEOUT when a barrier wait
 * ran out, MAP_ERR_CAPACITY) are returned by the next call or map_batch_sync. */
map_status map_batch_integrate(map_batch_t *batch, const scan_desc *scans, void *stream);

/* With MAP_BATCH_STREAMS the step is n_maps integrate_scan calls, each on
 * its own stream of the batch, run concurrently and joined to `stream`;
 * per-map results are those of integrate_scan (map_frame_stats included).
 * A map whose call is refused (bad arguments) is left as it was, the other
 * maps are still fused, and the first refusal is returned.  With
 * MAP_BATCH_GRAPH as well, the same calls are captured and replayed as one
 * graph launch (identical results); the capture and the graph update run on
 * the host before the step's first kernel starts, where the plain streams
 * form has the GPU working from its first launch on. */

/* Wait for the step in flight and report its errors. */
map_status map_batch_sync(map_batch_t *batch, void *stream);

/* The launch configuration in use (0 while still tuning). */
map_status map_batch_config(map_batch_t *batch, int32_t *threads_per_block, int32_t *items_per_thread,
                            int32_t *tuned);

/* Fix the launch configuration (0..5; -1 = tune). */
map_status map_batch_set_config(map_batch_t *batch, int32_t config_index);

/* Failure test hook: the next batch launch lets one CTA leave at once, so
 * the first grid barrier cannot complete; every other CTA gives up after
 * spin_limit polls and the step reports MAP_ERR_TIMEOUT. */
map_status map_batch_test_timeout(map_batch_t *batch, uint64_t spin_limit);

const char *map_batch_last_error(map_batch_t *batch);

/* ---- host-side inspection and checkpoint helpers (synchronising) ---- */

/* Wait for the map's work on `stream` and report latched device errors. */
map_status map_sync(map_t *map, void *stream);

/* Counters of the last integrate_scan (MAP_STAT_*); out has room for
 * MAP_STAT_COUNT int64 values.  Synchronises `stream`. */
map_status map_get_frame_stats(map_t *map, int64_t *out, void *stream);

/* Allocated block coordinates (host int32[cap][3], unsorted); *count
 * receives the number of allocated blocks even when cap is smaller. */
map_status map_get_blocks(map_t *map, int32_t *coords_host, int64_t cap, int64_t *count);

/* Read n blocks into host arrays (FP32 whatever the storage):
 * D[n][512], W[n][512], logP[n][C][512], label[n][512] (each may be NULL);
 * voxel index x + 8 y + 64 z.  found[n] (may be NULL) is 1 for allocated
 * blocks; others read as zeros / uniform. */
map_status map_read_blocks(map_t *map, const int32_t *coords_host, int64_t n, float *D, float *W,
                           float *logP, uint8_t *label, uint8_t *found);

/* Read the gradients g_i of n blocks (distance_mode 1; MAP_ERR_STATE
 * otherwise) into host G[n][3][512] (x, y, z planes, FP32 whatever the
 * storage; zero before a voxel's first normal and for unallocated blocks). */
map_status map_read_gradients(map_t *map, const int32_t *coords_host, int64_t n, float *G);

/* Write n blocks from host arrays (allocating them when new): D, W
 * [n][512]; logP [n][C][512] or NULL (uniform).  The label plane is
 * recomputed as the argmax.  Marks nothing dirty (call map_remesh_all). */
map_status map_write_blocks(map_t *map, const int32_t *coords_host, int64_t n, const float *D, const float *W,
                            const float *logP);

/* ---- phase profiling (CUDA events on the caller's stream) ---- */

/* Phases of one integrate_scan, in launch order (one kernel each, after the resets).
 * The class update and the re-meshing run concurrently (two streams, both
 * after the TSDF kernel); each reports its own duration, so a scan takes
 * less than the sum of its phases.  Recording puts an event between every
 * two kernels, which also keeps the TSDF and re-meshing kernels from being
 * scheduled before their predecessor ends (unrecorded scans let them). */
enum {
    MAP_PHASE_RESET = 0,      /* range-image and counter resets: empty in the steady state (the
                                 previous scan's per-point kernel resets this scan's set)     */
    MAP_PHASE_POINTS = 1,     /* per point: range-image winner (Sec. III-C.1), band allocation;
                                 the normal image in the non-projective mode                  */
    MAP_PHASE_TSDF = 2,       /* projective TSDF update (Sec. III-C.2), re-mesh queue          */
    MAP_PHASE_SEMANTIC = 3,   /* Bayesian class fusion (Eq. bayesian_filter)                  */
    MAP_PHASE_MESH = 4,       /* incremental marching cubes                                   */
    MAP_PHASE_COUNT = 5
};

/* Start recording per-phase events for up to max_frames subsequent
 * integrate_scan calls (earlier recording is discarded). */
map_status map_profile_begin(map_t *map, int32_t max_frames);

/* Concurrency of a scan's last two phases: 1 (default) runs the class update
 * on a second stream beside the re-meshing (it reads no class), joined before
 * integrate_scan returns; 0 runs the class update after the re-meshing on the
 * scan's stream, so each phase has the GPU to itself (to time the kernels
 * alone).  MAP_ERR_ARG for other values.  The results are the same. */
map_status map_set_concurrent_phases(map_t *map, int32_t concurrent);

/* Stop recording; synchronises.  ms_out[max_frames][MAP_PHASE_COUNT]
 * receives each recorded frame's phase durations in milliseconds,
 * stats_out[max_frames][MAP_STAT_COUNT] (may be NULL) its per-frame
 * counters (indices 0..8 of MAP_STAT_*), and *n_frames the number of
 * frames recorded. */
map_status map_profile_end(map_t *map, float *ms_out, int64_t *stats_out, int32_t *n_frames);

/* Most recent error message for this map (or a global one for map = NULL). */
const char *map_last_error(map_t *map);

/* Build-time helpers used by host tests (no GPU needed):
 * the marching-cubes table the kernels use, as triangles of cube-edge ids
 * (table[256][MAP_MC_MAXTRI][3], -1 padded; cube edge e = axis * 4 + d_a1 +
 * 2 d_a2 with a1, a2 the next axes cyclically); and the class palette. */
enum { MAP_MC_MAXTRI = 8 };
int32_t map_mc_table(int8_t *table_out);
int32_t map_palette(int32_t n_classes, uint8_t *rgb_out);

#ifdef __cplusplus
}
#endif
#endif /* SEMTSDF_H */
