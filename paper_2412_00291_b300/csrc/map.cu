// C ABI of libsemtsdf: map lifetime, per-frame orchestration on the caller's
// stream, mesh extraction, queries, alignment and host inspection helpers.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <algorithm>

#include "../../include/semtsdf.h"
#include "batch.h"
#include "kernels.h"

using namespace stsdf;

struct map_t {
    map_config cfg;
    int C = 0;
    MapDev md{};
    FrameDev fd{};
    DevState *st = nullptr;
    // Per-scan buffers, two of each: a scan uses one set while its per-point
    // kernel resets the other for the next scan (no memsets between scans).
    unsigned long long *ctr_pair = nullptr;
    unsigned long long *ctr_buf[2] = {};
    unsigned long long *win_buf[2] = {};
    long long win_dirty[2] = {};     // leading range-image entries that may hold a winner
    bool ctr_clean[2] = {true, true};
    int fcur = 1;                    // set m->fd points at; the next scan uses the other
    // second mesh arena for compaction
    float4 *av_alt = nullptr;
    int64_t *ak_alt = nullptr;
    ushort4 *at_alt = nullptr;
    GatherBufs gb{};
    int nchunks = 0;
    // host views (pinned) of the last frame's counters and device state; when
    // h_ctr_slot >= 0 the counters are those of that ring entry
    unsigned long long *h_ctr = nullptr;
    int h_ctr_slot = -1;
    DevState *h_st = nullptr;
    long long *h_totals = nullptr;
    // Ring of per-frame device-state copies: bounds how far the host runs ahead
    // (at most RING frames in flight) and gives it a view of the mesh-arena
    // cursor that is at most RING frames old.
    static constexpr int RING = 8;
    static constexpr size_t CTR_BYTES = CT_COUNT * sizeof(unsigned long long);
    static constexpr size_t REC_BYTES = CTR_BYTES + sizeof(DevState);
    // A scan ends with a device-side snapshot of its counters and the device
    // state into d_ring[slot] ([counters | state]); a download stream copies it
    // to h_ring[slot] off the scan stream (a copy there would hold the next
    // scan's kernels for the whole transfer).
    unsigned char *h_ring = nullptr;   // [RING][REC_BYTES]
    unsigned char *d_ring = nullptr;   // [RING][REC_BYTES]
    cudaStream_t dl = nullptr;
    cudaEvent_t ev_snap = nullptr;
    cudaEvent_t ev_ring[RING] = {};
    // the class update runs on a second stream beside the re-meshing (the mesh
    // does not read class labels); fork after the TSDF kernel, join before return
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    long long ring_frame[RING] = {};
    long long absorbed = -1;        // ring entries up to this frame have been read
    int ring_epoch[RING] = {};
    int epoch = 0;                  // bumped by every compaction
    double known_fill = 0.0;         // largest used fraction of any arena partition
    long long known_frame = -1;
    double max_append = 0.0;         // largest per-frame growth of that fraction
    // staging for host inputs
    // integrate_scan_host: two staging sets, filled on a copy stream, so that a
    // scan's upload overlaps the previous scan's kernels
    float *stage_pts[2] = {};
    int32_t *stage_lab[2] = {};
    float *stage_probs[2] = {};
    int stage_next = 0;
    cudaStream_t cp = nullptr;
    cudaEvent_t ev_copied[2] = {}, ev_used[2] = {};
    // extracted mesh
    long long out_vcap = 0, out_tcap = 0;
    float *out_pos = nullptr;
    uint8_t *out_col = nullptr;
    int64_t *out_keys = nullptr;
    int32_t *out_tri = nullptr;
    int32_t *out_anchor = nullptr;
    // class palette (rgb per class, on the device as uchar4)
    uint8_t palette[256 * 3];
    uchar4 *pal_dev = nullptr;
    // non-projective mode: pixel-ray tables (float pairs) for the current
    // intrinsics, uploaded from a pinned copy when the intrinsics change
    float4 *row_dir = nullptr, *col_dir = nullptr;
    float4 *nrm = nullptr;           // [max_pixels] the scan's normal image
    float4 *h_dir = nullptr;
    long long h_dir_cap = 0;
    cudaEvent_t ev_dir = nullptr;
    lidar_intrinsics dir_for{};
    bool dir_valid = false;
    // traversability scratch (grown on demand) and the last extract_mesh's size
    TravDev trav{};
    long long trav_nv_cap = 0;
    // map quality scratch: grids of the welded vertices and of the ground truth, accumulators
    GridDev q_map{}, q_gt{};
    long long q_map_cap = 0, q_gt_cap = 0;
    QualityAcc *q_acc = nullptr;
    unsigned long long *q_conf = nullptr;
    // camera class update: hit ranges of the last image (when the caller passes none)
    float *cam_range = nullptr;
    long long cam_range_cap = 0;
    int *cam_bounds = nullptr;      // box of the allocated blocks (ray-cast bound)
    bool ext_valid = false;
    long long ext_nv = 0, ext_nt = 0;
    // alignment scratch
    double *gn_T = nullptr, *gn_acc = nullptr;
    double *qb_part = nullptr;   // pose-gradient partial sums of query_sdf_backward
    int frame = 0;
    bool mesh_per_frame = true;     // incremental re-meshing in every integrate_scan
    bool concurrent = true;         // class update beside the re-meshing (second stream)
    int grid_integrate = 0, grid_mesh = 0, grid_semantic = 0;
    // phase profiling: (MAP_PHASE_COUNT + 1) events per recorded frame
    std::vector<cudaEvent_t> prof_ev;
    std::vector<char> prof_serial;              // per recorded frame: phases run one after the other
    int prof_cap = 0, prof_n = 0;
    unsigned long long *prof_stats = nullptr;   // device [prof_cap][CT_COUNT]
    long long launches = 0;                     // kernels launched by this map
    // parity instrumentation: decision records of the last scan (map_set_decision_record)
    int *dbg_point = nullptr, *dbg_vox = nullptr;
    long long dbg_frame = -1;                   // frame whose decisions the buffers hold
    long long dbg_n = 0, dbg_np = 0;            // its point and pixel counts
    std::string err;
};

static std::string g_err;

namespace stsdf {
void noalloc_prepare_device();   // noalloc.cu: loads its static scratch array on the current device
}

static map_status fail(map_t *m, map_status s, const std::string &msg) {
    if (m) m->err = msg;
    else g_err = msg;
    return s;
}

#define CU(call)                                                                                    \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess)                                                                      \
            return fail(m, MAP_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));       \
    } while (0)

static map_status launch_check(map_t *m, const char *what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(m, MAP_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    return MAP_OK;
}

extern "C" map_status map_config_default(map_config *cfg) {
    if (!cfg) return fail(nullptr, MAP_ERR_ARG, "null config");
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->voxel_size = 0.1;
    cfg->truncation = 0.3;
    cfg->n_classes = 20;
    cfg->weight_mode = 0;
    cfg->p_hit = 0.9;
    cfg->logp_floor = -30.0;
    cfg->lik_floor = 1e-6;
    cfg->storage = 0;
    cfg->max_blocks = 262144;
    cfg->hash_capacity = 1 << 20;
    cfg->max_points = 262144;
    cfg->max_pixels = 262144;
    cfg->mesh_vertex_capacity = 32ll << 20;
    cfg->mesh_triangle_capacity = 64ll << 20;
    return MAP_OK;
}

static void prof_clear(map_t *m) {
    for (cudaEvent_t e : m->prof_ev) cudaEventDestroy(e);
    m->prof_ev.clear();
    if (m->prof_stats) cudaFree(m->prof_stats);
    m->prof_stats = nullptr;
    m->prof_cap = m->prof_n = 0;
}

static void free_all(map_t *m) {
    prof_clear(m);
    void *ptrs[] = {m->md.hs, m->md.dstamp_slot, m->md.dw32, m->md.dw16, m->md.lp32,
                    m->md.lp16, m->md.label, m->md.slot_key, m->md.slot_frame, m->md.nbr, m->md.seg, m->md.av, m->md.ak, m->md.at,
                    m->av_alt, m->ak_alt, m->at_alt, m->st, m->ctr_pair, m->d_ring, m->win_buf[0], m->win_buf[1],
                    m->fd.touched, m->fd.dirty, m->fd.sem_list, m->gb.voff, m->gb.toff, m->gb.bsum_v, m->gb.bsum_t,
                    m->gb.totals, m->stage_pts[0], m->stage_lab[0], m->stage_probs[0], m->stage_pts[1],
                    m->stage_lab[1], m->stage_probs[1], m->out_pos, m->out_col,
                    m->out_keys, m->out_tri, m->out_anchor, m->gn_T, m->gn_acc, m->qb_part, m->pal_dev,
                    m->md.g32, m->md.g16, m->nrm, m->row_dir, m->col_dir, m->trav.vkeys, m->trav.vfirst,
                    m->trav.rep, m->trav.nacc, m->trav.vcell, m->trav.ckeys, m->trav.ccount, m->trav.cstart,
                    m->trav.cfill, m->trav.spos, m->trav.snrm, m->trav.cursor, m->q_map.ckeys, m->q_map.ccount,
                    m->q_map.cstart, m->q_map.cfill, m->q_map.spts, m->q_map.slot, m->q_map.cursor, m->q_gt.ckeys,
                    m->q_gt.ccount, m->q_gt.cstart, m->q_gt.cfill, m->q_gt.spts, m->q_gt.slot, m->q_gt.cursor,
                    m->q_acc, m->q_conf, m->cam_range, m->cam_bounds};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (m->h_ctr) cudaFreeHost(m->h_ctr);
    if (m->h_st) cudaFreeHost(m->h_st);
    if (m->h_totals) cudaFreeHost(m->h_totals);
    if (m->h_ring) cudaFreeHost(m->h_ring);
    if (m->h_dir) cudaFreeHost(m->h_dir);
    if (m->ev_dir) cudaEventDestroy(m->ev_dir);
    for (int b = 0; b < 2; ++b) {
        if (m->ev_copied[b]) cudaEventDestroy(m->ev_copied[b]);
        if (m->ev_used[b]) cudaEventDestroy(m->ev_used[b]);
    }
    if (m->cp) cudaStreamDestroy(m->cp);
    for (auto &e : m->ev_ring)
        if (e) cudaEventDestroy(e);
    if (m->ev_fork) cudaEventDestroy(m->ev_fork);
    if (m->ev_join) cudaEventDestroy(m->ev_join);
    if (m->side) cudaStreamDestroy(m->side);
    if (m->ev_snap) cudaEventDestroy(m->ev_snap);
    if (m->dl) cudaStreamDestroy(m->dl);
    if (m->dbg_point) cudaFree(m->dbg_point);
    if (m->dbg_vox) cudaFree(m->dbg_vox);
    m->dbg_point = m->dbg_vox = nullptr;
}

template <typename T>
static cudaError_t dalloc(T **p, size_t count) {
    return cudaMalloc((void **)p, count * sizeof(T) + 16);
}

extern "C" map_status map_create(const map_config *cfg_in, map_t **out) {
    map_t *m = nullptr;
    if (!cfg_in || !out) return fail(nullptr, MAP_ERR_ARG, "null argument");
    const map_config &c = *cfg_in;
    if (!(c.voxel_size > 0.0) || !(c.truncation > 0.0) || c.truncation > 15.0 * c.voxel_size)
        return fail(nullptr, MAP_ERR_ARG, "need 0 < truncation <= 15 voxel_size");
    if (c.n_classes < 2 || c.n_classes > 64) return fail(nullptr, MAP_ERR_ARG, "n_classes must be in [2, 64]");
    if (c.weight_mode < 0 || c.weight_mode > 1 || c.storage < 0 || c.storage > 1 || c.distance_mode < 0 ||
        c.distance_mode > 1)
        return fail(nullptr, MAP_ERR_ARG, "bad weight_mode, storage or distance_mode");
    if (!(c.p_hit > 0.0 && c.p_hit < 1.0) || !(c.lik_floor > 0.0))
        return fail(nullptr, MAP_ERR_ARG, "need 0 < p_hit < 1 and lik_floor > 0");
    if (c.max_blocks < 1 || c.max_blocks > (1ll << 22) || c.hash_capacity < 2 || c.max_points < 1 ||
        c.max_pixels < 1 || c.max_points > (1ll << 31) - 1 || c.mesh_vertex_capacity < 1 ||
        c.mesh_triangle_capacity < 1 || c.mesh_vertex_capacity > (1ll << 31) - 1 ||
        c.mesh_triangle_capacity > (1ll << 31) - 1)
        return fail(nullptr, MAP_ERR_ARG, "capacity out of range");
    if (c.distance_mode == 1 && c.max_pixels > (1ll << 23))
        return fail(nullptr, MAP_ERR_ARG, "non-projective mode: max_pixels <= 2^23");
    if (map_mc_table(nullptr) != 0) return fail(nullptr, MAP_ERR_STATE, "marching-cubes table generation failed");

    m = new map_t();
    m->cfg = c;
    m->C = c.n_classes;
    uint64_t cap = 1;
    while (cap < (uint64_t)c.hash_capacity) cap <<= 1;
    if ((long long)cap < 2 * c.max_blocks) {
        while ((long long)cap < 2 * c.max_blocks) cap <<= 1;
    }
    m->cfg.hash_capacity = (int64_t)cap;
    const long long nb = c.max_blocks, nvox = nb * BV;
    MapDev &md = m->md;
    md.mask = cap - 1;
    md.max_blocks = (int)nb;
    md.C = c.n_classes;
    md.storage = c.storage;
    {
        // log-probability record per voxel padded to whole 16-byte chunks (the unit of the
        // vector and staged accesses): 20 classes take 80 B in FP32, 48 B in FP16
        const int per_chunk = c.storage == 0 ? 4 : 8;
        md.CP = ((c.n_classes + per_chunk - 1) / per_chunk) * per_chunk;
    }
    md.nu = (float)c.voxel_size;
    md.av_cap = c.mesh_vertex_capacity;
    md.at_cap = c.mesh_triangle_capacity;
    cudaError_t e = cudaSuccess;
#define ALLOC(p, n)                                                                    \
    do {                                                                               \
        e = dalloc(&(p), (size_t)(n));                                                 \
        if (e != cudaSuccess) {                                                        \
            std::string msg = std::string("device allocation failed: ") + #p;         \
            free_all(m);                                                               \
            delete m;                                                                  \
            return fail(nullptr, MAP_ERR_NOMEM, msg);                                  \
        }                                                                              \
    } while (0)
    ALLOC(md.hs, cap);
    ALLOC(md.dstamp_slot, nb);
    if (c.storage == 0) {
        ALLOC(md.dw32, nvox);
        ALLOC(md.lp32, nvox * md.CP);
    } else {
        ALLOC(md.dw16, nvox);
        ALLOC(md.lp16, nvox * md.CP);
    }
    ALLOC(md.label, nvox);
    if (c.distance_mode == 1) {
        if (c.storage == 0) ALLOC(md.g32, nvox * 3);
        else ALLOC(md.g16, nvox * 3);
        ALLOC(m->nrm, c.max_pixels);
        ALLOC(m->row_dir, c.max_pixels);
        ALLOC(m->col_dir, c.max_pixels);
    }
    ALLOC(md.slot_key, nb);
    ALLOC(md.slot_frame, nb);
    ALLOC(md.nbr, nb * 16);
    ALLOC(md.seg, nb);
    ALLOC(md.av, c.mesh_vertex_capacity);
    ALLOC(md.ak, c.mesh_vertex_capacity);
    ALLOC(md.at, c.mesh_triangle_capacity);
    ALLOC(m->av_alt, c.mesh_vertex_capacity);
    ALLOC(m->ak_alt, c.mesh_vertex_capacity);
    ALLOC(m->at_alt, c.mesh_triangle_capacity);
    ALLOC(m->st, 1);
    ALLOC(m->ctr_pair, 2 * CT_COUNT);
    ALLOC(m->d_ring, map_t::RING * map_t::REC_BYTES);
    m->ctr_buf[0] = m->ctr_pair;
    m->ctr_buf[1] = m->ctr_pair + CT_COUNT;
    md.st = m->st;
    FrameDev &fd = m->fd;
    ALLOC(m->win_buf[0], c.max_pixels);
    ALLOC(m->win_buf[1], c.max_pixels);
    fd.win = m->win_buf[1];
    ALLOC(fd.touched, nb);
    ALLOC(fd.dirty, nb);
    fd.sem_cap = std::min<long long>(nvox, 1ll << 25);
    ALLOC(fd.sem_list, fd.sem_cap);
    fd.ctr = m->ctr_buf[1];
    m->nchunks = (int)((nb + 1023) / 1024);
    ALLOC(m->gb.voff, nb);
    ALLOC(m->gb.toff, nb);
    ALLOC(m->gb.bsum_v, m->nchunks);
    ALLOC(m->gb.bsum_t, m->nchunks);
    ALLOC(m->gb.totals, 2);
    ALLOC(m->gn_T, 16);
    ALLOC(m->gn_acc, (size_t)GN_ACC_ROWS * GN_ACC_STRIDE);
    ALLOC(m->qb_part, (size_t)QB_PART_DOUBLES);
    ALLOC(m->pal_dev, 256);
    md.pal = m->pal_dev;
#undef ALLOC
    if (cudaMallocHost(&m->h_ctr, CT_COUNT * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMallocHost(&m->h_st, sizeof(DevState)) != cudaSuccess ||
        cudaMallocHost(&m->h_totals, 2 * sizeof(long long)) != cudaSuccess ||
        cudaMallocHost(&m->h_ring, map_t::RING * map_t::REC_BYTES) != cudaSuccess) {
        free_all(m);
        delete m;
        return fail(nullptr, MAP_ERR_NOMEM, "pinned host allocation failed");
    }
    std::memset(m->h_ctr, 0, CT_COUNT * sizeof(unsigned long long));
    std::memset(m->h_st, 0, sizeof(DevState));
    std::memset(m->h_ring, 0, map_t::RING * map_t::REC_BYTES);
    for (auto &e : m->ev_ring) cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    if (cudaStreamCreateWithFlags(&m->cp, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&m->ev_copied[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&m->ev_copied[1], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&m->ev_used[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&m->ev_used[1], cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithFlags(&m->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&m->dl, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&m->ev_snap, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&m->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&m->ev_join, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&m->ev_dir, cudaEventDisableTiming) != cudaSuccess) {
        free_all(m);
        delete m;
        return fail(nullptr, MAP_ERR_CUDA, "stream / event creation failed");
    }
    for (int i = 0; i < map_t::RING; ++i) m->ring_frame[i] = -1;

    cudaStream_t s = 0;
    cudaMemsetAsync(md.hs, 0xFF, cap * sizeof(HashSlot), s);   // key EMPTY_KEY, slot -1, stamp -1
    cudaMemsetAsync(md.dstamp_slot, 0xFF, nb * sizeof(int), s);
    cudaMemsetAsync(md.slot_frame, 0xFF, nb * sizeof(int), s);
    cudaMemsetAsync(md.nbr, 0xFF, nb * 16 * sizeof(int), s);
    // no gradient before a voxel's first normal
    if (md.g32) cudaMemsetAsync(md.g32, 0, (size_t)nvox * 3 * sizeof(float), s);
    if (md.g16) cudaMemsetAsync(md.g16, 0, (size_t)nvox * 3 * sizeof(__half), s);
    {
        DevState init;
        std::memset(&init, 0, sizeof(init));
        for (int p = 0; p < ARENA_PARTS; ++p) {
            arena_partition(0, (unsigned long long)c.mesh_vertex_capacity, p, init.arena_v_base[p], init.arena_v_end[p]);
            arena_partition(0, (unsigned long long)c.mesh_triangle_capacity, p, init.arena_t_base[p], init.arena_t_end[p]);
            init.arena_v[p] = init.arena_v_base[p];
            init.arena_t[p] = init.arena_t_base[p];
        }
        cudaMemcpy(m->st, &init, sizeof(init), cudaMemcpyHostToDevice);
    }
    cudaMemsetAsync(m->ctr_pair, 0, 2 * map_t::CTR_BYTES, s);
    cudaMemsetAsync(m->win_buf[0], 0xFF, (size_t)c.max_pixels * sizeof(unsigned long long), s);
    cudaMemsetAsync(m->win_buf[1], 0xFF, (size_t)c.max_pixels * sizeof(unsigned long long), s);
    launch_init_pool(md, s);
    // tables
    std::vector<int8_t> tri(256 * MAP_MC_MAXTRI * 3);
    map_mc_table(tri.data());
    std::vector<uint8_t> ntri(256, 0);
    for (int cs = 0; cs < 256; ++cs)
        for (int j = 0; j < MAP_MC_MAXTRI; ++j)
            if (tri[(cs * MAP_MC_MAXTRI + j) * 3] >= 0) ntri[cs] = (uint8_t)(j + 1);
    map_palette(c.n_classes, m->palette);
    {
        std::vector<uchar4> pal(256, make_uchar4(0, 0, 0, 0));
        for (int l = 0; l < c.n_classes; ++l)
            pal[l] = make_uchar4(m->palette[3 * l], m->palette[3 * l + 1], m->palette[3 * l + 2], 0);
        cudaMemcpy(m->pal_dev, pal.data(), 256 * sizeof(uchar4), cudaMemcpyHostToDevice);
    }
    if (mesh_upload_tables(tri.data(), ntri.data()) != 0) {
        free_all(m);
        delete m;
        return fail(nullptr, MAP_ERR_CUDA, "marching-cubes table upload failed");
    }
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    alloc_kernel_attributes();
    integrate_kernel_attributes();
    mesh_kernel_attributes();
    m->grid_integrate = sms * integrate_blocks_per_sm(c.storage, c.n_classes, c.distance_mode);
    // two waves of the class update's resident CTAs (measured best beside the re-meshing: one
    // wave leaves the list's tail to too few warps, more waves queue CTAs that only start as
    // earlier ones retire)
    m->grid_semantic = 2 * sms * semantic_blocks_per_sm(c.storage, c.n_classes);
    // 4 re-meshing CTAs per SM (the padded staging admits no more)
    m->grid_mesh = sms * std::min(4, mesh_blocks_per_sm());
    e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        std::string msg = std::string("map initialisation failed: ") + cudaGetErrorString(e);
        free_all(m);
        delete m;
        return fail(nullptr, MAP_ERR_CUDA, msg);
    }
    // extract_mesh_noalloc's static scratch array is placed on this device now,
    // while allocating is allowed, so that the call itself allocates nothing
    noalloc_prepare_device();
    *out = m;
    return MAP_OK;
}

extern "C" map_status map_destroy(map_t *m) {
    if (!m) return fail(nullptr, MAP_ERR_ARG, "null map");
    cudaDeviceSynchronize();
    free_all(m);
    delete m;
    return MAP_OK;
}

// Pixel-ray tables of the non-projective mode for intrinsics L (Sec. III-C.1
// read backwards: beam v at polar angle theta0 + v dtheta, column u at azimuth
// pi - u dphi), each sine and cosine an FP64 value split into a float pair.
// Uploaded when the intrinsics differ from the last upload's; the pinned copy
// is rewritten only after that upload has completed.
static map_status upload_pixel_rays(map_t *m, const lidar_intrinsics *L) {
    if (m->dir_valid && m->dir_for.H == L->H && m->dir_for.W == L->W && m->dir_for.fov_up == L->fov_up &&
        m->dir_for.fov_down == L->fov_down)
        return MAP_OK;
    CU(cudaEventSynchronize(m->ev_dir));
    const long long need = (long long)L->H + L->W;
    if (need > m->h_dir_cap) {
        if (m->h_dir) cudaFreeHost(m->h_dir);
        m->h_dir = nullptr;
        m->h_dir_cap = 0;
        if (cudaMallocHost(&m->h_dir, need * sizeof(float4)) != cudaSuccess)
            return fail(m, MAP_ERR_NOMEM, "pinned host allocation failed");
        m->h_dir_cap = need;
    }
    auto split = [](double x, float &hi, float &lo) {
        hi = (float)x;
        lo = (float)(x - (double)hi);
    };
    const double theta0 = M_PI / 2.0 - L->fov_up, dtheta = (L->fov_up - L->fov_down) / (L->H - 1);
    const double dphi = 2.0 * M_PI / L->W;
    for (int v = 0; v < L->H; ++v) {
        const double th = theta0 + (double)v * dtheta;
        float4 &q = m->h_dir[v];
        split(std::sin(th), q.x, q.y);
        split(std::cos(th), q.z, q.w);
    }
    for (int u = 0; u < L->W; ++u) {
        const double ph = M_PI - (double)u * dphi;
        float4 &q = m->h_dir[L->H + u];
        split(std::cos(ph), q.x, q.y);
        split(std::sin(ph), q.z, q.w);
    }
    CU(cudaMemcpyAsync(m->row_dir, m->h_dir, L->H * sizeof(float4), cudaMemcpyHostToDevice, m->cp));
    CU(cudaMemcpyAsync(m->col_dir, m->h_dir + L->H, L->W * sizeof(float4), cudaMemcpyHostToDevice, m->cp));
    CU(cudaEventRecord(m->ev_dir, m->cp));
    m->dir_for = *L;
    m->dir_valid = true;
    return MAP_OK;
}

// Pose checks of a scan (no map needed): a proper rigid transform, and every
// voxel the scan can reach (points up to r_max plus the band's tau) inside
// the coordinate range of block and mesh-vertex keys.  Returns MAP_OK or the
// status, with the reason in *why.
static map_status check_scan_pose(double nu, double tau, const lidar_intrinsics *L, const double *T,
                                  const char **why) {
    if (!L || !T) {
        *why = "null intrinsics or pose";
        return MAP_ERR_ARG;
    }
    if (!(L->fov_up > L->fov_down) || !(L->r_max > L->r_min) || !(L->r_min >= 0.0) || !std::isfinite(L->r_max)) {
        *why = "need fov_up > fov_down and 0 <= r_min < r_max (finite)";
        return MAP_ERR_ARG;
    }
    double R[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) R[3 * r + c] = T[4 * r + c];
    for (int i = 0; i < 16; ++i)
        if (!std::isfinite(T[i])) {
            *why = "non-finite pose";
            return MAP_ERR_BAD_POSE;
        }
    // R^T R = I, det R = +1, last row (0, 0, 0, 1)
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += R[3 * k + a] * R[3 * k + b];
            if (std::fabs(s - (a == b ? 1.0 : 0.0)) > 1e-6) {
                *why = "rotation not orthonormal";
                return MAP_ERR_BAD_POSE;
            }
        }
    const double det = R[0] * (R[4] * R[8] - R[5] * R[7]) - R[1] * (R[3] * R[8] - R[5] * R[6]) +
                       R[2] * (R[3] * R[7] - R[4] * R[6]);
    if (det < 0.0 || T[12] != 0.0 || T[13] != 0.0 || T[14] != 0.0 || T[15] != 1.0) {
        *why = "not a proper rigid transform";
        return MAP_ERR_BAD_POSE;
    }
    for (int k = 0; k < 3; ++k)
        if ((std::fabs(T[4 * k + 3]) + L->r_max + tau) / nu + 1.0 >= (double)MAX_VOXEL_COORD) {
            *why = "the scan reaches voxels beyond the map's coordinate range (|t| + r_max + tau < "
                   "(2^19 - 16) voxel_size on every axis)";
            return MAP_ERR_BAD_POSE;
        }
    return MAP_OK;
}

extern "C" map_status map_check_scan_pose(const map_config *cfg, const lidar_intrinsics *L,
                                          const double T_world_lidar[16]) {
    if (!cfg || !(cfg->voxel_size > 0.0) || !(cfg->truncation > 0.0))
        return fail(nullptr, MAP_ERR_ARG, "need a config with voxel_size > 0 and truncation > 0");
    const char *why = nullptr;
    const map_status st = check_scan_pose(cfg->voxel_size, cfg->truncation, L, T_world_lidar, &why);
    return st == MAP_OK ? MAP_OK : fail(nullptr, st, why);
}

static map_status make_scan_const(map_t *m, const lidar_intrinsics *L, int64_t n, const double *T, int has_probs,
                                  ScanConst &sc) {
    if (!L || !T) return fail(m, MAP_ERR_ARG, "null intrinsics or pose");
    if (L->H < 2 || L->W < 1 || (long long)L->H * L->W > m->cfg.max_pixels)
        return fail(m, MAP_ERR_ARG, "H * W out of range (H >= 2, H * W <= max_pixels)");
    if (n < 0 || n > m->cfg.max_points) return fail(m, MAP_ERR_ARG, "n out of range (<= max_points)");
    {
        const char *why = nullptr;
        const map_status pst = check_scan_pose(m->cfg.voxel_size, m->cfg.truncation, L, T, &why);
        if (pst != MAP_OK) return fail(m, pst, why);
    }
    double R[9], t[3];
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) R[3 * r + c] = T[4 * r + c];
        t[r] = T[4 * r + 3];
    }
    const double nu = m->cfg.voxel_size, tau = m->cfg.truncation;
    const double dtheta = (L->fov_up - L->fov_down) / (L->H - 1);
    std::memset(&sc, 0, sizeof(sc));
    sc.H = L->H;
    sc.W = L->W;
    sc.C = m->C;
    sc.n = (int)n;
    sc.inv_dphi = (float)(L->W / (2.0 * M_PI));
    sc.inv_dtheta = (float)(1.0 / dtheta);
    sc.theta0 = (float)(M_PI / 2.0 - L->fov_up);
    sc.r_min = (float)L->r_min;
    sc.r_max = (float)L->r_max;
    for (int i = 0; i < 9; ++i) sc.Rv[i] = (float)(R[i] / nu);
    for (int k = 0; k < 3; ++k) sc.tv[k] = (float)(t[k] / nu + 0.5);
    sc.tau = (float)tau;
    sc.inv_2tau = (float)(1.0 / (2.0 * tau));
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) sc.Rt[3 * r + c] = (float)R[3 * c + r];
    for (int k = 0; k < 3; ++k) {
        const double tv = t[k] / nu;
        const double fl = std::floor(tv);
        const double f = tv - fl;
        sc.k[k] = (int)fl;
        sc.fhi[k] = (float)f;
        sc.flo[k] = (float)(f - (double)sc.fhi[k]);
    }
    const double nu2 = nu * nu;
    sc.nu = (float)nu;
    sc.nu2hi = (float)nu2;
    sc.nu2lo = (float)(nu2 - (double)sc.nu2hi);
    sc.log_phit = (float)std::log(m->cfg.p_hit);
    sc.log_pmiss = (float)std::log((1.0 - m->cfg.p_hit) / (m->C - 1));
    sc.lik_floor = (float)m->cfg.lik_floor;
    sc.logp_floor = (float)m->cfg.logp_floor;
    sc.weight_mode = m->cfg.weight_mode;
    sc.frame = m->frame;
    sc.has_probs = has_probs;
    sc.probs_vec4 = 0;
    if (m->cfg.distance_mode == 1) {
        map_status st = upload_pixel_rays(m, L);
        if (st != MAP_OK) return st;
        sc.dist_mode = 1;
        sc.row_dir = m->row_dir;
        sc.col_dir = m->col_dir;
        sc.nrm = m->nrm;
    }
    return MAP_OK;
}

// Largest used fraction of any mesh-arena partition in a device-state copy.
static double arena_fill(const DevState &d) {
    double f = 0.0;
    for (int p = 0; p < ARENA_PARTS; ++p) {
        const double sv = (double)(d.arena_v_end[p] - d.arena_v_base[p]);
        const double st = (double)(d.arena_t_end[p] - d.arena_t_base[p]);
        if (sv > 0) f = std::max(f, (double)(d.arena_v[p] - d.arena_v_base[p]) / sv);
        if (st > 0) f = std::max(f, (double)(d.arena_t[p] - d.arena_t_base[p]) / st);
    }
    return f;
}

// The device state and the counters held by a ring entry.
static const DevState &ring_state(const map_t *m, int slot) {
    return *reinterpret_cast<const DevState *>(m->h_ring + (size_t)slot * map_t::REC_BYTES + map_t::CTR_BYTES);
}
static const unsigned long long *ring_ctr(const map_t *m, int slot) {
    return reinterpret_cast<const unsigned long long *>(m->h_ring + (size_t)slot * map_t::REC_BYTES);
}

// Fold a completed ring entry into the host's view of the arena fill.
static void absorb(map_t *m, int slot) {
    if (m->ring_frame[slot] < 0 || m->ring_epoch[slot] != m->epoch) return;
    if (m->ring_frame[slot] > m->known_frame) {
        const double f = arena_fill(ring_state(m, slot));
        if (m->known_frame >= 0 && f >= m->known_fill)
            m->max_append = std::max(m->max_append, (f - m->known_fill) / (double)(m->ring_frame[slot] - m->known_frame));
        m->known_fill = f;
        m->known_frame = m->ring_frame[slot];
    }
}

// Before frame f: read the completed ring entries.  They complete in frame
// order (one download stream), so the scan starts at the oldest entry not yet
// read and stops at the first still in flight; the entry of frame f - RING,
// whose slot frame f reuses, is waited for (the frames-in-flight bound).
static void poll_stats(map_t *m) {
    const long long reuse = (long long)m->frame - map_t::RING;
    for (long long f = std::max(m->absorbed + 1, reuse); f < m->frame; ++f) {
        const int slot = (int)(f % map_t::RING);
        if (f >= 0 && m->ring_frame[slot] == f) {
            if (f == reuse) cudaEventSynchronize(m->ev_ring[slot]);
            else if (cudaEventQuery(m->ev_ring[slot]) != cudaSuccess) break;
            absorb(m, slot);
        }
        m->absorbed = f;    // read, or a batched step (no ring entry)
    }
}

// Compact when a partition could pass 3/4 of its space before the host sees it
// again (per-partition growth estimated at twice the largest seen).
static bool need_compaction(const map_t *m) {
    const double lag = (double)(m->frame - m->known_frame) + 1.0;
    return m->known_fill + 2.0 * lag * m->max_append > 0.75;
}

static map_status compact_arena(map_t *m, cudaStream_t s) {
    m->launches += 4;
    launch_seg_scan(m->md, m->gb, m->md.max_blocks, s);
    launch_seg_gather(m->md, m->gb, m->md.max_blocks, 0, m->av_alt, m->ak_alt, m->at_alt, nullptr, nullptr, nullptr,
                      nullptr, nullptr, s);
    launch_set_cursors(m->md, m->gb, s);
    std::swap(m->md.av, m->av_alt);
    std::swap(m->md.ak, m->ak_alt);
    std::swap(m->md.at, m->at_alt);
    // readings taken before this point describe the old arena
    m->epoch++;
    m->known_fill = 0.0;
    m->known_frame = m->frame - 1;
    return launch_check(m, "arena compaction");
}

static map_status run_frame(map_t *m, const lidar_intrinsics *L, const float *pts, const int32_t *labels,
                            const float *probs, int64_t n, const double *T, cudaStream_t s) {
    ScanConst sc;
    map_status st = make_scan_const(m, L, n, T, probs != nullptr, sc);
    if (st != MAP_OK) return st;
    sc.pts = pts;
    sc.labels = labels;
    sc.probs = probs;
    sc.probs_vec4 = probs && (m->C % 4 == 0) && (((uintptr_t)probs & 15) == 0);
    // inside a stream capture (a batch step replayed from a graph): no phase
    // timing, and the download and its ring event go into the graph (below)
    cudaStreamCaptureStatus cap_status = cudaStreamCaptureStatusNone;
    CU(cudaStreamIsCapturing(s, &cap_status));
    const bool capturing = cap_status != cudaStreamCaptureStatusNone;
    poll_stats(m);
    if (need_compaction(m)) {
        st = compact_arena(m, s);
        if (st != MAP_OK) return st;
    }
    const long long np = (long long)L->H * L->W;
    // this scan's range-image and counter set; the per-point kernel resets the other
    const int cur = m->fcur ^ 1, nxt = m->fcur;
    m->fcur = cur;
    m->fd.win = m->win_buf[cur];
    m->fd.ctr = m->ctr_buf[cur];
    FrameDev fd = m->fd;
    fd.win_next = m->win_buf[nxt];
    fd.win_next_n = m->win_dirty[nxt];
    fd.ctr_next = m->ctr_buf[nxt];
    cudaEvent_t *ev = nullptr;
    unsigned long long *ev_stats = nullptr;
    if (!capturing && m->prof_n < m->prof_cap) {
        ev_stats = m->prof_stats + (size_t)m->prof_n * CT_COUNT;
        m->prof_serial[m->prof_n] = m->concurrent ? 0 : 1;
        ev = &m->prof_ev[(size_t)m->prof_n++ * (MAP_PHASE_COUNT + 1)];
    }
    if (ev) CU(cudaEventRecord(ev[0], s));
    // only when the previous scan did not leave this set clean (first use after
    // a failed call): the resets the per-point kernel otherwise does ahead
    if (m->win_dirty[cur] > 0)
        CU(cudaMemsetAsync(fd.win, 0xFF, std::min(m->win_dirty[cur], (long long)m->cfg.max_pixels) * sizeof(unsigned long long), s));
    if (!m->ctr_clean[cur]) CU(cudaMemsetAsync(fd.ctr, 0, map_t::CTR_BYTES, s));
    if (ev) CU(cudaEventRecord(ev[1], s));
    m->win_dirty[cur] = np;
    m->ctr_clean[cur] = false;
    launch_points(pts, sc, m->md, fd, s);
    if (fd.dbg_point) {
        m->dbg_frame = m->frame;
        m->dbg_n = n;
        m->dbg_np = np;
    }
    m->win_dirty[nxt] = 0;
    m->ctr_clean[nxt] = true;
    if (sc.dist_mode) {
        // pixel-ray tables uploaded (a capturing caller has waited for them before the capture)
        if (!capturing) CU(cudaStreamWaitEvent(s, m->ev_dir, 0));
        launch_normals(sc, m->fd, s);
        m->launches += 1;
    }
    if (ev) CU(cudaEventRecord(ev[2], s));
    launch_integrate(sc, m->md, m->fd, m->grid_integrate, s);
    if (ev) CU(cudaEventRecord(ev[3], s));
    if (m->concurrent) {
        // class update on the side stream, re-meshing on the caller's, concurrently
        CU(cudaEventRecord(m->ev_fork, s));
        CU(cudaStreamWaitEvent(m->side, m->ev_fork, 0));
        launch_semantic(sc, m->md, m->fd, m->grid_semantic, m->side);
        if (ev) CU(cudaEventRecord(ev[4], m->side));
        if (m->mesh_per_frame) launch_mesh(m->md, m->fd, m->grid_mesh, s);
        if (ev) CU(cudaEventRecord(ev[5], s));
        CU(cudaEventRecord(m->ev_join, m->side));
        CU(cudaStreamWaitEvent(s, m->ev_join, 0));
    } else {
        // one after the other on the caller's stream: re-meshing (a programmatic dependent of the
        // TSDF grid, as above), then the class update
        if (m->mesh_per_frame) launch_mesh(m->md, m->fd, m->grid_mesh, s);
        if (ev) CU(cudaEventRecord(ev[5], s));
        launch_semantic(sc, m->md, m->fd, m->grid_semantic, s);
        if (ev) CU(cudaEventRecord(ev[4], s));
    }
    m->launches += m->mesh_per_frame ? 4 : 3;
    if (ev_stats)
        CU(cudaMemcpyAsync(ev_stats, m->fd.ctr, CT_COUNT * sizeof(unsigned long long), cudaMemcpyDeviceToDevice, s));
    st = launch_check(m, "integrate_scan kernels");
    if (st != MAP_OK) return st;
    // snapshot [counters | state] on the device, download it beside the next scan
    const int slot = m->frame % map_t::RING;
    unsigned char *rec = m->d_ring + (size_t)slot * map_t::REC_BYTES;
    launch_snapshot(m->fd.ctr, m->st, rec, s);
    m->launches += 1;
    if (capturing) {
        // in the graph, on this stream; the ring event as an event-record node, so that the
        // host's later queries of it see each replay
        CU(cudaMemcpyAsync(m->h_ring + (size_t)slot * map_t::REC_BYTES, rec, map_t::REC_BYTES,
                           cudaMemcpyDeviceToHost, s));
        CU(cudaEventRecordWithFlags(m->ev_ring[slot], s, cudaEventRecordExternal));
    } else {
        CU(cudaEventRecord(m->ev_snap, s));
        CU(cudaStreamWaitEvent(m->dl, m->ev_snap, 0));
        CU(cudaMemcpyAsync(m->h_ring + (size_t)slot * map_t::REC_BYTES, rec, map_t::REC_BYTES,
                           cudaMemcpyDeviceToHost, m->dl));
        CU(cudaEventRecord(m->ev_ring[slot], m->dl));
    }
    m->h_ctr_slot = slot;
    m->ring_frame[slot] = m->frame;
    m->ring_epoch[slot] = m->epoch;
    m->frame++;
    return MAP_OK;
}

extern "C" map_status integrate_scan(map_t *m, const lidar_intrinsics *L, const float *points_dev,
                                     const int32_t *labels_dev, const float *probs_dev, int64_t n,
                                     const double T_world_lidar[16], void *stream) {
    if (!m) return fail(nullptr, MAP_ERR_ARG, "null map");
    if (n > 0 && (!points_dev || ((labels_dev == nullptr) == (probs_dev == nullptr))))
        return fail(m, MAP_ERR_ARG, "need points and exactly one of labels / probs");
    return run_frame(m, L, points_dev, labels_dev, probs_dev, n, T_world_lidar, (cudaStream_t)stream);
}

extern "C" map_status integrate_scan_host(map_t *m, const lidar_intrinsics *L, const float *points_host,
                                          const int32_t *labels_host, const float *probs_host, int64_t n,
                                          const double T_world_lidar[16], void *stream) {
    if (!m) return fail(nullptr, MAP_ERR_ARG, "null map");
    if (n > 0 && (!points_host || ((labels_host == nullptr) == (probs_host == nullptr))))
        return fail(m, MAP_ERR_ARG, "need points and exactly one of labels / probs");
    if (n < 0 || n > m->cfg.max_points) return fail(m, MAP_ERR_ARG, "n out of range (<= max_points)");
    cudaStream_t s = (cudaStream_t)stream;
    const long long cap = m->cfg.max_points;
    // alternate staging sets: this scan's upload (copy stream) waits only for the
    // scan that last read the same set, so it overlaps the previous scan's kernels
    const int b = m->stage_next;
    m->stage_next ^= 1;
    if (!m->stage_pts[b]) CU(cudaMalloc(&m->stage_pts[b], cap * 3 * sizeof(float)));
    if (labels_host && !m->stage_lab[b]) CU(cudaMalloc(&m->stage_lab[b], cap * sizeof(int32_t)));
    if (probs_host && !m->stage_probs[b]) CU(cudaMalloc(&m->stage_probs[b], cap * m->C * sizeof(float)));
    CU(cudaStreamWaitEvent(m->cp, m->ev_used[b], 0));
    if (n > 0) {
        CU(cudaMemcpyAsync(m->stage_pts[b], points_host, n * 3 * sizeof(float), cudaMemcpyHostToDevice, m->cp));
        if (labels_host)
            CU(cudaMemcpyAsync(m->stage_lab[b], labels_host, n * sizeof(int32_t), cudaMemcpyHostToDevice, m->cp));
        else
            CU(cudaMemcpyAsync(m->stage_probs[b], probs_host, n * m->C * sizeof(float), cudaMemcpyHostToDevice,
                               m->cp));
    }
    CU(cudaEventRecord(m->ev_copied[b], m->cp));
    CU(cudaStreamWaitEvent(s, m->ev_copied[b], 0));
    const map_status st = run_frame(m, L, m->stage_pts[b], labels_host ? m->stage_lab[b] : nullptr,
                                    probs_host ? m->stage_probs[b] : nullptr, n, T_world_lidar, s);
    CU(cudaEventRecord(m->ev_used[b], s));
    return st;
}

extern "C" map_status map_remesh_all(map_t *m, void *stream) {
    if (!m) return fail(nullptr, MAP_ERR_ARG, "null map");
    cudaStream_t s = (cudaStream_t)stream;
    // every block is re-meshed and rewrites its segment, so the old arena
    // contents are dropped rather than compacted: cursors back to empty
    CU(cudaMemsetAsync(m->gb.totals, 0, 2 * sizeof(long long), s));
    launch_set_cursors(m->md, m->gb, s);
    m->epoch++;
    m->known_fill = 0.0;
    m->known_frame = m->frame - 1;
    CU(cudaMemsetAsync(m->fd.ctr, 0, CT_COUNT * sizeof(unsigned long long), s));
    launch_list_all(m->md, m->fd, m->frame, s);
    launch_mesh(m->md, m->fd, m->grid_mesh, s);
    m->launches += 3;
    map_status st = launch_check(m, "map_remesh_all");
    if (st != MAP_OK) return st;
    // map_get_frame_stats now reports this pass (blocks meshed, vertices, triangles)
    CU(cudaMemcpyAsync(m->h_ctr, m->fd.ctr, CT_COUNT * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    m->h_ctr_slot = -1;
    return MAP_OK;
}

extern "C" map_status map_set_concurrent_phases(map_t *m, int32_t concurrent) {
    if (!m) return fail(nullptr, MAP_ERR_ARG, "null map");
    if (concurrent != 0 && concurrent != 1) return fail(m, MAP_ERR_ARG, "concurrent must be 0 or 1");
    m->concurrent = concurrent == 1;
    return MAP_OK;
}

extern "C" map_status map_set_incremental_mesh(map_t *m, int32_t enabled) {
    if (!m || (enabled != 0 && enabled != 1)) return fail(m, MAP_ERR_ARG, "enabled must be 0 or 1");
    m->mesh_per_frame = enabled == 1;
    return MAP_OK;
}

static map_status device_errors_of(map_t *m, const DevState &d) {
    if (d.err & ERR_TIMEOUT) return fail(m, MAP_ERR_TIMEOUT, "a device-side wait gave up");
    if (d.err) {
        char buf[128];
        std::snprintf(buf, sizeof buf, "device capacity exceeded (error bits 0x%x)", d.err);
        return fail(m, MAP_ERR_CAPACITY, buf);
    }
    return MAP_OK;
}

static map_status device_errors(map_t *m) {
    if (m->h_st->err & ERR_TIMEOUT) return fail(m, MAP_ERR_TIMEOUT, "a device-side wait gave up");
    if (m->h_st->err) {
        char buf[128];
        std::snprintf(buf, sizeof buf, "device capacity exceeded (error bits 0x%x)", m->h_st->err);
        return fail(m, MAP_ERR_CAPACITY, buf);
    }
    return MAP_OK;
}

extern "C" int64_t map_frame_count(map_t *m) { return m ? (int64_t)m->frame : -1; }

extern "C" map_status map_frame_stats(map_t *m, int64_t frame, int64_t *out) {
    if (!m || !out) return fail(m, MAP_ERR_ARG, "null argument");
    if (frame < 0 || frame >= m->frame || frame < m->frame - map_t::RING)
        return fail(m, MAP_ERR_ARG, "frame out of range (one of the last 8 integrated scans)");
    const int slot = (int)(frame % map_t::RING);
    if (m->ring_frame[slot] != frame) return fail(m, MAP_ERR_ARG, "frame no longer held");
    CU(cudaEventSynchronize(m->ev_ring[slot]));
    for (int i = 0; i < MAP_STAT_COUNT; ++i) out[i] = 0;
    const unsigned long long *c = ring_ctr(m, slot);
    const DevState &d = ring_state(m, slot);
    for (int i = 0; i < CT_MT + 1; ++i) out[i] = (int64_t)c[i];
    out[MAP_STAT_TOTAL_BLOCKS] = (int64_t)std::min<unsigned long long>(d.pool_count, m->md.max_blocks);
    out[MAP_STAT_ERROR_BITS] = (int64_t)d.err;
    out[MAP_STAT_KERNEL_LAUNCHES] = (int64_t)m->launches;
    return device_errors_of(m, d);
}

extern "C" map_status map_sync(map_t *m, void *stream) {
    if (!m) return fail(nullptr, MAP_ERR_ARG, "null map");
    cudaStream_t s = (cudaStream_t)stream;
    CU(cudaMemcpyAsync(m->h_st, m->st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    m->known_fill = arena_fill(*m->h_st);
    m->known_frame = m->frame - 1;
    return device_errors(m);
}

extern "C" map_status map_get_frame_stats(map_t *m, int64_t *out, void *stream) {
    if (!m || !out) return fail(m, MAP_ERR_ARG, "null argument");
    map_status st = map_sync(m, stream);
    if (m->h_ctr_slot >= 0) {
        CU(cudaEventSynchronize(m->ev_ring[m->h_ctr_slot]));
        std::memcpy(m->h_ctr, ring_ctr(m, m->h_ctr_slot), map_t::CTR_BYTES);
    }
    for (int i = 0; i < MAP_STAT_COUNT; ++i) out[i] = 0;
    for (int i = 0; i < CT_MT + 1; ++i) out[i] = (int64_t)m->h_ctr[i];
    out[MAP_STAT_TOTAL_BLOCKS] = (int64_t)std::min<unsigned long long>(m->h_st->pool_count, m->md.max_blocks);
    out[MAP_STAT_ERROR_BITS] = (int64_t)m->h_st->err;
    out[MAP_STAT_KERNEL_LAUNCHES] = (int64_t)m->launches;
    return st;
}

extern "C" map_status extract_mesh(map_t *m, mesh_view *out, void *stream) {
    if (!m || !out) return fail(m, MAP_ERR_ARG, "null argument");
    cudaStream_t s = (cudaStream_t)stream;
    launch_seg_scan(m->md, m->gb, m->md.max_blocks, s);
    CU(cudaMemcpyAsync(m->h_totals, m->gb.totals, 2 * sizeof(long long), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    const long long nv = m->h_totals[0], nt = m->h_totals[1];
    if (nv > m->out_vcap) {
        if (m->out_pos) cudaFree(m->out_pos);
        if (m->out_col) cudaFree(m->out_col);
        if (m->out_keys) cudaFree(m->out_keys);
        m->out_pos = nullptr;
        m->out_col = nullptr;
        m->out_keys = nullptr;
        m->out_vcap = 0;
        CU(cudaMalloc(&m->out_pos, nv * 3 * sizeof(float) + 16));
        CU(cudaMalloc(&m->out_col, nv * 4 + 16));
        CU(cudaMalloc(&m->out_keys, nv * sizeof(int64_t) + 16));
        m->out_vcap = nv;
    }
    if (nt > m->out_tcap) {
        if (m->out_tri) cudaFree(m->out_tri);
        if (m->out_anchor) cudaFree(m->out_anchor);
        m->out_tri = nullptr;
        m->out_anchor = nullptr;
        m->out_tcap = 0;
        CU(cudaMalloc(&m->out_tri, nt * 3 * sizeof(int32_t) + 16));
        CU(cudaMalloc(&m->out_anchor, nt * 3 * sizeof(int32_t) + 16));
        m->out_tcap = nt;
    }
    launch_seg_gather(m->md, m->gb, m->md.max_blocks, 1, nullptr, nullptr, nullptr, m->out_pos, m->out_col,
                      m->out_keys, m->out_tri, m->out_anchor, s);
    map_status st = launch_check(m, "extract_mesh");
    if (st != MAP_OK) return st;
    m->ext_valid = true;
    m->ext_nv = nv;
    m->ext_nt = nt;
    out->n_vertices = nv;
    out->n_triangles = nt;
    out->positions = m->out_pos;
    out->colors = m->out_col;
    out->vertex_keys = m->out_keys;
    out->triangles = m->out_tri;
    out->triangle_anchors = m->out_anchor;
    return MAP_OK;
}

extern "C" map_status integrate_labels_camera(map_t *m, const camera_intrinsics *cam, const int32_t *labels_dev,
                                              const float *probs_dev, const double T_world_cam[16], float *range_dev,
                                              void *stream) {
    if (!m || !cam || !T_world_cam || ((labels_dev == nullptr) == (probs_dev == nullptr)))
        return fail(m, MAP_ERR_ARG, "need intrinsics, a pose and exactly one of labels / probs");
    if (cam->width < 1 || cam->height < 1 || (long long)cam->width * cam->height > (1ll << 26) ||
        !(cam->fx > 0.0) || !(cam->fy > 0.0) || !(cam->r_max > 0.0) || !(cam->r_max < 1e4))
        return fail(m, MAP_ERR_ARG, "bad camera intrinsics (1 <= W*H <= 2^26, fx, fy > 0, 0 < r_max < 1e4)");
    for (int i = 0; i < 16; ++i)
        if (!std::isfinite(T_world_cam[i])) return fail(m, MAP_ERR_BAD_POSE, "non-finite camera pose");
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double q = 0.0;
            for (int k = 0; k < 3; ++k) q += T_world_cam[4 * k + a] * T_world_cam[4 * k + b];
            if (std::fabs(q - (a == b ? 1.0 : 0.0)) > 1e-6) return fail(m, MAP_ERR_BAD_POSE, "rotation not orthonormal");
        }
    for (int k = 0; k < 3; ++k)
        if ((std::fabs(T_world_cam[4 * k + 3]) + cam->r_max) / m->cfg.voxel_size + 1.0 >= (double)MAX_VOXEL_COORD)
            return fail(m, MAP_ERR_BAD_POSE, "the camera reaches voxels beyond the map's coordinate range "
                                             "(|t| + r_max < (2^19 - 16) voxel_size on every axis)");
    cudaStream_t s = (cudaStream_t)stream;
    const long long np = (long long)cam->width * cam->height;
    float *range = range_dev;
    if (!range) {
        if (np > m->cam_range_cap) {
            CU(cudaStreamSynchronize(s));
            if (m->cam_range) cudaFree(m->cam_range);
            m->cam_range = nullptr;
            m->cam_range_cap = 0;
            CU(cudaMalloc(&m->cam_range, np * sizeof(float)));
            m->cam_range_cap = np;
        }
        range = m->cam_range;
    }
    CamConst cc;
    cc.W = cam->width;
    cc.H = cam->height;
    const double nu = m->cfg.voxel_size;
    cc.max_steps = (int)std::min(1e8, 3.0 * cam->r_max / nu + 8.0);
    cc.fx = (float)cam->fx;
    cc.fy = (float)cam->fy;
    cc.cx = (float)cam->cx;
    cc.cy = (float)cam->cy;
    cc.inv_fx = (float)(1.0 / cam->fx);
    cc.inv_fy = (float)(1.0 / cam->fy);
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) cc.R[3 * r + c] = (float)T_world_cam[4 * r + c];
        cc.c[r] = (float)T_world_cam[4 * r + 3];
    }
    cc.nu = (float)nu;
    cc.inv_nu = (float)(1.0 / nu);
    cc.r_max = (float)cam->r_max;
    // class-update constants: the likelihood model of the scans, per pixel of the image
    ScanConst sc;
    std::memset(&sc, 0, sizeof(sc));
    sc.C = m->C;
    sc.tau = (float)m->cfg.truncation;
    sc.log_phit = (float)std::log(m->cfg.p_hit);
    sc.log_pmiss = (float)std::log((1.0 - m->cfg.p_hit) / (m->C - 1));
    sc.lik_floor = (float)m->cfg.lik_floor;
    sc.logp_floor = (float)m->cfg.logp_floor;
    sc.has_probs = probs_dev != nullptr;
    sc.probs_vec4 = probs_dev && (m->C % 4 == 0) && (((uintptr_t)probs_dev & 15) == 0);
    sc.labels = labels_dev;
    sc.probs = probs_dev;
    CU(cudaMemsetAsync(m->fd.ctr, 0, CT_COUNT * sizeof(unsigned long long), s));
    if (!m->cam_bounds) CU(cudaMalloc(&m->cam_bounds, 6 * sizeof(int)));
    CU(cudaMemsetAsync(m->cam_bounds, 0x7F, 3 * sizeof(int), s));        // min: 0x7f7f7f7f
    CU(cudaMemsetAsync(m->cam_bounds + 3, 0x80, 3 * sizeof(int), s));    // max: 0x80808080 (< any block)
    launch_camera(cc, sc, m->md, m->fd, range, m->cam_bounds, m->grid_semantic, s);
    m->launches += 4;
    map_status st = launch_check(m, "integrate_labels_camera");
    if (st != MAP_OK) return st;
    // map_get_frame_stats now reports this image (MAP_STAT_VOXELS_SEMANTIC)
    CU(cudaMemcpyAsync(m->h_ctr, m->fd.ctr, CT_COUNT * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    m->h_ctr_slot = -1;
    return MAP_OK;
}

extern "C" map_status map_trav_params_default(trav_params *p) {
    if (!p) return fail(nullptr, MAP_ERR_ARG, "null parameters");
    p->radius = 0.25;
    p->max_height_diff = 0.6;
    p->max_steepness = 20.0 * M_PI / 180.0;
    p->max_roughness = 30.0 * M_PI / 180.0;
    p->class_mask = ~0ull;
    return MAP_OK;
}

static void trav_free(TravDev &t) {
    void *ptrs[] = {t.vkeys, t.vfirst, t.rep, t.nacc, t.vcell, t.ckeys, t.ccount, t.cstart, t.cfill, t.spos, t.snrm,
                    t.cursor};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    t = TravDev{};
}

// Traversability / welding scratch for meshes of up to nv vertices (grows; synchronises `s` to grow).
static map_status trav_ensure(map_t *m, long long nv, cudaStream_t s) {
    TravDev &b = m->trav;
    if (nv <= m->trav_nv_cap) return MAP_OK;
    CU(cudaStreamSynchronize(s));
    trav_free(b);
    m->trav_nv_cap = 0;
    uint64_t cap = 1024;
    while ((long long)cap < 2 * nv) cap <<= 1;
    cudaError_t e = cudaSuccess;
    auto A = [&](auto **q, size_t count) {
        if (e == cudaSuccess) e = cudaMalloc((void **)q, count * sizeof(**q) + 16);
    };
    A(&b.vkeys, cap);
    A(&b.vfirst, cap);
    A(&b.ckeys, cap);
    A(&b.ccount, cap);
    A(&b.cstart, cap);
    A(&b.cfill, cap);
    A(&b.rep, (size_t)nv);
    A(&b.nacc, (size_t)nv);
    A(&b.vcell, (size_t)nv);
    A(&b.spos, (size_t)nv);
    A(&b.snrm, (size_t)nv);
    A(&b.cursor, 1);
    if (e != cudaSuccess) {
        trav_free(b);
        return fail(m, MAP_ERR_NOMEM, "mesh scratch allocation failed");
    }
    b.vmask = b.cmask = cap - 1;
    m->trav_nv_cap = nv;
    return MAP_OK;
}

static void grid_free(GridDev &g) {
    void *ptrs[] = {g.ckeys, g.ccount, g.cstart, g.cfill, g.spts, g.slot, g.cursor};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    g = GridDev{};
}

// A point grid for clouds of up to n points (grows); returns false on allocation failure.
static bool grid_ensure(GridDev &g, long long &cap_n, long long n) {
    if (n <= cap_n) return true;
    grid_free(g);
    cap_n = 0;
    uint64_t cap = 1024;
    while ((long long)cap < 2 * n) cap <<= 1;
    cudaError_t e = cudaSuccess;
    auto A = [&](auto **q, size_t count) {
        if (e == cudaSuccess) e = cudaMalloc((void **)q, count * sizeof(**q) + 16);
    };
    A(&g.ckeys, cap);
    A(&g.ccount, cap);
    A(&g.cstart, cap);
    A(&g.cfill, cap);
    A(&g.spts, (size_t)n);
    A(&g.slot, (size_t)n);
    A(&g.cursor, 1);
    if (e != cudaSuccess) {
        grid_free(g);
        return false;
    }
    g.cmask = cap - 1;
    cap_n = n;
    return true;
}

static map_status grid_reset(map_t *m, GridDev &g, double cell, cudaStream_t s) {
    const size_t tab = (size_t)(g.cmask + 1);
    CU(cudaMemsetAsync(g.ckeys, 0xFF, tab * sizeof(uint64_t), s));
    CU(cudaMemsetAsync(g.ccount, 0, tab * sizeof(int), s));
    CU(cudaMemsetAsync(g.cfill, 0, tab * sizeof(int), s));
    CU(cudaMemsetAsync(g.cursor, 0, sizeof(unsigned long long), s));
    g.err = &m->st->err;
    g.inv_cell = (float)(1.0 / (cell * (1.0 + 1e-5)));
    return MAP_OK;
}

extern "C" map_status map_quality(map_t *m, const float *gt_points_dev, const int32_t *gt_labels_dev, int64_t n_gt,
                                  double trunc, quality_report *out, int64_t *confusion, void *stream) {
    if (!m || !out || n_gt < 1 || !gt_points_dev || !gt_labels_dev || !(trunc > 0.0) || !(trunc < 1e3))
        return fail(m, MAP_ERR_ARG, "bad quality arguments (need n_gt >= 1, 0 < trunc < 1e3)");
    if (!m->ext_valid || m->ext_nv < 1) return fail(m, MAP_ERR_STATE, "no extracted mesh (call extract_mesh first)");
    cudaStream_t s = (cudaStream_t)stream;
    const long long nv = m->ext_nv;
    const int C = m->C;
    map_status st = trav_ensure(m, nv, s);
    if (st != MAP_OK) return st;
    if (!grid_ensure(m->q_map, m->q_map_cap, nv) || !grid_ensure(m->q_gt, m->q_gt_cap, n_gt))
        return fail(m, MAP_ERR_NOMEM, "quality scratch allocation failed");
    if (!m->q_acc) CU(cudaMalloc(&m->q_acc, sizeof(QualityAcc)));
    if (!m->q_conf) CU(cudaMalloc(&m->q_conf, 64 * 64 * sizeof(unsigned long long)));
    TravDev &b = m->trav;
    b.err = &m->st->err;
    CU(cudaMemsetAsync(b.vkeys, 0xFF, (size_t)(b.vmask + 1) * sizeof(uint64_t), s));
    CU(cudaMemsetAsync(b.vfirst, 0x7F, (size_t)(b.vmask + 1) * sizeof(int), s));
    st = grid_reset(m, m->q_map, trunc, s);
    if (st == MAP_OK) st = grid_reset(m, m->q_gt, trunc, s);
    if (st != MAP_OK) return st;
    CU(cudaMemsetAsync(m->q_acc, 0, sizeof(QualityAcc), s));
    CU(cudaMemsetAsync(m->q_conf, 0, (size_t)C * C * sizeof(unsigned long long), s));
    launch_weld(b, m->out_keys, nv, s);
    launch_quality(m->q_map, m->q_gt, b.rep, m->out_pos, m->out_col, nv, gt_points_dev, gt_labels_dev, n_gt,
                   (float)trunc, C, m->q_acc, m->q_conf, s);
    m->launches += 10;
    st = launch_check(m, "map_quality");
    if (st != MAP_OK) return st;
    QualityAcc a;
    std::vector<unsigned long long> conf((size_t)C * C);
    CU(cudaMemcpyAsync(&a, m->q_acc, sizeof(a), cudaMemcpyDeviceToHost, s));
    CU(cudaMemcpyAsync(conf.data(), m->q_conf, conf.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    st = map_sync(m, stream);
    if (st != MAP_OK) return st;
    out->n_map = (int64_t)a.n_map;
    out->n_gt = (int64_t)a.n_gt;
    out->n_labeled = (int64_t)a.n_labeled;
    out->re = a.n_map ? std::sqrt(a.sum_d2_map / (double)a.n_map) : 0.0;
    out->cd = (a.n_map && a.n_gt) ? 0.5 * a.sum_d_map / (double)a.n_map + 0.5 * a.sum_d_gt / (double)a.n_gt : 0.0;
    out->rc = a.n_gt ? (double)a.n_gt_covered / (double)a.n_gt : 0.0;
    // mIoU over the classes that occur, accuracy over the labelled vertices
    double iou_sum = 0.0, tp_sum = 0.0, all = 0.0;
    int occ = 0;
    for (int c = 0; c < C; ++c) {
        double tp = (double)conf[(size_t)c * C + c], row = 0.0, colsum = 0.0;
        for (int k = 0; k < C; ++k) {
            row += (double)conf[(size_t)c * C + k];
            colsum += (double)conf[(size_t)k * C + c];
        }
        const double den = row + colsum - tp;
        if (den > 0) {
            iou_sum += tp / den;
            ++occ;
        }
        tp_sum += tp;
        all += row;
    }
    out->miou = occ ? iou_sum / occ : 0.0;
    out->acc = all > 0 ? tp_sum / all : 0.0;
    out->n_correct = (int64_t)tp_sum;
    if (confusion)
        for (size_t i = 0; i < conf.size(); ++i) confusion[i] = (int64_t)conf[i];
    return MAP_OK;
}

extern "C" map_status map_traversability(map_t *m, const trav_params *p, float *props_dev, uint8_t *trav_dev,
                                         void *stream) {
    if (!m || !p || (m->ext_nv > 0 && (!props_dev || !trav_dev))) return fail(m, MAP_ERR_ARG, "bad arguments");
    if (!(p->radius > 0.0) || !(p->radius < 1e4)) return fail(m, MAP_ERR_ARG, "need 0 < radius < 1e4 m");
    if (!m->ext_valid) return fail(m, MAP_ERR_STATE, "no extracted mesh (call extract_mesh first)");
    cudaStream_t s = (cudaStream_t)stream;
    const long long nv = m->ext_nv, nt = m->ext_nt;
    if (nv == 0) return MAP_OK;
    map_status st = trav_ensure(m, nv, s);
    if (st != MAP_OK) return st;
    TravDev &b = m->trav;
    b.err = &m->st->err;
    b.inv_cell = (float)(1.0 / (p->radius * (1.0 + 1e-5)));
    const size_t tab = (size_t)(b.vmask + 1);
    CU(cudaMemsetAsync(b.vkeys, 0xFF, tab * sizeof(uint64_t), s));
    CU(cudaMemsetAsync(b.vfirst, 0x7F, tab * sizeof(int), s));
    CU(cudaMemsetAsync(b.ckeys, 0xFF, tab * sizeof(uint64_t), s));
    CU(cudaMemsetAsync(b.ccount, 0, tab * sizeof(int), s));
    CU(cudaMemsetAsync(b.cfill, 0, tab * sizeof(int), s));
    CU(cudaMemsetAsync(b.nacc, 0, (size_t)nv * sizeof(float4), s));
    CU(cudaMemsetAsync(b.cursor, 0, sizeof(unsigned long long), s));
    TravParamsDev pd;
    pd.r2 = (float)(p->radius * p->radius);
    pd.t_hd = (float)p->max_height_diff;
    pd.t_s = (float)p->max_steepness;
    pd.t_r = (float)p->max_roughness;
    pd.class_mask = p->class_mask;
    launch_traversability(b, pd, m->out_pos, m->out_col, m->out_keys, m->out_tri, nv, nt,
                          reinterpret_cast<float4 *>(props_dev), trav_dev, s);
    m->launches += nt > 0 ? 7 : 6;
    return launch_check(m, "map_traversability");
}

extern "C" map_status query_sdf(map_t *m, const float *xyz_dev, int64_t n, float *sdf_dev, uint8_t *valid_dev,
                                void *stream) {
    if (!m || n < 0 || (n > 0 && (!xyz_dev || !sdf_dev))) return fail(m, MAP_ERR_ARG, "bad query arguments");
    launch_query(m->md, xyz_dev, n, sdf_dev, valid_dev, (cudaStream_t)stream);
    return launch_check(m, "query_sdf");
}

extern "C" map_status query_sdf_backward(map_t *m, const float *xyz_dev, const float *grad_sdf_dev, int64_t n,
                                         float *grad_xyz_dev, double *pose_grad_dev, void *stream) {
    if (!m || n < 0 || (n > 0 && (!xyz_dev || !grad_sdf_dev || !grad_xyz_dev)))
        return fail(m, MAP_ERR_ARG, "bad backward arguments");
    launch_query_bwd(m->md, xyz_dev, grad_sdf_dev, n, grad_xyz_dev, pose_grad_dev, m->qb_part, (cudaStream_t)stream);
    return launch_check(m, "query_sdf_backward");
}

extern "C" map_status map_align_scan(map_t *m, const float *points_dev, int64_t n, const double T0[16], int32_t iters,
                                     double T_out[16], void *stream) {
    if (!m || n < 0 || !T0 || !T_out || iters < 0 || (n > 0 && !points_dev))
        return fail(m, MAP_ERR_ARG, "bad alignment arguments");
    cudaStream_t s = (cudaStream_t)stream;
    CU(cudaMemcpyAsync(m->gn_T, T0, 16 * sizeof(double), cudaMemcpyHostToDevice, s));
    const int parts = gn_terms_grid(n);
    for (int it = 0; it < iters; ++it) {
        launch_gn_terms(m->md, points_dev, n, m->gn_T, m->gn_acc, s);
        launch_gn_step(m->gn_T, m->gn_acc, parts, s);
    }
    map_status st = launch_check(m, "map_align_scan");
    if (st != MAP_OK) return st;
    CU(cudaMemcpyAsync(T_out, m->gn_T, 16 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    return MAP_OK;
}

extern "C" map_status map_get_blocks(map_t *m, int32_t *coords_host, int64_t cap, int64_t *count) {
    if (!m || !count || cap < 0 || (cap > 0 && !coords_host)) return fail(m, MAP_ERR_ARG, "bad arguments");
    unsigned long long *d_cnt = nullptr;
    int32_t *d_coords = nullptr;
    CU(cudaMalloc(&d_cnt, sizeof(unsigned long long)));
    CU(cudaMemset(d_cnt, 0, sizeof(unsigned long long)));
    CU(cudaMalloc(&d_coords, (size_t)m->md.max_blocks * 3 * sizeof(int32_t)));
    launch_collect_blocks(m->md, d_coords, d_cnt, 0);
    unsigned long long cnt = 0;
    cudaError_t e = cudaMemcpy(&cnt, d_cnt, sizeof(cnt), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && cap > 0)
        e = cudaMemcpy(coords_host, d_coords, (size_t)std::min<long long>(cap, (long long)cnt) * 3 * sizeof(int32_t),
                       cudaMemcpyDeviceToHost);
    cudaFree(d_cnt);
    cudaFree(d_coords);
    if (e != cudaSuccess) return fail(m, MAP_ERR_CUDA, cudaGetErrorString(e));
    *count = (int64_t)cnt;
    return MAP_OK;
}

extern "C" map_status map_read_blocks(map_t *m, const int32_t *coords, int64_t n, float *D, float *W, float *logP,
                                      uint8_t *label, uint8_t *found) {
    if (!m || n < 0 || (n > 0 && !coords)) return fail(m, MAP_ERR_ARG, "bad arguments");
    if (n == 0) return MAP_OK;
    std::vector<uint64_t> keys(n);
    for (int64_t i = 0; i < n; ++i) keys[i] = pack_block(coords[3 * i], coords[3 * i + 1], coords[3 * i + 2]);
    uint64_t *dk = nullptr;
    float *dD = nullptr, *dW = nullptr, *dL = nullptr;
    uint8_t *dlab = nullptr, *dfound = nullptr;
    const size_t nv = (size_t)n * BV;
    cudaError_t e = cudaMalloc(&dk, n * sizeof(uint64_t));
    if (e == cudaSuccess && D) e = cudaMalloc(&dD, nv * sizeof(float));
    if (e == cudaSuccess && W) e = cudaMalloc(&dW, nv * sizeof(float));
    if (e == cudaSuccess && logP) e = cudaMalloc(&dL, nv * m->C * sizeof(float));
    if (e == cudaSuccess && label) e = cudaMalloc(&dlab, nv);
    if (e == cudaSuccess && found) e = cudaMalloc(&dfound, n);
    if (e == cudaSuccess) e = cudaMemcpy(dk, keys.data(), n * sizeof(uint64_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        for (int64_t off = 0; off < n; off += 65535) {
            const int cnt = (int)std::min<int64_t>(65535, n - off);
            launch_read_blocks(m->md, dk + off, cnt, dD ? dD + off * BV : nullptr, dW ? dW + off * BV : nullptr,
                               dL ? dL + off * BV * m->C : nullptr, dlab ? dlab + off * BV : nullptr,
                               dfound ? dfound + off : nullptr, nullptr, 0);
        }
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && D) e = cudaMemcpy(D, dD, nv * sizeof(float), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && W) e = cudaMemcpy(W, dW, nv * sizeof(float), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && logP) e = cudaMemcpy(logP, dL, nv * m->C * sizeof(float), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && label) e = cudaMemcpy(label, dlab, nv, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && found) e = cudaMemcpy(found, dfound, n, cudaMemcpyDeviceToHost);
    void *ptrs[] = {dk, dD, dW, dL, dlab, dfound};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (e != cudaSuccess) return fail(m, MAP_ERR_CUDA, cudaGetErrorString(e));
    return MAP_OK;
}

extern "C" map_status map_read_gradients(map_t *m, const int32_t *coords, int64_t n, float *G) {
    if (!m || n < 0 || (n > 0 && (!coords || !G))) return fail(m, MAP_ERR_ARG, "bad arguments");
    if (m->cfg.distance_mode != 1) return fail(m, MAP_ERR_STATE, "the map keeps no gradients (projective mode)");
    if (n == 0) return MAP_OK;
    std::vector<uint64_t> keys(n);
    for (int64_t i = 0; i < n; ++i) keys[i] = pack_block(coords[3 * i], coords[3 * i + 1], coords[3 * i + 2]);
    uint64_t *dk = nullptr;
    float *dG = nullptr;
    cudaError_t e = cudaMalloc(&dk, n * sizeof(uint64_t));
    if (e == cudaSuccess) e = cudaMalloc(&dG, (size_t)n * 3 * BV * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(dk, keys.data(), n * sizeof(uint64_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        for (int64_t off = 0; off < n; off += 65535) {
            const int cnt = (int)std::min<int64_t>(65535, n - off);
            launch_read_blocks(m->md, dk + off, cnt, nullptr, nullptr, nullptr, nullptr, nullptr, dG + off * 3 * BV, 0);
        }
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(G, dG, (size_t)n * 3 * BV * sizeof(float), cudaMemcpyDeviceToHost);
    if (dk) cudaFree(dk);
    if (dG) cudaFree(dG);
    if (e != cudaSuccess) return fail(m, MAP_ERR_CUDA, cudaGetErrorString(e));
    return MAP_OK;
}

extern "C" map_status map_write_blocks(map_t *m, const int32_t *coords, int64_t n, const float *D, const float *W,
                                       const float *logP) {
    if (!m || n < 0 || (n > 0 && (!coords || !D || !W))) return fail(m, MAP_ERR_ARG, "bad arguments");
    float *dD = nullptr, *dW = nullptr, *dL = nullptr;
    const size_t nv = (size_t)n * BV;
    cudaError_t e = cudaMalloc(&dD, nv * sizeof(float) + 16);
    if (e == cudaSuccess) e = cudaMalloc(&dW, nv * sizeof(float) + 16);
    if (e == cudaSuccess && logP) e = cudaMalloc(&dL, nv * m->C * sizeof(float) + 16);
    if (e == cudaSuccess) e = cudaMemcpy(dD, D, nv * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dW, W, nv * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && logP) e = cudaMemcpy(dL, logP, nv * m->C * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        for (int64_t i = 0; i < n; ++i)
            launch_write_block(m->md, pack_block(coords[3 * i], coords[3 * i + 1], coords[3 * i + 2]), dD + i * BV,
                               dW + i * BV, dL ? dL + i * BV * m->C : nullptr, 0);
        launch_link_all(m->md, 0);
        e = cudaDeviceSynchronize();
    }
    if (dD) cudaFree(dD);
    if (dW) cudaFree(dW);
    if (dL) cudaFree(dL);
    if (e != cudaSuccess) return fail(m, MAP_ERR_CUDA, cudaGetErrorString(e));
    cudaMemcpy(m->h_st, m->st, sizeof(DevState), cudaMemcpyDeviceToHost);
    return device_errors(m);
}

extern "C" map_status map_profile_begin(map_t *m, int32_t max_frames) {
    if (!m || max_frames < 0) return fail(m, MAP_ERR_ARG, "bad arguments");
    prof_clear(m);
    m->prof_ev.resize((size_t)max_frames * (MAP_PHASE_COUNT + 1));
    m->prof_serial.assign((size_t)max_frames, 0);
    for (auto &e : m->prof_ev) CU(cudaEventCreate(&e));
    if (max_frames > 0) {
        CU(cudaMalloc(&m->prof_stats, (size_t)max_frames * CT_COUNT * sizeof(unsigned long long)));
        CU(cudaMemset(m->prof_stats, 0, (size_t)max_frames * CT_COUNT * sizeof(unsigned long long)));
    }
    m->prof_cap = max_frames;
    m->prof_n = 0;
    return MAP_OK;
}

extern "C" map_status map_profile_end(map_t *m, float *ms_out, int64_t *stats_out, int32_t *n_frames) {
    if (!m || !n_frames) return fail(m, MAP_ERR_ARG, "bad arguments");
    const int n = m->prof_n;
    for (int f = 0; f < n; ++f) {
        cudaEvent_t *ev = &m->prof_ev[(size_t)f * (MAP_PHASE_COUNT + 1)];
        CU(cudaEventSynchronize(ev[MAP_PHASE_COUNT]));
        CU(cudaEventSynchronize(ev[MAP_PHASE_SEMANTIC + 1]));
        for (int ph = 0; ph < MAP_PHASE_COUNT; ++ph) {
            // the class update and the re-meshing both start at the end of the TSDF kernel, or,
            // one after the other, the class update at the end of the re-meshing
            int from = ph == MAP_PHASE_MESH ? MAP_PHASE_SEMANTIC : ph;
            if (m->prof_serial[f] && ph == MAP_PHASE_SEMANTIC) from = MAP_PHASE_MESH + 1;
            float ms = 0.f;
            CU(cudaEventElapsedTime(&ms, ev[from], ev[ph + 1]));
            if (ms_out) ms_out[(size_t)f * MAP_PHASE_COUNT + ph] = ms;
        }
    }
    if (stats_out && n > 0)
        CU(cudaMemcpy(stats_out, m->prof_stats, (size_t)n * CT_COUNT * sizeof(unsigned long long),
                      cudaMemcpyDeviceToHost));
    *n_frames = n;
    prof_clear(m);
    return MAP_OK;
}

extern "C" map_status map_set_decision_record(map_t *m, int32_t enable) {
    if (!m) return fail(nullptr, MAP_ERR_ARG, "null map");
    if (enable != 0 && enable != 1) return fail(m, MAP_ERR_ARG, "enable must be 0 or 1");
    CU(cudaDeviceSynchronize());
    if (!enable) {
        if (m->dbg_point) cudaFree(m->dbg_point);
        if (m->dbg_vox) cudaFree(m->dbg_vox);
        m->dbg_point = m->dbg_vox = nullptr;
    } else if (!m->dbg_point) {
        if (m->cfg.max_pixels > (1ll << 23)) return fail(m, MAP_ERR_ARG, "decision record: max_pixels <= 2^23");
        if (cudaMalloc(&m->dbg_point, (size_t)m->cfg.max_points * sizeof(int)) != cudaSuccess ||
            cudaMalloc(&m->dbg_vox, (size_t)m->cfg.max_blocks * BV * sizeof(int)) != cudaSuccess) {
            if (m->dbg_point) cudaFree(m->dbg_point);
            m->dbg_point = nullptr;
            cudaGetLastError();
            return fail(m, MAP_ERR_NOMEM, "decision record: device allocation failed");
        }
    }
    m->fd.dbg_point = m->dbg_point;
    m->fd.dbg_vox = m->dbg_vox;
    m->dbg_frame = -1;
    return MAP_OK;
}

extern "C" map_status map_read_decision_record(map_t *m, int32_t *point_pix, int64_t n_points, uint64_t *winner,
                                               int64_t n_pixels, int32_t *touched, int64_t touched_cap,
                                               int64_t *n_touched, int32_t *voxel_rec) {
    if (!m || !n_touched) return fail(m, MAP_ERR_ARG, "null map or count");
    if (!m->dbg_point || m->dbg_frame < 0 || m->dbg_frame != m->frame - 1)
        return fail(m, MAP_ERR_STATE, "no decision record of the last scan (map_set_decision_record, then a scan)");
    if ((point_pix && n_points != m->dbg_n) || (winner && n_pixels != m->dbg_np))
        return fail(m, MAP_ERR_ARG, "point or pixel count differs from the recorded scan's");
    CU(cudaDeviceSynchronize());
    unsigned long long ctr[CT_COUNT];
    CU(cudaMemcpy(ctr, m->fd.ctr, sizeof(ctr), cudaMemcpyDeviceToHost));
    const long long nt = (long long)std::min<unsigned long long>(ctr[CT_TOUCHED], (unsigned long long)m->cfg.max_blocks);
    *n_touched = nt;
    if (point_pix && n_points > 0)
        CU(cudaMemcpy(point_pix, m->dbg_point, n_points * sizeof(int32_t), cudaMemcpyDeviceToHost));
    if (winner && n_pixels > 0)
        CU(cudaMemcpy(winner, m->fd.win, n_pixels * sizeof(uint64_t), cudaMemcpyDeviceToHost));
    if (touched && nt > 0) {
        if (touched_cap < nt) return fail(m, MAP_ERR_CAPACITY, "touched_cap below the touched-block count");
        int32_t *dc = nullptr, *dv = nullptr;
        CU(cudaMalloc(&dc, nt * 3 * sizeof(int32_t)));
        if (cudaMalloc(&dv, nt * BV * sizeof(int32_t)) != cudaSuccess) {
            cudaFree(dc);
            return fail(m, MAP_ERR_NOMEM, "decision record: gather buffer");
        }
        launch_dbg_gather(m->md, m->fd.touched, nt, m->dbg_vox, dc, dv, 0);
        cudaError_t e = cudaMemcpy(touched, dc, nt * 3 * sizeof(int32_t), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && voxel_rec) e = cudaMemcpy(voxel_rec, dv, nt * BV * sizeof(int32_t), cudaMemcpyDeviceToHost);
        cudaFree(dc);
        cudaFree(dv);
        if (e != cudaSuccess) return fail(m, MAP_ERR_CUDA, cudaGetErrorString(e));
    }
    return MAP_OK;
}

extern "C" const char *map_last_error(map_t *m) { return m ? m->err.c_str() : g_err.c_str(); }

// ===========================================================================
// Batched persistent integration (one cooperative launch for many maps)
// ===========================================================================
struct map_batch_t {
    std::vector<map_t *> maps;
    int flags = 0;
    BatchCtl *ctl = nullptr;          // device
    BatchState *out_dev = nullptr;    // device
    BatchState *out_host = nullptr;   // pinned
    int grid[kNumBatchConfigs] = {};
    cudaGraph_t graph[kNumBatchConfigs] = {};
    cudaGraphExec_t exec[kNumBatchConfigs] = {};
    cudaGraphNode_t knode[kNumBatchConfigs] = {};
    int fixed_cfg = -1;               // set by map_batch_set_config
    int chosen = -1;                  // autotuner's choice
    int trials = 3;                   // timed steps per configuration
    std::vector<float> samples[kNumBatchConfigs];
    cudaEvent_t ev_a = nullptr, ev_b = nullptr, ev_done = nullptr;
    cudaStream_t cap = nullptr;       // private stream the graphs are captured on (never executes work)
    int pending_cfg = -1;             // configuration of the step in flight (timed when tuning)
    bool pending = false;
    bool pending_streams = false;     // the step in flight ran on the per-map streams
    std::vector<cudaStream_t> mstream;   // MAP_BATCH_STREAMS: one stream per map
    std::vector<cudaEvent_t> mdone;      // ... and the event that joins it to the caller's stream
    cudaEvent_t ev_fork = nullptr;
    // MAP_BATCH_STREAMS | MAP_BATCH_GRAPH: the executable graph of the streams step, updated in
    // place from each step's capture (instantiated again when the step's shape changes)
    cudaGraphExec_t sexec = nullptr;
    long long s_steps = 0, s_instantiations = 0;
    unsigned long long fault_spin = 0;   // test hook: next launch lets CTA 0 leave at once
    BatchArgs args;                      // host staging of the kernel parameters
    std::string err;
};

static map_status bfail(map_batch_t *b, map_status st, const std::string &msg) {
    if (b) b->err = msg;
    g_err = msg;
    return st;
}

#define BCU(call)                                                                                    \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess)                                                                       \
            return bfail(b, MAP_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));      \
    } while (0)

extern "C" map_status map_batch_create(map_t *const *maps, int32_t n_maps, int32_t flags, map_batch_t **out) {
    map_batch_t *b = nullptr;
    if (!maps || !out || n_maps < 1 || n_maps > BATCH_MAX)
        return bfail(nullptr, MAP_ERR_ARG, "need 1 <= n_maps <= 48 and non-null pointers");
    for (int i = 0; i < n_maps; ++i) {
        if (!maps[i]) return bfail(nullptr, MAP_ERR_ARG, "null map in batch");
        if (maps[i]->cfg.distance_mode != 0 && !(flags & MAP_BATCH_STREAMS))
            return bfail(nullptr, MAP_ERR_ARG, "the batch kernel takes projective-distance maps only");
    }
    int coop = 0, dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (!coop) return bfail(nullptr, MAP_ERR_STATE, "device does not support cooperative launches");
    b = new map_batch_t();
    b->maps.assign(maps, maps + n_maps);
    b->flags = flags;
    for (int c = 0; c < kNumBatchConfigs; ++c) {
        int bps = 0;
        cudaError_t e = batch_occupancy(c, bps);
        if (e != cudaSuccess || bps < 1) {
            map_batch_destroy(b);
            return bfail(nullptr, MAP_ERR_CUDA, std::string("batch kernel occupancy: ") + cudaGetErrorString(e));
        }
        b->grid[c] = bps * sms;
    }
    if (cudaMalloc(&b->ctl, sizeof(BatchCtl)) != cudaSuccess ||
        cudaMalloc(&b->out_dev, BATCH_MAX * sizeof(BatchState)) != cudaSuccess ||
        cudaMallocHost(&b->out_host, BATCH_MAX * sizeof(BatchState)) != cudaSuccess) {
        map_batch_destroy(b);
        return bfail(nullptr, MAP_ERR_NOMEM, "batch allocation failed");
    }
    if (cudaEventCreate(&b->ev_a) != cudaSuccess || cudaEventCreate(&b->ev_b) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_done, cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) {
        map_batch_destroy(b);
        return bfail(nullptr, MAP_ERR_CUDA, "batch capture stream");
    }
    if (!(flags & MAP_BATCH_AUTOTUNE)) b->fixed_cfg = kNumBatchConfigs - 2;   // 8 warps, 2 items per thread
    if (flags & MAP_BATCH_STREAMS) {
        b->mstream.assign(n_maps, nullptr);
        b->mdone.assign(n_maps, nullptr);
        bool ok = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) == cudaSuccess;
        for (int i = 0; ok && i < n_maps; ++i)
            ok = cudaStreamCreateWithFlags(&b->mstream[i], cudaStreamNonBlocking) == cudaSuccess &&
                 cudaEventCreateWithFlags(&b->mdone[i], cudaEventDisableTiming) == cudaSuccess;
        if (!ok) {
            map_batch_destroy(b);
            return bfail(nullptr, MAP_ERR_CUDA, "batch per-map streams");
        }
    }
    *out = b;
    return MAP_OK;
}

extern "C" map_status map_batch_destroy(map_batch_t *b) {
    if (!b) return bfail(nullptr, MAP_ERR_ARG, "null batch");
    cudaDeviceSynchronize();
    for (int c = 0; c < kNumBatchConfigs; ++c) {
        if (b->exec[c]) cudaGraphExecDestroy(b->exec[c]);
        if (b->graph[c]) cudaGraphDestroy(b->graph[c]);
    }
    if (b->sexec) cudaGraphExecDestroy(b->sexec);
    if (b->ctl) cudaFree(b->ctl);
    if (b->out_dev) cudaFree(b->out_dev);
    if (b->out_host) cudaFreeHost(b->out_host);
    if (b->ev_a) cudaEventDestroy(b->ev_a);
    if (b->ev_b) cudaEventDestroy(b->ev_b);
    if (b->ev_done) cudaEventDestroy(b->ev_done);
    if (b->cap) cudaStreamDestroy(b->cap);
    for (cudaStream_t st : b->mstream)
        if (st) cudaStreamDestroy(st);
    for (cudaEvent_t e : b->mdone)
        if (e) cudaEventDestroy(e);
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    delete b;
    return MAP_OK;
}

// Wait for the step in flight and fold its per-map results into the maps.
static map_status batch_retire(map_batch_t *b) {
    if (!b->pending) return MAP_OK;
    BCU(cudaEventSynchronize(b->ev_done));
    b->pending = false;
    if (b->pending_streams) {           // the maps' own calls have recorded their results
        b->pending_streams = false;
        return MAP_OK;
    }
    const int timed_cfg = b->pending_cfg;
    b->pending_cfg = -1;
    BatchCtl ctl;
    BCU(cudaMemcpy(&ctl, b->ctl, sizeof(ctl), cudaMemcpyDeviceToHost));
    // a step that timed out wrote no results; the maps keep their last readings
    if (ctl.err & ERR_TIMEOUT) return bfail(b, MAP_ERR_TIMEOUT, "batch launch: a grid barrier timed out");
    if (timed_cfg >= 0) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, b->ev_a, b->ev_b) == cudaSuccess) b->samples[timed_cfg].push_back(ms);
    }
    for (size_t i = 0; i < b->maps.size(); ++i) {
        map_t *m = b->maps[i];
        *m->h_st = b->out_host[i].st;
        std::memcpy(m->h_ctr, b->out_host[i].ctr, sizeof(b->out_host[i].ctr));
        m->h_ctr_slot = -1;
        const double f = arena_fill(*m->h_st);
        if (m->known_frame >= 0 && m->frame - 1 > m->known_frame && f >= m->known_fill)
            m->max_append = std::max(m->max_append, (f - m->known_fill) / (double)(m->frame - 1 - m->known_frame));
        m->known_fill = f;
        m->known_frame = m->frame - 1;
    }
    return MAP_OK;
}

static int batch_pick_config(map_batch_t *b) {
    if (b->fixed_cfg >= 0) return b->fixed_cfg;
    if (b->chosen >= 0) return b->chosen;
    int best = -1, fewest = 1 << 30;
    for (int c = 0; c < kNumBatchConfigs; ++c)
        if ((int)b->samples[c].size() < fewest) {
            fewest = (int)b->samples[c].size();
            best = c;
        }
    if (fewest < b->trials) return best;
    // every configuration timed: keep the one with the lowest median step time
    float best_ms = 1e30f;
    for (int c = 0; c < kNumBatchConfigs; ++c) {
        std::vector<float> v = b->samples[c];
        std::sort(v.begin(), v.end());
        const float med = v[v.size() / 2];
        if (med < best_ms) {
            best_ms = med;
            b->chosen = c;
        }
    }
    return b->chosen;
}

extern "C" map_status map_batch_integrate(map_batch_t *b, const scan_desc *scans, void *stream) {
    if (!b || !scans) return bfail(b, MAP_ERR_ARG, "null batch or scans");
    cudaStream_t s = (cudaStream_t)stream;
    map_status st = batch_retire(b);
    if (st != MAP_OK) return st;
    const int n = (int)b->maps.size();
    if (b->flags & MAP_BATCH_STREAMS) {
        for (int i = 0; i < n; ++i)
            if (scans[i].map != b->maps[i]) return bfail(b, MAP_ERR_ARG, "scans[i].map must be the batch's i-th map");
        // With MAP_BATCH_GRAPH the step is captured on the batch's private stream and
        // replayed as one graph launch on the caller's stream.
        const bool graph = (b->flags & MAP_BATCH_GRAPH) != 0;
        cudaStream_t origin = s;
        if (graph) {
            // uploads a capture cannot wait for (pixel-ray tables) are done and waited for first
            for (int i = 0; i < n; ++i) {
                map_t *m = b->maps[i];
                if (m->cfg.distance_mode != 1 || scans[i].n <= 0) continue;
                if (upload_pixel_rays(m, &scans[i].lidar) != MAP_OK) continue;   // refused again below
                BCU(cudaEventSynchronize(m->ev_dir));
            }
            BCU(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed));
            origin = b->cap;
        }
        map_status first = MAP_OK;
        std::string cuda_err;
        auto step = [&]() {
            cudaError_t e = cudaEventRecord(b->ev_fork, origin);
            for (int i = 0; i < n && e == cudaSuccess; ++i) {
                const scan_desc &d = scans[i];
                map_t *m = b->maps[i];
                e = cudaStreamWaitEvent(b->mstream[i], b->ev_fork, 0);
                if (e != cudaSuccess) break;
                map_status st_i = MAP_OK;
                if (d.n > 0 && (!d.points_dev || ((d.labels_dev == nullptr) == (d.probs_dev == nullptr))))
                    st_i = fail(m, MAP_ERR_ARG, "need points and exactly one of labels / probs");
                else
                    st_i = run_frame(m, &d.lidar, d.points_dev, d.labels_dev, d.probs_dev, d.n, d.T_world_lidar,
                                     b->mstream[i]);
                if (st_i != MAP_OK && first == MAP_OK) {
                    first = st_i;
                    b->err = m->err;
                }
                // join every map's stream, also after an error (what was enqueued completes before the
                // caller's stream goes on)
                e = cudaEventRecord(b->mdone[i], b->mstream[i]);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(origin, b->mdone[i], 0);
            }
            if (e != cudaSuccess) cuda_err = cudaGetErrorString(e);
        };
        step();
        if (graph) {
            cudaGraph_t g = nullptr;
            const cudaError_t ec = cudaStreamEndCapture(b->cap, &g);
            if (ec != cudaSuccess || !cuda_err.empty()) {
                if (g) cudaGraphDestroy(g);
                return bfail(b, MAP_ERR_CUDA, "streams step capture: " +
                                                  (cuda_err.empty() ? std::string(cudaGetErrorString(ec)) : cuda_err));
            }
            bool updated = false;
            if (b->sexec) {
                cudaGraphExecUpdateResultInfo info;
                updated = cudaGraphExecUpdate(b->sexec, g, &info) == cudaSuccess;
                if (!updated) {
                    cudaGetLastError();
                    cudaGraphExecDestroy(b->sexec);
                    b->sexec = nullptr;
                }
            }
            cudaError_t el = cudaSuccess;
            if (!updated) {
                el = cudaGraphInstantiate(&b->sexec, g, 0);
                b->s_instantiations++;
            }
            cudaGraphDestroy(g);
            if (el == cudaSuccess) el = cudaGraphLaunch(b->sexec, s);
            if (el != cudaSuccess)
                return bfail(b, MAP_ERR_CUDA, std::string("streams step graph: ") + cudaGetErrorString(el));
            b->s_steps++;
        } else if (!cuda_err.empty()) {
            return bfail(b, MAP_ERR_CUDA, "streams step: " + cuda_err);
        }
        BCU(cudaEventRecord(b->ev_done, s));
        b->pending = true;
        b->pending_streams = true;
        if (first != MAP_OK) return bfail(b, first, b->err);
        return MAP_OK;
    }
    BatchArgs &args = b->args;   // copied into the launch (or the graph node) by the calls below
    std::memset(&args, 0, sizeof(args));
    for (int i = 0; i < n; ++i) {
        map_t *m = b->maps[i];
        const scan_desc &d = scans[i];
        if (d.map != m) return bfail(b, MAP_ERR_ARG, "scans[i].map must be the batch's i-th map");
        if (d.n > 0 && (!d.points_dev || ((d.labels_dev == nullptr) == (d.probs_dev == nullptr))))
            return bfail(b, MAP_ERR_ARG, "need points and exactly one of labels / probs");
        ScanConst sc;
        st = make_scan_const(m, &d.lidar, d.n, d.T_world_lidar, d.probs_dev != nullptr, sc);
        if (st != MAP_OK) return bfail(b, st, m->err);
        sc.probs_vec4 = d.probs_dev && (m->C % 4 == 0) && (((uintptr_t)d.probs_dev & 15) == 0);
        if (need_compaction(m)) {
            st = compact_arena(m, s);
            if (st != MAP_OK) return bfail(b, st, m->err);
        }
        BatchItem &it = args.it[i];
        it.sc = sc;
        it.md = m->md;
        it.fd = m->fd;      // the batch kernel resets this set's range image and counters itself
        it.fd.dbg_point = it.fd.dbg_vox = nullptr;   // no decision record in the batched form
        m->win_dirty[m->fcur] = m->cfg.max_pixels;
        it.sc.pts = d.points_dev;
        it.sc.labels = d.labels_dev;
        it.sc.probs = d.probs_dev;
    }
    // the warp-staged class update when every map has 20 classes, one storage type, and labels or
    // 16-byte-aligned probability rows
    {
        bool staged = true;
        for (int i = 0; i < n && staged; ++i) {
            const BatchItem &it = args.it[i];
            staged = it.sc.C == 20 && it.md.storage == args.it[0].md.storage && (!it.sc.has_probs || it.sc.probs_vec4);
        }
        args.sem_staged = staged && n > 0 ? (args.it[0].md.storage == 0 ? 1 : 2) : 0;
        bool one_floor = true;
        for (int i = 1; i < n; ++i) one_floor = one_floor && args.it[i].sc.lik_floor == args.it[0].sc.lik_floor;
        args.sem_rows_once = args.sem_staged && one_floor ? 1 : 0;
    }
    args.n = n;
    args.ctl = b->ctl;
    args.out = b->out_dev;
    args.tri = mesh_table_tri();
    args.ntri = mesh_table_ntri();
    args.fault_skip_cta0 = b->fault_spin ? 1 : 0;
    args.spin_limit = b->fault_spin;
    b->fault_spin = 0;
    const int cfg = batch_pick_config(b);
    const bool timing = b->fixed_cfg < 0 && b->chosen < 0;
    if (timing) BCU(cudaEventRecord(b->ev_a, s));
    if (b->flags & MAP_BATCH_GRAPH) {
        if (!b->exec[cfg]) {
            // capture barrier reset + launch + result copy once per configuration, on the
            // private stream (the caller's stream may be the legacy default stream)
            BCU(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
            cudaError_t e0 = cudaMemsetAsync(b->ctl, 0, sizeof(BatchCtl), b->cap);
            cudaError_t e = launch_batch(cfg, b->grid[cfg], args, b->cap);
            cudaError_t e2 = cudaMemcpyAsync(b->out_host, b->out_dev, BATCH_MAX * sizeof(BatchState),
                                             cudaMemcpyDeviceToHost, b->cap);
            BCU(cudaStreamEndCapture(b->cap, &b->graph[cfg]));
            BCU(e0);
            BCU(e);
            BCU(e2);
            size_t nn = 0;
            BCU(cudaGraphGetNodes(b->graph[cfg], nullptr, &nn));
            std::vector<cudaGraphNode_t> nodes(nn);
            BCU(cudaGraphGetNodes(b->graph[cfg], nodes.data(), &nn));
            for (auto nd : nodes) {
                cudaGraphNodeType t;
                cudaGraphNodeGetType(nd, &t);
                if (t == cudaGraphNodeTypeKernel) b->knode[cfg] = nd;
            }
            BCU(cudaGraphInstantiate(&b->exec[cfg], b->graph[cfg], 0));
        } else {
            cudaKernelNodeParams kp;
            BCU(cudaGraphKernelNodeGetParams(b->knode[cfg], &kp));
            void *params[] = {(void *)&args};
            kp.kernelParams = params;
            kp.extra = nullptr;
            BCU(cudaGraphExecKernelNodeSetParams(b->exec[cfg], b->knode[cfg], &kp));
        }
        BCU(cudaGraphLaunch(b->exec[cfg], s));
    } else {
        BCU(cudaMemsetAsync(b->ctl, 0, sizeof(BatchCtl), s));
        BCU(launch_batch(cfg, b->grid[cfg], args, s));
        BCU(cudaMemcpyAsync(b->out_host, b->out_dev, n * sizeof(BatchState), cudaMemcpyDeviceToHost, s));
    }
    if (timing) {
        BCU(cudaEventRecord(b->ev_b, s));
        b->pending_cfg = cfg;
    }
    BCU(cudaEventRecord(b->ev_done, s));
    b->pending = true;
    for (map_t *m : b->maps) {
        m->frame++;
        m->launches += 1;
    }
    return MAP_OK;
}

extern "C" map_status map_batch_sync(map_batch_t *b, void *stream) {
    if (!b) return bfail(nullptr, MAP_ERR_ARG, "null batch");
    map_status st = batch_retire(b);
    if (st != MAP_OK) return st;
    for (map_t *m : b->maps) {
        st = device_errors(m);
        if (st != MAP_OK) return bfail(b, st, m->err);
    }
    (void)stream;
    return MAP_OK;
}

extern "C" map_status map_batch_config(map_batch_t *b, int32_t *threads_per_block, int32_t *items_per_thread,
                                       int32_t *tuned) {
    if (!b) return bfail(nullptr, MAP_ERR_ARG, "null batch");
    const int c = b->fixed_cfg >= 0 ? b->fixed_cfg : b->chosen;
    if (threads_per_block) *threads_per_block = c >= 0 ? 32 * kBatchConfigs[c].warps : 0;
    if (items_per_thread) *items_per_thread = c >= 0 ? kBatchConfigs[c].vpt : 0;
    if (tuned) *tuned = b->fixed_cfg < 0 && b->chosen >= 0;
    return MAP_OK;
}

extern "C" map_status map_batch_set_config(map_batch_t *b, int32_t cfg) {
    if (!b || cfg < -1 || cfg >= kNumBatchConfigs) return bfail(b, MAP_ERR_ARG, "bad configuration index");
    b->fixed_cfg = cfg;
    return MAP_OK;
}

extern "C" map_status map_batch_test_timeout(map_batch_t *b, uint64_t spin_limit) {
    if (!b || spin_limit == 0) return bfail(b, MAP_ERR_ARG, "need a batch and a positive spin limit");
    b->fault_spin = spin_limit;
    return MAP_OK;
}

extern "C" const char *map_batch_last_error(map_batch_t *b) { return b ? b->err.c_str() : g_err.c_str(); }

// Internal accessors for translation units that add entry points around a map.
namespace stsdf {
const MapDev *map_device_view(const map_t *m) { return &m->md; }
void map_set_error(map_t *m, const char *msg) { m->err = msg; }
}  // namespace stsdf
