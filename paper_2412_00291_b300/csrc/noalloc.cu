// extract_mesh_noalloc: mesh extraction that allocates no memory at all.
//
// extract_mesh grows map-owned output buffers with cudaMalloc and keeps its
// scan scratch in map-owned memory.  Some callers cannot allocate: a real-time
// loop that must never block on the allocator (cudaMalloc/cudaFree can
// synchronise the whole device), or a framework that hands the library only
// the memory it reserved up front.  This entry point runs the same gather
// kernels, writes into buffers the caller passes in, and keeps its scratch in
// one file-scope device array of fixed size (held by every GPU that loads the
// library, until the process exits).
#include <cstdio>
#include <mutex>

#include "../../include/semtsdf.h"
#include "kernels.h"

namespace stsdf {
const MapDev *map_device_view(const map_t *m);
void map_set_error(map_t *m, const char *msg);
}  // namespace stsdf

using namespace stsdf;

namespace {

constexpr long long kMaxSlots = 1ll << 19;            // pool blocks the scratch can index
constexpr long long kChunk = 1024;                    // slots per CTA of the first scan pass
constexpr long long kMaxChunks = kMaxSlots / kChunk;
// per-slot vertex and triangle offsets, per-chunk sums, two totals (8.4 MB)
constexpr long long kScratchWords = 2 * kMaxSlots + 2 * kMaxChunks + 2;

static __device__ __align__(256) long long g_extract_scratch[kScratchWords];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
long long *g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (host code cannot use the symbol itself as a device pointer).
map_status scratch_address(map_t *m, long long **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        map_set_error(m, "extract_mesh_noalloc: no usable current device");
        return MAP_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_extract_scratch);
        if (e != cudaSuccess || !p) {
            char buf[160];
            std::snprintf(buf, sizeof buf, "extract_mesh_noalloc: cudaGetSymbolAddress failed: %s",
                          cudaGetErrorString(e));
            map_set_error(m, buf);
            return MAP_ERR_CUDA;
        }
        g_scratch_addr[dev] = (long long *)p;
    }
    *out = g_scratch_addr[dev];
    return MAP_OK;
}

}  // namespace

extern "C" map_status extract_mesh_noalloc(map_t *map, float *positions, uint8_t *colors, int64_t *vertex_keys,
                                           int32_t *triangles, int32_t *triangle_anchors, int64_t vertex_capacity,
                                           int64_t triangle_capacity, int64_t *n_vertices, int64_t *n_triangles,
                                           void *stream) {
    if (!map || !n_vertices || !n_triangles || vertex_capacity < 0 || triangle_capacity < 0 ||
        (vertex_capacity > 0 && (!positions || !colors || !vertex_keys)) ||
        (triangle_capacity > 0 && (!triangles || !triangle_anchors))) {
        if (map) map_set_error(map, "extract_mesh_noalloc: null pointer or negative capacity");
        return MAP_ERR_ARG;
    }
    const MapDev &md = *map_device_view(map);
    if ((long long)md.max_blocks > kMaxSlots) {
        char buf[160];
        std::snprintf(buf, sizeof buf,
                      "extract_mesh_noalloc: pool of %d blocks exceeds the %lld-block static scratch",
                      md.max_blocks, kMaxSlots);
        map_set_error(map, buf);
        return MAP_ERR_ARG;
    }
    long long *scr = nullptr;
    map_status st = scratch_address(map, &scr);
    if (st != MAP_OK) return st;
    // Every word the kernels read is written earlier in the same call (offsets
    // of slots below the pool count, all chunk sums, both totals), so nothing
    // needs clearing.
    GatherBufs g;
    g.voff = scr;
    g.toff = scr + kMaxSlots;
    g.bsum_v = scr + 2 * kMaxSlots;
    g.bsum_t = g.bsum_v + kMaxChunks;
    g.totals = g.bsum_t + kMaxChunks;
    cudaStream_t s = (cudaStream_t)stream;
    launch_seg_scan(md, g, md.max_blocks, s);
    long long tot[2] = {0, 0};
    cudaError_t e = cudaMemcpyAsync(tot, g.totals, sizeof(tot), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        map_set_error(map, cudaGetErrorString(e));
        return MAP_ERR_CUDA;
    }
    *n_vertices = tot[0];
    *n_triangles = tot[1];
    if (tot[0] > vertex_capacity || tot[1] > triangle_capacity) {
        char buf[160];
        std::snprintf(buf, sizeof buf, "extract_mesh_noalloc: mesh needs %lld vertices and %lld triangles", tot[0],
                      tot[1]);
        map_set_error(map, buf);
        return MAP_ERR_CAPACITY;
    }
    launch_seg_gather(md, g, md.max_blocks, 1, nullptr, nullptr, nullptr, positions, colors, vertex_keys, triangles,
                      triangle_anchors, s);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        map_set_error(map, cudaGetErrorString(e));
        return MAP_ERR_CUDA;
    }
    return MAP_OK;
}
