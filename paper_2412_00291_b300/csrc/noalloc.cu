// extract_mesh_noalloc: mesh extraction that allocates no memory at all.
//
// extract_mesh grows map-owned output buffers with cudaMalloc and keeps its
// scan scratch in map-owned memory.  Some callers cannot allocate: a real-time
// loop that must never block on the allocator (cudaMalloc/cudaFree can
// synchronise the whole device), or a framework that hands the library only
// the memory it reserved up front.  This entry point runs the same gather
// kernels, writes into buffers the caller passes in, and keeps its scratch in
// one file-scope device array of fixed size.  The array lives in this file's
// device module, which the CUDA runtime loads on a device when the array is
// first used there (lazy module loading, the default): map_create looks its
// address up on the map's device, so the array (8.4 MB) is taken when a map
// is created there and stays until the process exits; extract_mesh_noalloc
// itself then allocates nothing.
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

// Device address of the scratch array on device `dev` (the current device),
// looked up once per device (host code cannot use the symbol itself as a
// device pointer).  The first lookup on a device loads this file's module
// there, which places the array in that device's memory.
cudaError_t scratch_lookup(int dev, long long **out) {
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_extract_scratch);
        if (e != cudaSuccess) return e;
        if (!p) return cudaErrorInvalidSymbol;
        g_scratch_addr[dev] = (long long *)p;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

// Device holding `p` (device or managed memory), or -1 for host memory or an
// unknown pointer.
int owner_device(const void *p) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();   // clear the sticky-free error of a failed query
        return -1;
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) return -1;
    return a.device;
}

}  // namespace

namespace stsdf {
// Called by map_create with the map's device current: loads the scratch array
// there ahead of any extract_mesh_noalloc call (errors are left to that call).
void noalloc_prepare_device() {
    int dev = -1;
    long long *p = nullptr;
    if (cudaGetDevice(&dev) == cudaSuccess && scratch_lookup(dev, &p) != cudaSuccess) cudaGetLastError();
}
}  // namespace stsdf

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
    // the map, the five buffers and the scratch array must all be on the current device
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        map_set_error(map, "extract_mesh_noalloc: no usable current device");
        return MAP_ERR_CUDA;
    }
    if (owner_device(md.hs) != dev) {
        map_set_error(map, "extract_mesh_noalloc: the map was created on another device than the current one");
        return MAP_ERR_ARG;
    }
    const void *bufs[5] = {positions, colors, vertex_keys, triangles, triangle_anchors};
    const long long caps[5] = {vertex_capacity, vertex_capacity, vertex_capacity, triangle_capacity,
                               triangle_capacity};
    for (int i = 0; i < 5; ++i)
        if (caps[i] > 0 && owner_device(bufs[i]) != dev) {
            map_set_error(map, "extract_mesh_noalloc: an output buffer is not device memory of the current device");
            return MAP_ERR_ARG;
        }
    long long *scr = nullptr;
    cudaError_t le = scratch_lookup(dev, &scr);
    if (le != cudaSuccess) {
        char buf[160];
        std::snprintf(buf, sizeof buf, "extract_mesh_noalloc: cudaGetSymbolAddress failed: %s",
                      cudaGetErrorString(le));
        map_set_error(map, buf);
        return MAP_ERR_CUDA;
    }
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
