// Types shared by the batched persistent kernel (k_batch.cu) and its host side (map.cu).
#pragma once

#include "common.cuh"

namespace stsdf {

constexpr int BATCH_MAX = 48;   // maps per launch (their descriptors travel as kernel parameters)

// One map's scan in a batch step.
struct BatchItem {
    ScanConst sc;
    MapDev md;
    FrameDev fd;
};

// Grid barrier and status of one batch launch (zeroed before each launch).
struct BatchCtl {
    unsigned int bar_count, bar_gen;
    unsigned int err;
    unsigned int pad;
};

// Per-map state returned to the host after a batch step.
struct BatchState {
    DevState st;
    unsigned long long ctr[CT_COUNT];
};

struct BatchArgs {
    BatchItem it[BATCH_MAX];
    int n;
    int fault_skip_cta0;     // test hook: CTA 0 leaves at once, the first barrier times out
    int sem_staged;          // class update: 0 one voxel per thread, 1 / 2 warp-staged (FP32 / FP16 records)
    int sem_rows_once;       // warp-staged: each (map, point) probability row staged and taken to log2
                             // once per warp round (every map with the same likelihood floor)
    unsigned long long spin_limit;   // polls before a barrier wait gives up (0: default)
    BatchCtl *ctl;
    BatchState *out;
    const int8_t *tri;
    const uint8_t *ntri;
};
static_assert(sizeof(BatchArgs) < 32000, "batch descriptors must fit the kernel parameter space");

// Launch configurations the autotuner chooses from: warps per CTA (threads
// per block / 32) and items per thread per sweep of the point and class phases.
struct BatchConfig {
    int warps, vpt;
};
constexpr int kNumBatchConfigs = 6;
extern const BatchConfig kBatchConfigs[kNumBatchConfigs];

cudaError_t batch_occupancy(int cfg, int &blocks_per_sm);
cudaError_t launch_batch(int cfg, int grid, const BatchArgs &args, cudaStream_t s);
const int8_t *mesh_table_tri();
const uint8_t *mesh_table_ntri();

}  // namespace stsdf
