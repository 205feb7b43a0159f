// Measurement preprocessing (Sec. III-C.1), second half: the per-pixel table
// of the range image whose winners k_points (k_alloc.cu) decided.
#include "frame_bodies.cuh"

namespace stsdf {

__global__ void __launch_bounds__(256) k_pixels(const float *__restrict__ pts, const int32_t *__restrict__ labels,
                                                const float *__restrict__ probs, ScanConst sc, FrameDev fd) {
    pixel_item(pts, labels, probs, sc, fd, blockIdx.x * blockDim.x + threadIdx.x);
}

void launch_pixels(const float *pts, const int32_t *labels, const float *probs, const ScanConst &sc,
                   const FrameDev &fd, cudaStream_t s) {
    const long long np = (long long)sc.H * sc.W;
    k_pixels<<<(unsigned)((np + 255) / 256), 256, 0, s>>>(pts, labels, probs, sc, fd);
}

}  // namespace stsdf
