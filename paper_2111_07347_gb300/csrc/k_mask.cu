// Two-stage (masked) indexing, arXiv 2111.07347 Section 4.3: the dominant matrix
// reflections are removed with a mask made from the average of all patterns, thresholded,
// then cleaned by erosions (noise-like features) and dilations (tails of intense peaks);
// the masked patterns are then indexed against the precipitate library.
//
// frame_sum_kernel: one thread per pixel adds the pixel over the frames in frame order, in
//   FP64 (exact for u16 frames; a fixed order for f32), optionally onto a previous sum, so
//   a scan may be summed chunk by chunk with the same result.
// threshold_kernel / morph_kernel: the binary image (sum > threshold * n) and one 3 x 3
//   erosion or dilation step (pixels outside the image count as unset); the kept pixels
//   are the complement of the final image.
#include "tm_internal.h"

namespace tmgb {
namespace {

template <typename T>
__global__ void frame_sum_kernel(const T* __restrict__ frames, int64_t n, int64_t hw, int accumulate,
                                 double* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < hw; i += (int64_t)gridDim.x * blockDim.x) {
        double s = accumulate ? out[i] : 0.0;
        const T* p = frames + i;
        int64_t f = 0;
        for (; f + 8 <= n; f += 8) {                     // loads issued ahead, adds in frame order
            T v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = __ldg(p + (f + u) * hw);
#pragma unroll
            for (int u = 0; u < 8; ++u) s += (double)v[u];
        }
        for (; f < n; ++f) s += (double)__ldg(p + f * hw);
        out[i] = s;
    }
}

__global__ void threshold_kernel(const double* __restrict__ sum, int64_t hw, double thr_n, uint8_t* __restrict__ b) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < hw; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = sum[i] > thr_n ? 1 : 0;
}

// One 3 x 3 step: dilate = any neighbour set, erode = all nine set (outside = unset);
// invert writes the complement of the result.
__global__ void morph_kernel(const uint8_t* __restrict__ in, int H, int W, int dilate, int invert,
                             uint8_t* __restrict__ out) {
    const int64_t hw = (int64_t)H * W;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < hw; i += (int64_t)gridDim.x * blockDim.x) {
        const int y = (int)(i / W), x = (int)(i - (int64_t)y * W);
        int any = 0, all = 1;
        for (int dy = -1; dy <= 1; ++dy) {
            for (int dx = -1; dx <= 1; ++dx) {
                const int yy = y + dy, xx = x + dx;
                const int v = (yy >= 0 && yy < H && xx >= 0 && xx < W) ? in[(int64_t)yy * W + xx] : 0;
                any |= v;
                all &= v;
            }
        }
        int r = dilate ? any : all;
        if (invert) r = !r;
        out[i] = (uint8_t)r;
    }
}

__global__ void invert_kernel(const uint8_t* __restrict__ in, int64_t hw, uint8_t* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < hw; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = in[i] ? 0 : 1;
}

int grid_for(int64_t items, int threads, int num_sms) {
    const int64_t g = (items + threads - 1) / threads;
    const int64_t cap = (int64_t)num_sms * 8;
    return (int)(g < cap ? (g > 0 ? g : 1) : cap);
}

}  // namespace

cudaError_t launch_frame_sum(const void* frames, int dtype, int64_t n, int H, int W, int accumulate, double* out,
                             int num_sms, cudaStream_t st) {
    const int64_t hw = (int64_t)H * W;
    if (hw <= 0) return cudaSuccess;
    const int threads = 256;
    const int grid = grid_for(hw, threads, num_sms);
    if (dtype == TM_DTYPE_U16)
        frame_sum_kernel<uint16_t><<<grid, threads, 0, st>>>((const uint16_t*)frames, n, hw, accumulate, out);
    else
        frame_sum_kernel<float><<<grid, threads, 0, st>>>((const float*)frames, n, hw, accumulate, out);
    return cudaGetLastError();
}

cudaError_t launch_matrix_mask(const double* sum, int H, int W, double thr_n, int n_open, int n_dilate,
                               uint8_t* mask, uint8_t* scratch, int num_sms, cudaStream_t st) {
    const int64_t hw = (int64_t)H * W;
    if (hw <= 0) return cudaSuccess;
    const int threads = 256;
    const int grid = grid_for(hw, threads, num_sms);
    // ping-pong between scratch and mask so that the last step writes the kept pixels to mask
    const int steps = 2 * n_open + n_dilate;
    uint8_t* bufs[2] = {scratch, mask};
    int cur = steps % 2 == 0 ? 0 : 1;                     // after `steps` flips the image lands in scratch
    threshold_kernel<<<grid, threads, 0, st>>>(sum, hw, thr_n, bufs[cur]);
    for (int s = 0; s < steps; ++s) {
        const int dil = s >= n_open;
        morph_kernel<<<grid, threads, 0, st>>>(bufs[cur], H, W, dil, 0, bufs[cur ^ 1]);
        cur ^= 1;
    }
    invert_kernel<<<grid, threads, 0, st>>>(bufs[cur], hw, mask);
    return cudaGetLastError();
}

}  // namespace tmgb
