// Two-stage (masked) indexing, arXiv 2111.07347 Section 4.3: the dominant matrix
// reflections are removed with a mask made from the average of all patterns, thresholded,
// then cleaned by erosions (noise-like features) and dilations (tails of intense peaks);
// the masked patterns are then indexed against the precipitate library.
//
// frame_sum_kernel: one thread per pixel adds the pixel over the frames in frame order, in
//   FP64 (exact for u16 frames; a fixed order for f32), optionally onto a previous sum, so
//   a scan may be summed chunk by chunk with the same result.  For u16 frames, whose sums
//   are exact integers in any order, groups of frames are summed in parallel in 64-bit
//   integers and the partials added, which keeps the whole GPU busy.
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

// u16 frames: the sums are integers below 2^53, exact in any order, so groups of frames are
// summed in parallel (partial [groups][hw]) and the partials added afterwards.
__global__ void frame_sum_u16_groups_kernel(const uint16_t* __restrict__ frames, int64_t n, int64_t hw, int groups,
                                            double* __restrict__ partial) {
    const int64_t per = (n + groups - 1) / groups;
    const int64_t total = (int64_t)groups * hw;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int gi = (int)(t / hw);
        const int64_t i = t - (int64_t)gi * hw;
        const int64_t f0 = gi * per, f1 = min(n, f0 + per);
        uint64_t s = 0;                                     // exact: at most 65535 per frame
        const uint16_t* p = frames + i;
        int64_t f = f0;
        for (; f + 16 <= f1; f += 16) {                     // 16 loads in flight per thread
            uint32_t v[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) v[u] = __ldg(p + (f + u) * hw);
#pragma unroll
            for (int u = 0; u < 16; ++u) s += v[u];
        }
        for (; f < f1; ++f) s += __ldg(p + f * hw);
        partial[t] = (double)s;
    }
}

__global__ void add_partials_kernel(const double* __restrict__ partial, int64_t hw, int groups, int accumulate,
                                    double* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < hw; i += (int64_t)gridDim.x * blockDim.x) {
        double s = accumulate ? out[i] : 0.0;
        for (int gi = 0; gi < groups; ++gi) s += partial[(int64_t)gi * hw + i];
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
    const int64_t cap = (int64_t)num_sms * 8;               // 8 CTAs of 256 threads: a full SM
    return (int)(g < cap ? (g > 0 ? g : 1) : cap);
}

}  // namespace

int frame_sum_groups(int64_t n, int64_t hw, int num_sms) {
    // enough threads to fill the GPU (2048 resident threads per SM), at least 64 frames per group
    int64_t g = (int64_t)num_sms * 2048 / (hw > 0 ? hw : 1);
    if (g > n / 64) g = n / 64;
    if (g > 64) g = 64;
    return (int)(g < 1 ? 1 : g);
}

size_t frame_sum_scratch_bytes(int dtype, int64_t n, int H, int W, int num_sms) {
    const int64_t hw = (int64_t)H * W;
    if (dtype != TM_DTYPE_U16) return 0;
    const int g = frame_sum_groups(n, hw, num_sms);
    return g > 1 ? (size_t)g * hw * sizeof(double) : 0;
}

cudaError_t launch_frame_sum(const void* frames, int dtype, int64_t n, int H, int W, int accumulate, double* out,
                             double* scratch, int num_sms, cudaStream_t st) {
    const int64_t hw = (int64_t)H * W;
    if (hw <= 0) return cudaSuccess;
    const int threads = 256;
    if (dtype == TM_DTYPE_U16) {
        const int groups = frame_sum_groups(n, hw, num_sms);
        if (groups > 1 && scratch) {
            frame_sum_u16_groups_kernel<<<grid_for((int64_t)groups * hw, threads, num_sms), threads, 0, st>>>(
                (const uint16_t*)frames, n, hw, groups, scratch);
            add_partials_kernel<<<grid_for(hw, threads, num_sms), threads, 0, st>>>(scratch, hw, groups, accumulate, out);
            return cudaGetLastError();
        }
        frame_sum_kernel<uint16_t><<<grid_for(hw, threads, num_sms), threads, 0, st>>>((const uint16_t*)frames, n, hw,
                                                                                       accumulate, out);
    } else {
        frame_sum_kernel<float><<<grid_for(hw, threads, num_sms), threads, 0, st>>>((const float*)frames, n, hw,
                                                                                    accumulate, out);
    }
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
