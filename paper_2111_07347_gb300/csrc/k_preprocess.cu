// Background removal and smoothing before the polar transform (arXiv 2111.07347, Section 3.1:
// the diffuse background of each pattern was removed with a difference of Gaussians and the
// result smoothed by a Gaussian blur).  Separable Gaussian filters with the edge pixel
// repeated outside the frame: a row pass, then a column pass, each output a sum over the
// 2R + 1 offsets in ascending order (FP32 multiply-adds), weights computed in double
// precision on the host.
//
// gauss_rows_kernel: one warp per image row; the row and a clamped halo of R pixels on each
//   side are staged in shared memory, lanes take the outputs; up to two filters per pass
//   (the two Gaussians of the difference share the row).
// gauss_cols_kernel: one CTA per 32-column strip of a frame; the strip of one or two inputs
//   is staged in shared memory (rows clamped on reading), lanes are columns (no bank
//   conflicts), warps split the rows; the difference of Gaussians (clipped at 0) is formed
//   in the same pass.
#include "tm_internal.h"

namespace tmgb {
namespace {

constexpr int kRowWarps = 8;
constexpr int kStrip = 32;

template <typename T>
__device__ __forceinline__ float as_float(T v) {
    return (float)v;
}

template <typename T>
__global__ void __launch_bounds__(32 * kRowWarps)
gauss_rows_kernel(const T* __restrict__ in, int64_t rows, int W, const float* __restrict__ w1, int r1,
                  const float* __restrict__ w2, int r2, float* __restrict__ out1, float* __restrict__ out2) {
    extern __shared__ float sm[];
    const int R = max(r1, w2 ? r2 : 0);
    const int nw1 = 2 * r1 + 1, nw2 = w2 ? 2 * r2 + 1 : 0;
    float* sw1 = sm;                                         // [nw1]
    float* sw2 = sw1 + nw1;                                  // [nw2]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float* row_s = sw2 + nw2 + warp * (W + 2 * R);           // [W + 2R]: pixel j - R, clamped
    for (int i = threadIdx.x; i < nw1; i += blockDim.x) sw1[i] = w1[i];
    for (int i = threadIdx.x; i < nw2; i += blockDim.x) sw2[i] = w2[i];
    __syncthreads();
    for (int64_t r = (int64_t)blockIdx.x * kRowWarps + warp; r < rows; r += (int64_t)gridDim.x * kRowWarps) {
        const T* src = in + (size_t)r * W;
        for (int j = lane; j < W + 2 * R; j += 32) row_s[j] = as_float(__ldg(src + min(max(j - R, 0), W - 1)));
        __syncwarp();
        for (int x = lane; x < W; x += 32) {
            float a = 0.0f;
            const float* p = row_s + x + (R - r1);
            for (int i = 0; i < nw1; ++i) a = fmaf(sw1[i], p[i], a);
            out1[(size_t)r * W + x] = a;
            if (w2) {
                float b = 0.0f;
                const float* q = row_s + x + (R - r2);
                for (int i = 0; i < nw2; ++i) b = fmaf(sw2[i], q[i], b);
                out2[(size_t)r * W + x] = b;
            }
        }
        __syncwarp();
    }
}

// dog: out = max(a - b, 0) with a the column filter of in1 by w1 and b that of in2 by w2;
// else out = a.
__global__ void __launch_bounds__(256)
gauss_cols_kernel(const float* __restrict__ in1, const float* __restrict__ in2, int64_t n, int H, int W,
                  const float* __restrict__ w1, int r1, const float* __restrict__ w2, int r2, int dog,
                  float* __restrict__ out) {
    extern __shared__ float sm[];
    const int nw1 = 2 * r1 + 1, nw2 = dog ? 2 * r2 + 1 : 0;
    float* sw1 = sm;
    float* sw2 = sw1 + nw1;
    float* s1 = sw2 + nw2;                                   // [H][kStrip]
    float* s2 = s1 + (size_t)H * kStrip;                     // [H][kStrip] (dog)
    for (int i = threadIdx.x; i < nw1; i += blockDim.x) sw1[i] = w1[i];
    for (int i = threadIdx.x; i < nw2; i += blockDim.x) sw2[i] = w2[i];
    const int strips = (W + kStrip - 1) / kStrip;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int64_t t = blockIdx.x; t < n * strips; t += gridDim.x) {
        const int64_t p = t / strips;
        const int x0 = (int)(t - p * strips) * kStrip;
        const int x = x0 + lane;
        const bool col = x < W;
        const size_t base = (size_t)p * H * W;
        __syncthreads();                                     // previous strip's reads are done
        for (int y = warp; y < H; y += nwarps) {
            s1[y * kStrip + lane] = col ? __ldg(in1 + base + (size_t)y * W + x) : 0.0f;
            if (dog) s2[y * kStrip + lane] = col ? __ldg(in2 + base + (size_t)y * W + x) : 0.0f;
        }
        __syncthreads();
        if (!col) continue;
        for (int y = warp; y < H; y += nwarps) {
            float a = 0.0f;
            for (int i = 0; i < nw1; ++i) a = fmaf(sw1[i], s1[min(max(y + i - r1, 0), H - 1) * kStrip + lane], a);
            float v = a;
            if (dog) {
                float b = 0.0f;
                for (int i = 0; i < nw2; ++i) b = fmaf(sw2[i], s2[min(max(y + i - r2, 0), H - 1) * kStrip + lane], b);
                v = fmaxf(a - b, 0.0f);
            }
            out[base + (size_t)y * W + x] = v;
        }
    }
}

int grid_of(int64_t items, int per_block) {
    const int64_t g = (items + per_block - 1) / per_block;
    const int64_t cap = (int64_t)device_sms() * 16;
    return (int)(g < 1 ? 1 : (g < cap ? g : cap));
}

}  // namespace

size_t gauss_cols_smem(int H, int r1, int r2, int dog) {
    return ((size_t)(2 * r1 + 1) + (dog ? 2 * r2 + 1 : 0) + (size_t)H * kStrip * (dog ? 2 : 1)) * sizeof(float);
}

cudaError_t launch_gauss_rows(const void* in, int dtype, int64_t rows, int W, const float* w1, int r1, const float* w2,
                              int r2, float* out1, float* out2, cudaStream_t st) {
    if (rows <= 0) return cudaSuccess;
    const int R = w2 ? (r1 > r2 ? r1 : r2) : r1;
    const size_t smem = ((size_t)(2 * r1 + 1) + (w2 ? 2 * r2 + 1 : 0) + (size_t)kRowWarps * (W + 2 * R)) * sizeof(float);
    const int grid = grid_of(rows, kRowWarps);
    cudaError_t e;
    if (dtype == TM_DTYPE_U16) {
        e = kernel_occupancy((const void*)gauss_rows_kernel<uint16_t>, 32 * kRowWarps, smem, nullptr);
        if (e != cudaSuccess) return e;
        gauss_rows_kernel<uint16_t><<<grid, 32 * kRowWarps, smem, st>>>((const uint16_t*)in, rows, W, w1, r1, w2, r2,
                                                                        out1, out2);
    } else {
        e = kernel_occupancy((const void*)gauss_rows_kernel<float>, 32 * kRowWarps, smem, nullptr);
        if (e != cudaSuccess) return e;
        gauss_rows_kernel<float><<<grid, 32 * kRowWarps, smem, st>>>((const float*)in, rows, W, w1, r1, w2, r2, out1,
                                                                     out2);
    }
    return cudaGetLastError();
}

cudaError_t launch_gauss_cols(const float* in1, const float* in2, int64_t n, int H, int W, const float* w1, int r1,
                              const float* w2, int r2, int dog, float* out, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const size_t smem = gauss_cols_smem(H, r1, r2, dog);
    const cudaError_t e = kernel_occupancy((const void*)gauss_cols_kernel, 256, smem, nullptr);
    if (e != cudaSuccess) return e;
    const int64_t strips = (int64_t)n * ((W + kStrip - 1) / kStrip);
    gauss_cols_kernel<<<grid_of(strips, 1), 256, smem, st>>>(in1, in2, n, H, W, w1, r1, w2, r2, dog, out);
    return cudaGetLastError();
}

}  // namespace tmgb
