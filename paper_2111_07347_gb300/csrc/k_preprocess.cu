// Background removal and smoothing before the polar transform (arXiv 2111.07347, Section 3.1:
// the diffuse background of each pattern was removed with a difference of Gaussians and the
// result smoothed by a Gaussian blur).  Separable Gaussian filters with the edge pixel
// repeated outside the frame: a row pass, then a column pass, each output a sum over the
// 2R + 1 offsets in ascending order (FP32 multiply-adds), weights computed in double
// precision on the host and zero-padded to a multiple of four taps.
//
// Each thread computes eight consecutive outputs.  Taps go four at a time: the four inputs
// that enter the thread's window and the four weights are read once from shared memory and
// feed 32 multiply-adds (the window's other inputs stay in registers), so shared memory
// serves a quarter of an operand per multiply-add.
// gauss_rows_kernel: one warp per image row (256 outputs per pass over the row); the row and
//   a clamped halo are staged in shared memory with one padding word every eight, so the
//   lanes' stride-8 reads fall in distinct banks; up to two filters per pass (the two
//   Gaussians of the difference share the row).
// gauss_cols_kernel: one CTA per 32-column strip of a frame; the strip of one or two inputs
//   is staged in shared memory (rows clamped on reading), lanes are columns, each thread takes
//   eight consecutive rows; the difference of Gaussians (clipped at 0) is formed in the same
//   pass.
#include "tm_internal.h"

namespace tmgb {
namespace {

constexpr int kRowWarps = 8;
constexpr int kStrip = 32;
constexpr int kOut = 8;                                     // outputs per thread
constexpr int kTap = 4;                                     // taps per step (weights padded to it)

template <typename T>
__device__ __forceinline__ float as_float(T v) {
    return (float)v;
}

__host__ __device__ inline int padded_taps(int r) { return ((2 * r + 1 + kTap - 1) / kTap) * kTap; }

// Shared-memory index of row element e with one padding word every eight.
__device__ __forceinline__ int skew(int e) { return e + (e >> 3); }

// acc[j] += sum_t w[t] x[base + j + t] over t < nt (nt a multiple of kTap); x(e) reads
// element e.  The window of kOut + kTap inputs slides by kTap per step.
template <typename F>
__device__ __forceinline__ void conv8(float (&acc)[kOut], const float* __restrict__ w, int nt, int base, F x) {
    float a[kOut];
#pragma unroll
    for (int j = 0; j < kOut; ++j) a[j] = x(base + j);
    for (int t0 = 0; t0 < nt; t0 += kTap) {
        float b[kTap], wt[kTap];
#pragma unroll
        for (int u = 0; u < kTap; ++u) {
            b[u] = x(base + kOut + t0 + u);
            wt[u] = w[t0 + u];
        }
#pragma unroll
        for (int u = 0; u < kTap; ++u) {
#pragma unroll
            for (int j = 0; j < kOut; ++j) acc[j] = fmaf(wt[u], j + u < kOut ? a[j + u] : b[j + u - kOut], acc[j]);
        }
#pragma unroll
        for (int j = 0; j < kOut; ++j) a[j] = j + kTap < kOut ? a[j + kTap] : b[j + kTap - kOut];
    }
}

template <typename T>
__global__ void __launch_bounds__(32 * kRowWarps)
gauss_rows_kernel(const T* __restrict__ in, int64_t rows, int W, const float* __restrict__ w1, int r1,
                  const float* __restrict__ w2, int r2, float* __restrict__ out1, float* __restrict__ out2) {
    extern __shared__ float sm[];
    const int R = max(r1, w2 ? r2 : 0);
    const int nt1 = padded_taps(r1), nt2 = w2 ? padded_taps(r2) : 0;
    float* sw1 = sm;                                         // [nt1]
    float* sw2 = sw1 + nt1;                                  // [nt2]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int span = 32 * kOut;                              // outputs per pass over the row
    const int chunks = (W + span - 1) / span;
    const int ne = chunks * span + 2 * R + kOut + kTap;      // staged elements (pixel e - R, clamped)
    float* row_s = sw2 + nt2 + warp * skew(ne);
    for (int i = threadIdx.x; i < nt1; i += blockDim.x) sw1[i] = w1[i];
    for (int i = threadIdx.x; i < nt2; i += blockDim.x) sw2[i] = w2[i];
    __syncthreads();
    for (int64_t r = (int64_t)blockIdx.x * kRowWarps + warp; r < rows; r += (int64_t)gridDim.x * kRowWarps) {
        const T* src = in + (size_t)r * W;
        for (int e = lane; e < ne; e += 32) row_s[skew(e)] = as_float(__ldg(src + min(max(e - R, 0), W - 1)));
        __syncwarp();
        for (int c = 0; c < chunks; ++c) {
            const int x0 = c * span + kOut * lane;           // the thread's first output
            float acc[kOut];
#pragma unroll
            for (int j = 0; j < kOut; ++j) acc[j] = 0.0f;
            conv8(acc, sw1, nt1, x0 + (R - r1), [&](int e) { return row_s[skew(e)]; });
#pragma unroll
            for (int j = 0; j < kOut; ++j)
                if (x0 + j < W) out1[(size_t)r * W + x0 + j] = acc[j];
            if (w2) {
#pragma unroll
                for (int j = 0; j < kOut; ++j) acc[j] = 0.0f;
                conv8(acc, sw2, nt2, x0 + (R - r2), [&](int e) { return row_s[skew(e)]; });
#pragma unroll
                for (int j = 0; j < kOut; ++j)
                    if (x0 + j < W) out2[(size_t)r * W + x0 + j] = acc[j];
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
    const int nt1 = padded_taps(r1), nt2 = dog ? padded_taps(r2) : 0;
    float* sw1 = sm;
    float* sw2 = sw1 + nt1;
    float* s1 = sw2 + nt2;                                   // [H][kStrip]
    float* s2 = s1 + (size_t)H * kStrip;                     // [H][kStrip] (dog)
    for (int i = threadIdx.x; i < nt1; i += blockDim.x) sw1[i] = w1[i];
    for (int i = threadIdx.x; i < nt2; i += blockDim.x) sw2[i] = w2[i];
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
        for (int y0 = kOut * warp; y0 < H; y0 += kOut * nwarps) {
            float a[kOut];
#pragma unroll
            for (int j = 0; j < kOut; ++j) a[j] = 0.0f;
            conv8(a, sw1, nt1, y0 - r1, [&](int e) { return s1[min(max(e, 0), H - 1) * kStrip + lane]; });
            if (dog) {
                float b[kOut];
#pragma unroll
                for (int j = 0; j < kOut; ++j) b[j] = 0.0f;
                conv8(b, sw2, nt2, y0 - r2, [&](int e) { return s2[min(max(e, 0), H - 1) * kStrip + lane]; });
#pragma unroll
                for (int j = 0; j < kOut; ++j) a[j] = fmaxf(a[j] - b[j], 0.0f);
            }
#pragma unroll
            for (int j = 0; j < kOut; ++j)
                if (y0 + j < H) out[base + (size_t)(y0 + j) * W + x] = a[j];
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
    return ((size_t)padded_taps(r1) + (dog ? padded_taps(r2) : 0) + (size_t)H * kStrip * (dog ? 2 : 1)) * sizeof(float);
}

int gauss_padded_taps(int r) { return padded_taps(r); }

cudaError_t launch_gauss_rows(const void* in, int dtype, int64_t rows, int W, const float* w1, int r1, const float* w2,
                              int r2, float* out1, float* out2, cudaStream_t st) {
    if (rows <= 0) return cudaSuccess;
    const int R = w2 ? (r1 > r2 ? r1 : r2) : r1;
    const int span = 32 * kOut, ne = ((W + span - 1) / span) * span + 2 * R + kOut + kTap;
    const size_t smem = ((size_t)padded_taps(r1) + (w2 ? padded_taps(r2) : 0) + (size_t)kRowWarps * (ne + (ne >> 3))) *
                        sizeof(float);
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
