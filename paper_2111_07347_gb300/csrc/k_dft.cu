// Angular DFT of the polar images and survivor compaction for the BF16 tensor-core path.
//
// The paper notes (Section 2.2, complexity paragraph) that the azimuthal cross-correlation
// can be computed through an FFT along phi instead of sliding the template.  The BF16 path
// uses the correlation theorem along theta: with X^[r, m] = sum_theta X[r, theta]
// e^{-2 pi i m theta / n}, the correlation of template k with pattern P at shift s is
//   C[k, s] = sum_{m=0}^{n/2} (w_m / n) Re( G[k, m] e^{2 pi i m s / n} ),
//   G[k, m] = sum_r conj(T^_k[r, m]) P^[r, m]                (w = 1 at m = 0, n/2; else 2).
// This file computes P^ (divided by |P|) for the radii the libraries use, in FP32, stored
// as half precision (values are bounded by sqrt(n_theta)), one CTA per pattern.
#include <cuda_fp16.h>

#include "tm_internal.h"

namespace tmgb {
namespace {

// grid-stride over patterns; thread handles (radius slot, frequency m)
__global__ void __launch_bounds__(256)
dft_kernel(const float* __restrict__ polar, const float* __restrict__ pnorm, int64_t n, int n_r, int n_theta,
           const int32_t* __restrict__ radii, int n_rad, int n_freq, const float2* __restrict__ twiddle,
           __half2* __restrict__ out) {
    extern __shared__ float sm[];
    float* rows = sm;                                  // [n_rad][n_theta]
    float2* tw = (float2*)(rows + (size_t)n_rad * n_theta);  // [n_theta]: (cos, sin) of 2 pi j / n
    for (int i = threadIdx.x; i < n_theta; i += blockDim.x) tw[i] = twiddle[i];
    for (int64_t p = blockIdx.x; p < n; p += gridDim.x) {
        __syncthreads();
        const float* src = polar + (size_t)p * n_r * n_theta;
        for (int i = threadIdx.x; i < n_rad * n_theta; i += blockDim.x) {
            const int a = i / n_theta, th = i - a * n_theta;
            rows[i] = src[(size_t)radii[a] * n_theta + th];
        }
        __syncthreads();
        const float pn = pnorm[p];
        const float inv = pn > 0.0f ? 1.0f / pn : 0.0f;
        __half2* o = out + (size_t)p * n_rad * n_freq;
        for (int idx = threadIdx.x; idx < n_rad * n_freq; idx += blockDim.x) {
            const int a = idx / n_freq, m = idx - a * n_freq;
            const float* row = rows + (size_t)a * n_theta;
            float re = 0.0f, im = 0.0f;
            const float2 step = tw[m];                 // e^{2 pi i m / n}
            int j = 0;                                 // (m * theta) mod n_theta at block starts
            for (int th0 = 0; th0 < n_theta; th0 += 32) {
                float2 w = tw[j];                      // exact restart every 32 angles
                const int th1 = min(th0 + 32, n_theta);
                for (int th = th0; th < th1; ++th) {
                    const float v = row[th];           // same address across the warp: broadcast
                    re = fmaf(v, w.x, re);
                    im = fmaf(-v, w.y, im);
                    const float wx = w.x * step.x - w.y * step.y;
                    w.y = fmaf(w.x, step.y, w.y * step.x);
                    w.x = wx;
                }
                j = (int)(((int64_t)m * th1) % n_theta);
            }
            o[idx] = __floats2half2_rn(re * inv, im * inv);
        }
    }
}

// Survivors of the pre-filter mask in the library's dense order (templates sorted by spot
// count, so a warp of the tensor-core kernel holds templates of similar cost).
__global__ void __launch_bounds__(512)
compact_kernel(const uint32_t* __restrict__ mask, int64_t n, int K, int words, const int32_t* __restrict__ order,
               int keep, int32_t* __restrict__ list) {
    __shared__ int wsum[16];
    __shared__ int base_s;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t p = blockIdx.x; p < n; p += gridDim.x) {
        const uint32_t* mrow = mask + (size_t)p * words;
        if (threadIdx.x == 0) base_s = 0;
        __syncthreads();
        for (int d0 = 0; d0 < K; d0 += blockDim.x) {
            const int d = d0 + threadIdx.x;
            int k = -1;
            bool on = false;
            if (d < K) {
                k = order[d];
                on = (mrow[k >> 5] >> (k & 31)) & 1u;
            }
            const unsigned b = __ballot_sync(0xffffffffu, on);
            if (lane == 0) wsum[warp] = __popc(b);
            __syncthreads();
            int before = base_s;
            for (int w = 0; w < warp; ++w) before += wsum[w];
            before += __popc(b & ((1u << lane) - 1u));
            if (on && before < keep) list[(size_t)p * keep + before] = k;
            __syncthreads();
            if (threadIdx.x == 0) {
                int t = 0;
                for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += wsum[w];
                base_s += t;
            }
            __syncthreads();
        }
    }
}

}  // namespace

cudaError_t launch_dft(const float* polar, const float* pnorm, int64_t n, int n_r, int n_theta, const int32_t* radii,
                       int n_rad, int n_freq, const float2* twiddle, void* out, int num_sms, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const size_t smem = (size_t)n_rad * n_theta * 4 + (size_t)n_theta * 8;
    if (smem > 200 * 1024) return cudaErrorInvalidValue;
    int per_sm = 1;
    const cudaError_t e = kernel_occupancy((const void*)dft_kernel, 256, smem, &per_sm);
    if (e != cudaSuccess) return e;
    int64_t grid = (int64_t)num_sms * (per_sm > 0 ? per_sm : 1);
    if (grid > n) grid = n;
    dft_kernel<<<(int)grid, 256, smem, st>>>(polar, pnorm, n, n_r, n_theta, radii, n_rad, n_freq, twiddle,
                                             (__half2*)out);
    return cudaGetLastError();
}

cudaError_t launch_compact(const uint32_t* mask, int64_t n, int K, const int32_t* order, int keep, int32_t* list,
                           cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int grid = (int)(n < 65536 ? n : 65536);
    compact_kernel<<<grid, 512, 0, st>>>(mask, n, K, (K + 31) / 32, order, keep, list);
    return cudaGetLastError();
}

}  // namespace tmgb
