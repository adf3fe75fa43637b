// Stage 2: the azimuthally integrated pre-filter (arXiv 2111.07347, Section 2.2 and
// Fig. 3): the polar image and every template are integrated over the azimuth, the
// integrated image is correlated with the integrated library (one matrix-vector product
// per pattern; here one matrix-matrix product per batch) and only the best-correlated
// templates go on to full matching.
//
//   score[p][k] = R_P[p] . R_T[k] / (|R_P[p]| |R_T[k]|)        (0 if a norm is 0)
//   keep the ceil(f K) largest per pattern, ties to the lower k  -> bit mask [p][K/32]
//
// The scores are a tiled FP32 SIMT product (n_r = 128 is far too short a contraction
// to pay for tensor-core staging); the selection is an exact 4-pass radix select over
// order-preserving integer keys, one CTA per pattern.
#include "tm_internal.h"

namespace tmgb {
namespace {

__global__ void radial_norm_kernel(const float* __restrict__ radial, int64_t n, int n_r,
                                   float* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t p = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (p >= n) return;
    float s = 0.0f;
    for (int j = lane; j < n_r; j += 32) {
        const float v = radial[(size_t)p * n_r + j];
        s = fmaf(v, v, s);
    }
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[p] = sqrtf(s);
}

constexpr int PT = 64, KT = 64, RC = 16;   // tile: 64 patterns x 64 templates, 16-deep chunks

__global__ void __launch_bounds__(256)
prefilter_scores_kernel(const float* __restrict__ radial, const float* __restrict__ rpn, int64_t n,
                        int n_r, RadialLib lib, float* __restrict__ score) {
    __shared__ float sp[RC][PT + 4];
    __shared__ float st[RC][KT + 4];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;    // 16 x 16 threads, 4 x 4 each
    const int64_t p0 = (int64_t)blockIdx.y * PT;
    const int k0 = blockIdx.x * KT;
    float acc[4][4] = {};
    for (int r0 = 0; r0 < n_r; r0 += RC) {
        for (int i = threadIdx.x; i < RC * PT; i += 256) {
            const int rr = i % RC, pp = i / RC;
            const int64_t p = p0 + pp;
            sp[rr][pp] = (p < n && r0 + rr < n_r) ? radial[(size_t)p * n_r + r0 + rr] : 0.0f;
        }
        for (int i = threadIdx.x; i < RC * KT; i += 256) {
            const int rr = i % RC, kk = i / RC;
            const int k = k0 + kk;
            st[rr][kk] = (k < lib.K && r0 + rr < n_r) ? lib.radial[(size_t)k * n_r + r0 + rr] : 0.0f;
        }
        __syncthreads();
        #pragma unroll
        for (int rr = 0; rr < RC; ++rr) {
            float a[4], b[4];
            #pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = sp[rr][ty * 4 + i];
            #pragma unroll
            for (int i = 0; i < 4; ++i) b[i] = st[rr][tx * 4 + i];
            #pragma unroll
            for (int i = 0; i < 4; ++i)
                #pragma unroll
                for (int jj = 0; jj < 4; ++jj) acc[i][jj] = fmaf(a[i], b[jj], acc[i][jj]);
        }
        __syncthreads();
    }
    #pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t p = p0 + ty * 4 + i;
        if (p >= n) continue;
        const float np_ = rpn[p];
        #pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            const int k = k0 + tx * 4 + jj;
            if (k >= lib.K) continue;
            const float d = np_ * lib.rnorm[k];
            score[(size_t)p * lib.K + k] = d > 0.0f ? __fdiv_rn(acc[i][jj], d) : 0.0f;
        }
    }
}

__device__ __forceinline__ uint32_t order_key(float x) {
    const uint32_t u = __float_as_uint(x);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);     // larger float -> larger key
}

constexpr int SEL_THREADS = 512;

__global__ void __launch_bounds__(SEL_THREADS)
prefilter_select_kernel(const float* __restrict__ score, int64_t n, int K, int keep,
                        uint32_t* __restrict__ mask) {
    extern __shared__ uint32_t keys[];              // [K]
    __shared__ uint32_t hist[256];
    __shared__ uint32_t s_prefix, s_remaining, s_wsum[SEL_THREADS / 32];
    const int words = (K + 31) >> 5;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t p = blockIdx.x; p < n; p += gridDim.x) {
        for (int k = threadIdx.x; k < K; k += blockDim.x) keys[k] = order_key(score[(size_t)p * K + k]);
        if (threadIdx.x == 0) { s_prefix = 0; s_remaining = (uint32_t)keep; }
        __syncthreads();
        uint32_t pmask = 0;
        for (int pass = 0; pass < 4; ++pass) {
            const int shift = 24 - 8 * pass;
            for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
            __syncthreads();
            const uint32_t prefix = s_prefix;
            for (int k = threadIdx.x; k < K; k += blockDim.x) {
                const uint32_t key = keys[k];
                if ((key & pmask) == prefix) atomicAdd(&hist[(key >> shift) & 255u], 1u);
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                uint32_t rem = s_remaining, cum = 0;
                int b = 255;
                for (; b > 0; --b) {
                    if (cum + hist[b] >= rem) break;
                    cum += hist[b];
                }
                s_remaining = rem - cum;
                s_prefix = prefix | ((uint32_t)b << shift);
            }
            pmask |= 255u << shift;
            __syncthreads();
        }
        const uint32_t T = s_prefix;          // key of the keep-th largest score
        const uint32_t need = s_remaining;    // how many entries equal to T are kept
        // keep keys > T, and the first `need` keys == T in ascending k
        uint32_t taken = 0;
        for (int base = 0; base < words * 32; base += blockDim.x) {
            const int k = base + threadIdx.x;
            const uint32_t key = k < K ? keys[k] : 0u;
            const bool eq = k < K && key == T;
            const uint32_t ball = __ballot_sync(0xffffffffu, eq);
            if (lane == 0) s_wsum[warp] = __popc(ball);
            __syncthreads();
            uint32_t before = taken;
            for (int w = 0; w < warp; ++w) before += s_wsum[w];
            before += __popc(ball & ((1u << lane) - 1u));
            const bool kept = k < K && (key > T || (eq && before < need));
            const uint32_t word = __ballot_sync(0xffffffffu, kept);
            if (lane == 0 && (k >> 5) < words) mask[(size_t)p * words + (k >> 5)] = word;
            uint32_t tot = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += s_wsum[w];
            taken += tot;
            __syncthreads();
        }
    }
}

}  // namespace

cudaError_t launch_radial_norm(const float* radial, int64_t n, int n_r, float* out, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int64_t blocks = (n + 7) / 8;
    radial_norm_kernel<<<(unsigned)blocks, 256, 0, st>>>(radial, n, n_r, out);
    return cudaGetLastError();
}

cudaError_t launch_prefilter_scores(const float* radial, const float* radial_norm, int64_t n, int n_r,
                                    const RadialLib& lib, float* score, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    dim3 grid((lib.K + KT - 1) / KT, (unsigned)((n + PT - 1) / PT));
    prefilter_scores_kernel<<<grid, 256, 0, st>>>(radial, radial_norm, n, n_r, lib, score);
    return cudaGetLastError();
}

cudaError_t launch_prefilter_select(const float* score, int64_t n, int K, int keep, uint32_t* mask,
                                    cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const size_t smem = (size_t)K * sizeof(uint32_t);
    if (smem > 200 * 1024) return cudaErrorInvalidValue;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(prefilter_select_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int grid = (int)(n < 65536 ? n : 65536);
    prefilter_select_kernel<<<grid, SEL_THREADS, smem, st>>>(score, n, K, keep, mask);
    return cudaGetLastError();
}

}  // namespace tmgb
