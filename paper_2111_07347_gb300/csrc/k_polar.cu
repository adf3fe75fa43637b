// Stage 1: gamma / constant subtraction of the raw frame and bilinear resampling onto
// the polar grid about the direct beam (arXiv 2111.07347, Section 2.2, Fig. 2 (a)-(c);
// the gamma and subtraction of Sections 2.2 and 4.3).  By-products for later stages:
// the image norm sqrt(sum P'^2) of Eq. 1 and the azimuthal sums R_P[j] used by the
// pre-filter (Section 2.2, Fig. 3).
//
// One CTA per pattern (grid-stride).  Thread k owns polar column k; rows are walked in
// order, so the writes of a row are coalesced.  Tap positions and the fractions fx, 1-fx,
// fy, 1-fy come from a table built on the host in double precision for the call's centre
// (storing 1-fx avoids the cancellation of forming it in float when fx is near 1), so
// each bilinear weight is within a few float ulps of its exact value.  Reductions run in a fixed order: the result does not
// depend on the grid size or on other patterns of the batch.
#include "tm_internal.h"

namespace tmgb {
namespace {

struct Gamma {
    int mode;            // 0: sqrt (gamma = 0.5), 1: identity, 2: powf
    float g, sub;
    __device__ __forceinline__ float operator()(float v) const {
        v = fmaxf(v, 0.0f);
        float r = mode == 0 ? sqrtf(v) : (mode == 1 ? v : powf(v, g));
        return r - sub;
    }
};

template <typename T>
__device__ __forceinline__ float tap(const T* frame, int H, int W, int x, int y, const Gamma& gm) {
    if ((unsigned)x >= (unsigned)W || (unsigned)y >= (unsigned)H) return 0.0f;  // zero outside
    return gm((float)__ldg(frame + (size_t)y * W + x));
}

// Tap of a sample at offset (dx, dy) = (r cos theta, r sin theta) from a per-pattern centre
// (cx, cy): the offsets come from the host in double precision split as hi + lo floats;
// x = cx + dx is formed with an error-free sum so that the fraction is accurate far below
// float resolution before it is rounded.
__device__ __forceinline__ void centre_tap(float c, float hi, float lo, int& i0, float& f, float& g) {
    const float s = c + hi;
    const float bb = s - c;
    const float err = (c - (s - bb)) + (hi - bb);               // s + err == c + hi exactly
    float base = floorf(s);
    float fh = s - base;                                        // exact
    float fl = err + lo;
    float fr = fh + fl;
    if (fr < 0.0f) { base -= 1.0f; fh += 1.0f; fr = fh + fl; }
    else if (fr >= 1.0f) { base += 1.0f; fh -= 1.0f; fr = fh + fl; }
    i0 = (int)base;
    f = fr;
    g = (1.0f - fh) - fl;
}

template <typename T>
__global__ void __launch_bounds__(1024)
polar_kernel(const T* __restrict__ frames, int64_t n, int H, int W,
             const int32_t* __restrict__ txy, const float4* __restrict__ tw, Gamma gm, int n_r, int n_theta,
             const uint8_t* __restrict__ keep_row, float* __restrict__ polar, float* __restrict__ pnorm,
             float* __restrict__ radial, const float2* __restrict__ centres, const float4* __restrict__ toff) {
    extern __shared__ float smem[];
    const int nw = blockDim.x >> 5;
    float* part = smem;                         // [n_r][nw] row partial sums
    float* red = smem + (size_t)n_r * nw;       // [blockDim] norm partials
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int U = 4;                        // rows in flight per thread

    for (int64_t p = blockIdx.x; p < n; p += gridDim.x) {
        const T* frame = frames + (size_t)p * H * W;
        float* out = polar + (size_t)p * n_r * n_theta;
        float2 cen = make_float2(0.0f, 0.0f);
        if (centres) cen = __ldg(centres + p);
        float s2 = 0.0f, c2 = 0.0f;             // Kahan sum of P'^2 for this thread
        for (int j0 = 0; j0 < n_r; j0 += U) {
            float rowsum[U];
#pragma unroll
            for (int u = 0; u < U; ++u) rowsum[u] = 0.0f;
            for (int k = threadIdx.x; k < n_theta; k += blockDim.x) {
                float v[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int j = j0 + u;
                    v[u] = 0.0f;
                    if (j < n_r) {
                        const int idx = j * n_theta + k;
                        int x0, y0;
                        float4 f;                                   // fx, 1 - fx, fy, 1 - fy
                        if (centres) {
                            const float4 o = __ldg(toff + idx);     // dx hi, dx lo, dy hi, dy lo
                            centre_tap(cen.x, o.x, o.y, x0, f.x, f.y);
                            centre_tap(cen.y, o.z, o.w, y0, f.z, f.w);
                        } else {
                            const int xy = __ldg(txy + idx);
                            x0 = (int)(int16_t)(xy & 0xffff);
                            y0 = xy >> 16;
                            f = __ldg(tw + idx);
                        }
                        const float v00 = tap(frame, H, W, x0, y0, gm);
                        const float v10 = tap(frame, H, W, x0 + 1, y0, gm);
                        const float v01 = tap(frame, H, W, x0, y0 + 1, gm);
                        const float v11 = tap(frame, H, W, x0 + 1, y0 + 1, gm);
                        v[u] = f.w * (f.y * v00 + f.x * v10) + f.z * (f.y * v01 + f.x * v11);
                    }
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int j = j0 + u;
                    if (j < n_r) {
                        if (!keep_row || keep_row[j]) out[j * n_theta + k] = v[u];
                        const float y = fmaf(v[u], v[u], -c2);
                        const float t = s2 + y;
                        c2 = (t - s2) - y;
                        s2 = t;
                        rowsum[u] += v[u];
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                float r = rowsum[u];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
                if (lane == 0 && j0 + u < n_r) part[(j0 + u) * nw + warp] = r;
            }
        }
        red[threadIdx.x] = s2;
        __syncthreads();
        // fixed-order tree over the block (blockDim is a multiple of 32)
        for (int w = 1; w < (int)blockDim.x; w <<= 1) {
            const int i = threadIdx.x;
            if ((i & (2 * w - 1)) == 0 && i + w < (int)blockDim.x) red[i] += red[i + w];
            __syncthreads();
        }
        if (threadIdx.x == 0 && pnorm) pnorm[p] = sqrtf(red[0]);
        if (radial) {
            for (int j = threadIdx.x; j < n_r; j += blockDim.x) {
                float s = 0.0f;
                for (int w = 0; w < nw; ++w) s += part[j * nw + w];
                radial[(size_t)p * n_r + j] = s;
            }
        }
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_polar(const void* frames, int dtype, int64_t n, int H, int W,
                         const PolarTable& tab, double gamma, double subtract, int n_r,
                         int n_theta, float* polar, float* pnorm, float* radial,
                         cudaStream_t st, const uint8_t* keep_row, const float2* centres, const float4* offsets) {
    if (n <= 0) return cudaSuccess;
    Gamma gm;
    gm.mode = gamma == 0.5 ? 0 : (gamma == 1.0 ? 1 : 2);
    gm.g = (float)gamma;
    gm.sub = (float)subtract;
    int threads = ((n_theta + 31) / 32) * 32;
    if (threads > 1024) threads = 1024;
    const int nw = threads / 32;
    const size_t smem = ((size_t)n_r * nw + threads) * sizeof(float);
    if (smem > 48 * 1024) {
        cudaError_t e;
        if (dtype == TM_DTYPE_U16)
            e = cudaFuncSetAttribute(polar_kernel<uint16_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        else
            e = cudaFuncSetAttribute(polar_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int64_t grid64 = n < 65535 * 16 ? n : 65535 * 16;
    const int grid = (int)grid64;
    if (dtype == TM_DTYPE_U16)
        polar_kernel<uint16_t><<<grid, threads, smem, st>>>((const uint16_t*)frames, n, H, W, tab.xy, tab.w, gm, n_r, n_theta, keep_row, polar, pnorm, radial, centres, offsets);
    else
        polar_kernel<float><<<grid, threads, smem, st>>>((const float*)frames, n, H, W, tab.xy, tab.w, gm, n_r, n_theta, keep_row, polar, pnorm, radial, centres, offsets);
    return cudaGetLastError();
}

}  // namespace tmgb
