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

// The same tap from a frame staged in shared memory.
template <typename T>
__device__ __forceinline__ float tap(T* frame, int H, int W, int x, int y, const Gamma& gm) {
    if ((unsigned)x >= (unsigned)W || (unsigned)y >= (unsigned)H) return 0.0f;
    return gm((float)frame[y * W + x]);
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

// Staged variant: the CTA first copies the whole frame into shared memory with coalesced
// 16-byte loads, then every tap is a shared-memory read.  Rows are split over R groups of
// warps (thread (g, k): rows j = g, g + R, ...), so a CTA has R x 32 ceil(n_theta / 32)
// threads.  Used when the frame fits in shared memory.
template <typename T>
__global__ void __launch_bounds__(1024)
polar_staged_kernel(const T* __restrict__ frames, int64_t n, int H, int W,
                    const int32_t* __restrict__ txy, const float4* __restrict__ tw, Gamma gm, int n_r, int n_theta,
                    int R, const uint8_t* __restrict__ keep_row, float* __restrict__ polar,
                    float* __restrict__ pnorm, float* __restrict__ radial, const float2* __restrict__ centres,
                    const float4* __restrict__ toff) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int cols = blockDim.x / R;                     // threads per row group (multiple of 32)
    const int g = threadIdx.x / cols, k0 = threadIdx.x - g * cols;
    const int nw = blockDim.x >> 5;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const size_t fbytes = (size_t)H * W * sizeof(T);
    T* sF = (T*)smem_raw;
    float* part = (float*)(smem_raw + ((fbytes + 15) & ~(size_t)15));   // [n_r][nw]
    float* red = part + (size_t)n_r * nw;                               // [blockDim]

    for (int64_t p = blockIdx.x; p < n; p += gridDim.x) {
        const T* frame = frames + (size_t)p * H * W;
        __syncthreads();
        if ((((uintptr_t)frame) & 15) == 0) {
            const size_t nv = fbytes / 16;
            const uint4* src = (const uint4*)frame;
            uint4* dst = (uint4*)sF;
            for (size_t i = threadIdx.x; i < nv; i += blockDim.x) dst[i] = __ldg(src + i);
            for (size_t i = nv * 16 / sizeof(T) + threadIdx.x; i < (size_t)H * W; i += blockDim.x) sF[i] = frame[i];
        } else {
            for (size_t i = threadIdx.x; i < (size_t)H * W; i += blockDim.x) sF[i] = frame[i];
        }
        __syncthreads();
        float* out = polar + (size_t)p * n_r * n_theta;
        float2 cen = make_float2(0.0f, 0.0f);
        if (centres) cen = __ldg(centres + p);
        float s2 = 0.0f, c2 = 0.0f;                      // Kahan sum of P'^2 for this thread
        for (int j = g; j < n_r; j += R) {
            float rowsum = 0.0f;
            for (int k = k0; k < n_theta; k += cols) {
                const int idx = j * n_theta + k;
                int x0, y0;
                float4 f;                                // fx, 1 - fx, fy, 1 - fy
                if (centres) {
                    const float4 o = __ldg(toff + idx);
                    centre_tap(cen.x, o.x, o.y, x0, f.x, f.y);
                    centre_tap(cen.y, o.z, o.w, y0, f.z, f.w);
                } else {
                    const int xy = __ldg(txy + idx);
                    x0 = (int)(int16_t)(xy & 0xffff);
                    y0 = xy >> 16;
                    f = __ldg(tw + idx);
                }
                const float v00 = tap(sF, H, W, x0, y0, gm);
                const float v10 = tap(sF, H, W, x0 + 1, y0, gm);
                const float v01 = tap(sF, H, W, x0, y0 + 1, gm);
                const float v11 = tap(sF, H, W, x0 + 1, y0 + 1, gm);
                const float v = f.w * (f.y * v00 + f.x * v10) + f.z * (f.y * v01 + f.x * v11);
                if (!keep_row || keep_row[j]) out[idx] = v;
                const float y = fmaf(v, v, -c2);
                const float t = s2 + y;
                c2 = (t - s2) - y;
                s2 = t;
                rowsum += v;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) rowsum += __shfl_xor_sync(0xffffffffu, rowsum, o);
            if (lane == 0) part[j * nw + warp] = rowsum;  // warps of other groups leave theirs for row j
        }
        red[threadIdx.x] = s2;
        __syncthreads();
        for (int w = 1; w < (int)blockDim.x; w <<= 1) {
            const int i = threadIdx.x;
            if ((i & (2 * w - 1)) == 0 && i + w < (int)blockDim.x) red[i] += red[i + w];
            __syncthreads();
        }
        if (threadIdx.x == 0 && pnorm) pnorm[p] = sqrtf(red[0]);
        if (radial) {
            // row j's partials come from the warps of group j % R only
            const int wpg = cols >> 5;
            for (int j = threadIdx.x; j < n_r; j += blockDim.x) {
                const int g0 = j % R;
                float s = 0.0f;
                for (int w = 0; w < wpg; ++w) s += part[j * nw + g0 * wpg + w];
                radial[(size_t)p * n_r + j] = s;
            }
        }
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
    const size_t esz = dtype == TM_DTYPE_U16 ? 2 : 4;
    const size_t fbytes = (size_t)H * W * esz;
    const int cols = ((n_theta + 31) / 32) * 32;
    if (cols <= 512) {
        // staged: frame in shared memory, rows split over R groups of warps
        const int R = cols <= 256 ? 4 : 2;
        const int threads = R * cols;
        const int nw = threads / 32;
        const size_t smem = ((fbytes + 15) & ~(size_t)15) + ((size_t)n_r * nw + threads) * sizeof(float);
        if (smem <= 200 * 1024) {
            cudaError_t e;
            if (dtype == TM_DTYPE_U16)
                e = cudaFuncSetAttribute(polar_staged_kernel<uint16_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            else
                e = cudaFuncSetAttribute(polar_staged_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            int per_sm = 1;
            if (dtype == TM_DTYPE_U16)
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, polar_staged_kernel<uint16_t>, threads, smem);
            else
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, polar_staged_kernel<float>, threads, smem);
            int dev = 0, sms = 148;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            int64_t grid = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
            if (grid > n) grid = n;
            if (dtype == TM_DTYPE_U16)
                polar_staged_kernel<uint16_t><<<(int)grid, threads, smem, st>>>(
                    (const uint16_t*)frames, n, H, W, tab.xy, tab.w, gm, n_r, n_theta, R, keep_row, polar, pnorm,
                    radial, centres, offsets);
            else
                polar_staged_kernel<float><<<(int)grid, threads, smem, st>>>(
                    (const float*)frames, n, H, W, tab.xy, tab.w, gm, n_r, n_theta, R, keep_row, polar, pnorm,
                    radial, centres, offsets);
            return cudaGetLastError();
        }
    }
    int threads = cols;
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
