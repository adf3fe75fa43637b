// Stage 1: gamma / constant subtraction of the raw frame and bilinear resampling onto
// the polar grid about the direct beam (arXiv 2111.07347, Section 2.2, Fig. 2 (a)-(c);
// the gamma and subtraction of Sections 2.2 and 4.3).  By-products for later stages:
// the image norm sqrt(sum P'^2) of Eq. 1 and the azimuthal sums R_P[j] used by the
// pre-filter (Section 2.2, Fig. 3).
//
// One CTA per pattern (grid-stride over patterns).  The CTA's threads form R row groups of
// `cols` threads (a multiple of 32); thread (g, k0) owns polar columns k0, k0 + cols, ... of
// rows g, g + R, ..., four rows at a time, so the stores of a row are coalesced and four
// samples are in flight per thread.
//
// Staged form (frame fits in shared memory): the CTA first copies the frame into shared
// memory with 16-byte global loads; rows are padded to an odd number of 32-bit words, so
// samples on an arc (same x, different y) fall in different banks.  Otherwise the taps
// are read from global memory.
//
// Tap positions and bilinear fractions come from a table built on the host in double
// precision for the call's centre.  The fractions are stored as 23-bit fixed point q, so
// that both weights come out of float arithmetic exactly: with y = 1 + q 2^-23 (formed by
// bit assembly), fx = y - 1 and 1 - fx = 2 - y, both exact; each weight is then within
// 2^-24 of the double-precision value.  A sample whose four taps are all inside the
// frame takes a fast path with one bounds test and the subtraction applied once
// (the weights sum to exactly 1); edge samples test each tap (zero outside).
// For u16 frames the gamma of the pixel values below 4096 (all of them at the counts of an
// electron diffraction pattern) is tabulated once per CTA in shared memory, g(v) - c from
// the same correctly rounded sqrtf / powf, so a tap is one table read; larger values are
// computed directly.
// Reductions run in a fixed order: the result does not depend on the grid size or on
// other patterns of the batch.
#include <math.h>

#include <algorithm>

#include "tm_internal.h"

namespace tmgb {
namespace {

constexpr double kPi = 3.14159265358979323846;

constexpr int kLut = 4096;                  // u16 values with a tabulated gamma

// Gamma without the subtraction (negative inputs clamp to 0).  MODE 0: v^0.5 (correctly
// rounded sqrtf), 1: v, 2: v^g (powf).
template <int MODE>
__device__ __forceinline__ float gamma_of(float v, float g) {
    v = fmaxf(v, 0.0f);
    if (MODE == 1) return v;
    if (MODE == 0) return sqrtf(v);
    return powf(v, g);
}

template <bool SMEM, typename T>
__device__ __forceinline__ T load_px(const T* p) {
    if (SMEM) return *p;
    return __ldg(p);
}

// Pixel mask (Section 4.3, masked indexing): pixels whose mask byte is 0 read as 0.
// Global taps: the mask has the frame's layout (row pitch W).
template <bool SMEM, typename T>
__device__ __forceinline__ T load_px_masked(const T* p, const T* frame, const uint8_t* pmask) {
    const T v = load_px<SMEM>(p);
    if (SMEM || !pmask) return v;
    return __ldg(pmask + (p - frame)) ? v : T(0);
}

// A 16-byte vector of pixels starting at pixel 16 i / sizeof(T) of the frame, masked.
__device__ __forceinline__ uint32_t keep_pair(uint32_t mb) {   // mask bytes at bits 0..7, 8..15
    return ((mb & 0xffu) ? 0x0000ffffu : 0u) | ((mb & 0xff00u) ? 0xffff0000u : 0u);
}
__device__ __forceinline__ void mask_vector(uint4& v, const uint8_t* pmask, int i) {
    // u16 frames: 8 pixels per vector (the float variant below takes 4)
    const uint2 m = __ldg(reinterpret_cast<const uint2*>(pmask) + i);
    v.x &= keep_pair(m.x);
    v.y &= keep_pair(m.x >> 16);
    v.z &= keep_pair(m.y);
    v.w &= keep_pair(m.y >> 16);
}
__device__ __forceinline__ void mask_vector4(uint4& v, const uint8_t* pmask, int i) {
    const uint32_t m = __ldg(reinterpret_cast<const uint32_t*>(pmask) + i);
    v.x = (m & 0xffu) ? v.x : 0u;
    v.y = (m & 0xff00u) ? v.y : 0u;
    v.z = (m & 0xff0000u) ? v.z : 0u;
    v.w = (m & 0xff000000u) ? v.w : 0u;
}

// g(v) - sub of one raw pixel.  u16: from the table lut[v] = g(v) - sub (filled with the same
// functions), computed directly for v >= kLut.
template <int MODE>
__device__ __forceinline__ float tap_value(uint16_t v, const float* lut, float2 g, float sub) {
    if (v < kLut) return lut[v];
    const float f = (float)v;
    return gamma_of<MODE>(f < g.y ? 0.0f : f, g.x) - sub;
}
template <int MODE>
__device__ __forceinline__ float tap_value(float v, const float* lut, float2 g, float sub) {
    return gamma_of<MODE>(v < g.y ? 0.0f : v, g.x) - sub;
}

__device__ __forceinline__ bool all_in_lut(uint16_t a, uint16_t b, uint16_t c, uint16_t d) {
    return ((a | b | c | d) & ~(kLut - 1)) == 0;
}
__device__ __forceinline__ bool all_in_lut(float, float, float, float) { return false; }

// Weights (f, 1 - f) from the 23-bit fixed-point fraction q (q < 2^23): both exact.
__device__ __forceinline__ void fixed_weights(uint32_t q, float& f, float& g) {
    const float y = __uint_as_float(0x3F800000u | q);       // 1 + q 2^-23
    f = y - 1.0f;
    g = 2.0f - y;
}

// Bilinear sample of the gamma-corrected, subtracted frame at (x0 + fx, y0 + fy); the frame
// has row pitch `pitch` elements; taps outside [0, W) x [0, H) contribute zero.
template <typename T, int MODE, bool SMEM>
__device__ __forceinline__ float bilinear(const T* frame, int pitch, int H, int W, int x0, int y0, float fx,
                                          float gx, float fy, float gy, const float* lut, float2 g, float sub,
                                          const uint8_t* pmask) {
    if ((unsigned)x0 < (unsigned)(W - 1) && (unsigned)y0 < (unsigned)(H - 1)) {
        const T* p = frame + y0 * pitch + x0;
        const T a = load_px_masked<SMEM>(p, frame, pmask), b = load_px_masked<SMEM>(p + 1, frame, pmask);
        const T c = load_px_masked<SMEM>(p + pitch, frame, pmask), d = load_px_masked<SMEM>(p + pitch + 1, frame, pmask);
        float v00, v10, v01, v11;
        if (all_in_lut(a, b, c, d)) {
            v00 = lut[(int)a];
            v10 = lut[(int)b];
            v01 = lut[(int)c];
            v11 = lut[(int)d];
        } else {
            v00 = tap_value<MODE>(a, lut, g, sub);
            v10 = tap_value<MODE>(b, lut, g, sub);
            v01 = tap_value<MODE>(c, lut, g, sub);
            v11 = tap_value<MODE>(d, lut, g, sub);
        }
        return gy * (gx * v00 + fx * v10) + fy * (gx * v01 + fx * v11);
    }
    float v[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const int x = x0 + (t & 1), y = y0 + (t >> 1);
        v[t] = 0.0f;
        if ((unsigned)x < (unsigned)W && (unsigned)y < (unsigned)H)
            v[t] = tap_value<MODE>(load_px_masked<SMEM>(frame + y * pitch + x, frame, pmask), lut, g, sub);
    }
    return gy * (gx * v[0] + fx * v[1]) + fy * (gx * v[2] + fx * v[3]);
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

// Sum of a[u] over the 32 lanes for four rows u at once (6 shuffles instead of 20): after
// the exchange the lanes 8u hold the total of row u.  Fixed order: deterministic.
__device__ __forceinline__ float warp_sum4(const float a[4], int lane) {
    const bool hi = lane & 16;
    const float b0 = (hi ? a[2] : a[0]) + __shfl_xor_sync(0xffffffffu, hi ? a[0] : a[2], 16);
    const float b1 = (hi ? a[3] : a[1]) + __shfl_xor_sync(0xffffffffu, hi ? a[1] : a[3], 16);
    const bool h8 = lane & 8;
    float c = (h8 ? b1 : b0) + __shfl_xor_sync(0xffffffffu, h8 ? b0 : b1, 8);
    c += __shfl_xor_sync(0xffffffffu, c, 4);
    c += __shfl_xor_sync(0xffffffffu, c, 2);
    c += __shfl_xor_sync(0xffffffffu, c, 1);
    return c;                                   // row (lane >> 3) when (lane & 7) == 0
}

// One polar sample (table entry idx): tap position and weights from the fixed table, or
// from the per-pattern centre plus the offset table.
template <typename T, int MODE, bool STAGED, bool CENTRES>
__device__ __forceinline__ float sample(const T* frame, int pitch, int H, int W, int idx,
                                       const int32_t* __restrict__ txy, const uint2* __restrict__ tq,
                                       const float4* __restrict__ toff, float2 cen, const float* lut, float2 g,
                                       float sub, const uint8_t* pmask) {
    int x0, y0;
    float fx, gx, fy, gy;
    if (CENTRES) {
        const float4 o = __ldg(toff + idx);                      // dx hi, dx lo, dy hi, dy lo
        centre_tap(cen.x, o.x, o.y, x0, fx, gx);
        centre_tap(cen.y, o.z, o.w, y0, fy, gy);
    } else {
        const int xy = __ldg(txy + idx);
        const uint2 q = __ldg(tq + idx);
        x0 = (int)(int16_t)(xy & 0xffff);
        y0 = xy >> 16;
        fixed_weights(q.x, fx, gx);
        fixed_weights(q.y, fy, gy);
    }
    return bilinear<T, MODE, STAGED>(frame, pitch, H, W, x0, y0, fx, gx, fy, gy, lut, g, sub, pmask);
}

constexpr int kMaxThreads = 768;            // 80 registers per thread at one CTA per SM

template <typename T, int MODE, bool STAGED, bool CENTRES>
__global__ void __launch_bounds__(kMaxThreads, 1)
polar_kernel(const T* __restrict__ frames, int64_t n, int H, int W, int pitch, const int32_t* __restrict__ txy,
             const uint2* __restrict__ tq, float2 g, float sub, int n_r, int n_theta, int R,
             const uint8_t* __restrict__ keep_row, const uint8_t* __restrict__ pmask, float* __restrict__ polar,
             float* __restrict__ pnorm,
             float* __restrict__ radial, const float2* __restrict__ centres, const float4* __restrict__ toff) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int cols = blockDim.x / R;                     // threads per row group (multiple of 32)
    const int grp = threadIdx.x / cols, k0 = threadIdx.x - grp * cols;
    const int nw = blockDim.x >> 5;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const size_t fbytes = STAGED ? (size_t)H * pitch * sizeof(T) : 0;
    constexpr bool kHasLut = sizeof(T) == 2;
    T* sF = (T*)smem_raw;
    float* lut = (float*)(smem_raw + ((fbytes + 15) & ~(size_t)15));   // [kLut] for u16 frames
    float* part = lut + (kHasLut ? kLut : 0);                           // [n_r][nw]
    float* red = part + (size_t)n_r * nw;                               // [blockDim]
    if (kHasLut) {
        for (int i = threadIdx.x; i < kLut; i += blockDim.x) {
            const float f = (float)i;
            lut[i] = gamma_of<MODE>(f < g.y ? 0.0f : f, g.x) - sub;
        }
        __syncthreads();
    }
    const int my_rows = grp < n_r ? (n_r - grp + R - 1) / R : 0;        // rows grp, grp + R, ...
    const int rstride = R * n_theta;                                    // table step between them

    for (int64_t p = blockIdx.x; p < n; p += gridDim.x) {
        const T* gframe = frames + (size_t)p * H * W;
        const T* frame = gframe;
        if (STAGED) {
            __syncthreads();                             // previous pattern's reads are done
            const bool vec = (((uintptr_t)gframe) & 15) == 0 && (W * sizeof(T)) % 16 == 0;
            if (vec) {
                const int vr = (int)(W * sizeof(T) / 16);           // 16-byte vectors per row
                const int nv = H * vr;
                const uint4* src = (const uint4*)gframe;
                constexpr int B = 8;                                // loads in flight per thread
                for (int i0 = threadIdx.x; i0 < nv; i0 += B * blockDim.x) {
                    uint4 v[B];
#pragma unroll
                    for (int b = 0; b < B; ++b) {
                        const int i = i0 + b * blockDim.x;
                        if (i < nv) {
                            v[b] = __ldg(src + i);
                            if (pmask) {
                                if (sizeof(T) == 2) mask_vector(v[b], pmask, i);
                                else mask_vector4(v[b], pmask, i);
                            }
                        }
                    }
#pragma unroll
                    for (int b = 0; b < B; ++b) {
                        const int i = i0 + b * blockDim.x;
                        if (i < nv) {
                            const int y = i / vr, xv = i - y * vr;
                            uint32_t* d = (uint32_t*)(sF + (size_t)y * pitch) + xv * 4;
                            d[0] = v[b].x;
                            d[1] = v[b].y;
                            d[2] = v[b].z;
                            d[3] = v[b].w;
                        }
                    }
                }
            } else {
                for (int e = threadIdx.x; e < H * W; e += blockDim.x) {
                    const int y = e / W;
                    sF[(size_t)y * pitch + (e - y * W)] = (!pmask || pmask[e]) ? gframe[e] : T(0);
                }
            }
            __syncthreads();
            frame = sF;
        }
        float* out = polar + (size_t)p * n_r * n_theta;
        float2 cen = make_float2(0.0f, 0.0f);
        if (CENTRES) cen = __ldg(centres + p);
        const int pf = STAGED ? pitch : W;
        float s2 = 0.0f, c2 = 0.0f;                      // Kahan sum of P'^2 for this thread
        for (int b = 0; b < my_rows; b += 4) {           // warp-uniform
            const int nu = my_rows - b;                  // rows left in this batch (>= 1)
            const int j0 = grp + R * b;
            unsigned keep = 0;                           // rows of the batch whose values are stored
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (u < nu && (!keep_row || keep_row[j0 + R * u])) keep |= 1u << u;
            float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
            for (int k = k0; k < n_theta; k += cols) {
                const int idx0 = j0 * n_theta + k;
                float v[4];
                if (nu >= 4) {
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        v[u] = sample<T, MODE, STAGED, CENTRES>(frame, pf, H, W, idx0 + u * rstride, txy, tq, toff,
                                                                cen, lut, g, sub, pmask);
                } else {
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        v[u] = u < nu ? sample<T, MODE, STAGED, CENTRES>(frame, pf, H, W, idx0 + u * rstride, txy, tq,
                                                                         toff, cen, lut, g, sub, pmask)
                                      : 0.0f;
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (u < nu) {
                        if ((keep >> u) & 1u) out[idx0 + u * rstride] = v[u];
                        const float y = fmaf(v[u], v[u], -c2);
                        const float t = s2 + y;
                        c2 = (t - s2) - y;
                        s2 = t;
                        acc[u] += v[u];
                    }
                }
            }
            const float r = warp_sum4(acc, lane);
            const int u = lane >> 3;
            if ((lane & 7) == 0 && u < nu) part[(j0 + R * u) * nw + warp] = r;
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
            // row j's partials come from the warps of group j % R only
            const int wpg = cols >> 5;
            for (int j = threadIdx.x; j < n_r; j += blockDim.x) {
                const int g0 = j % R;
                float s = 0.0f;
                for (int w = 0; w < wpg; ++w) s += part[j * nw + g0 * wpg + w];
                radial[(size_t)p * n_r + j] = s;
            }
        }
        if (!STAGED) __syncthreads();                    // part / red reused by the next pattern
    }
}

template <typename T, int MODE, bool STAGED, bool CENTRES>
cudaError_t launch_one(const T* frames, int64_t n, int H, int W, int pitch, const PolarTable& tab, float2 g, float sub,
                       int n_r, int n_theta, int R, int threads, size_t smem, const uint8_t* keep_row,
                       const uint8_t* pmask, float* polar, float* pnorm, float* radial, const float2* centres,
                       const float4* offsets, cudaStream_t st) {
    auto kern = polar_kernel<T, MODE, STAGED, CENTRES>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 1, dev = 0, sms = 148;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t grid = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
    if (grid > n) grid = n;
    kern<<<(int)grid, threads, smem, st>>>(frames, n, H, W, pitch, tab.xy, tab.q, g, sub, n_r, n_theta, R, keep_row,
                                           pmask, polar, pnorm, radial, centres, offsets);
    return cudaGetLastError();
}

template <typename T, bool STAGED>
cudaError_t launch_mode(int mode, const T* frames, int64_t n, int H, int W, int pitch, const PolarTable& tab,
                        float2 g, float sub, int n_r, int n_theta, int R, int threads, size_t smem,
                        const uint8_t* keep_row, const uint8_t* pmask, float* polar, float* pnorm, float* radial,
                        const float2* centres, const float4* offsets, cudaStream_t st) {
    if (mode == 0)
        return (centres ? launch_one<T, 0, STAGED, true> : launch_one<T, 0, STAGED, false>)(frames, n, H, W, pitch, tab, g, sub, n_r, n_theta, R, threads, smem, keep_row,
                                        pmask, polar, pnorm, radial, centres, offsets, st);
    if (mode == 1)
        return (centres ? launch_one<T, 1, STAGED, true> : launch_one<T, 1, STAGED, false>)(frames, n, H, W, pitch, tab, g, sub, n_r, n_theta, R, threads, smem, keep_row,
                                        pmask, polar, pnorm, radial, centres, offsets, st);
    return (centres ? launch_one<T, 2, STAGED, true> : launch_one<T, 2, STAGED, false>)(frames, n, H, W, pitch, tab, g, sub, n_r, n_theta, R, threads, smem, keep_row,
                                    pmask, polar, pnorm, radial, centres, offsets, st);
}

template <typename T>
cudaError_t launch_typed(const T* frames, int64_t n, int H, int W, const PolarTable& tab, int mode, float2 g,
                         float sub, int n_r, int n_theta, float* polar, float* pnorm, float* radial, cudaStream_t st,
                         const uint8_t* keep_row, const float2* centres, const float4* offsets, const uint8_t* pmask) {
    const int cols = ((n_theta + 31) / 32) * 32;
    if (cols <= kMaxThreads) {
        // staged: rows padded to an odd number of 32-bit words
        int words = (int)((W * sizeof(T) + 3) / 4);
        if (words % 2 == 0) ++words;
        const int pitch = (int)(words * 4 / sizeof(T));
        const int R = std::max(1, std::min(4, kMaxThreads / cols));
        const int threads = R * cols;
        const int nw = threads / 32;
        const size_t fbytes = ((size_t)H * pitch * sizeof(T) + 15) & ~(size_t)15;
        const size_t lut = sizeof(T) == 2 ? kLut * sizeof(float) : 0;
        const size_t smem = fbytes + lut + ((size_t)n_r * nw + threads) * sizeof(float);
        if (smem <= 200 * 1024)
            return launch_mode<T, true>(mode, frames, n, H, W, pitch, tab, g, sub, n_r, n_theta, R, threads, smem,
                                        keep_row, pmask, polar, pnorm, radial, centres, offsets, st);
    }
    const int threads = cols < kMaxThreads ? cols : kMaxThreads;
    const size_t smem = (sizeof(T) == 2 ? kLut * sizeof(float) : 0) + ((size_t)n_r * (threads / 32) + threads) * sizeof(float);
    if (smem > 200 * 1024) return cudaErrorInvalidValue;
    return launch_mode<T, false>(mode, frames, n, H, W, W, tab, g, sub, n_r, n_theta, 1, threads, smem, keep_row,
                                 pmask, polar, pnorm, radial, centres, offsets, st);
}

}  // namespace

void build_polar_taps(int H, int W, int n_r, int n_theta, double dr, double cx, double cy, int32_t* xy, uint2* q) {
    (void)H;
    for (int j = 0; j < n_r; ++j) {
        const double r = j * dr;
        for (int k = 0; k < n_theta; ++k) {
            const double th = 2.0 * kPi * k / n_theta;
            const double x = cx + r * cos(th), y = cy + r * sin(th);
            double x0 = floor(x), y0 = floor(y);
            double fx = x - x0, fy = y - y0;
            int64_t qx = llround(fx * 8388608.0), qy = llround(fy * 8388608.0);
            if (qx >= 8388608) { qx = 0; x0 += 1.0; }          // fraction rounds up to the next tap
            if (qy >= 8388608) { qy = 0; y0 += 1.0; }
            // taps outside [-2, size + 1] contribute zero either way; clamp into int16
            if (x0 < -2.0 || x0 > (double)W + 1.0) { x0 = std::min(std::max(x0, -2.0), (double)W + 1.0); qx = 0; }
            if (y0 < -2.0 || y0 > (double)H + 1.0) { y0 = std::min(std::max(y0, -2.0), (double)H + 1.0); qy = 0; }
            const size_t i = (size_t)j * n_theta + k;
            xy[i] = (int32_t)((uint32_t)(uint16_t)(int16_t)(int)x0 | ((uint32_t)(int16_t)(int)y0 << 16));
            q[i] = make_uint2((uint32_t)qx, (uint32_t)qy);
        }
    }
}

cudaError_t launch_polar(const void* frames, int dtype, int64_t n, int H, int W,
                         const PolarTable& tab, double gamma, double subtract, int n_r,
                         int n_theta, float* polar, float* pnorm, float* radial,
                         cudaStream_t st, const uint8_t* keep_row, const float2* centres, const float4* offsets,
                         const uint8_t* pixel_mask, double threshold) {
    if (n <= 0) return cudaSuccess;
    const int mode = gamma == 0.5 ? 0 : (gamma == 1.0 ? 1 : 2);
    // threshold: pixels v < threshold read as 0.  As a float t with v < t exactly when
    // v < threshold for every float v (t rounded up when the float is below threshold).
    float thr = -INFINITY;
    if (threshold > 0.0) {
        thr = (float)threshold;
        if ((double)thr < threshold) thr = nextafterf(thr, INFINITY);
    }
    const float2 g = make_float2((float)gamma, thr);
    if (dtype == TM_DTYPE_U16)
        return launch_typed<uint16_t>((const uint16_t*)frames, n, H, W, tab, mode, g, (float)subtract, n_r,
                                      n_theta, polar, pnorm, radial, st, keep_row, centres, offsets, pixel_mask);
    return launch_typed<float>((const float*)frames, n, H, W, tab, mode, g, (float)subtract, n_r, n_theta,
                               polar, pnorm, radial, st, keep_row, centres, offsets, pixel_mask);
}

}  // namespace tmgb
