// Stage 1: gamma / constant subtraction of the raw frame and bilinear resampling onto
// the polar grid about the direct beam (arXiv 2111.07347, Section 2.2, Fig. 2 (a)-(c);
// the gamma and subtraction of Sections 2.2 and 4.3).  By-products for later stages:
// the image norm sqrt(sum P'^2) of Eq. 1 and the azimuthal sums R_P[j] used by the
// pre-filter (Section 2.2, Fig. 3).
//
// One CTA per pattern (grid-stride over patterns).  The CTA's threads form R row groups of
// `cols` threads (a multiple of 32).  A warp samples a patch of 8 consecutive angles by 4
// consecutive rows (lane = 8 sub + kl): the warp-in-group wg, lane (sub, kl) of group g owns
// columns 8 wg + kl, 8 wg + kl + cols / 4, ... of rows sub + 4 g, sub + 4 (g + R), ..., four
// rows at a time, so four samples are in flight per thread and a store writes 32-byte runs.
//
// Staged form (frame fits in shared memory): the CTA first copies the frame into shared
// memory with 16-byte global loads (its next frame having been prefetched into L2 while the
// previous one was sampled).  The taps of a warp's patch cover a small 2-D region of
// the frame; rows are padded to 9 (mod 32) 32-bit words, which puts such regions' words in
// distinct banks more often than a plain odd pitch (whose banks repeat every two pixels along
// one diagonal direction): 1.5 instead of 2.7 shared-memory wavefronts per tap load on a
// 256 x 256 frame.  Otherwise the taps are read from global memory.
//
// Tap positions come from fixed-point ray stepping: along the ray of angle theta_k the
// sample of row j sits at x = cx + j dr cos(theta_k), kept as a signed 32.32 fixed-point
// integer X = CX + j DX, with DX = round(dr cos(theta_k) 2^32) built on the host in double
// precision (one pair per angle, 16 B, instead of a table entry per sample).  The integer
// part of X is the tap column x0; the top 23 bits of the fraction (rounded, the carry
// going into x0) give the bilinear weight exactly: with y = 1 + q 2^-23 (formed by bit
// assembly), fx = y - 1 is exact, and the sample is formed as interpolations a + fx (b - a).
// The position error is at most (j + 1) 2^-33 px before the rounding to 23 bits, each weight
// within 2^-24 (+ that) of the double-precision value.  A per-pattern centre enters only
// through CX, converted exactly from its float value.  A sample whose four taps are all
// inside the frame takes a fast path with one bounds test; edge samples test each tap (zero
// outside).
// For u16 frames the gamma of the pixel values below 4096 (all of them at the counts of an
// electron diffraction pattern) is tabulated once per CTA in shared memory, g(v) - c from
// the same correctly rounded sqrtf / powf, so a tap is one table read; larger values are
// computed directly.  The staging notes whether any pixel of the frame is that large, and
// frames without one take a path with no per-tap range test.
// The norm's squares are added four at a time (one sample per row of a batch), then into the
// thread's compensated (Kahan) sum.
// Reductions run in a fixed order: the result does not depend on the grid size or on
// other patterns of the batch.
#include <math.h>

#include <algorithm>

#include "tm_device.h"
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

// Weight f = q 2^-23 from the 23-bit fixed-point fraction q (q < 2^23), exact.
__device__ __forceinline__ float fixed_weight(uint32_t q) {
    return __uint_as_float(0x3F800000u | q) - 1.0f;          // (1 + q 2^-23) - 1
}

// a + f (b - a): the interpolation between two taps.
__device__ __forceinline__ float lerp(float a, float b, float f) { return fmaf(f, b - a, a); }

// Bilinear sample of the gamma-corrected, subtracted frame at (x0 + fx, y0 + fy); the frame
// has row pitch `pitch` elements; taps outside [0, W) x [0, H) contribute zero.
// CHECK = false: the caller knows that all four taps lie inside the frame.  LUT_ONLY: every
// pixel of the frame is below the gamma table's end.
template <typename T, int MODE, bool SMEM, bool LUT_ONLY, bool CHECK>
__device__ __forceinline__ float bilinear(const T* frame, int pitch, int H, int W, int x0, int y0, float fx,
                                          float fy, const float* lut, float2 g, float sub, const uint8_t* pmask) {
    if (!CHECK || ((unsigned)x0 < (unsigned)(W - 1) && (unsigned)y0 < (unsigned)(H - 1))) {
        const T* p = frame + y0 * pitch + x0;
        const T a = load_px_masked<SMEM>(p, frame, pmask), b = load_px_masked<SMEM>(p + 1, frame, pmask);
        const T c = load_px_masked<SMEM>(p + pitch, frame, pmask), d = load_px_masked<SMEM>(p + pitch + 1, frame, pmask);
        float v00, v10, v01, v11;
        if (LUT_ONLY || all_in_lut(a, b, c, d)) {
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
        return lerp(lerp(v00, v10, fx), lerp(v01, v11, fx), fy);
    }
    float v[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const int x = x0 + (t & 1), y = y0 + (t >> 1);
        v[t] = 0.0f;
        if ((unsigned)x < (unsigned)W && (unsigned)y < (unsigned)H) {
            const T raw = load_px_masked<SMEM>(frame + y * pitch + x, frame, pmask);
            v[t] = LUT_ONLY ? lut[(int)raw] : tap_value<MODE>(raw, lut, g, sub);
        }
    }
    return lerp(lerp(v[0], v[1], fx), lerp(v[2], v[3], fx), fy);
}

// Sum of a[u] over the 8 lanes of each group of eight (lanes 8 sub .. 8 sub + 7) for four
// values u at once (4 shuffles instead of 12): afterwards the even lanes kl of a group hold
// the total of u = 2 ((kl >> 2) & 1) + ((kl >> 1) & 1).  Fixed order: deterministic.
__device__ __forceinline__ float group8_sum4(const float a[4], int lane) {
    const bool h4 = lane & 4;
    const float b0 = (h4 ? a[2] : a[0]) + __shfl_xor_sync(0xffffffffu, h4 ? a[0] : a[2], 4);
    const float b1 = (h4 ? a[3] : a[1]) + __shfl_xor_sync(0xffffffffu, h4 ? a[1] : a[3], 4);
    const bool h2 = lane & 2;
    float c = (h2 ? b1 : b0) + __shfl_xor_sync(0xffffffffu, h2 ? b0 : b1, 2);
    c += __shfl_xor_sync(0xffffffffu, c, 1);
    return c;
}

constexpr long long kRound = 1ll << 8;     // half of the last kept fraction bit (2^-24 of a pixel)

// One polar sample at the fixed-point position (X, Y) (32.32, rounding bias included).
template <typename T, int MODE, bool STAGED, bool LUT_ONLY, bool CHECK>
__device__ __forceinline__ float sample_at(const T* frame, int pitch, int H, int W, long long X, long long Y,
                                          const float* lut, float2 g, float sub, const uint8_t* pmask) {
    return bilinear<T, MODE, STAGED, LUT_ONLY, CHECK>(frame, pitch, H, W, (int)(X >> 32), (int)(Y >> 32),
                                                     fixed_weight((uint32_t)X >> 9), fixed_weight((uint32_t)Y >> 9),
                                                     lut, g, sub, pmask);
}

// Whether the four taps of a sample at fixed-point (X, Y) lie inside the frame.
__device__ __forceinline__ bool taps_inside(long long X, long long Y, int H, int W) {
    return (unsigned)(int)(X >> 32) < (unsigned)(W - 1) && (unsigned)(int)(Y >> 32) < (unsigned)(H - 1);
}

constexpr int kMaxThreads = 768;            // 80 registers per thread at one CTA per SM

// One column of the thread's rows (batches of four), from the fixed-point position (X, Y) of
// its first row row0 and the step (SX, SY) to its next row (rows row0, row0 + rstep, ...).
// my_rows: the lane's rows; wrows: the most rows of a lane of the warp (the loop bound, so
// the loop is warp-uniform).  keepm: bit i set when the lane's i-th row is stored (rows past
// 64 read keep_row).  CHECK = false when the whole column lies inside the frame.
template <typename T, int MODE, bool STAGED, bool LUT_ONLY, bool CHECK>
__device__ __forceinline__ void polar_column(const T* frame, int pf, int H, int W, long long X, long long Y,
                                             long long SX, long long SY, int k, bool active, int my_rows, int wrows,
                                             int row0, int rstep, int n_theta, int lane, int warp, int nw, int kk,
                                             unsigned long long keepm, const uint8_t* __restrict__ keep_row,
                                             const uint8_t* pmask, const float* lut, float2 g, float sub,
                                             float* __restrict__ out, float* part, float& s2, float& c2) {
    for (int b = 0; b < wrows; b += 4) {                                // warp-uniform
        const int nu = my_rows - b;                                     // this lane's rows left (may be <= 0)
        const int j0 = row0 + rstep * b;
        float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        if (active && nu > 0) {
            unsigned kb;                                                // rows of the batch that are stored
            if (b + 4 <= 64) {
                kb = (unsigned)(keepm >> b) & 15u;
            } else {
                kb = 0u;
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (u < nu && (!keep_row || keep_row[j0 + rstep * u])) kb |= 1u << u;
            }
            float v[4];
            // stores of the kept rows, the row sums' inputs, and the batch's squares (zeros past
            // the lane's rows) added to the norm in one compensated step
            auto tail = [&]() {
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if ((kb >> u) & 1u) out[(size_t)(j0 + rstep * u) * n_theta + k] = v[u];
                    acc[u] = v[u];
                }
                const float q = fmaf(v[3], v[3], fmaf(v[2], v[2], fmaf(v[1], v[1], v[0] * v[0])));
                const float y = q - c2;
                const float t = s2 + y;
                c2 = (t - s2) - y;
                s2 = t;
            };
            if (nu >= 4) {
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    v[u] = sample_at<T, MODE, STAGED, LUT_ONLY, CHECK>(frame, pf, H, W, X, Y, lut, g, sub, pmask);
                    X += SX;
                    Y += SY;
                }
                tail();
            } else {
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    v[u] = u < nu ? sample_at<T, MODE, STAGED, LUT_ONLY, CHECK>(frame, pf, H, W, X, Y, lut, g, sub,
                                                                               pmask)
                                  : 0.0f;
                    X += SX;
                    Y += SY;
                }
                tail();
            }
        }
        const float r = group8_sum4(acc, lane);
        const int kl = lane & 7;
        const int u = ((kl >> 2) & 1) * 2 + ((kl >> 1) & 1);          // the value this lane's sum is of
        if ((kl & 1) == 0 && u < nu) {
            float* dst = part + (j0 + rstep * u) * nw + warp;
            *dst = kk ? *dst + r : r;
        }
    }
}

// The polar rows of one pattern: the lane takes columns k0, k0 + kstep, ... of rows row0,
// row0 + rstep, ..., four rows at a time.  Stores the kept rows, adds P'^2 to the thread's
// Kahan sum and leaves each row's partial sums per warp in part[row][warp].
template <typename T, int MODE, bool STAGED, bool LUT_ONLY>
__device__ __forceinline__ void polar_rows(const T* frame, int pf, int H, int W, long long cxb, long long cyb,
                                           const longlong2* __restrict__ rays, int n_r, int n_theta, int row0,
                                           int rstep, int wrows, int kstep, int k0, int lane, int warp, int nw,
                                           unsigned long long keepm, const uint8_t* __restrict__ keep_row,
                                           const uint8_t* pmask, const float* lut, float2 g, float sub,
                                           float* __restrict__ out, float* part, float& s2, float& c2) {
    const int my_rows = row0 < n_r ? (n_r - row0 + rstep - 1) / rstep : 0;
    for (int kk = 0; kk < n_theta; kk += kstep) {                       // block-uniform
        const int k = kk + k0;
        const bool active = k < n_theta;
        long long X = cxb, Y = cyb, SX = 0, SY = 0;
        bool inside = true;
        if (active) {
            const longlong2 d = __ldg(rays + k);
            X += (long long)row0 * d.x;
            Y += (long long)row0 * d.y;
            SX = (long long)rstep * d.x;
            SY = (long long)rstep * d.y;
            // the column is a segment, so its samples are inside when both ends are
            const long long last = my_rows > 0 ? (long long)(my_rows - 1) : 0;
            inside = taps_inside(X, Y, H, W) && taps_inside(X + last * SX, Y + last * SY, H, W);
        }
        if (__all_sync(0xffffffffu, inside))
            polar_column<T, MODE, STAGED, LUT_ONLY, false>(frame, pf, H, W, X, Y, SX, SY, k, active, my_rows, wrows,
                                                           row0, rstep, n_theta, lane, warp, nw, kk, keepm, keep_row,
                                                           pmask, lut, g, sub, out, part, s2, c2);
        else
            polar_column<T, MODE, STAGED, LUT_ONLY, true>(frame, pf, H, W, X, Y, SX, SY, k, active, my_rows, wrows,
                                                          row0, rstep, n_theta, lane, warp, nw, kk, keepm, keep_row,
                                                          pmask, lut, g, sub, out, part, s2, c2);
    }
}

// Copies one frame into shared memory (row pitch `pitch` elements), masked pixels as 0, and
// returns the OR of the staged 32-bit words (u16: whether a pixel reaches the gamma table's
// end).
template <typename T>
__device__ __forceinline__ uint32_t stage_frame(const T* __restrict__ gframe, T* sF, int H, int W, int pitch,
                                                const uint8_t* __restrict__ pmask) {
    uint32_t hi_bits = 0;
    const bool vec = (((uintptr_t)gframe) & 15) == 0 && (W * sizeof(T)) % 16 == 0;
    if (vec) {
        const int vr = (int)(W * sizeof(T) / 16);           // 16-byte vectors per row
        const int nv = H * vr;
        const uint4* src = (const uint4*)gframe;
        constexpr int B = 4;                                // loads in flight per thread (the frame is in L2)
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
                    hi_bits |= v[b].x | v[b].y | v[b].z | v[b].w;
                }
            }
        }
    } else {
        for (int e = threadIdx.x; e < H * W; e += blockDim.x) {
            const int y = e / W;
            const T v = (!pmask || pmask[e]) ? gframe[e] : T(0);
            sF[(size_t)y * pitch + (e - y * W)] = v;
            if (sizeof(T) == 2) hi_bits |= (uint32_t)v;
        }
    }
    return hi_bits;
}

// ---------------------------------------------------------------- bulk (TMA) staging
// Copies one frame into shared memory with the bulk-copy engine (one cp.async.bulk per row,
// rows `pitch` elements apart, every row start and length a multiple of 16 bytes), completing
// on the mbarrier `bar` (phase `parity`), then returns the OR of the staged words as
// stage_frame does.  False (uniformly over the CTA) when the wait ran out.
template <typename T>
__device__ __forceinline__ bool stage_frame_bulk(const T* __restrict__ gframe, T* sF, int H, int W, int pitch,
                                                 uint64_t* bar, uint32_t parity, uint32_t& hi_bits) {
    const uint32_t row_bytes = (uint32_t)(W * sizeof(T));
    fence_proxy_async_smem();                            // earlier reads of sF before the copies' writes
    if (threadIdx.x == 0) mbar_arrive_expect_tx(bar, row_bytes * (uint32_t)H);
    for (int y = threadIdx.x; y < H; y += blockDim.x)
        bulk_g2s(sF + (size_t)y * pitch, gframe + (size_t)y * W, row_bytes, bar);
    const bool ok = mbar_wait_bounded(bar, parity);
    if (__syncthreads_or(!ok)) return false;
    hi_bits = 0;
    const int vr = (int)(row_bytes / 16);
    for (int i = threadIdx.x; i < H * vr; i += blockDim.x) {
        const int y = i / vr, xv = i - y * vr;
        const uint4 v = *(const uint4*)((const char*)(sF + (size_t)y * pitch) + 16 * xv);
        hi_bits |= v.x | v.y | v.z | v.w;
    }
    return true;
}

template <typename T, int MODE, bool STAGED>
__global__ void __launch_bounds__(kMaxThreads, 1)
polar_kernel(const T* __restrict__ frames, int64_t n, int H, int W, int pitch, const longlong2* __restrict__ rays,
             long long cxb, long long cyb, float2 g, float sub, int n_r, int n_theta, int R,
             const uint8_t* __restrict__ keep_row, const uint8_t* __restrict__ pmask, float* __restrict__ polar,
             float* __restrict__ pnorm, float* __restrict__ radial, const float2* __restrict__ centres, int bulk,
             unsigned* __restrict__ err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int cols = blockDim.x / R;                     // threads per row group (multiple of 32)
    const int grp = threadIdx.x / cols, t_in = threadIdx.x - grp * cols;
    const int nw = blockDim.x >> 5;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // the warp's patch: 8 angles (lane & 7) by 4 rows (lane >> 3)
    const int k0 = 8 * (t_in >> 5) + (lane & 7), kstep = cols >> 2;
    const int row0 = (lane >> 3) + 4 * grp, rstep = 4 * R;
    const int wrows = 4 * grp < n_r ? (n_r - 4 * grp + rstep - 1) / rstep : 0;   // lane sub = 0: the most
    const size_t fbytes = STAGED ? (size_t)H * pitch * sizeof(T) : 0;
    constexpr bool kHasLut = sizeof(T) == 2;
    // rows of this thread that are stored (its first 64 rows; later ones read keep_row)
    unsigned long long keepm = 0ull;
    if (row0 < n_r) {
        const int my_rows = (n_r - row0 + rstep - 1) / rstep;
        for (int i = 0; i < my_rows && i < 64; ++i)
            if (!keep_row || keep_row[row0 + rstep * i]) keepm |= 1ull << i;
    }
    // the gamma table first (offset 0), so that a staged table offset addresses it directly
    T* sF = (T*)smem_raw;
    float* lut = (float*)(smem_raw + ((fbytes + 15) & ~(size_t)15));   // [kLut] for u16 frames
    float* part = lut + (kHasLut ? kLut : 0);                           // [n_r][nw]
    float* red = part + (size_t)n_r * nw;                               // [blockDim]
    uint64_t* bar = (uint64_t*)(((uintptr_t)(red + blockDim.x) + 7) & ~(uintptr_t)7);   // bulk staging
    if (STAGED && bulk && threadIdx.x == 0) mbar_init1(bar);
    uint32_t staged = 0;                                                // frames staged by bulk copies
    if (kHasLut) {
        for (int i = threadIdx.x; i < kLut; i += blockDim.x) {
            const float f = (float)i;
            lut[i] = gamma_of<MODE>(f < g.y ? 0.0f : f, g.x) - sub;
        }
        __syncthreads();
    }

    for (int64_t p = blockIdx.x; p < n; p += gridDim.x) {
        const T* gframe = frames + (size_t)p * H * W;
        const T* frame = gframe;
        bool big = true;                                 // some pixel may lie beyond the gamma table
        if (STAGED) {
            __syncthreads();                             // previous pattern's reads are done
            uint32_t hi_bits = 0;
            if (bulk) {
                if (!stage_frame_bulk<T>(gframe, sF, H, W, pitch, bar, staged & 1u, hi_bits)) {
                    // the copy did not land in time: report it, let it finish (bounded), stop
                    if (threadIdx.x == 0) {
                        atomicOr(err, 2u);
                        mbar_wait_bounded(bar, staged & 1u);
                    }
                    __syncthreads();
                    return;
                }
                ++staged;
            } else {
                hi_bits = stage_frame<T>(gframe, sF, H, W, pitch, pmask);
            }
            // u16 words: a pixel >= kLut sets a bit of 0xF000 in its half
            big = __syncthreads_or(kHasLut ? (hi_bits & 0xF000F000u) != 0 : 1) != 0;
            frame = sF;
            // bring the CTA's next frame into L2 while this one is sampled, so that its staging
            // reads L2 rather than HBM (one 128-byte line per thread and step)
            const int64_t pnext = p + gridDim.x;
            if (pnext < n) {
                const char* nf = reinterpret_cast<const char*>(frames + (size_t)pnext * H * W);
                const size_t nbytes = (size_t)H * W * sizeof(T);
                for (size_t off = (size_t)threadIdx.x * 128; off < nbytes; off += (size_t)blockDim.x * 128)
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(nf + off));
            }
        }
        float* out = polar + (size_t)p * n_r * n_theta;
        long long cx = cxb, cy = cyb;
        if (centres) {                                   // exact: c 2^32 is an integer-valued float
            const float2 c = __ldg(centres + p);
            cx = __float2ll_rn(c.x * 4294967296.0f) + kRound;
            cy = __float2ll_rn(c.y * 4294967296.0f) + kRound;
        }
        const int pf = STAGED ? pitch : W;
        float s2 = 0.0f, c2 = 0.0f;                      // Kahan sum of P'^2 for this thread
        if (kHasLut && STAGED && !big)
            polar_rows<T, MODE, STAGED, true>(frame, pf, H, W, cx, cy, rays, n_r, n_theta, row0, rstep, wrows, kstep,
                                              k0, lane, warp, nw, keepm, keep_row, pmask, lut, g, sub, out, part, s2,
                                              c2);
        else
            polar_rows<T, MODE, STAGED, false>(frame, pf, H, W, cx, cy, rays, n_r, n_theta, row0, rstep, wrows,
                                               kstep, k0, lane, warp, nw, keepm, keep_row, pmask, lut, g, sub, out,
                                               part, s2, c2);
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
            // row j's partials come from the warps of group (j / 4) % R only
            const int wpg = cols >> 5;
            for (int j = threadIdx.x; j < n_r; j += blockDim.x) {
                const int g0 = (j >> 2) % R;
                float s = 0.0f;
                for (int w = 0; w < wpg; ++w) s += part[j * nw + g0 * wpg + w];
                radial[(size_t)p * n_r + j] = s;
            }
        }
        if (!STAGED) __syncthreads();                    // part / red reused by the next pattern
    }
}

template <typename T, int MODE, bool STAGED>
cudaError_t launch_one(const T* frames, int64_t n, int H, int W, int pitch, const longlong2* rays, long long cxb,
                       long long cyb, float2 g, float sub, int n_r, int n_theta, int R, int threads, size_t smem,
                       const uint8_t* keep_row, const uint8_t* pmask, float* polar, float* pnorm, float* radial,
                       const float2* centres, int bulk, unsigned* err, cudaStream_t st) {
    auto kern = polar_kernel<T, MODE, STAGED>;
    int per_sm = 1;
    const cudaError_t e = kernel_occupancy((const void*)kern, threads, smem, &per_sm);
    if (e != cudaSuccess) return e;
    int64_t grid = (int64_t)device_sms() * (per_sm > 0 ? per_sm : 1);
    if (grid > n) grid = n;
    kern<<<(int)grid, threads, smem, st>>>(frames, n, H, W, pitch, rays, cxb, cyb, g, sub, n_r, n_theta, R, keep_row,
                                           pmask, polar, pnorm, radial, centres, bulk, err);
    return cudaGetLastError();
}

template <typename T, bool STAGED>
cudaError_t launch_mode(int mode, const T* frames, int64_t n, int H, int W, int pitch, const longlong2* rays,
                        long long cxb, long long cyb, float2 g, float sub, int n_r, int n_theta, int R, int threads,
                        size_t smem, const uint8_t* keep_row, const uint8_t* pmask, float* polar, float* pnorm,
                        float* radial, const float2* centres, int bulk, unsigned* err, cudaStream_t st) {
    auto f = mode == 0 ? launch_one<T, 0, STAGED> : (mode == 1 ? launch_one<T, 1, STAGED> : launch_one<T, 2, STAGED>);
    return f(frames, n, H, W, pitch, rays, cxb, cyb, g, sub, n_r, n_theta, R, threads, smem, keep_row, pmask, polar,
             pnorm, radial, centres, bulk, err, st);
}

template <typename T>
cudaError_t launch_typed(const T* frames, int64_t n, int H, int W, const longlong2* rays, long long cxb, long long cyb,
                         int mode, float2 g, float sub, int n_r, int n_theta, float* polar, float* pnorm, float* radial,
                         cudaStream_t st, const uint8_t* keep_row, const float2* centres, const uint8_t* pmask,
                         unsigned* err) {
    const int cols = ((n_theta + 31) / 32) * 32;
    if (cols <= kMaxThreads) {
        // staged: rows padded to 4 (mod 32) 32-bit words when the frame's rows are whole
        // 16-byte units (then the rows are copied by the bulk-copy engine), else to 9 (mod 32);
        // both spread a warp's taps over the banks alike (1.5 shared-memory wavefronts per tap
        // load on a 256 x 256 frame, replayed on the CPU over every warp's patch); an odd pitch
        // if neither fits
        const int words = (int)((W * sizeof(T) + 3) / 4);
        const int R = std::max(1, std::min(4, kMaxThreads / cols));
        const int threads = R * cols;
        const int nw = threads / 32;
        const size_t lut = sizeof(T) == 2 ? kLut * sizeof(float) : 0;
        auto smem_of = [&](int pw) {
            return (((size_t)H * pw * 4 + 15) & ~(size_t)15) + lut + ((size_t)n_r * nw + threads) * sizeof(float) + 16;
        };
        const bool rows16 = (W * sizeof(T)) % 16 == 0 && ((uintptr_t)frames & 15) == 0;
        int pw = words + (((rows16 ? 4 : 9) - words % 32) + 32) % 32;
        if (smem_of(pw) > 200 * 1024) pw = words | 1;
        const int pitch = (int)(pw * 4 / sizeof(T));
        const size_t smem = smem_of(pw);
        const int bulk = rows16 && (pw % 4) == 0 && !pmask && err != nullptr;
        if (smem <= 200 * 1024)
            return launch_mode<T, true>(mode, frames, n, H, W, pitch, rays, cxb, cyb, g, sub, n_r, n_theta, R, threads,
                                        smem, keep_row, pmask, polar, pnorm, radial, centres, bulk, err, st);
    }
    const int threads = cols < kMaxThreads ? cols : kMaxThreads;
    const size_t smem = (sizeof(T) == 2 ? kLut * sizeof(float) : 0) + ((size_t)n_r * (threads / 32) + threads) * sizeof(float);
    if (smem > 200 * 1024) return cudaErrorInvalidValue;
    return launch_mode<T, false>(mode, frames, n, H, W, W, rays, cxb, cyb, g, sub, n_r, n_theta, 1, threads, smem,
                                 keep_row, pmask, polar, pnorm, radial, centres, 0, err, st);
}

}  // namespace

void build_polar_rays(int n_theta, double dr, longlong2* rays) {
    for (int k = 0; k < n_theta; ++k) {
        const double th = 2.0 * kPi * k / n_theta;
        rays[k].x = llround(dr * cos(th) * 4294967296.0);
        rays[k].y = llround(dr * sin(th) * 4294967296.0);
    }
}

cudaError_t launch_polar(const void* frames, int dtype, int64_t n, int H, int W, const longlong2* rays, double cx,
                         double cy, double gamma, double subtract, int n_r, int n_theta, float* polar, float* pnorm,
                         float* radial, cudaStream_t st, const uint8_t* keep_row, const float2* centres,
                         const uint8_t* pixel_mask, double threshold, unsigned* err) {
    if (n <= 0) return cudaSuccess;
    // positions stay within 2^31 px in the 32.32 format (the caller bounds n_r dr as well)
    if (!(fabs(cx) < 1073741824.0 && fabs(cy) < 1073741824.0)) return cudaErrorInvalidValue;
    const int mode = gamma == 0.5 ? 0 : (gamma == 1.0 ? 1 : 2);
    // threshold: pixels v < threshold read as 0.  As a float t with v < t exactly when
    // v < threshold for every float v (t rounded up when the float is below threshold).
    float thr = -INFINITY;
    if (threshold > 0.0) {
        thr = (float)threshold;
        if ((double)thr < threshold) thr = nextafterf(thr, INFINITY);
    }
    const float2 g = make_float2((float)gamma, thr);
    const long long cxb = llround(cx * 4294967296.0) + kRound, cyb = llround(cy * 4294967296.0) + kRound;
    if (dtype == TM_DTYPE_U16)
        return launch_typed<uint16_t>((const uint16_t*)frames, n, H, W, rays, cxb, cyb, mode, g, (float)subtract, n_r,
                                      n_theta, polar, pnorm, radial, st, keep_row, centres, pixel_mask, err);
    return launch_typed<float>((const float*)frames, n, H, W, rays, cxb, cyb, mode, g, (float)subtract, n_r, n_theta,
                               polar, pnorm, radial, st, keep_row, centres, pixel_mask, err);
}

}  // namespace tmgb
