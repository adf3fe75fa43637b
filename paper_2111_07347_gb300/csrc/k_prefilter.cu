// Stage 2: the azimuthally integrated pre-filter (arXiv 2111.07347, Section 2.2 and
// Fig. 3): the polar image and every template are integrated over the azimuth, the
// integrated image is correlated with the integrated library (one matrix-vector product
// per pattern) and only the best-correlated templates go on to full matching.
//
//   score[p][k] = R_P[p] . R_T[k] / (|R_P[p]| |R_T[k]|)        (0 if a norm is 0)
//   keep the ceil(f K) largest per pattern, ties to the lower k  -> bit mask [p][K/32]
//
// R_T[k] is zero outside the library's few distinct spot radii (9 rows of 128 for FCC), so
// the product runs over those rows only, in ascending order: the same FP32 sums as the
// full-length product, whose other terms add exact zeros.  One CTA takes PB patterns: it
// forms their scores in shared memory (the library's rows are read once for PB patterns)
// and selects from there, so the scores need not reach global memory.  The selection is
// exact: a radix select over order-preserving integer keys whose digits (up to 11 bits)
// start at the highest bit in which the pattern's keys differ (cosine scores share their sign
// and most exponent bits; the keys' range comes with the scores).  One warp finds each digit's
// bin by a two-level scan of the histogram; the passes stop once every key of the boundary's
// bin is kept or the bin holds at most 256 keys, which one warp then finishes bit by bit in
// registers over the bits in which they differ.
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

__device__ __forceinline__ uint32_t order_key(float x) {
    const uint32_t u = __float_as_uint(x);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);     // larger float -> larger key
}

constexpr int SEL_THREADS = 512;
constexpr int SEL_BINS = 2048;                             // digits of at most 11 bits
constexpr int SEL_CAND = 256;                              // candidates finished by one warp
constexpr int MAX_PB = 2;

struct SelShared {
    uint32_t kmin[MAX_PB], kmax[MAX_PB];                    // range of each pattern's keys
    uint32_t prefix, remaining, bincount, ncand, T, need, neq;
    uint32_t wsum[SEL_THREADS / 32];
};

// Running min / max of a thread's keys into sh (lane 0 of each warp after a warp reduce).
__device__ __forceinline__ void range_publish(uint32_t lo, uint32_t hi, uint32_t* kmin, uint32_t* kmax) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(kmin, lo);
        atomicMax(kmax, hi);
    }
}

// Warp 0: the bin of hist[0, nb) (nb a power of two <= 2048) where the count taken from the
// top bin down first reaches rem (>= 1, <= the total).  Level 1: lane l sums its c = nb / 32
// bins and a suffix scan over lanes finds the lane whose run holds the bin; level 2: the lanes
// split that run (two bins each, from the top) and a prefix scan finds the bin.  Writes the
// bin's prefix bits, what is left to take inside it and its count to sh.
__device__ __forceinline__ void find_bin(const uint32_t* hist, uint32_t nb, uint32_t rem, uint32_t prefix, int shift,
                                         SelShared& sh, int lane) {
    const uint32_t c = nb >= 32u ? nb >> 5 : 1u;
    const uint32_t b0 = (uint32_t)lane * c;
    uint32_t t = 0u;
    if (b0 < nb) {
        if (c >= 4u) {
            for (uint32_t i = 0; i < c; i += 4) {
                const uint4 a = *reinterpret_cast<const uint4*>(hist + b0 + i);
                t += a.x + a.y + a.z + a.w;
            }
        } else {
            for (uint32_t i = 0; i < c; ++i) t += hist[b0 + i];
        }
    }
    uint32_t sfx = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_down_sync(0xffffffffu, sfx, o);
        if (lane + o < 32) sfx += v;
    }
    const unsigned hit = __ballot_sync(0xffffffffu, b0 < nb && sfx >= rem && sfx - t < rem);
    const int L = hit ? __ffs(hit) - 1 : 0;                 // exactly one lane
    const uint32_t above = __shfl_sync(0xffffffffu, sfx - t, L);
    // level 2 over bins [L c, L c + c): lane i takes bins top - 2 i and top - 2 i - 1
    const int top = L * (int)c + (int)c - 1, bot = L * (int)c;
    const int hi_b = top - 2 * lane, lo_b = hi_b - 1;
    const uint32_t hh = hi_b >= bot ? hist[hi_b] : 0u;
    const uint32_t hl = lo_b >= bot ? hist[lo_b] : 0u;
    const uint32_t q = hh + hl;
    uint32_t inc = q;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += v;
    }
    const uint32_t exc = inc - q;
    if (hi_b >= bot && above + inc >= rem && above + exc < rem) {
        uint32_t cum = above + exc;
        int bin = hi_b;
        uint32_t cnt = hh;
        if (cum + hh < rem) {
            cum += hh;
            bin = lo_b;
            cnt = hl;
        }
        sh.prefix = prefix | ((uint32_t)bin << shift);
        sh.remaining = rem - cum;
        sh.bincount = cnt;
    }
}

// The `keep` largest of keys[0, K) (ties to the lower index) as bits of mrow[ceil(K/32)].
// [kmin, kmax] is the keys' range.  Called by the whole block with uniform arguments after a
// barrier that follows the last write of keys; ends with a barrier.
//   Block-wide histogram passes of up to 11 bits (starting at the highest bit in which the
//   keys differ) narrow the boundary to one bin; once that bin holds at most SEL_CAND keys
//   they are gathered and warp 0 finishes bit by bit with ballots over registers.  The
//   threshold T and the number `need` of keys equal to T that are kept then give the mask.
__device__ __forceinline__ void select_keep(const uint32_t* keys, int K, int keep, uint32_t kmin, uint32_t kmax,
                                            uint32_t* hist, uint32_t* cand, SelShared& sh,
                                            uint32_t* __restrict__ mrow) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int words = (K + 31) >> 5;
    if (keep <= 0 || keep >= K) {
        for (int w = tid; w < words; w += blockDim.x) {
            const int left = K - 32 * w;
            mrow[w] = keep <= 0 ? 0u : (left >= 32 ? 0xffffffffu : (1u << left) - 1u);
        }
        __syncthreads();
        return;
    }
    uint32_t T, need, neq;                                  // neq: keys equal to T (0: unknown)
    if (kmin == kmax) {
        T = kmin;                                           // all equal: the first `keep` indices
        need = (uint32_t)keep;
        neq = (uint32_t)K;
    } else {
        const int bits = 32 - __clz(kmin ^ kmax);           // the keys differ in bits [0, bits)
        uint32_t prefix = bits == 32 ? 0u : (kmin >> bits) << bits;
        uint32_t pmask = bits == 32 ? 0u : 0xffffffffu << bits;
        uint32_t rem = (uint32_t)keep;                      // still to take among the candidates
        int left = bits;
        uint32_t nbin = 0u;
        for (;;) {
            const int d = min(11, left);
            const int shift = left - d;
            const uint32_t nb = 1u << d, dm = nb - 1u;
            for (uint32_t i = tid; i < nb; i += blockDim.x) hist[i] = 0u;
            __syncthreads();
            for (int k = tid; k < K; k += blockDim.x) {
                const uint32_t x = keys[k];
                if ((x & pmask) == prefix) atomicAdd(&hist[(x >> shift) & dm], 1u);
            }
            __syncthreads();
            if (warp == 0) find_bin(hist, nb, rem, prefix, shift, sh, lane);
            __syncthreads();
            prefix = sh.prefix;
            rem = sh.remaining;
            nbin = sh.bincount;
            pmask |= dm << shift;
            left = shift;
            if (nbin == rem || left == 0 || nbin <= (uint32_t)SEL_CAND) break;
        }
        if (nbin == rem) {                                  // every key of the bin is kept
            T = prefix;
            need = 0xffffffffu;
            neq = 0u;
        } else if (left == 0) {                             // the bin is one key value
            T = prefix;
            need = rem;
            neq = nbin;
        } else {
            // gather the bin's keys (order does not matter) and finish in warp 0's registers
            if (tid == 0) sh.ncand = 0u;
            __syncthreads();
            for (int k0 = warp * 32; k0 < K; k0 += blockDim.x) {            // warp-uniform trip count
                const int k = k0 + lane;
                const uint32_t x = k < K ? keys[k] : 0u;
                const bool in = k < K && (x & pmask) == prefix;
                const unsigned b = __ballot_sync(0xffffffffu, in);
                if (b) {
                    uint32_t base = 0u;
                    if (lane == 0) base = atomicAdd(&sh.ncand, (uint32_t)__popc(b));
                    base = __shfl_sync(0xffffffffu, base, 0);
                    const uint32_t at = base + __popc(b & ((1u << lane) - 1u));
                    if (in && at < (uint32_t)SEL_CAND) cand[at] = x;
                }
            }
            __syncthreads();
            if (warp == 0) {
                const uint32_t nc = min(sh.ncand, (uint32_t)SEL_CAND);
                const int slots = (int)((nc + 31u) >> 5);   // registers in use per lane
                uint32_t r[SEL_CAND / 32];
                unsigned play = 0u;                         // bit i: r[i] still a candidate
                uint32_t vor = 0u, vand = 0xffffffffu;
#pragma unroll
                for (int i = 0; i < SEL_CAND / 32; ++i) {
                    const uint32_t idx = (uint32_t)(lane + 32 * i);
                    r[i] = idx < nc ? cand[idx] : 0u;
                    if (idx < nc) {
                        play |= 1u << i;
                        vor |= r[i];
                        vand &= r[i];
                    }
                }
                // bits in which every candidate agrees are taken as they are; the others are
                // decided from the highest down, keeping the side that holds the rem-th key
                vor = __reduce_or_sync(0xffffffffu, vor);
                vand = __reduce_and_sync(0xffffffffu, vand);
                const uint32_t low = (1u << left) - 1u;     // left <= 31 here
                const uint32_t diff = (vor ^ vand) & low;
                uint32_t tv = prefix | (vand & low & ~(diff ? (2u << (31 - __clz(diff))) - 1u : 0u));
                uint32_t rr = rem;
                for (int bit = diff ? 31 - __clz(diff) : -1; bit >= 0; --bit) {
                    unsigned with = 0u;
                    uint32_t c1 = 0u;
#pragma unroll
                    for (int i = 0; i < SEL_CAND / 32; ++i) {
                        if (i >= slots) break;
                        const bool one = ((play >> i) & 1u) && ((r[i] >> bit) & 1u);
                        if (one) with |= 1u << i;
                        c1 += __popc(__ballot_sync(0xffffffffu, one));
                    }
                    if (c1 >= rr) {
                        play = with;
                        tv |= 1u << bit;
                    } else {
                        rr -= c1;
                        play &= ~with;
                    }
                }
                uint32_t ne = 0u;
#pragma unroll
                for (int i = 0; i < SEL_CAND / 32; ++i) {
                    if (i >= slots) break;
                    ne += __popc(__ballot_sync(0xffffffffu, (play >> i) & 1u));
                }
                if (lane == 0) {
                    sh.T = tv;
                    sh.need = rr;
                    sh.neq = ne;
                }
            }
            __syncthreads();
            T = sh.T;
            need = sh.need;
            neq = sh.neq;
        }
    }
    const int per = (words + nw - 1) / nw;
    const int w0 = warp * per, w1 = min(words, w0 + per);
    if (need == 0xffffffffu || (neq != 0u && need >= neq)) {
        // every key equal to T is kept: kept = key >= T
        for (int w = w0; w < w1; ++w) {
            const int k = 32 * w + lane;
            const uint32_t word = __ballot_sync(0xffffffffu, k < K && keys[k] >= T);
            if (lane == 0) mrow[w] = word;
        }
        __syncthreads();
        return;
    }
    // kept = key > T, or key == T among the first `need` such keys in index order; each warp
    // writes a contiguous run of words
    uint32_t cnt = 0u;
    for (int w = w0; w < w1; ++w) {
        const int k = 32 * w + lane;
        cnt += __popc(__ballot_sync(0xffffffffu, k < K && keys[k] == T));
    }
    if (lane == 0) sh.wsum[warp] = cnt;
    __syncthreads();
    uint32_t before = 0u;
    for (int w = 0; w < warp; ++w) before += sh.wsum[w];
    for (int w = w0; w < w1; ++w) {
        const int k = 32 * w + lane;
        const uint32_t key = k < K ? keys[k] : 0u;
        const bool eq = k < K && key == T;
        const uint32_t eqb = __ballot_sync(0xffffffffu, eq);
        const uint32_t rank = before + __popc(eqb & ((1u << lane) - 1u));
        const bool kept = k < K && (key > T || (eq && rank < need));
        const uint32_t word = __ballot_sync(0xffffffffu, kept);
        if (lane == 0) mrow[w] = word;
        before += __popc(eqb);
    }
    __syncthreads();
}

// PB patterns per CTA: scores into shared memory as keys, then one selection per pattern.
// The library's radial sums are [K][n_pad] (n_pad = n_rad rounded up to 4, zero-padded), read
// as float4; the patterns' sums at the radii go to shared memory in the same padded form.
template <int PB>
__global__ void __launch_bounds__(SEL_THREADS)
prefilter_kernel(const float* __restrict__ radial, const float* __restrict__ rpn, int64_t n, int n_r,
                 RadialLib lib, int keep, uint32_t* __restrict__ mask, float* __restrict__ score) {
    extern __shared__ __align__(16) uint32_t keys[];        // rp [PB][n_pad], then keys [PB][K]
    __shared__ __align__(16) uint32_t hist[SEL_BINS];
    __shared__ uint32_t cand[SEL_CAND];
    __shared__ SelShared sh;
    const int K = lib.K, n_rad = lib.n_rad, n_pad = (n_rad + 3) & ~3, words = (K + 31) >> 5;
    float* rp = (float*)keys;
    uint32_t* kb = keys + PB * n_pad;
    for (int64_t p0 = (int64_t)blockIdx.x * PB; p0 < n; p0 += (int64_t)gridDim.x * PB) {
        if (threadIdx.x < PB) {
            sh.kmin[threadIdx.x] = 0xffffffffu;
            sh.kmax[threadIdx.x] = 0u;
        }
        for (int i = threadIdx.x; i < PB * n_pad; i += blockDim.x) {
            const int b = i / n_pad, j = i - b * n_pad;
            const int64_t p = p0 + b;
            rp[i] = (p < n && j < n_rad) ? __ldg(radial + (size_t)p * n_r + __ldg(lib.radii + j)) : 0.0f;
        }
        float np_[PB];
#pragma unroll
        for (int b = 0; b < PB; ++b) np_[b] = p0 + b < n ? __ldg(rpn + p0 + b) : 0.0f;
        __syncthreads();
        uint32_t lo[PB], hi[PB];
#pragma unroll
        for (int b = 0; b < PB; ++b) { lo[b] = 0xffffffffu; hi[b] = 0u; }
        for (int k = threadIdx.x; k < K; k += blockDim.x) {
            float acc[PB];
#pragma unroll
            for (int b = 0; b < PB; ++b) acc[b] = 0.0f;
            const float4* t4 = reinterpret_cast<const float4*>(lib.radc + (size_t)k * n_pad);
            for (int j4 = 0; j4 < n_pad; j4 += 4) {
                const float4 t = __ldg(t4 + (j4 >> 2));
#pragma unroll
                for (int b = 0; b < PB; ++b) {
                    const float4 r = *reinterpret_cast<const float4*>(rp + b * n_pad + j4);
                    // ascending radii; the padding adds exact zeros
                    acc[b] = fmaf(r.x, t.x, acc[b]);
                    acc[b] = fmaf(r.y, t.y, acc[b]);
                    acc[b] = fmaf(r.z, t.z, acc[b]);
                    acc[b] = fmaf(r.w, t.w, acc[b]);
                }
            }
            const float rk = __ldg(lib.rnorm + k);
#pragma unroll
            for (int b = 0; b < PB; ++b) {
                const float d = np_[b] * rk;
                const float sc = d > 0.0f ? __fdiv_rn(acc[b], d) : 0.0f;
                const uint32_t key = order_key(sc);
                kb[b * K + k] = key;
                lo[b] = min(lo[b], key);
                hi[b] = max(hi[b], key);
                if (score && p0 + b < n) score[(size_t)(p0 + b) * K + k] = sc;
            }
        }
#pragma unroll
        for (int b = 0; b < PB; ++b) range_publish(lo[b], hi[b], &sh.kmin[b], &sh.kmax[b]);
        __syncthreads();
#pragma unroll 1
        for (int b = 0; b < PB; ++b)
            if (p0 + b < n)
                select_keep(kb + (size_t)b * K, K, keep, sh.kmin[b], sh.kmax[b], hist, cand, sh,
                            mask + (size_t)(p0 + b) * words);
    }
}

// Selection alone, over scores already in global memory (the BF16 path's candidates).
__global__ void __launch_bounds__(SEL_THREADS)
prefilter_select_kernel(const float* __restrict__ score, int64_t n, int K, int keep,
                        uint32_t* __restrict__ mask) {
    extern __shared__ __align__(16) uint32_t keys[];        // [K]
    __shared__ __align__(16) uint32_t hist[SEL_BINS];
    __shared__ uint32_t cand[SEL_CAND];
    __shared__ SelShared sh;
    const int words = (K + 31) >> 5;
    for (int64_t p = blockIdx.x; p < n; p += gridDim.x) {
        if (threadIdx.x == 0) {
            sh.kmin[0] = 0xffffffffu;
            sh.kmax[0] = 0u;
        }
        __syncthreads();
        uint32_t lo = 0xffffffffu, hi = 0u;
        for (int k = threadIdx.x; k < K; k += blockDim.x) {
            const uint32_t key = order_key(__ldg(score + (size_t)p * K + k));
            keys[k] = key;
            lo = min(lo, key);
            hi = max(hi, key);
        }
        range_publish(lo, hi, &sh.kmin[0], &sh.kmax[0]);
        __syncthreads();
        select_keep(keys, K, keep, sh.kmin[0], sh.kmax[0], hist, cand, sh, mask + (size_t)p * words);
    }
}

cudaError_t allow_smem(const void* fn, size_t smem) { return kernel_occupancy(fn, SEL_THREADS, smem, nullptr); }

constexpr size_t kSelSmemMax = 200 * 1024;                  // dynamic part, beside hist and sh

}  // namespace

cudaError_t launch_radial_norm(const float* radial, int64_t n, int n_r, float* out, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int64_t blocks = (n + 7) / 8;
    radial_norm_kernel<<<(unsigned)blocks, 256, 0, st>>>(radial, n, n_r, out);
    return cudaGetLastError();
}

cudaError_t launch_prefilter(const float* radial, const float* radial_norm, int64_t n, int n_r, const RadialLib& lib,
                             int keep, uint32_t* mask, float* score, cudaStream_t st) {
    if (n <= 0 || lib.K <= 0) return cudaSuccess;
    const size_t per = (size_t)lib.K * 4 + (size_t)((lib.n_rad + 3) & ~3) * 4;
    // two patterns per CTA while their keys stay within 100 KB (three CTAs fit an SM)
    const int pb = 2 * per <= 100 * 1024 ? 2 : 1;
    const size_t smem = pb * per;
    if (smem > kSelSmemMax) return cudaErrorInvalidValue;
    const int64_t groups = (n + pb - 1) / pb;
    const unsigned grid = (unsigned)(groups < (1 << 20) ? groups : (1 << 20));
    cudaError_t e;
    if (pb == 2) {
        e = allow_smem((const void*)prefilter_kernel<2>, smem);
        if (e != cudaSuccess) return e;
        prefilter_kernel<2><<<grid, SEL_THREADS, smem, st>>>(radial, radial_norm, n, n_r, lib, keep, mask, score);
    } else {
        e = allow_smem((const void*)prefilter_kernel<1>, smem);
        if (e != cudaSuccess) return e;
        prefilter_kernel<1><<<grid, SEL_THREADS, smem, st>>>(radial, radial_norm, n, n_r, lib, keep, mask, score);
    }
    return cudaGetLastError();
}

cudaError_t launch_prefilter_select(const float* score, int64_t n, int K, int keep, uint32_t* mask,
                                    cudaStream_t st) {
    if (n <= 0 || K <= 0) return cudaSuccess;
    const size_t smem = (size_t)K * sizeof(uint32_t);
    if (smem > kSelSmemMax) return cudaErrorInvalidValue;
    cudaError_t e = allow_smem((const void*)prefilter_select_kernel, smem);
    if (e != cudaSuccess) return e;
    const int grid = (int)(n < 65536 ? n : 65536);
    prefilter_select_kernel<<<grid, SEL_THREADS, smem, st>>>(score, n, K, keep, mask);
    return cudaGetLastError();
}

}  // namespace tmgb
