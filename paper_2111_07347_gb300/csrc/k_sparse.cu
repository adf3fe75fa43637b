// Stage 3: the correlation index Q of Eq. 1 for every template at every azimuthal shift
// with wraparound, the best shift per template, and the fused top-N (arXiv 2111.07347,
// Section 2.2: templates are sparse, so the numerator is a sum over the template's spots;
// the denominators are precomputed; the template is slid along the azimuth with
// wraparound; the maximum Q and its angle are kept per template; the top N templates are
// returned).
//
// Design (GB300):
// * Shared memory holds only the polar rows the library uses (its distinct spot radii --
//   a few to a few tens of the 128 rows); column c of a row holds P'[c mod Nθ], so a warp
//   reading 32 or 64 consecutive shifts never splits at the wrap.  Three layouts, the
//   first that fits:
//   - dual: every row twice, the second copy shifted by one column, pitch Nθ + 64 NB2.  A spot
//     at column t reads float2 pairs at even columns of the copy (t & 1): lane L of 64-wide
//     shift block b takes shifts 64 b + 2 L + {0, 1} with ONE 8-byte load and two FMAs;
//   - wrap-free: one copy, pitch Nθ + 32 NB; block b of lane L reads column t + 32 b + L
//     (one 4-byte load and one FMA per shift);
//   - wrapped: one copy padded by 32 columns; a block past the wrap reads Nθ columns earlier
//     (a select per block).
//   The library stores, per spot, its shared-memory offset in the dual and wrap-free
//   layouts, so no address is decoded in the inner loop.
// * A persistent CTA takes patterns (or tiles of up to 4 patterns) from a global counter and
//   stages their rows (with bulk copies on an mbarrier when the layout allows), prefetching
//   into L2 the rows of the patterns one tile per CTA further on, which some CTA takes soon;
//   its warps take 32-template mask words from a shared counter.  One warp scores one template: the lanes hold all its
//   shifts in registers; the template's spots arrive in one lane-parallel load and are
//   broadcast by shuffles.  The bound is the shared-memory load path (4 bytes per
//   multiply-add).
// * The best shift is only resolved (lowest shift among equal maxima) when the template
//   can enter the warp's top-N, or when per-template results are requested.
// * Unmasked top-N (the common case), exact branch and bound: a first pass bounds every
//   template over three windows of shifts (from per-row window maxima of the pattern) and
//   stores the bound / (|P| |T|) rounded up to FP16; the templates are visited in spot-count
//   order (largest first) with each word's bound entries lane-adjacent, so the pass neither
//   diverges much nor scatters its loads.  A tile's patterns share this pass: each bound entry
//   is loaded once and applied to the tile's window tables.  Each warp scores first the
//   templates of highest bound among those it bounded (the seeds); the N-th best Q over all
//   warps' lists is a lower bound of the final N-th best, and every template whose stored
//   bound is below it is dropped without a look at its spots.  The others are gathered into
//   one list and scored, fewest spots first.
// Results do not depend on scheduling: a template's sum runs over its spots in CSR order
// and ranking uses the total order (Q desc, template asc).
#include <cuda_fp16.h>
#include <float.h>
#include <limits.h>

#include "tm_device.h"
#include "tm_internal.h"

namespace tmgb {

namespace {

// Shift blocks per template are rounded up to one of a few unrolled kernels.
__host__ __device__ constexpr int round_nb(int nb) {
    return nb <= 4 ? nb : nb <= 6 ? 6 : nb <= 8 ? 8 : nb <= 12 ? 12 : nb <= 16 ? 16 : nb <= 24 ? 24 : 32;
}

constexpr int kMaxThreads = 512;            // block sizes: 128, 256 (default) or 512
constexpr int kStageUnroll = 4;             // row-staging chunks unrolled (their loads overlap)
constexpr int kBoundUnroll = 4;             // bound loop over a template's spots unrolled
constexpr int kMaxWarps = kMaxThreads / 32;
constexpr int kSeedsMax = 16;              // templates of highest bound scored first, per warp (at most)

}  // namespace

// Row pitch (floats) of a layout, column c holding P'[c mod n_theta] (second dual copy:
// P'[(c + 1) mod n_theta]).  Dual: pairs at even columns t' + 2 L + 64 b + {0, 1} for
// t' = t & ~1 and b < NB2, so n_theta + 64 NB2 columns (even, for 8-byte alignment).
// Wrap-free: t + 32 b + L for b < NB, so n_theta + 32 NB.  Wrapped: blocks past the wrap read
// n_theta columns earlier, so n_theta + 32 columns and every column below 32 NB suffice.
int sparse_pitch(int n_theta, int layout) {
    if (layout == TM_LAYOUT_DUAL) {
        const int p = n_theta + 64 * round_nb((n_theta + 63) / 64);
        return p + (p & 1);
    }
    const int nb = round_nb((n_theta + 31) / 32);
    if (layout == TM_LAYOUT_WF) return n_theta + 32 * nb;
    const int a = n_theta + 32, b = 32 * nb;
    return a > b ? a : b;
}

int sparse_rows(int n_rad, int layout) { return layout == TM_LAYOUT_DUAL ? 2 * n_rad : n_rad; }

namespace {

__device__ __forceinline__ float max4(const float4& a) { return fmaxf(fmaxf(a.x, a.y), fmaxf(a.z, a.w)); }
__device__ __forceinline__ float4 abs4(const float4& a) {
    return make_float4(fabsf(a.x), fabsf(a.y), fabsf(a.z), fabsf(a.w));
}

__device__ __forceinline__ bool better(float qa, int ka, float qb, int kb) {
    return qa > qb || (qa == qb && ka < kb);
}

// Order-preserving integer key of a float (for atomicMax on scores).
__device__ __forceinline__ unsigned score_key(float x) {
    const unsigned u = __float_as_uint(x);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float key_score(unsigned k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// Row (among the library's distinct radii) and column t of a spot word.  Dual and wrap-free
// words hold the offset row * pitch + column (column < pitch); (off + 1/2) / pitch in float
// is off by far less than 1/(2 pitch), so its floor is the row exactly.  Dual: rows n_rad..
// are the copy shifted by one column, which holds the spots of odd t at column t - 1.
template <int LAYOUT>
__device__ __forceinline__ void spot_row_col(int px, float inv_pitch, int pitch, int n_rad, int& row, int& t) {
    if (LAYOUT == TM_LAYOUT_WRAP) {
        t = px & 0x7ff;
        row = (px >> 11) & 0x1fff;
        return;
    }
    const int off = LAYOUT == TM_LAYOUT_DUAL ? (int)((unsigned)px & 0xffffu) : (int)((unsigned)px >> 16);
    const int rr = (int)(((float)off + 0.5f) * inv_pitch);
    t = off - rr * pitch;
    row = rr;
    if (LAYOUT == TM_LAYOUT_DUAL && rr >= n_rad) {
        row = rr - n_rad;
        t += 1;
    }
}

// ---------------------------------------------------------------- per-layout spot updates
// acc holds V values per lane (V = 2 NB for the dual layout, NB otherwise); value v of lane L
// is shift shift_of(v, L).  FIRST initialises instead of accumulating.

template <int LAYOUT>
__device__ __forceinline__ int shift_of(int v, int lane) {
    return LAYOUT == TM_LAYOUT_DUAL ? 64 * (v >> 1) + 2 * lane + (v & 1) : 32 * v + lane;
}

// Dual and wrap-free layouts: px holds the spot's shared-memory offset (bits 0..15 dual,
// 16..31 wrap-free).
template <int V, int LAYOUT, bool FIRST>
__device__ __forceinline__ void add_spot(float (&acc)[V], const float* __restrict__ sP, int px, float I, int lane) {
    if (LAYOUT == TM_LAYOUT_DUAL) {
        const float2* p = reinterpret_cast<const float2*>(sP + (px & 0xffff)) + lane;
#pragma unroll
        for (int b = 0; b < V / 2; ++b) {
            const float2 v = p[32 * b];
            acc[2 * b] = FIRST ? I * v.x : fmaf(I, v.x, acc[2 * b]);
            acc[2 * b + 1] = FIRST ? I * v.y : fmaf(I, v.y, acc[2 * b + 1]);
        }
    } else {
        const float* p = sP + ((unsigned)px >> 16) + lane;
#pragma unroll
        for (int b = 0; b < V; ++b) acc[b] = FIRST ? I * p[32 * b] : fmaf(I, p[32 * b], acc[b]);
    }
}

// Wrapped layout: px = t | row << 11 | w << 24, w the first 32-wide block past the wrap.
template <int V, bool FIRST>
__device__ __forceinline__ void add_spot_wrapped(float (&acc)[V], const float* __restrict__ sP, int px, float I,
                                                 int pitch, int n_theta, int lane) {
    const int t = px & 0x7ff;
    const int row = (px >> 11) & 0x1fff;
    const int w = (int)((unsigned)px >> 24);
    const float* p1 = sP + row * pitch + t + lane;
    const float* p2 = p1 - n_theta;                           // blocks b >= w: wrapped
#pragma unroll
    for (int b = 0; b < V; ++b) {
        const float v = (b < w ? p1 : p2)[32 * b];
        acc[b] = FIRST ? I * v : fmaf(I, v, acc[b]);
    }
}

// Correlation C(s) of one template for all its shifts (warp-collective).  NB = shift blocks
// (64 wide for the dual layout, else 32).  Returns the warp-wide maximum; when it reaches
// thr_c, shift_out is the lowest shift attaining it and `resolved` is set.  FULL: the
// template is slid over all n_theta shifts.
template <int NB, int LAYOUT, bool FULL>
__device__ __forceinline__ float score_template(const float* __restrict__ sP, const int2* __restrict__ spots, int beg,
                                                int cnt_all, int S, int n_theta, int pitch, int lane, float thr_c,
                                                int& shift_out, bool& resolved) {
    constexpr int V = LAYOUT == TM_LAYOUT_DUAL ? 2 * NB : NB;
    resolved = false;
    int cnt = min(32, cnt_all);
    int2 mine = make_int2(0, 0);
    if (lane < cnt) mine = __ldg(spots + beg + lane);             // one lane-parallel load
    float acc[V];
    if (cnt <= 0) {                                               // no spot on the grid: C = 0, no read
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v] = 0.0f;
        cnt = 0;
    }
    if (cnt > 0) {
        const int px = __shfl_sync(0xffffffffu, mine.x, 0);
        const float I = __int_as_float(__shfl_sync(0xffffffffu, mine.y, 0));
        if (LAYOUT == TM_LAYOUT_WRAP) add_spot_wrapped<V, true>(acc, sP, px, I, pitch, n_theta, lane);
        else add_spot<V, LAYOUT, true>(acc, sP, px, I, lane);
    }
    const int end = beg + cnt_all;
    for (int i0 = beg, j = 1;;) {
        for (; j < cnt; ++j) {
            const int px = __shfl_sync(0xffffffffu, mine.x, j);
            const float I = __int_as_float(__shfl_sync(0xffffffffu, mine.y, j));
            if (LAYOUT == TM_LAYOUT_WRAP) add_spot_wrapped<V, false>(acc, sP, px, I, pitch, n_theta, lane);
            else add_spot<V, LAYOUT, false>(acc, sP, px, I, lane);
        }
        i0 += 32;
        if (i0 >= end) break;
        cnt = min(32, end - i0);
        if (lane < cnt) mine = __ldg(spots + i0 + lane);
        j = 0;
    }
    // Every value holds C(shift mod Nθ), computed by the same operations as the shift it
    // repeats (column c of a row holds P'[c mod Nθ]); so for a template slid over all Nθ
    // shifts the maximum needs no lane mask.  Otherwise shifts >= S are masked.
    float best = -FLT_MAX;
    if (FULL) {
#pragma unroll
        for (int v = 0; v < V; ++v) best = fmaxf(best, acc[v]);
    } else {
#pragma unroll
        for (int v = 0; v < V; ++v)
            if (shift_of<LAYOUT>(v, lane) < S) best = fmaxf(best, acc[v]);
    }
    if (!__any_sync(0xffffffffu, best >= thr_c)) return best;    // cannot enter the top-N
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = fmaxf(best, __shfl_xor_sync(0xffffffffu, best, o));
    if (best >= thr_c) {
        int s = INT_MAX;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const int sv = shift_of<LAYOUT>(v, lane);
            if (sv < S && acc[v] == best) s = min(s, sv);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s = min(s, __shfl_xor_sync(0xffffffffu, s, o));
        shift_out = s;
        resolved = true;
    }
    return best;
}

template <int NBMAX, int LAYOUT>
__device__ __forceinline__ float score_dispatch(const float* sP, const int2* spots, int beg, int cnt, int S,
                                                int n_theta, int pitch, int lane, float thr_c, int& s, bool& res) {
    constexpr int W = LAYOUT == TM_LAYOUT_DUAL ? 64 : 32;
    res = false;
    if (S == n_theta && round_nb((n_theta + W - 1) / W) == NBMAX)   // the common case, tested first
        return score_template<NBMAX, LAYOUT, true>(sP, spots, beg, cnt, S, n_theta, pitch, lane, thr_c, s, res);
    const int nb = (S + W - 1) / W;
#define TMGB_SCORE(NBV)                                                                                          \
    return score_template<(NBMAX >= NBV ? NBV : 1), LAYOUT, false>(sP, spots, beg, cnt, S, n_theta, pitch, lane, \
                                                                   thr_c, s, res)
    if (nb <= 1) TMGB_SCORE(1);
    if (nb <= 2) TMGB_SCORE(2);
    if (nb <= 3) TMGB_SCORE(3);
    if (nb <= 4) TMGB_SCORE(4);
    if (NBMAX >= 6 && nb <= 6) TMGB_SCORE(6);
    if (NBMAX >= 8 && nb <= 8) TMGB_SCORE(8);
    if (NBMAX >= 12 && nb <= 12) TMGB_SCORE(12);
    if (NBMAX >= 16 && nb <= 16) TMGB_SCORE(16);
    if (NBMAX >= 24 && nb <= 24) TMGB_SCORE(24);
    TMGB_SCORE(32);
#undef TMGB_SCORE
}

template <int NBMAX, int LAYOUT>
__global__ void __launch_bounds__(kMaxThreads, (LAYOUT == TM_LAYOUT_DUAL ? 2 * NBMAX : NBMAX) <= 12 ? 2 : 1)
sparse_kernel(const SparseCall c) {
    extern __shared__ __align__(16) float smem[];
    const int n_theta = c.n_theta, pitch = c.pitch;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int kWarps = blockDim.x >> 5;
    const int N = c.top_n;
    float* sP = smem;                                        // [rows][pitch]
    float* lq = sP + (size_t)(LAYOUT == TM_LAYOUT_DUAL ? 2 : 1) * c.max_rad * pitch;   // [kWarps][N]
    int* lk = (int*)(lq + kWarps * N);                       // [kWarps][N]
    int* ls = lk + kWarps * N;                               // [kWarps][N]
    int* lcnt = ls + kWarps * N;                             // [kWarps]
    int* counter = lcnt + kWarps;                            // [1]
    int* s_pattern = counter + 1;                            // [1]
    unsigned* s_thr = (unsigned*)(s_pattern + 1);            // [1] best of the warps' N-th scores (key)
    float* s_rmax = (float*)(s_thr + 1);                     // [max_rad] row maxima of P'
    float* s_rabs = s_rmax + c.max_rad;                      // [max_rad] row maxima of |P'|
    // window maxima for the pruning bound: s_cw[row][j] is the maximum of P' over the columns
    // [32 j, 32 (j + ncov)) (chunk maxima held one per lane, so at most 32 chunks per row)
    const int ncov = prune_ncov(n_theta), nchw = prune_nchw(n_theta);
    const int nq = nchw + ncov - 1;
    // patterns per tile (bounded together by the unmasked top-N pass) and the tables and lists
    // kept per pattern of a tile
    const int T = c.tile > 1 ? min(c.tile, kSparseTile) : 1;
    const int TS = T > 1 ? kSparseTile : 1;
    const int tstride = c.max_rad * nchw;
    float* s_cw = s_rabs + c.max_rad;                        // [TS][max_rad][nchw]
    // per-warp seed lists (bound / (|P| |T|) descending, template ids), [TS][kWarps][kSeedsMax]
    float* s_seedq = s_cw + (size_t)TS * tstride;
    int* s_seedk = reinterpret_cast<int*>(s_seedq + TS * kWarps * kSeedsMax);
    int* s_ncand = s_seedk + TS * kWarps * kSeedsMax;       // [1] candidates after the seeds
    float* s_tpn = reinterpret_cast<float*>(s_ncand + 1);    // [TS] |P| of the tile's patterns
    unsigned* s_tpmax = reinterpret_cast<unsigned*>(s_tpn + TS);   // [TS] max |P'| (float bits)
    uint64_t* s_bar = reinterpret_cast<uint64_t*>(((uintptr_t)(s_tpmax + TS) + 7) & ~(uintptr_t)7);   // row copies
    // polar rows staged by bulk copies (single-copy layouts; every segment 16-byte aligned)
    const bool bulk = c.bulk && LAYOUT != TM_LAYOUT_DUAL && (pitch & 3) == 0 && (n_theta & 3) == 0;
    uint32_t n_bulk = 0;                                     // bulk stagings so far (mbarrier phase)
    if (bulk && threadIdx.x == 0) mbar_init1(s_bar);
    const int kSeeds = c.seeds_per_warp > 0 ? min(c.seeds_per_warp, kSeedsMax) : 8;
    const float inv_pitch = 1.0f / (float)pitch;
    unsigned long long work = 0;                             // multiply-adds of this warp (lane 0)

    for (;;) {
        __syncthreads();                                     // previous tile fully done
        if (threadIdx.x == 0) *s_pattern = atomicAdd(c.pattern_counter, T);
        __syncthreads();
        const int64_t p0 = *s_pattern;
        if (p0 >= c.n) break;
        const int nt = (int)min((int64_t)T, c.n - p0);
        for (int li = 0; li < c.n_libs; ++li) {
            const SparseLib L = c.lib[li];
            const bool windows = L.bspot != nullptr;         // window bounds (else whole-row bounds)
            // Unmasked pruned top-N over a tile of patterns: the window tables of all of them first,
            // then one bound pass over the library that reads each bound entry once for the whole
            // tile; the patterns are then scored one by one from their stored bounds.
            const bool tiled = T > 1 && c.hits && !c.q_out[li] && L.nonneg && c.seed_bits && c.seed_cand &&
                               !c.mask[li] && windows && L.ell != nullptr;
            if (tiled) {
                if (threadIdx.x < TS) {
                    s_tpmax[threadIdx.x] = 0u;
                    s_tpn[threadIdx.x] = threadIdx.x < nt ? __ldg(c.pnorm + p0 + threadIdx.x) : 0.0f;
                }
                if (threadIdx.x == 0) *counter = 0;
                for (int tl = 0; tl < nt; ++tl) {
                    uint32_t* sb = c.seed_bits + ((size_t)blockIdx.x * kSparseTile + tl) * c.seed_words;
                    for (int i = threadIdx.x; i < L.words; i += blockDim.x) sb[i] = 0u;
                }
                if (lane < kSeeds)
                    for (int tl = 0; tl < TS; ++tl) {
                        s_seedq[(tl * kWarps + warp) * kSeedsMax + lane] = -INFINITY;
                        s_seedk[(tl * kWarps + warp) * kSeedsMax + lane] = -1;
                    }
                __syncthreads();
                // window tables: per library row of each pattern, the maxima of the 32-column chunks
                // q < nq of P'[c mod Nθ] (lane q keeps chunk q; warp-uniform trip count), then of the
                // chunks each window start covers; and the pattern's max |P'|.  With Nθ a multiple
                // of 8 (at most 512) and 16-byte aligned rows, a chunk is four 8-column pieces
                // (mod Nθ), whose maxima the lanes take with 16-byte loads.
                const int npc = n_theta >> 3;
                const bool pieces = bulk && (n_theta & 7) == 0 && npc <= 64;
                for (int it = warp; it < nt * L.n_rad; it += kWarps) {
                    const int tl = it / L.n_rad, rr = it - tl * L.n_rad;
                    const float* row =
                        c.polar + (size_t)(p0 + tl) * c.n_r * n_theta + (size_t)__ldg(L.radii + rr) * n_theta;
                    float ma = 0.0f, mq = -INFINITY;
                    if (pieces) {
                        float pm[2] = {-INFINITY, -INFINITY};        // pieces lane and lane + 32
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            if (lane + 32 * h < npc) {
                                const float4* q4 = reinterpret_cast<const float4*>(row) + 2 * (lane + 32 * h);
                                const float4 a = __ldg(q4), b = __ldg(q4 + 1);
                                pm[h] = fmaxf(max4(a), max4(b));
                                ma = fmaxf(ma, fmaxf(max4(abs4(a)), max4(abs4(b))));
                            }
                        }
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const int pc = (4 * lane + i) % npc;
                            const float v0 = __shfl_sync(0xffffffffu, pm[0], pc & 31);
                            const float v1 = __shfl_sync(0xffffffffu, pm[1], pc & 31);
                            mq = fmaxf(mq, pc >= 32 ? v1 : v0);
                        }
                    }
#pragma unroll kStageUnroll
                    for (int c0 = 0; c0 < (pieces ? 0 : 32 * nq); c0 += 32) {
                        int sc = c0 + lane;
                        while (sc >= n_theta) sc -= n_theta;
                        const float v = __ldg(row + sc);
                        ma = fmaxf(ma, fabsf(v));
                        float m = v;
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
                        if (lane == (c0 >> 5)) mq = m;
                    }
                    float w = -INFINITY;
                    for (int i = 0; i < ncov; ++i) {
                        const float o = __shfl_sync(0xffffffffu, mq, (lane + i) & 31);
                        if (lane + i < nq) w = fmaxf(w, o);
                    }
                    if (lane < nchw) s_cw[tl * tstride + rr * nchw + lane] = w;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) ma = fmaxf(ma, __shfl_xor_sync(0xffffffffu, ma, o));
                    if (lane == 0) atomicMax(s_tpmax + tl, __float_as_uint(ma));   // (ma >= 0)
                }
                __syncthreads();
                float rpn[kSparseTile], tpm[kSparseTile];     // 1 / |P| (0: |P| = 0) and max |P'|
#pragma unroll
                for (int tl = 0; tl < kSparseTile; ++tl) {
                    rpn[tl] = s_tpn[tl] > 0.0f ? 1.0f / s_tpn[tl] : 0.0f;
                    tpm[tl] = __uint_as_float(s_tpmax[tl]);
                }
                // the bound pass of every pattern of the tile (tables of patterns past nt are left
                // over from earlier tiles: their sums are formed and not used)
                for (;;) {
                    int wd = 0;
                    if (lane == 0) wd = atomicAdd(counter, 1);
                    wd = __shfl_sync(0xffffffffu, wd, 0);
                    if (wd >= L.words) break;
                    const int rem = L.K - wd * 32;
                    int4 meta_l = make_int4(0, 0, 0, 0);
                    if (lane < rem) meta_l = __ldg(L.smeta + wd * 32 + lane);
                    const int cnt_l = meta_l.y & 0xffff;
                    const int2* bs = L.ell + __ldg(L.ellw + wd) + lane;
                    float u[kSparseTile][3];
#pragma unroll
                    for (int tl = 0; tl < kSparseTile; ++tl) u[tl][0] = u[tl][1] = u[tl][2] = 0.0f;
#pragma unroll kBoundUnroll
                    for (int i = 0; i < cnt_l; ++i) {
                        const int2 e = __ldg(bs + 32 * i);
                        const float I = __int_as_float(e.x);
                        const int j0 = e.y & 0xffff;
                        const int j1 = j0 + ((e.y >> 16) & 0xff), j2 = j0 + (int)((unsigned)e.y >> 24);
#pragma unroll
                        for (int tl = 0; tl < kSparseTile; ++tl) {
                            const float* tb = s_cw + tl * tstride;
                            u[tl][0] = fmaf(I, tb[j0], u[tl][0]);
                            u[tl][1] = fmaf(I, tb[j1], u[tl][1]);
                            u[tl][2] = fmaf(I, tb[j2], u[tl][2]);
                        }
                    }
                    // the rounding margin of the bound as in the single-pattern pass; bound / (|P| |T|)
                    // as a product with the reciprocals (one division per template for the tile),
                    // whose few roundings stay far inside the 1e-5 relative margin the stored bounds
                    // are compared with
                    const float tn = __int_as_float(meta_l.z);
                    const float mrg = (2.0f * (float)cnt_l + 40.0f) * 5.9604645e-8f * __int_as_float(meta_l.w);
                    const float rtn = tn > 0.0f ? 1.0f / tn : 0.0f;
#pragma unroll
                    for (int tl = 0; tl < kSparseTile; ++tl) {
                        if (tl >= nt) break;                 // uniform
                        __half* qbt = c.seed_qub + ((size_t)blockIdx.x * kSparseTile + tl) * c.seed_words * 32;
                        float qb = -INFINITY;
                        if (lane < rem) {
                            if (rtn > 0.0f && rpn[tl] > 0.0f) {
                                qb = (fmaxf(fmaxf(u[tl][0], u[tl][1]), u[tl][2]) + mrg * tpm[tl]) * rtn * rpn[tl];
                                qbt[wd * 32 + lane] = __float2half_ru(qb);
                            } else {
                                qbt[wd * 32 + lane] = __ushort_as_half((unsigned short)0x7c00);   // +inf
                            }
                        }
                        // the word's best bound enters the warp's seed list (lowest lane on ties)
                        // only when it beats the list's last entry
                        float mq = qb;
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) mq = fmaxf(mq, __shfl_xor_sync(0xffffffffu, mq, o));
                        float* sq = s_seedq + (tl * kWarps + warp) * kSeedsMax;
                        int* sk = s_seedk + (tl * kWarps + warp) * kSeedsMax;
                        if (mq > sq[kSeeds - 1]) {           // uniform (the list is the warp's own)
                            const int ml = __ffs(__ballot_sync(0xffffffffu, qb == mq)) - 1;
                            if (lane == 0) {
                                int i = kSeeds - 1;
                                while (i > 0 && mq > sq[i - 1]) { sq[i] = sq[i - 1]; sk[i] = sk[i - 1]; --i; }
                                sq[i] = mq;
                                sk[i] = wd * 32 + ml;
                            }
                            __syncwarp();
                        }
                    }
                    __syncwarp();
                }
                __syncthreads();
            }
            for (int t = 0; t < nt; ++t) {
                const int64_t p = p0 + t;
                const float* src = c.polar + (size_t)p * c.n_r * n_theta;
                const float pn = __ldg(c.pnorm + p);
                // bring the same rows of pattern p + T gridDim.x into L2: patterns are taken in order,
                // so the CTA that takes it soon finds them there (one 128-byte line per thread)
                if (p + (int64_t)T * gridDim.x < c.n) {
                    const int lines = (n_theta * (int)sizeof(float) + 127) >> 7;
                    const float* nsrc = c.polar + (size_t)(p + (int64_t)T * gridDim.x) * c.n_r * n_theta;
                    for (int i = threadIdx.x; i < L.n_rad * lines; i += blockDim.x) {
                        const int r0 = i / lines, l = i - r0 * lines;
                        const char* a =
                            reinterpret_cast<const char*>(nsrc + (size_t)__ldg(L.radii + r0) * n_theta) + 128 * l;
                        asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
                    }
                }
                // the library's polar rows (dual layout: a second copy shifted by one column); column c of
                // a row holds P'[c mod Nθ]: with bulk copies, segments of at most Nθ columns
                const int rows = (LAYOUT == TM_LAYOUT_DUAL ? 2 : 1) * L.n_rad;
                if (bulk) {
                    const int nseg = (pitch + n_theta - 1) / n_theta;
                    fence_proxy_async_smem();                    // earlier reads of sP before the copies
                    if (threadIdx.x == 0)
                        mbar_arrive_expect_tx(s_bar, (uint32_t)(L.n_rad * pitch * 4) + (c.test_stall ? 16u : 0u));
                    for (int it = threadIdx.x; it < L.n_rad * nseg; it += blockDim.x) {
                        const int rr = it / nseg, c0 = (it - rr * nseg) * n_theta;
                        bulk_g2s(sP + (size_t)rr * pitch + c0, src + (size_t)__ldg(L.radii + rr) * n_theta,
                                 (uint32_t)(min(n_theta, pitch - c0) * 4), s_bar);
                    }
                    const bool ok = mbar_wait_bounded(s_bar, n_bulk & 1u);
                    if (__syncthreads_or(!ok)) {
                        // the copies did not land in time: report it, let them finish (bounded), stop
                        if (threadIdx.x == 0) {
                            atomicOr(c.error, 4u);
                            mbar_wait_bounded(s_bar, n_bulk & 1u);
                        }
                        __syncthreads();
                        return;
                    }
                    ++n_bulk;
                }
                // row maxima (and window tables) from the staged rows; a tile's patterns need neither
                for (int rr = warp; rr < ((bulk && tiled) ? 0 : rows); rr += kWarps) {
                    const int r0 = rr < L.n_rad ? rr : rr - L.n_rad;
                    const int sh = rr < L.n_rad ? 0 : 1;
                    const float* row = src + (size_t)__ldg(L.radii + r0) * n_theta;
                    float* dst = sP + (size_t)rr * pitch;
                    float mx = -INFINITY, ma = 0.0f;
                    // copy-0 rows also take the maxima of the 32-column chunks q < nq of
                    // P'[c mod Nθ] (lane q keeps chunk q); warp-uniform trip count
                    const bool first = rr < L.n_rad;
                    const bool chunks = first && windows && !tiled;   // (windows imply nq <= 32)
                    const int ncol = bulk ? (chunks ? 32 * nq : n_theta) : (chunks ? max(pitch, 32 * nq) : pitch);
                    float mq = -INFINITY;
#pragma unroll kStageUnroll
                    for (int c0 = 0; c0 < ncol; c0 += 32) {
                        const int col = c0 + lane;
                        int sc = col + sh;
                        while (sc >= n_theta) sc -= n_theta;
                        const bool valid = bulk || col < pitch || chunks;
                        float v;
                        if (bulk) {
                            v = dst[sc];                         // (staged: column sc < Nθ holds P'[sc])
                        } else {
                            v = valid ? __ldg(row + sc) : -INFINITY;
                            if (col < pitch) dst[col] = v;
                        }
                        if (valid) {
                            mx = fmaxf(mx, v);
                            ma = fmaxf(ma, fabsf(v));
                        }
                        if (chunks) {
                            float m = v;
#pragma unroll
                            for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
                            if (lane == (c0 >> 5)) mq = m;
                        }
                    }
                    if (chunks) {
                        float w = -INFINITY;
                        for (int i = 0; i < ncov; ++i) {
                            const float o = __shfl_sync(0xffffffffu, mq, (lane + i) & 31);
                            if (lane + i < nq) w = fmaxf(w, o);
                        }
                        if (lane < nchw) s_cw[rr * nchw + lane] = w;
                    }
                    if (first) {
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) {
                            mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
                            ma = fmaxf(ma, __shfl_xor_sync(0xffffffffu, ma, o));
                        }
                        if (lane == 0) { s_rmax[rr] = mx; s_rabs[rr] = ma; }
                    }
                }
                if (threadIdx.x == 0) { *counter = 0; *s_thr = score_key(-INFINITY); }
                if (threadIdx.x < kWarps) lcnt[threadIdx.x] = 0;
                __syncthreads();
                const int2* spots = LAYOUT == TM_LAYOUT_WRAP ? L.spot : L.spot2;
                float pmax = 0.0f;                               // max |P'| over the library's rows
                for (int rr = lane; rr < L.n_rad; rr += 32) pmax = fmaxf(pmax, s_rabs[rr]);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) pmax = fmaxf(pmax, __shfl_xor_sync(0xffffffffu, pmax, o));
                const uint32_t* mrow = c.mask[li] ? c.mask[li] + (size_t)p * L.words : nullptr;
                float* qo = c.q_out[li] ? c.q_out[li] + (size_t)p * L.K : nullptr;
                int32_t* so = c.s_out[li] ? c.s_out[li] + (size_t)p * L.K : nullptr;
                float* wq = lq + warp * N;
                int* wk = lk + warp * N;
                int* ws = ls + warp * N;
                const bool use_thr = !qo && c.hits;
                const bool prune = use_thr && L.nonneg;
                float qthr = -INFINITY;                          // the warp's N-th best Q once its list is full
                // per-lane metadata of word wd's templates {first spot, spots | shifts << 16, norm bits,
                // intensity-sum bits} (one load) and the mask of the word's templates to score
                auto word_meta = [&](int wd, uint32_t& m, int4& meta_l, int& rem) {
                    m = mrow ? __ldg(mrow + wd) : 0xffffffffu;
                    rem = L.K - wd * 32;
                    if (rem < 32) m &= (1u << rem) - 1u;
                    meta_l = make_int4(0, 1 << 16, 0, 0);
                    if (lane < rem && ((m >> lane) & 1u)) meta_l = __ldg(L.meta + wd * 32 + lane);
                };
                // exact pruning (intensities >= 0): each lane bounds its template's best correlation
                // over each of three windows of shifts, C(s) <= sum_i I_i max P'[r_i][visited
                // columns] (a superset of the visited columns: whole 32-column chunks), or with
                // windows too wide for the chunk table over the whole row; plus a margin for the
                // rounding of both sums
                // (2^-24 per operation; sum_i |I_i P'| <= isum * pmax).  bs[i * bstride] holds the
                // window entries of the template's spot i.
                auto lane_bound = [&](const int4& meta_l, const int2* bs, int bstride) -> float {
                    const int cnt_l = meta_l.y & 0xffff;
                    float ub = 0.0f, u0 = 0.0f, u1 = 0.0f, u2 = 0.0f;
                    if (windows) {
                        // per spot: its intensity and the table entries of its three windows
#pragma unroll kBoundUnroll
                        for (int i = 0; i < cnt_l; ++i) {
                            const int2 w = __ldg(bs + i * bstride);
                            const float I = __int_as_float(w.x);
                            const int j0 = w.y & 0xffff;
                            u0 = fmaf(I, s_cw[j0], u0);
                            u1 = fmaf(I, s_cw[j0 + ((w.y >> 16) & 0xff)], u1);
                            u2 = fmaf(I, s_cw[j0 + (int)((unsigned)w.y >> 24)], u2);
                        }
                        ub = fmaxf(fmaxf(u0, u1), u2);
                    } else {
                        for (int i = 0; i < cnt_l; ++i) {
                            const int2 w = __ldg(spots + meta_l.x + i);
                            int row, t;
                            spot_row_col<LAYOUT>(w.x, inv_pitch, pitch, L.n_rad, row, t);
                            ub = fmaf(__int_as_float(w.y), s_rmax[row], ub);
                        }
                    }
                    return ub + (2.0f * (float)cnt_l + 40.0f) * 5.9604645e-8f * __int_as_float(meta_l.w) * pmax;
                };
                // score template k (warp-collective) and keep it in the warp's top-N when it enters
                auto score_one = [&](int k, int beg, int cs, float tn, float ubm) {
                    const int cnt = cs & 0xffff, S = (int)((unsigned)cs >> 16);
                    const float d = pn * tn;
                    // Every warp's N-th best score is a lower bound of the pattern's final N-th
                    // best, and so is the best of them (s_thr).  A template below it cannot
                    // enter the top-N.
                    const float thr = use_thr ? fmaxf(qthr, key_score(*(volatile unsigned*)s_thr)) : -INFINITY;
                    // the template is skipped when its bound stays below thr * d (then Q < thr)
                    if (thr > -INFINITY && d > 0.0f) {
                        const float td = thr * d;
                        if (ubm < td - fabsf(td) * 4.8e-7f) return;
                    }
                    // a template whose correlation stays below the threshold (in correlation
                    // units, with a margin for the division's rounding) cannot enter the
                    // top-N, so its best shift is not resolved
                    float thr_c = -FLT_MAX;
                    if (use_thr && thr > -INFINITY && d > 0.0f) {
                        const float t = thr * d;
                        thr_c = t - fabsf(t) * 1e-6f;
                    }
                    int s = 0;
                    bool resolved = false;
                    const float best =
                        score_dispatch<NBMAX, LAYOUT>(sP, spots, beg, cnt, S, n_theta, pitch, lane, thr_c, s, resolved);
                    if (c.work) work += (unsigned long long)cnt * (unsigned long long)S;
                    if (!resolved) return;
                    float q;
                    if (d > 0.0f) q = __fdiv_rn(best, d);
                    else { q = 0.0f; s = 0; }
                    if (lane == 0) {
                        if (qo) { qo[k] = q; so[k] = s; }
                        if (c.hits) {
                            const int cnt_l = lcnt[warp];
                            if (cnt_l < N || better(q, k, wq[N - 1], wk[N - 1])) {
                                int i = cnt_l < N ? cnt_l : N - 1;
                                while (i > 0 && better(q, k, wq[i - 1], wk[i - 1])) {
                                    wq[i] = wq[i - 1]; wk[i] = wk[i - 1]; ws[i] = ws[i - 1];
                                    --i;
                                }
                                wq[i] = q; wk[i] = k; ws[i] = s;
                                if (cnt_l < N) lcnt[warp] = cnt_l + 1;
                            }
                        }
                    }
                    __syncwarp();
                    if (use_thr) {
                        float nt = -INFINITY;
                        if (lane == 0 && lcnt[warp] >= N) {
                            nt = wq[N - 1];
                            atomicMax(s_thr, score_key(nt));
                        }
                        qthr = __shfl_sync(0xffffffffu, nt, 0);
                    }
                };
                // Seeding (pruned top-N only): a first pass bounds every template and keeps, per warp,
                // the seeds_per_warp templates of highest bound / (|P| |T|) (an upper bound of their Q; each
                // 32-template word offers its best).  They are scored first, so the top-N threshold
                // starts near its final value and the main pass skips almost every other template by
                // its bound.  Seeded templates are marked and not scored again.
                // (not with a template mask -- the pre-filter's survivors or the rescore candidates --,
                // where too few templates remain for the extra pass to pay)
                const bool seeding = prune && c.seed_bits && c.seed_cand && !mrow;
                // Both passes of the seeded search visit the templates in spot-count order (window
                // bounds only): bit words, stored bounds and seeds then refer to sorted positions,
                // results to library indices.
                const bool sorted = seeding && windows && L.ell != nullptr;
                const int4* smeta = sorted ? L.smeta : L.meta;
                const int tl = tiled ? t : 0;                    // the pattern's slot of the tile
                uint32_t* seedbits =
                    c.seed_bits ? c.seed_bits + ((size_t)blockIdx.x * kSparseTile + tl) * c.seed_words : nullptr;
                // every template's bound / (|P| |T|) from the seeding pass, rounded up to FP16, so the
                // main pass compares it with the threshold instead of bounding the template again
                __half* qbound =
                    c.seed_bits ? c.seed_qub + ((size_t)blockIdx.x * kSparseTile + tl) * c.seed_words * 32 : nullptr;
                if (seeding) {
                    float* sq = s_seedq + (tl * kWarps + warp) * kSeedsMax;
                    int* sk = s_seedk + (tl * kWarps + warp) * kSeedsMax;
                    if (!tiled) {                                // (tiled: bounded with the tile above)
                        if (lane < kSeeds) { sq[lane] = -INFINITY; sk[lane] = -1; }
                        for (int i = threadIdx.x; i < L.words; i += blockDim.x) seedbits[i] = 0u;
                        __syncwarp();
                        for (;;) {
                            int wd = 0;
                            if (lane == 0) wd = atomicAdd(counter, 1);
                            wd = __shfl_sync(0xffffffffu, wd, 0);
                            if (wd >= L.words) break;
                            uint32_t m;
                            int4 meta_l;
                            int rem;
                            const int2* bs = nullptr;
                            int bstride = 1;
                            if (sorted) {
                                rem = L.K - wd * 32;
                                m = rem < 32 ? (1u << rem) - 1u : 0xffffffffu;
                                meta_l = make_int4(0, 1 << 16, 0, 0);
                                if (lane < rem) meta_l = __ldg(smeta + wd * 32 + lane);
                                bs = L.ell + __ldg(L.ellw + wd) + lane;
                                bstride = 32;
                            } else {
                                word_meta(wd, m, meta_l, rem);
                                if (windows) bs = L.bspot + meta_l.x;
                            }
                            float qb = -INFINITY;
                            if (lane < rem && ((m >> lane) & 1u)) {
                                const float d_l = pn * __int_as_float(meta_l.z);
                                if (d_l > 0.0f) {
                                    qb = lane_bound(meta_l, bs, bstride) / d_l;
                                    qbound[wd * 32 + lane] = __float2half_ru(qb);
                                } else {
                                    // +inf: never skipped
                                    qbound[wd * 32 + lane] = __ushort_as_half((unsigned short)0x7c00);
                                }
                            }
                            float mq = qb;
                            int ml = lane;
#pragma unroll
                            for (int o = 16; o > 0; o >>= 1) {
                                const float oq = __shfl_xor_sync(0xffffffffu, mq, o);
                                const int ol = __shfl_xor_sync(0xffffffffu, ml, o);
                                if (oq > mq || (oq == mq && ol < ml)) { mq = oq; ml = ol; }
                            }
                            if (lane == 0 && mq > sq[kSeeds - 1]) {
                                int i = kSeeds - 1;
                                while (i > 0 && mq > sq[i - 1]) { sq[i] = sq[i - 1]; sk[i] = sk[i - 1]; --i; }
                                sq[i] = mq;
                                sk[i] = wd * 32 + ml;
                            }
                            __syncwarp();
                        }
                    }
                    __syncthreads();                             // the bit words are zero; every warp's seeds known
                    for (int i = 0; i < kSeeds; ++i) {
                        const int j = sk[i];
                        if (j < 0) break;
                        if (lane == 0) atomicOr(seedbits + (j >> 5), 1u << (j & 31));
                        const int4 mk = __ldg(smeta + j);
                        score_one(sorted ? __ldg(L.sperm + j) : j, mk.x, mk.y, __int_as_float(mk.z), INFINITY);
                    }
                    __syncthreads();
                    // the N-th best of all warps' lists (distinct templates) bounds the final N-th
                    // best from below: it becomes the shared threshold
                    if (warp == 0) {
                        const int total = kWarps * N;
                        unsigned long long taken = 0;            // entries taken by this lane (bit per slot)
                        float nth = -INFINITY;
                        int got = 0;
                        for (int j = 0; j < N; ++j) {
                            float bq = -INFINITY;
                            int bk = INT_MAX, bi = -1;
                            for (int ci = lane, slot = 0; ci < total; ci += 32, ++slot) {
                                const int w = ci / N, i = ci - w * N;
                                if (i >= lcnt[w] || ((taken >> slot) & 1ull)) continue;
                                if (bi < 0 || better(lq[ci], lk[ci], bq, bk)) { bq = lq[ci]; bk = lk[ci]; bi = ci; }
                            }
#pragma unroll
                            for (int o = 16; o > 0; o >>= 1) {
                                const float oq = __shfl_xor_sync(0xffffffffu, bq, o);
                                const int ok = __shfl_xor_sync(0xffffffffu, bk, o);
                                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                                if (oi >= 0 && (bi < 0 || better(oq, ok, bq, bk))) { bq = oq; bk = ok; bi = oi; }
                            }
                            if (bi < 0) break;
                            if ((bi & 31) == lane) taken |= 1ull << (bi >> 5);
                            nth = bq;
                            ++got;
                        }
                        if (lane == 0 && got == N) atomicMax(s_thr, score_key(nth));
                    }
                    if (threadIdx.x == 0) *s_ncand = 0;
                    __syncthreads();
                    // Candidates: the templates not seeded whose stored bound (rounded up) reaches the
                    // threshold, with a margin far above the rounding of the division (the threshold
                    // only rises, so a template dropped here would be dropped later as well).  Each
                    // thread tests 8 consecutive positions; a warp reserves its entries at once.
                    int* cand = c.seed_cand + (size_t)blockIdx.x * c.seed_words * 32;
                    {
                        const float thr0 = key_score(*(volatile unsigned*)s_thr);
                        const float cut = thr0 - fabsf(thr0) * 1e-5f;
                        // warp-uniform trip count (the scan below is warp-collective); lanes past the
                        // end keep nothing
                        for (int jw = 256 * warp; jw < 32 * L.words; jw += 8 * blockDim.x) {
                            const int j0 = jw + 8 * lane;
                            const bool in = j0 < 32 * L.words;
                            uint4 v = make_uint4(0u, 0u, 0u, 0u);
                            uint32_t sb = 0xffu;
                            if (in) {
                                v = *reinterpret_cast<const uint4*>(qbound + j0);
                                sb = (seedbits[j0 >> 5] >> (j0 & 31)) & 0xffu;
                            }
                            const uint32_t h[4] = {v.x, v.y, v.z, v.w};
                            uint32_t keep = 0;
#pragma unroll
                            for (int u = 0; u < 8; ++u) {
                                const float qb =
                                    __half2float(__ushort_as_half((unsigned short)(h[u >> 1] >> (16 * (u & 1)))));
                                const bool k_ok = j0 + u < L.K && !((sb >> u) & 1u) && !(thr0 > -INFINITY && qb < cut);
                                keep |= (uint32_t)k_ok << u;
                            }
                            const int cnt = __popc(keep);
                            int incl = cnt;
#pragma unroll
                            for (int o = 1; o < 32; o <<= 1) {
                                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                                if (lane >= o) incl += y;
                            }
                            int base = 0;
                            if (lane == 31 && incl) base = atomicAdd(s_ncand, incl);
                            base = __shfl_sync(0xffffffffu, base, 31) + incl - cnt;
                            while (keep) {
                                const int u = __ffs(keep) - 1;
                                keep &= keep - 1;
                                cand[base++] = j0 + u;
                            }
                        }
                    }
                    __syncthreads();
                    const int ncand = *s_ncand;
                    // Warp w takes candidates w, w + kWarps, ... counted from the end of the list, which
                    // follows the bound pass's order (most spots first), so the templates with the fewest
                    // spots come first: over a subtracted background they reach a high Q most often, and
                    // the threshold rises sooner.  One lane-parallel load of 32 of them, then each is tested
                    // against the current threshold by its stored bound and scored.
                    for (int b0 = warp; b0 < ncand; b0 += 32 * kWarps) {
                        const int ci = b0 + lane * kWarps;
                        int j_l = 0, k_l = 0;
                        int4 mk_l = make_int4(0, 0, 0, 0);
                        float qb_l = 0.0f;
                        if (ci < ncand) {
                            j_l = cand[ncand - 1 - ci];
                            mk_l = __ldg(smeta + j_l);
                            k_l = sorted ? __ldg(L.sperm + j_l) : j_l;
                            qb_l = __half2float(qbound[j_l]);
                        }
                        uint32_t mm = __ballot_sync(0xffffffffu, ci < ncand);
                        while (mm) {
                            const int bit = __ffs(mm) - 1;
                            mm &= mm - 1;
                            const float qb = __shfl_sync(0xffffffffu, qb_l, bit);
                            const float thr = fmaxf(qthr, key_score(*(volatile unsigned*)s_thr));
                            if (thr > -INFINITY && qb < thr - fabsf(thr) * 1e-5f) continue;
                            score_one(__shfl_sync(0xffffffffu, k_l, bit), __shfl_sync(0xffffffffu, mk_l.x, bit),
                                      __shfl_sync(0xffffffffu, mk_l.y, bit),
                                      __int_as_float(__shfl_sync(0xffffffffu, mk_l.z, bit)), INFINITY);
                        }
                    }
                }
                for (; !seeding;) {
                    int wd = 0;
                    if (lane == 0) wd = atomicAdd(counter, 1);
                    wd = __shfl_sync(0xffffffffu, wd, 0);
                    if (wd >= L.words) break;
                    uint32_t m;
                    int4 meta_l;
                    int rem;
                    word_meta(wd, m, meta_l, rem);
                    if (qo && lane < rem && !((m >> lane) & 1u)) {
                        qo[wd * 32 + lane] = -INFINITY;
                        so[wd * 32 + lane] = -1;
                    }
                    float ubm_l = INFINITY;
                    if (prune && lane < rem && ((m >> lane) & 1u))
                        ubm_l = lane_bound(meta_l, windows ? L.bspot + meta_l.x : nullptr, 1);
                    // drop, all lanes at once, the templates whose bound is already below the
                    // threshold (the threshold only rises, so the test in the loop would drop them
                    // as well); the loop then visits the others only
                    if (prune) {
                        const float thr0 = fmaxf(qthr, key_score(*(volatile unsigned*)s_thr));
                        if (thr0 > -INFINITY) {
                            const float d_l = pn * __int_as_float(meta_l.z);
                            const float td = thr0 * d_l;
                            m &= ~__ballot_sync(0xffffffffu, d_l > 0.0f && ubm_l < td - fabsf(td) * 4.8e-7f);
                        }
                    }
                    while (m) {
                        const int bit = __ffs(m) - 1;
                        m &= m - 1;
                        const int k = wd * 32 + bit;
                        score_one(k, __shfl_sync(0xffffffffu, meta_l.x, bit), __shfl_sync(0xffffffffu, meta_l.y, bit),
                                  __int_as_float(__shfl_sync(0xffffffffu, meta_l.z, bit)),
                                  __shfl_sync(0xffffffffu, ubm_l, bit));
                    }
                }
                __syncthreads();
                if (c.hits && warp == 0) {
                    tm_hit* out = c.hits + (size_t)li * c.hits_lib_stride + (size_t)p * N;
                    const int total = kWarps * N;
                    for (int j = 0; j < N; ++j) {
                        float bq = -INFINITY;
                        int bk = INT_MAX, bi = -1;
                        for (int ci = lane; ci < total; ci += 32) {
                            const int w = ci / N, i = ci - w * N;
                            if (i >= lcnt[w]) continue;
                            const int kk = lk[ci];
                            if (kk < 0) continue;
                            if (bi < 0 || better(lq[ci], kk, bq, bk)) { bq = lq[ci]; bk = kk; bi = ci; }
                        }
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) {
                            const float oq = __shfl_xor_sync(0xffffffffu, bq, o);
                            const int ok = __shfl_xor_sync(0xffffffffu, bk, o);
                            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                            if (oi >= 0 && (bi < 0 || better(oq, ok, bq, bk))) { bq = oq; bk = ok; bi = oi; }
                        }
                        if (lane == 0) {
                            tm_hit h;
                            if (bi >= 0) {
                                h.template_index = bk;
                                h.shift = ls[bi];
                                h.score = bq;
                                h.angle_deg = (float)ls[bi] * (360.0f / (float)n_theta);
                                h.mirror = (L.mirror && bk >= L.K0) ? 1 : 0;
                                lk[bi] = -1;
                            } else {
                                h.template_index = -1; h.shift = -1; h.score = -INFINITY;
                                h.angle_deg = 0.0f; h.mirror = 0;
                            }
                            out[j] = h;
                        }
                        __syncwarp();
                    }
                }
                __syncthreads();
            }
        }
    }
    if (c.work && lane == 0 && work) atomicAdd(c.work, work);
}

template <int NBMAX, int LAYOUT>
cudaError_t launch_nb(const SparseCall& c, int num_sms, size_t smem, cudaStream_t st) {
    const int threads = (c.threads == 128 || c.threads == 512) ? c.threads : 256;
    int per_sm = 0;
    cudaError_t e = kernel_occupancy((const void*)sparse_kernel<NBMAX, LAYOUT>, threads, smem, &per_sm);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int64_t grid = (int64_t)num_sms * per_sm;
    const int64_t tiles = (c.n + (c.tile > 1 ? c.tile : 1) - 1) / (c.tile > 1 ? c.tile : 1);
    if (grid > tiles) grid = tiles;
    SparseCall cc = c;
    if (cc.seed_bits && grid > cc.seed_ctas) cc.seed_bits = nullptr;   // per-CTA bit words not provided: no seeding
    e = cudaMemsetAsync(c.pattern_counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    sparse_kernel<NBMAX, LAYOUT><<<(int)grid, threads, smem, st>>>(cc);
    return cudaGetLastError();
}

// Shared-memory budgets of the layouts: the dual layout only when four CTAs still fit on an
// SM, the wrap-free one when at least two do.
constexpr size_t kDualBytes = 54 * 1024;
constexpr size_t kWrapFreeBytes = 100 * 1024;

}  // namespace

int sparse_max_ctas(int num_sms) { return num_sms * 8; }

size_t sparse_smem_bytes(int max_rad, int n_theta, int top_n, int* layout, int* pitch, int tile) {
    if (n_theta < 1 || n_theta > 1024 || top_n < 1 || top_n > TM_MAX_TOPN || max_rad < 1) return 0;
    const size_t ts = tile > 1 ? kSparseTile : 1;          // window tables and seed lists per pattern
    const size_t lists = (size_t)kMaxWarps * top_n * 12 + kMaxWarps * 4 + 16 + (size_t)max_rad * 8 + 16 +
                         ts * kMaxWarps * kSeedsMax * 8 + 8 + ts * 8 + 4 + 16;
    const int order[3] = {TM_LAYOUT_DUAL, TM_LAYOUT_WF, TM_LAYOUT_WRAP};
    const size_t limit[3] = {kDualBytes, kWrapFreeBytes, 232448};
    for (int i = 0; i < 3; ++i) {
        const int pch = sparse_pitch(n_theta, order[i]);
        const size_t rows = (size_t)sparse_rows(max_rad, order[i]);
        // per-spot offsets of the dual and wrap-free layouts are 16-bit
        if (order[i] != TM_LAYOUT_WRAP && rows * pch > 65535) continue;
        const size_t windows = ts * max_rad * prune_nchw(n_theta) * 4;   // float [ts][max_rad][nchw]
        const size_t b = rows * pch * 4 + lists + windows;
        if (b <= limit[i]) {
            if (layout) *layout = order[i];
            if (pitch) *pitch = pch;
            return b;
        }
    }
    return 0;
}

cudaError_t launch_sparse(const SparseCall& call, int num_sms, cudaStream_t st) {
    if (call.n <= 0) return cudaSuccess;
    int layout = TM_LAYOUT_WRAP, pitch = 0;
    SparseCall c = call;
    size_t smem = 0;
    if (c.tile > 1) smem = sparse_smem_bytes(c.max_rad, c.n_theta, c.top_n, &layout, &pitch, c.tile);
    if (!smem) {                                            // (tiles need their tables and lists)
        c.tile = 1;
        smem = sparse_smem_bytes(c.max_rad, c.n_theta, c.top_n, &layout, &pitch, 1);
    }
    if (!smem) return cudaErrorInvalidValue;
    c.pitch = pitch;
    if (layout == TM_LAYOUT_DUAL) {
        const int nb2 = (c.n_theta + 63) / 64;
        if (nb2 <= 3) return launch_nb<3, TM_LAYOUT_DUAL>(c, num_sms, smem, st);
        if (nb2 <= 6) return launch_nb<6, TM_LAYOUT_DUAL>(c, num_sms, smem, st);
        if (nb2 <= 12) return launch_nb<12, TM_LAYOUT_DUAL>(c, num_sms, smem, st);
        return launch_nb<16, TM_LAYOUT_DUAL>(c, num_sms, smem, st);
    }
    const int nbmax = (c.n_theta + 31) / 32;
    if (layout == TM_LAYOUT_WF) {
        if (nbmax <= 6) return launch_nb<6, TM_LAYOUT_WF>(c, num_sms, smem, st);
        if (nbmax <= 12) return launch_nb<12, TM_LAYOUT_WF>(c, num_sms, smem, st);
        if (nbmax <= 24) return launch_nb<24, TM_LAYOUT_WF>(c, num_sms, smem, st);
        return launch_nb<32, TM_LAYOUT_WF>(c, num_sms, smem, st);
    }
    if (nbmax <= 6) return launch_nb<6, TM_LAYOUT_WRAP>(c, num_sms, smem, st);
    if (nbmax <= 12) return launch_nb<12, TM_LAYOUT_WRAP>(c, num_sms, smem, st);
    if (nbmax <= 24) return launch_nb<24, TM_LAYOUT_WRAP>(c, num_sms, smem, st);
    return launch_nb<32, TM_LAYOUT_WRAP>(c, num_sms, smem, st);
}

}  // namespace tmgb
