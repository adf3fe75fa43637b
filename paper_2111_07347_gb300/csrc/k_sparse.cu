// Stage 3: the correlation index Q of Eq. 1 for every template at every azimuthal shift
// with wraparound, the best shift per template, and the fused top-N (arXiv 2111.07347,
// Section 2.2: templates are sparse, so the numerator is a sum over the template's spots;
// the denominators are precomputed; the template is slid along the azimuth with
// wraparound; the maximum Q and its angle are kept per template; the top N templates are
// returned).
//
// Design (GB300):
// * Shared memory holds only the polar rows the library uses (its distinct spot radii --
//   a few to a few tens of the 128 rows), column c of a row holding P'[c mod Nθ].  When the
//   rows fit twice over (pitch Nθ + 32 NB), shift block b of a spot at column t reads
//   columns t + 32 b + [0, 32) with no wrap test at all (one load and one FMA per block);
//   otherwise rows are padded by 32 columns and a block past the wrap reads 32 b - Nθ
//   further (a select per block).  Either way a warp's 32 consecutive shifts never split at
//   the wrap and never conflict on a bank.  The small footprint lets several CTAs share an
//   SM and leaves L1 to cache the library's spot lists.
// * A persistent CTA takes patterns from a global counter; its warps take 32-template
//   mask words from a shared counter.  One warp scores one template: lane L accumulates
//   shifts s = 32 b + L of every shift block b in registers; the template's spots arrive
//   in one lane-parallel load and are broadcast by shuffles; a spot costs, per block, one
//   shared-memory load and one FMA.  The bound is the shared-memory load path (one 4-byte
//   operand per multiply-add).
// * The best shift is only resolved (lowest shift among equal maxima) when the template
//   can enter the warp's top-N, or when per-template results are requested.
// Results do not depend on scheduling: a template's sum runs over its spots in CSR order
// and ranking uses the total order (Q desc, template asc).
#include <float.h>
#include <limits.h>

#include "tm_internal.h"

namespace tmgb {

namespace {

// Shift blocks per template are rounded up to one of a few unrolled kernels.
__host__ __device__ constexpr int round_nb(int nb) {
    return nb <= 4 ? nb : nb <= 6 ? 6 : nb <= 8 ? 8 : nb <= 12 ? 12 : nb <= 16 ? 16 : nb <= 24 ? 24 : 32;
}

constexpr int kMaxThreads = 512;            // block sizes: 128, 256 (default) or 512
constexpr int kMaxWarps = kMaxThreads / 32;

}  // namespace

// Row pitch of the polar rows in shared memory, column c holding P'[c mod n_theta].
// Wrap-free layout: block b of a spot at column t reads t + 32 b + [0, 32) for b < NB (NB the
// widest rounded block count), so the pitch is n_theta + 32 NB.  Wrapped layout: blocks past
// the wrap read n_theta columns earlier, so n_theta + 32 columns and every column 32 NB - 1
// suffice.
int sparse_pitch(int n_theta, bool wrap_free) {
    const int nb = round_nb((n_theta + 31) / 32);
    if (wrap_free) return n_theta + 32 * nb;
    const int a = n_theta + 32, b = 32 * nb;
    return a > b ? a : b;
}

namespace {

__device__ __forceinline__ bool better(float qa, int ka, float qb, int kb) {
    return qa > qb || (qa == qb && ka < kb);
}

// Adds spot (px, I) to the accumulators: block b of lane L holds shift 32 b + L.  FIRST
// initialises them instead.  px must be a real spot word: its wrap block w keeps every read
// inside the spot's row.
template <int NB, bool WF, bool FIRST>
__device__ __forceinline__ void add_spot(float (&acc)[NB], const float* __restrict__ sP, int px, float I, int pitch,
                                         int n_theta, int lane) {
    const int t = px & 0x7ff;
    const int row = (px >> 11) & 0x1fff;
    const float* p1 = sP + row * pitch + t + lane;
    if (WF) {
#pragma unroll
        for (int b = 0; b < NB; ++b) acc[b] = FIRST ? I * p1[32 * b] : fmaf(I, p1[32 * b], acc[b]);
    } else {
        const int w = (int)((unsigned)px >> 24);
        const float* p2 = p1 - n_theta;                       // blocks b >= w: wrapped
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const float v = (b < w ? p1 : p2)[32 * b];
            acc[b] = FIRST ? I * v : fmaf(I, v, acc[b]);
        }
    }
}

// Correlation C(s) of one template for all its shifts (warp-collective).  Returns the
// warp-wide maximum; when it reaches thr_c, *shift_out is the lowest shift attaining it
// and `resolved` is set.
template <int NB, bool WF, bool FULL = false>
__device__ __forceinline__ float score_template(const float* __restrict__ sP, const SparseLib& L, int beg, int end,
                                                int S, int n_theta, int pitch, int lane, float thr_c,
                                                int& shift_out, bool& resolved) {
    float acc[NB];
    int cnt = min(32, end - beg);
    if (cnt <= 0) {                                               // no spot on the grid: C = 0, no read
#pragma unroll
        for (int b = 0; b < NB; ++b) acc[b] = 0.0f;
        cnt = 0;
    }
    int2 mine = make_int2(0, 0);
    if (lane < cnt) mine = __ldg(L.spot + beg + lane);            // one lane-parallel load
    if (cnt > 0)
        add_spot<NB, WF, true>(acc, sP, __shfl_sync(0xffffffffu, mine.x, 0),
                               __int_as_float(__shfl_sync(0xffffffffu, mine.y, 0)), pitch, n_theta, lane);
    for (int i0 = beg, j = 1;;) {
        for (; j < cnt; ++j)
            add_spot<NB, WF, false>(acc, sP, __shfl_sync(0xffffffffu, mine.x, j),
                                    __int_as_float(__shfl_sync(0xffffffffu, mine.y, j)), pitch, n_theta, lane);
        i0 += 32;
        if (i0 >= end) break;
        cnt = min(32, end - i0);
        if (lane < cnt) mine = __ldg(L.spot + i0 + lane);
        j = 0;
    }
    // Every lane's block b holds C((32 b + lane) mod Nθ), computed by the same operations as the
    // shift it repeats (column c of a row holds P'[c mod Nθ]); so for a template slid over all
    // Nθ shifts (FULL: S == Nθ) the maximum needs no lane mask.  Otherwise shifts >= S are masked.
    float best = -FLT_MAX;
    if (FULL) {
#pragma unroll
        for (int b = 0; b < NB; ++b) best = fmaxf(best, acc[b]);
    } else {
#pragma unroll
        for (int b = 0; b < NB; ++b)
            if (32 * b + lane < S) best = fmaxf(best, acc[b]);
    }
    resolved = false;
    if (!__any_sync(0xffffffffu, best >= thr_c)) return best;    // cannot enter the top-N
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = fmaxf(best, __shfl_xor_sync(0xffffffffu, best, o));
    if (best >= thr_c) {
        int s = INT_MAX;
#pragma unroll
        for (int b = NB - 1; b >= 0; --b)
            if (32 * b + lane < S && acc[b] == best) s = 32 * b + lane;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s = min(s, __shfl_xor_sync(0xffffffffu, s, o));
        shift_out = s;
        resolved = true;
    }
    return best;
}

template <int NBMAX, bool WF>
__device__ __forceinline__ float score_dispatch(const float* sP, const SparseLib& L, int beg, int end, int S,
                                                int n_theta, int pitch, int lane, float thr_c, int& s, bool& res) {
    const int nb = (S + 31) >> 5;
    if (S == n_theta && round_nb(nb) == NBMAX)                 // the common case, tested first
        return score_template<NBMAX, WF, true>(sP, L, beg, end, S, n_theta, pitch, lane, thr_c, s, res);
    if (nb <= 1) return score_template<1, WF>(sP, L, beg, end, S, n_theta, pitch, lane, thr_c, s, res);
    if (nb <= 2) return score_template<2, WF>(sP, L, beg, end, S, n_theta, pitch, lane, thr_c, s, res);
    if (nb <= 3) return score_template<3, WF>(sP, L, beg, end, S, n_theta, pitch, lane, thr_c, s, res);
    if (nb <= 4) return score_template<4, WF>(sP, L, beg, end, S, n_theta, pitch, lane, thr_c, s, res);
    if (NBMAX >= 6 && nb <= 6) return score_template<(NBMAX >= 6 ? 6 : 1), WF>(sP, L, beg, end, S, n_theta, pitch, lane, thr_c, s, res);
    if (NBMAX >= 8 && nb <= 8) return score_template<(NBMAX >= 8 ? 8 : 1), WF>(sP, L, beg, end, S, n_theta, pitch, lane, thr_c, s, res);
    if (NBMAX >= 12 && nb <= 12) return score_template<(NBMAX >= 12 ? 12 : 1), WF>(sP, L, beg, end, S, n_theta, pitch, lane, thr_c, s, res);
    if (NBMAX >= 16 && nb <= 16) return score_template<(NBMAX >= 16 ? 16 : 1), WF>(sP, L, beg, end, S, n_theta, pitch, lane, thr_c, s, res);
    if (NBMAX >= 24 && nb <= 24) return score_template<(NBMAX >= 24 ? 24 : 1), WF>(sP, L, beg, end, S, n_theta, pitch, lane, thr_c, s, res);
    return score_template<(NBMAX >= 32 ? 32 : 1), WF>(sP, L, beg, end, S, n_theta, pitch, lane, thr_c, s, res);
}

template <int NBMAX, bool WF>
__global__ void __launch_bounds__(kMaxThreads, NBMAX <= 12 ? 2 : 1)
sparse_kernel(const SparseCall c) {
    extern __shared__ __align__(16) float smem[];
    const int n_theta = c.n_theta, pitch = c.pitch;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int kWarps = blockDim.x >> 5;
    const int N = c.top_n;
    float* sP = smem;                                        // [max_rad][pitch]
    float* lq = sP + (size_t)c.max_rad * pitch;              // [kWarps][N]
    int* lk = (int*)(lq + kWarps * N);                       // [kWarps][N]
    int* ls = lk + kWarps * N;                               // [kWarps][N]
    int* lcnt = ls + kWarps * N;                             // [kWarps]
    int* counter = lcnt + kWarps;                            // [1]
    int* s_pattern = counter + 1;                            // [1]

    for (;;) {
        __syncthreads();                                     // previous pattern fully done
        if (threadIdx.x == 0) *s_pattern = atomicAdd(c.pattern_counter, 1);
        __syncthreads();
        const int64_t p = *s_pattern;
        if (p >= c.n) break;
        const float* src = c.polar + (size_t)p * c.n_r * n_theta;
        const float pn = __ldg(c.pnorm + p);
        for (int li = 0; li < c.n_libs; ++li) {
            const SparseLib L = c.lib[li];
            // the library's polar rows, padded with wrapped columns
            for (int rr = warp; rr < L.n_rad; rr += kWarps) {
                const float* row = src + (size_t)__ldg(L.radii + rr) * n_theta;
                float* dst = sP + (size_t)rr * pitch;
                for (int col = lane; col < pitch; col += 32) {
                    int sc = col;
                    while (sc >= n_theta) sc -= n_theta;
                    dst[col] = __ldg(row + sc);
                }
            }
            if (threadIdx.x == 0) *counter = 0;
            if (threadIdx.x < kWarps) lcnt[threadIdx.x] = 0;
            __syncthreads();
            const uint32_t* mrow = c.mask[li] ? c.mask[li] + (size_t)p * L.words : nullptr;
            float* qo = c.q_out[li] ? c.q_out[li] + (size_t)p * L.K : nullptr;
            int32_t* so = c.s_out[li] ? c.s_out[li] + (size_t)p * L.K : nullptr;
            float* wq = lq + warp * N;
            int* wk = lk + warp * N;
            int* ws = ls + warp * N;
            const bool use_thr = !qo && c.hits;
            float qthr = -INFINITY;                          // the warp's N-th best Q once its list is full
            for (;;) {
                int wd = 0;
                if (lane == 0) wd = atomicAdd(counter, 1);
                wd = __shfl_sync(0xffffffffu, wd, 0);
                if (wd >= L.words) break;
                uint32_t m = mrow ? __ldg(mrow + wd) : 0xffffffffu;
                const int rem = L.K - wd * 32;
                if (rem < 32) m &= (1u << rem) - 1u;
                // per-lane metadata of the word's 32 templates (one round trip per word)
                const int kl = wd * 32 + lane;
                int beg_l = 0, end_l = 0, S_l = 1;
                float tn_l = 0.0f;
                if (lane < rem && ((m >> lane) & 1u)) {
                    beg_l = __ldg(L.off + kl);
                    end_l = __ldg(L.off + kl + 1);
                    S_l = __ldg(L.nshift + kl);
                    tn_l = __ldg(L.norm + kl);
                } else if (qo && lane < rem) {
                    qo[kl] = -INFINITY;
                    so[kl] = -1;
                }
                while (m) {
                    const int bit = __ffs(m) - 1;
                    m &= m - 1;
                    const int k = wd * 32 + bit;
                    const int beg = __shfl_sync(0xffffffffu, beg_l, bit);
                    const int end = __shfl_sync(0xffffffffu, end_l, bit);
                    const int S = __shfl_sync(0xffffffffu, S_l, bit);
                    const float tn = __shfl_sync(0xffffffffu, tn_l, bit);
                    const float d = pn * tn;
                    // a template whose correlation stays below the warp's N-th best (in
                    // correlation units, with a margin for the division's rounding) cannot
                    // enter the top-N, so its best shift is not resolved
                    float thr_c = -FLT_MAX;
                    if (use_thr && qthr > -INFINITY && d > 0.0f) {
                        const float t = qthr * d;
                        thr_c = t - fabsf(t) * 1e-6f;
                    }
                    int s = 0;
                    bool resolved = false;
                    const float best = score_dispatch<NBMAX, WF>(sP, L, beg, end, S, n_theta, pitch, lane, thr_c, s,
                                                                 resolved);
                    if (!resolved) continue;
                    float q;
                    if (d > 0.0f) q = __fdiv_rn(best, d);
                    else { q = 0.0f; s = 0; }
                    if (lane == 0) {
                        if (qo) { qo[k] = q; so[k] = s; }
                        if (c.hits) {
                            const int cnt = lcnt[warp];
                            if (cnt < N || better(q, k, wq[N - 1], wk[N - 1])) {
                                int i = cnt < N ? cnt : N - 1;
                                while (i > 0 && better(q, k, wq[i - 1], wk[i - 1])) {
                                    wq[i] = wq[i - 1]; wk[i] = wk[i - 1]; ws[i] = ws[i - 1];
                                    --i;
                                }
                                wq[i] = q; wk[i] = k; ws[i] = s;
                                if (cnt < N) lcnt[warp] = cnt + 1;
                            }
                        }
                    }
                    __syncwarp();
                    if (use_thr) {
                        float nt = -INFINITY;
                        if (lane == 0 && lcnt[warp] >= N) nt = wq[N - 1];
                        qthr = __shfl_sync(0xffffffffu, nt, 0);
                    }
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

template <int NBMAX, bool WF>
cudaError_t launch_nb(const SparseCall& c, int num_sms, size_t smem, cudaStream_t st) {
    const int threads = (c.threads == 128 || c.threads == 512) ? c.threads : 256;
    cudaError_t e = cudaFuncSetAttribute(sparse_kernel<NBMAX, WF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sparse_kernel<NBMAX, WF>, threads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int64_t grid = (int64_t)num_sms * per_sm;
    if (grid > c.n) grid = c.n;
    e = cudaMemsetAsync(c.pattern_counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    sparse_kernel<NBMAX, WF><<<(int)grid, threads, smem, st>>>(c);
    return cudaGetLastError();
}

}  // namespace

// Layout for a call: the wrap-free rows when they fit in kWrapFreeBytes (several CTAs per
// SM), else the wrapped rows; 0 when even those do not fit.
constexpr size_t kWrapFreeBytes = 100 * 1024;

size_t sparse_smem_bytes(int max_rad, int n_theta, int top_n, bool* wrap_free, int* pitch) {
    if (n_theta < 1 || n_theta > 1024 || top_n < 1 || top_n > TM_MAX_TOPN || max_rad < 1) return 0;
    const size_t lists = (size_t)kMaxWarps * top_n * 12 + kMaxWarps * 4 + 16;
    for (int wf = 1; wf >= 0; --wf) {
        const int pch = sparse_pitch(n_theta, wf != 0);
        const size_t b = (size_t)max_rad * pch * 4 + lists;
        if ((wf && b <= kWrapFreeBytes) || (!wf && b <= 232448)) {
            if (wrap_free) *wrap_free = wf != 0;
            if (pitch) *pitch = pch;
            return b;
        }
    }
    return 0;
}

cudaError_t launch_sparse(const SparseCall& call, int num_sms, cudaStream_t st) {
    if (call.n <= 0) return cudaSuccess;
    bool wf = false;
    int pitch = 0;
    const size_t smem = sparse_smem_bytes(call.max_rad, call.n_theta, call.top_n, &wf, &pitch);
    if (!smem) return cudaErrorInvalidValue;
    SparseCall c = call;
    c.pitch = pitch;
    const int nbmax = (c.n_theta + 31) / 32;
    if (wf) {
        if (nbmax <= 6) return launch_nb<6, true>(c, num_sms, smem, st);
        if (nbmax <= 12) return launch_nb<12, true>(c, num_sms, smem, st);
        if (nbmax <= 24) return launch_nb<24, true>(c, num_sms, smem, st);
        return launch_nb<32, true>(c, num_sms, smem, st);
    }
    if (nbmax <= 6) return launch_nb<6, false>(c, num_sms, smem, st);
    if (nbmax <= 12) return launch_nb<12, false>(c, num_sms, smem, st);
    if (nbmax <= 24) return launch_nb<24, false>(c, num_sms, smem, st);
    return launch_nb<32, false>(c, num_sms, smem, st);
}

}  // namespace tmgb
