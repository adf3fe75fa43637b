// Stage 3: the correlation index Q of Eq. 1 for every template at every azimuthal shift
// with wraparound, the best shift per template, and the fused top-N (arXiv 2111.07347,
// Section 2.2: templates are sparse, so the numerator is a sum over the template's spots;
// the denominators are precomputed; the template is slid along the azimuth with
// wraparound; the maximum Q and its angle are kept per template; the top N templates are
// returned).
//
// Design (GB300): a persistent CTA holds one pattern's polar image in shared memory with
// its rows extended by at least 32 wrapped columns (sparse_pitch), so a warp reading 32
// consecutive shifts of one spot never splits at the wrap and never conflicts on a bank.
// One warp scores one template: lane L accumulates shifts s = 32 b + L for every shift
// block b in registers; a spot costs one broadcast 8-byte load and, per block, one
// shared-memory load and one FMA.  The work bound is the shared-memory load path
// (one 4-byte operand per multiply-add).  Warps pull 32-template mask words from a
// shared counter; a per-warp sorted top-N list is merged at the end of the pattern.
// Results are independent of scheduling: the per-template sum runs over the spots in
// CSR order and ranking uses the total order (Q desc, template asc).
#include <float.h>
#include <limits.h>

#include "tm_internal.h"

namespace tmgb {

namespace {

// Shift blocks per template are rounded up to one of a few unrolled kernels.
__host__ __device__ constexpr int round_nb(int nb) {
    return nb <= 4 ? nb : nb <= 6 ? 6 : nb <= 8 ? 8 : nb <= 12 ? 12 : nb <= 16 ? 16 : nb <= 24 ? 24 : 32;
}

}  // namespace

// Row pitch of the polar image in shared memory.  Block b of a spot at column t reads
// columns t + 32 b + [0, 32) (or that minus n_theta once it wraps), so the pitch covers
// n_theta + 32 columns and every column 32 * NB - 1 that the widest rounded block count
// NB can touch; column c holds P'[c mod n_theta].
int sparse_pitch(int n_theta) {
    const int nb = round_nb((n_theta + 31) / 32);
    const int a = n_theta + 32, b = 32 * nb;
    return a > b ? a : b;
}

namespace {

__device__ __forceinline__ bool better(float qa, int ka, float qb, int kb) {
    return qa > qb || (qa == qb && ka < kb);
}

// Score template k against the polar image in shared memory (warp-collective).
template <int NB>
__device__ __forceinline__ void score_template(const float* __restrict__ sP, const SparseLib& L,
                                               int k, int n_theta, int lane, float& best_out,
                                               int& shift_out) {
    const int beg = __ldg(L.off + k), end = __ldg(L.off + k + 1);
    const int S = __ldg(L.nshift + k);
    float acc[NB];
    #pragma unroll
    for (int b = 0; b < NB; ++b) acc[b] = 0.0f;
    for (int i = beg; i < end; ++i) {
        const int2 sp = __ldg(L.spot + i);
        const int a = sp.x & 0xffffff;
        const int w = (int)((unsigned)sp.x >> 24);
        const float I = __int_as_float(sp.y);
        const float* p1 = sP + a + lane;           // blocks b < w: no wrap
        const float* p2 = p1 - n_theta;            // blocks b >= w: wrapped
        #pragma unroll
        for (int b = 0; b < NB; ++b) acc[b] = fmaf(I, (b < w ? p1 : p2)[32 * b], acc[b]);
    }
    float best = -FLT_MAX;
    int bs = INT_MAX;
    #pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int s = 32 * b + lane;
        if (s < S && acc[b] > best) { best = acc[b]; bs = s; }
    }
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int os = __shfl_xor_sync(0xffffffffu, bs, o);
        if (ob > best || (ob == best && os < bs)) { best = ob; bs = os; }
    }
    best_out = best;
    shift_out = bs;
}

template <int NBMAX>
__device__ __forceinline__ void score_dispatch(const float* sP, const SparseLib& L, int k,
                                               int n_theta, int lane, float& best, int& s) {
    const int nb = (__ldg(L.nshift + k) + 31) >> 5;
    if (nb <= 1) score_template<1>(sP, L, k, n_theta, lane, best, s);
    else if (nb <= 2) score_template<2>(sP, L, k, n_theta, lane, best, s);
    else if (nb <= 3) score_template<3>(sP, L, k, n_theta, lane, best, s);
    else if (nb <= 4) score_template<4>(sP, L, k, n_theta, lane, best, s);
    else if (NBMAX >= 6 && nb <= 6) score_template<(NBMAX >= 6 ? 6 : 1)>(sP, L, k, n_theta, lane, best, s);
    else if (NBMAX >= 8 && nb <= 8) score_template<(NBMAX >= 8 ? 8 : 1)>(sP, L, k, n_theta, lane, best, s);
    else if (NBMAX >= 12 && nb <= 12) score_template<(NBMAX >= 12 ? 12 : 1)>(sP, L, k, n_theta, lane, best, s);
    else if (NBMAX >= 16 && nb <= 16) score_template<(NBMAX >= 16 ? 16 : 1)>(sP, L, k, n_theta, lane, best, s);
    else if (NBMAX >= 24 && nb <= 24) score_template<(NBMAX >= 24 ? 24 : 1)>(sP, L, k, n_theta, lane, best, s);
    else score_template<(NBMAX >= 32 ? 32 : 1)>(sP, L, k, n_theta, lane, best, s);
}

template <int NBMAX>
__global__ void __launch_bounds__(1024)
sparse_kernel(const SparseCall c) {
    extern __shared__ __align__(16) float smem[];
    const int n_r = c.n_r, n_theta = c.n_theta, pitch = c.pitch;
    const int nw = blockDim.x >> 5;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int N = c.top_n;
    float* sP = smem;                                        // [n_r][pitch]
    float* lq = sP + (size_t)n_r * pitch;                    // [nw][N]
    int* lk = (int*)(lq + nw * N);                           // [nw][N]
    int* ls = lk + nw * N;                                   // [nw][N]
    int* lcnt = ls + nw * N;                                 // [nw]
    int* counter = lcnt + nw;                                // [1]

    for (int64_t p = blockIdx.x; p < c.n; p += gridDim.x) {
        __syncthreads();
        const float* src = c.polar + (size_t)p * n_r * n_theta;
        for (int j = warp; j < n_r; j += nw) {
            const float* row = src + (size_t)j * n_theta;
            float* dst = sP + (size_t)j * pitch;
            for (int col = lane; col < pitch; col += 32) {
                int sc = col;
                while (sc >= n_theta) sc -= n_theta;
                dst[col] = __ldg(row + sc);
            }
        }
        const float pn = __ldg(c.pnorm + p);
        for (int li = 0; li < c.n_libs; ++li) {
            const SparseLib L = c.lib[li];
            if (threadIdx.x == 0) *counter = 0;
            if (threadIdx.x < nw) lcnt[threadIdx.x] = 0;
            __syncthreads();
            const uint32_t* mrow = c.mask[li] ? c.mask[li] + (size_t)p * L.words : nullptr;
            float* qo = c.q_out[li] ? c.q_out[li] + (size_t)p * L.K : nullptr;
            int32_t* so = c.s_out[li] ? c.s_out[li] + (size_t)p * L.K : nullptr;
            const int32_t* crow = c.cand[li] ? c.cand[li] + (size_t)p * c.kc : nullptr;
            uint32_t m = 0;          // remaining bits of the current mask word (warp-uniform)
            int wd = 0;
            for (;;) {
                // next template: from the candidate list, or the next set bit of a mask word
                int k = -1;
                if (crow) {
                    int j = 0;
                    if (lane == 0) j = atomicAdd(counter, 1);
                    j = __shfl_sync(0xffffffffu, j, 0);
                    if (j >= c.kc) break;
                    k = __ldg(crow + j);
                    if (k < 0 || k >= L.K) continue;
                } else {
                    bool done = false;
                    while (m == 0) {
                        if (lane == 0) wd = atomicAdd(counter, 1);
                        wd = __shfl_sync(0xffffffffu, wd, 0);
                        if (wd >= L.words) { done = true; break; }
                        m = mrow ? __ldg(mrow + wd) : 0xffffffffu;
                        const int rem = L.K - wd * 32;
                        if (rem < 32) m &= (1u << rem) - 1u;
                        if (qo) {
                            const int kk = wd * 32 + lane;
                            if (lane < rem && !((m >> lane) & 1u)) { qo[kk] = -INFINITY; so[kk] = -1; }
                        }
                    }
                    if (done) break;
                    const int bit = __ffs(m) - 1;
                    m &= m - 1;
                    k = wd * 32 + bit;
                }
                float best;
                int s;
                score_dispatch<NBMAX>(sP, L, k, n_theta, lane, best, s);
                const float d = pn * __ldg(L.norm + k);
                float q;
                if (d > 0.0f) q = __fdiv_rn(best, d);
                else { q = 0.0f; s = 0; }
                if (lane == 0) {
                    if (qo) { qo[k] = q; so[k] = s; }
                    if (c.hits) {
                        float* wq = lq + warp * N;
                        int* wk = lk + warp * N;
                        int* ws = ls + warp * N;
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
            }
            __syncthreads();
            if (c.hits && warp == 0) {
                tm_hit* out = c.hits + (size_t)li * c.hits_lib_stride + (size_t)p * N;
                const int total = nw * N;
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

template <int NBMAX>
cudaError_t launch_nb(const SparseCall& c, int num_sms, size_t smem, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(sparse_kernel<NBMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    // 1024 threads when only one CTA fits per SM, else 512 (more CTAs per SM)
    int threads = smem > 110 * 1024 ? 1024 : 512;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sparse_kernel<NBMAX>, threads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) { threads = 512; e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sparse_kernel<NBMAX>, threads, smem); }
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int64_t grid = (int64_t)num_sms * per_sm;
    if (grid > c.n) grid = c.n;
    sparse_kernel<NBMAX><<<(int)grid, threads, smem, st>>>(c);
    return cudaGetLastError();
}

}  // namespace

size_t sparse_smem_bytes(int n_r, int n_theta, int top_n) {
    if (n_theta < 1 || n_theta > 1024 || top_n < 1 || top_n > TM_MAX_TOPN) return 0;
    const size_t nw = 32;   // lists sized for the largest block
    const size_t b = (size_t)n_r * sparse_pitch(n_theta) * 4 + nw * top_n * 12 + nw * 4 + 16;
    return b <= 232448 ? b : 0;
}

cudaError_t launch_sparse(const SparseCall& c, int num_sms, cudaStream_t st) {
    if (c.n <= 0) return cudaSuccess;
    const size_t smem = sparse_smem_bytes(c.n_r, c.n_theta, c.top_n);
    if (!smem) return cudaErrorInvalidValue;
    const int nbmax = (c.n_theta + 31) / 32;
    if (nbmax <= 6) return launch_nb<6>(c, num_sms, smem, st);
    if (nbmax <= 12) return launch_nb<12>(c, num_sms, smem, st);
    if (nbmax <= 24) return launch_nb<24>(c, num_sms, smem, st);
    return launch_nb<32>(c, num_sms, smem, st);
}

}  // namespace tmgb
