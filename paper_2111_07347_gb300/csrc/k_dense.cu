// BF16 tensor-core pre-score (tcgen05, TMEM accumulators) of the correlation index.
//
// The correlation of Eq. 1 along the azimuth is evaluated through the correlation theorem
// (the FFT cross-correlation alternative the paper names in Section 2.2's complexity
// paragraph):
//   C[k, s] = sum_{m=0}^{H} (w_m / n) Re( G[k, m] e^{2 pi i m s / n} ),  H = n / 2,
//   G[k, m] = sum_{spots i of k} I_i e^{+2 pi i m t_i / n} P^[r_i, m]   (= sum_r conj(T^) P^).
// Templates are sparse (a few spots), so G is built on CUDA cores from the spot list; the
// dense part -- the inverse transform over all frequencies for every shift, 2 x 192 x 384
// multiply-adds per template against 2 x 192 for the sparse sum's inner loop -- runs on
// the tensor cores.  A radix-2 split halves it: with E[s] the even-m part and O[s] the
// odd-m part of the sum for s < H, C[s] = E[s] + O[s] and C[s + H] = E[s] - O[s], so one
// 128 x 192 x 384 BF16 GEMM per 128 templates gives all n shifts (E and O live in TMEM
// columns [0, 192) and [192, 384)).
//
// CTA layout (one per SM, persistent over patterns; 672 threads):
//   warps 0-15 producers: four threads per row (one template) of G, eight frequencies each
//              per 64-element chunk, in BF16, into a 2-slot shared-memory ring
//              (128B-swizzled K-major); four warps per scheduler hide the latency of the
//              twiddle recurrence; each warp waits for a free slot on its own;
//   warp  20   TMEM allocation and the single MMA-issuing thread;
//   warps 16-19 epilogue: tcgen05.ld of E and O, max over all n shifts, one pre-score
//              per (pattern, template) written to global memory (the candidates are
//              then chosen by the exact radix select and rescored in FP32).
// The basis (w_m / n) cos / -sin for both halves stays resident in shared memory.
// Every mbarrier wait is bounded by the global timer (1 s); on timeout the CTA records an error
// in a device word, stops its roles uniformly, releases TMEM and returns.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <float.h>
#include <limits.h>

#include "tm_internal.h"

namespace tmgb {
namespace {

constexpr int kRows = 128;                 // templates per tile (MMA M)
constexpr int kN = 192;                    // shifts per half (MMA N), >= n_theta / 2
constexpr int kKB = 384;                   // K: 192 even-m + 192 odd-m elements
constexpr int kChunk = 64;                 // K per ring slot (one 128-byte swizzle row)
constexpr int kChunks = kKB / kChunk;      // 6
constexpr int kSlotBytes = kRows * 128;    // 16 KB
constexpr int kBasisChunkBytes = kN * 128; // 24 KB
constexpr int kProdWarps = 16;             // 4 threads per row, 8 frequencies each
constexpr int kProdThreads = kProdWarps * 32;
constexpr int kEpiWarp0 = kProdWarps;      // 4 epilogue warps
constexpr int kMmaWarp = kProdWarps + 4;
constexpr int kThreads = (kMmaWarp + 1) * 32;
constexpr unsigned long long kTimeoutNs = 1000000000ull;   // 1 s per wait

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t addr, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(addr), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t addr) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(addr) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t addr, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(addr), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait; false on timeout or when another role has aborted.
__device__ bool mbar_wait(uint32_t addr, uint32_t parity, volatile int* abort_flag) {
    uint64_t t0 = 0;
    for (uint32_t it = 0;; ++it) {
        if (mbar_try(addr, parity)) return true;
        if ((it & 255u) == 255u) {
            if (*abort_flag) return false;
            const uint64_t t = globaltimer();
            if (t0 == 0) t0 = t;
            else if (t - t0 > kTimeoutNs) return false;
        }
    }
}

__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void named_bar(int id, int count) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;                      // leading byte offset (unused for this layout)
    d |= (uint64_t)(1024 >> 4) << 32;            // stride byte offset between 8-row groups
    d |= (uint64_t)1 << 46;                      // descriptor version
    d |= (uint64_t)2 << 61;                      // 128-byte swizzle
    return d;
}

// Instruction descriptor: kind::f16, A = B = BF16, D = F32, both K-major, M = 128, N = 192.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

struct Smem {
    uint8_t* basis;       // kChunks x [kN rows x 128 B], swizzled
    uint8_t* ring;        // 2 x [kRows x 128 B], swizzled
    __half2* phat;        // [n_rad][n_freq]
    float2* tw;           // [n_theta]
    int16_t* rmap;        // [n_r]
    uint64_t* bar;        // full[2], empty[2], acc_full, acc_empty
    uint32_t* tmem_base;
    int* abort_flag;
    int* prod_stop;       // producers' uniform stop decision, published at pattern boundaries
    int* epi_stop;        // [2] epilogue's uniform stop decision, by tile parity
};

// Template row of tile t of (lib, pattern p), or -1 past the survivors.
__device__ __forceinline__ int row_template(const DenseCall& c, int li, int64_t p, int row) {
    if (row >= c.count[li]) return -1;
    const int32_t* lst = c.list[li];
    return lst ? lst[(size_t)p * c.count[li] + row] : c.lib[li].order[row];
}

__global__ void __launch_bounds__(kThreads, 1) dense_kernel(const DenseCall c) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    Smem s;
    s.basis = base;
    s.ring = s.basis + kChunks * kBasisChunkBytes;
    s.phat = (__half2*)(s.ring + 2 * kSlotBytes);
    s.tw = (float2*)(((uintptr_t)(s.phat + (size_t)c.n_rad * c.n_freq) + 15) & ~(uintptr_t)15);
    s.rmap = (int16_t*)(s.tw + c.n_theta);
    s.bar = (uint64_t*)(((uintptr_t)(s.rmap + c.n_r) + 15) & ~(uintptr_t)15);
    s.tmem_base = (uint32_t*)(s.bar + 6);
    s.abort_flag = (int*)(s.tmem_base + 1);
    s.prod_stop = s.abort_flag + 1;
    s.epi_stop = s.prod_stop + 1;
    volatile int* abort_flag = s.abort_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_theta = c.n_theta, H = n_theta / 2;
    const uint32_t bar_full0 = smem_u32(&s.bar[0]), bar_empty0 = smem_u32(&s.bar[2]);
    const uint32_t bar_accf = smem_u32(&s.bar[4]), bar_acce = smem_u32(&s.bar[5]);

    // ---- one-time setup
    for (int i = threadIdx.x; i < kChunks * kN * 8; i += blockDim.x) {
        const int cch = i / (kN * 8), rem = i - cch * kN * 8, n = rem >> 3, q = rem & 7;
        const uint4 v = *(const uint4*)((const __nv_bfloat16*)c.basis + (size_t)n * kKB + cch * kChunk + q * 8);
        *(uint4*)(s.basis + cch * kBasisChunkBytes + n * 128 + ((q ^ (n & 7)) << 4)) = v;
    }
    for (int i = threadIdx.x; i < n_theta; i += blockDim.x) s.tw[i] = c.twiddle[i];
    for (int i = threadIdx.x; i < c.n_r; i += blockDim.x) s.rmap[i] = (int16_t)c.rmap[i];
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&s.bar[0]), kProdThreads);
        mbar_init(smem_u32(&s.bar[1]), kProdThreads);
        mbar_init(smem_u32(&s.bar[2]), 1);
        mbar_init(smem_u32(&s.bar[3]), 1);
        mbar_init(bar_accf, 1);
        mbar_init(bar_acce, kRows);
        *s.abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(s.tmem_base)),
                     "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fence_proxy_async();           // basis stores -> visible to the tensor-core (async) proxy
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *s.tmem_base;

    if (warp < kProdWarps) {
        // ================================================================ producers
        const int row = threadIdx.x & (kRows - 1);
        const int quarter = threadIdx.x >> 7;                    // frequencies 8 q .. 8 q + 7 of a chunk
        uint32_t g = 0;                                         // global chunk counter
        bool stop = false;
        for (int64_t p = blockIdx.x; p < c.n; p += gridDim.x) {
            // all producer warps reach this point (a warp that saw a failed wait skips the rest
            // of its pattern instead of leaving); thread 0 publishes one stop decision
            named_bar(1, kProdThreads);                         // previous pattern's P^ no longer read
            if (threadIdx.x == 0) *s.prod_stop = *abort_flag;
            named_bar(1, kProdThreads);
            if (*(volatile int*)s.prod_stop) break;
            const __half2* src = (const __half2*)c.phat + (size_t)p * c.n_rad * c.n_freq;
            for (int i = threadIdx.x; i < c.n_rad * c.n_freq; i += kProdThreads) s.phat[i] = src[i];
            named_bar(1, kProdThreads);
            for (int li = 0; li < c.n_libs; ++li) {
                const DenseLib& L = c.lib[li];
                const int tiles = (c.count[li] + kRows - 1) / kRows;
                for (int t = 0; t < tiles; ++t) {
                    const int k = row_template(c, li, p, t * kRows + row);
                    int beg = 0, end = 0;
                    float inv_norm = 0.0f;
                    if (k >= 0) {
                        beg = L.off[k];
                        end = L.off[k + 1];
                        const float nk = L.norm[k];
                        inv_norm = nk > 0.0f ? 1.0f / nk : 0.0f;
                    }
                    for (int ch = 0; ch < kChunks; ++ch, ++g) {
                        const uint32_t slot = g & 1u, use = g >> 1;
                        // each warp waits for the slot on its own (no block-wide barrier per chunk);
                        // warps drift at most the ring depth apart, since a slot is only freed
                        // once every producer thread has filled it
                        if (stop) continue;                      // skipping to the pattern boundary
                        int ok = 1;
                        if (lane == 0) ok = mbar_wait(bar_empty0 + 8 * slot, (use & 1u) ^ 1u, abort_flag) ? 1 : 0;
                        ok = __shfl_sync(0xffffffffu, ok, 0);
                        if (!ok) { *abort_flag = 1; stop = true; continue; }
                        const int part = ch / 3;                   // 0: even m, 1: odd m
                        const int m0 = 2 * ((ch % 3) * 32 + quarter * 8) + part;
                        int nvalid = (H - m0) / 2 + 1;             // frequencies m0 + 2 jj <= H
                        if (m0 > H) nvalid = 0;
                        if (nvalid > 8) nvalid = 8;
                        float are[8], aim[8];
#pragma unroll
                        for (int jj = 0; jj < 8; ++jj) { are[jj] = 0.0f; aim[jj] = 0.0f; }
                        if (nvalid > 0) {
                            for (int i = beg; i < end; ++i) {
                                const int rt = L.rt[i];
                                const int r = rt & 0xffff, tt = rt >> 16;
                                const float I = __int_as_float(L.spot[i].y) * inv_norm;
                                const __half2* ph = s.phat + (size_t)s.rmap[r] * c.n_freq + m0;
                                float2 w = s.tw[(m0 * tt) % n_theta];
                                w.x *= I;
                                w.y *= I;
                                const float2 st = s.tw[(2 * tt) % n_theta];
#pragma unroll
                                for (int jj = 0; jj < 8; ++jj) {
                                    if (jj < nvalid) {
                                        const float2 pv = __half22float2(ph[2 * jj]);
                                        are[jj] = fmaf(w.x, pv.x, fmaf(-w.y, pv.y, are[jj]));
                                        aim[jj] = fmaf(w.x, pv.y, fmaf(w.y, pv.x, aim[jj]));
                                        const float wx = w.x * st.x - w.y * st.y;
                                        w.y = fmaf(w.x, st.y, w.y * st.x);
                                        w.x = wx;
                                    }
                                }
                            }
                        }
                        uint8_t* dst = s.ring + slot * kSlotBytes + row * 128;
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const int q = 2 * quarter + h;              // 16-byte chunk of the row
                            uint4 v;
                            __nv_bfloat162 b0 = __floats2bfloat162_rn(are[4 * h + 0], aim[4 * h + 0]);
                            __nv_bfloat162 b1 = __floats2bfloat162_rn(are[4 * h + 1], aim[4 * h + 1]);
                            __nv_bfloat162 b2 = __floats2bfloat162_rn(are[4 * h + 2], aim[4 * h + 2]);
                            __nv_bfloat162 b3 = __floats2bfloat162_rn(are[4 * h + 3], aim[4 * h + 3]);
                            v.x = *(uint32_t*)&b0;
                            v.y = *(uint32_t*)&b1;
                            v.z = *(uint32_t*)&b2;
                            v.w = *(uint32_t*)&b3;
                            *(uint4*)(dst + ((q ^ (row & 7)) << 4)) = v;
                        }
                        fence_proxy_async();
                        mbar_arrive(bar_full0 + 8 * slot);
                    }
                }
            }
        }
    } else if (warp == kMmaWarp) {
        // ================================================================ MMA issuer
        if (lane == 0 && !c.stall) {
            const uint32_t idesc = idesc_bf16(kRows, kN);
            const uint32_t ring0 = smem_u32(s.ring), basis0 = smem_u32(s.basis);
            uint32_t g = 0, tt = 0;
            bool stop = false;
            uint32_t last_bar = 0, last_par = 0;
            bool issued = false;
            for (int64_t p = blockIdx.x; p < c.n && !stop; p += gridDim.x) {
                for (int li = 0; li < c.n_libs && !stop; ++li) {
                    const int tiles = (c.count[li] + kRows - 1) / kRows;
                    for (int t = 0; t < tiles && !stop; ++t, ++tt) {
                        if (!mbar_wait(bar_acce, (tt & 1u) ^ 1u, abort_flag)) { *abort_flag = 1; stop = true; break; }
                        tc_fence_after();
                        for (int ch = 0; ch < kChunks; ++ch, ++g) {
                            const uint32_t slot = g & 1u, use = g >> 1;
                            if (!mbar_wait(bar_full0 + 8 * slot, use & 1u, abort_flag)) { *abort_flag = 1; stop = true; break; }
                            tc_fence_after();
                            const uint32_t d = tmem + (ch < 3 ? 0u : (uint32_t)kN);
#pragma unroll
                            for (int ks = 0; ks < kChunk / 16; ++ks) {
                                const uint64_t a = sdesc(ring0 + slot * kSlotBytes + ks * 32);
                                const uint64_t b = sdesc(basis0 + ch * kBasisChunkBytes + ks * 32);
                                mma_bf16(d, a, b, idesc, (ch % 3 == 0 && ks == 0) ? 0u : 1u);
                            }
                            mma_commit(bar_empty0 + 8 * slot);
                            last_bar = bar_empty0 + 8 * slot;
                            last_par = use & 1u;
                            issued = true;
                        }
                        if (stop) break;
                        mma_commit(bar_accf);
                    }
                }
            }
            if (stop && issued) {
                // let the MMAs already issued finish before TMEM is released
                volatile int never = 0;
                mbar_wait(last_bar, last_par, &never);
            }
        }
    } else {
        // ================================================================ epilogue (warps 16-19)
        const int ew = warp - kEpiWarp0;
        const int row = ew * 32 + lane;
        const uint32_t tbase = tmem + ((uint32_t)(ew * 32) << 16);
        uint32_t tt = 0;
        bool stop = false;
        for (int64_t p = blockIdx.x; p < c.n && !stop; p += gridDim.x) {
            for (int li = 0; li < c.n_libs && !stop; ++li) {
                const int tiles = (c.count[li] + kRows - 1) / kRows;
                float* out = c.pre[li] + (size_t)p * c.lib[li].K;
                for (int t = 0; t < tiles; ++t, ++tt) {
                    // row 0 waits and publishes one decision (a word per tile parity, so the
                    // next tile's write cannot overtake a slow reader of this one)
                    if (row == 0) {
                        const bool ok = mbar_wait(bar_accf, tt & 1u, abort_flag);
                        if (!ok) *abort_flag = 1;
                        s.epi_stop[tt & 1u] = (!ok || *abort_flag) ? 1 : 0;
                    }
                    named_bar(2, kRows);
                    if (*(volatile int*)&s.epi_stop[tt & 1u]) { stop = true; break; }
                    tc_fence_after();
                    float best = -FLT_MAX;
#pragma unroll 1
                    for (int cb = 0; cb < kN / 32; ++cb) {
                        float e[32], o[32];
                        tmem_ld32(tbase + cb * 32, e);
                        tmem_ld32(tbase + kN + cb * 32, o);
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            if (cb * 32 + j < H) best = fmaxf(best, fmaxf(e[j] + o[j], e[j] - o[j]));
                        }
                    }
                    tc_fence_before();
                    mbar_arrive(bar_acce);
                    const int k = row_template(c, li, p, t * kRows + row);
                    if (k >= 0) out[k] = best;
                }
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (*abort_flag && threadIdx.x == 0) atomicOr(c.error, 1u);
    if (warp == kMmaWarp) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
    }
}

}  // namespace

size_t dense_smem_bytes(int n_theta, int n_r, int n_rad, int n_freq) {
    size_t b = 1024;                                           // alignment slack
    b += (size_t)kChunks * kBasisChunkBytes + 2 * kSlotBytes;
    b += (size_t)n_rad * n_freq * 4 + 16 + (size_t)n_theta * 8 + (size_t)n_r * 2 + 16;
    b += 6 * 8 + 4 * 5 + 16;          // barriers, TMEM base, abort flag, stop words
    return b;
}

bool dense_supported(int n_theta) { return n_theta % 2 == 0 && n_theta / 2 <= kN && (n_theta / 2) / 2 + 1 <= kN / 2; }

int dense_basis_rows() { return kN; }
int dense_basis_cols() { return kKB; }

cudaError_t launch_dense(const DenseCall& c, int num_sms, cudaStream_t st) {
    if (c.n <= 0) return cudaSuccess;
    const size_t smem = dense_smem_bytes(c.n_theta, c.n_r, c.n_rad, c.n_freq);
    if (smem > 232448) return cudaErrorInvalidValue;
    const cudaError_t e = kernel_occupancy((const void*)dense_kernel, kThreads, smem, nullptr);
    if (e != cudaSuccess) return e;
    int64_t grid = num_sms;
    if (grid > c.n) grid = c.n;
    dense_kernel<<<(int)grid, kThreads, smem, st>>>(c);
    return cudaGetLastError();
}

}  // namespace tmgb
