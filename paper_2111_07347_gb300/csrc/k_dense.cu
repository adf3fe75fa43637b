// BF16 tensor-core pre-score, stage B: the inverse angular DFT on tcgen05 with the maximum
// over shifts fused into the epilogue.
//
// The correlation of Eq. 1 along the azimuth is evaluated through the correlation theorem
// (the FFT cross-correlation alternative the paper names in Section 2.2's complexity
// paragraph):
//   C[k, s] = sum_{m=0}^{H} (w_m / n) Re( G[k, m] e^{2 pi i m s / n} ),  H = n / 2,
//   G[k, m] = sum_r conj(T^_k[r, m]) P^[r, m],
// with T^ and P^ the angular DFTs of the template (divided by |T_k|) and of the polar pattern
// (divided by |P|), so C is Q directly.  Stage A (G, a GEMM per frequency over the radii) runs
// before this kernel and leaves G in global memory as BF16, frequency-major:
//   G[j][p][c][k]  (slot j, pattern p of the batch, c = 0 real / 1 imaginary, template k),
// slot j < 96 holding m = 2 j and slot j >= 96 holding m = 2 (j - 96) + 1.  A radix-2 split
// halves this kernel's work: with E[s] the even-m part and O[s] the odd-m part of the sum for
// s < H, C[s] = E[s] + O[s] and C[s + H] = E[s] - O[s], so max(C[s], C[s + H]) = E[s] + |O[s]|.
// Per (pattern, tile of 128 templates) one GEMM [128 x 384] x [384 x 192] gives E (TMEM columns
// 0..191, K = slots 0..95) and O (columns 192..383, K = slots 96..191).
//
// Operands: A = G read by TMA as MN-major tiles (template index contiguous; 64 K-rows of 2 x 64
// templates per ring slot, 128-byte swizzle); B = the inverse-DFT basis (w_m / n) cos / -sin,
// K-major, resident in shared memory.  CTA (persistent over (pattern, tile) units, 384 threads):
//   warp 0 lane 0  TMA producer into a 4-slot ring;
//   warp 1 lane 0  MMA issuer (tcgen05.mma.cta_group::1.kind::f16, BF16 x BF16 -> FP32 in TMEM);
//   warp 2         TMEM allocation;
//   warps 4-11     epilogue: two warps per TMEM lane quadrant (32 templates), each reading half
//                  of the shift columns of E and O (tcgen05.ld) and taking their maximum; the
//                  halves are combined in shared memory and one pre-score per (pattern, template)
//                  is written to global memory (masked-out templates: -NaN).
// Every mbarrier wait is bounded by the global timer (1 s); on timeout the CTA records an error
// in a device word, stops its roles, lets the copies and MMAs it issued finish, releases TMEM
// and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <float.h>
#include <math.h>

#include "tm_internal.h"

namespace tmgb {
namespace {

constexpr int kRows = 128;                 // templates per tile (MMA M)
constexpr int kN = 192;                    // shifts per half (MMA N), >= n_theta / 2
constexpr int kKB = 384;                   // K: 192 even-m + 192 odd-m (slot, re/im) elements
constexpr int kChunk = 64;                 // K rows per ring slot
constexpr int kChunks = kKB / kChunk;      // 6
constexpr int kBoxBytes = 64 * kChunk * 2; // 8 KB: 64 templates x 64 K rows
constexpr int kSlotBytes = 2 * kBoxBytes;  // 16 KB
constexpr int kStages = 4;
constexpr int kBasisChunkBytes = kN * 128; // 24 KB
constexpr int kEpiWarp0 = 4;
constexpr int kEpiWarps = 8;               // two per TMEM lane quadrant, each half of the shift columns
constexpr int kEpiThreads = kEpiWarps * 32;
constexpr int kThreads = (kEpiWarp0 + kEpiWarps) * 32;
constexpr unsigned long long kTimeoutNs = 1000000000ull;   // 1 s per wait

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

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

__device__ __forceinline__ void mbar_expect_tx(uint32_t addr, uint32_t bytes) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(addr),
                 "r"(bytes)
                 : "memory");
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

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void named_bar(int id, int count) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// 4-D tiled TMA load (coordinates innermost first) completing on an mbarrier.
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
        "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(mbar)
        : "memory");
}

// Shared-memory matrix descriptors (128-byte swizzle).  K-major: rows of 64 K-elements, 8-row
// groups 1024 B apart.  MN-major: rows of 64 MN-elements (one per K index), 8 K-rows 1024 B
// apart (stride dimension), 64-element MN blocks `mn_stride` bytes apart (leading dimension).
__device__ __forceinline__ uint64_t sdesc_kmajor(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}
__device__ __forceinline__ uint64_t sdesc_mnmajor(uint32_t saddr, uint32_t mn_stride) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((mn_stride >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor: kind::f16, A = B = BF16, D = F32, A MN-major (bit 15), B K-major.
__host__ __device__ constexpr uint32_t idesc_bf16_amn(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
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

__global__ void __launch_bounds__(kThreads, 1) dense_kernel(const __grid_constant__ CUtensorMap gmap, const DenseCall c) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* s_basis = base;                                   // kChunks x [kN rows x 128 B]
    uint8_t* s_ring = s_basis + kChunks * kBasisChunkBytes;    // kStages x 16 KB
    uint64_t* bar = (uint64_t*)(s_ring + kStages * kSlotBytes);  // full[S], empty[S], acc_full, acc_empty
    uint32_t* s_tmem = (uint32_t*)(bar + 2 * kStages + 2);
    int* s_abort = (int*)(s_tmem + 1);
    int* s_epi_stop = s_abort + 1;                             // [2], by unit parity
    float* s_part = (float*)(s_epi_stop + 2);                  // [2 halves][kRows] partial maxima
    volatile int* abort_flag = s_abort;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int H = c.n_theta / 2;
    const int tiles = (c.K + kRows - 1) / kRows;
    const int64_t units = c.n * (int64_t)tiles;
    const uint32_t bar_full0 = smem_u32(&bar[0]), bar_empty0 = smem_u32(&bar[kStages]);
    const uint32_t bar_accf = smem_u32(&bar[2 * kStages]), bar_acce = smem_u32(&bar[2 * kStages + 1]);

    // ---- one-time setup: the basis, swizzled (16-byte chunk q of row r at (q ^ (r & 7)))
    for (int i = threadIdx.x; i < kChunks * kN * 8; i += blockDim.x) {
        const int cch = i / (kN * 8), rem = i - cch * kN * 8, n = rem >> 3, q = rem & 7;
        const uint4 v = *(const uint4*)((const __nv_bfloat16*)c.basis + (size_t)n * kKB + cch * kChunk + q * 8);
        *(uint4*)(s_basis + cch * kBasisChunkBytes + n * 128 + ((q ^ (n & 7)) << 4)) = v;
    }
    if (threadIdx.x == 0) {
        for (int i = 0; i < kStages; ++i) {
            mbar_init(smem_u32(&bar[i]), 1);
            mbar_init(smem_u32(&bar[kStages + i]), 1);
        }
        mbar_init(bar_accf, 1);
        mbar_init(bar_acce, kEpiThreads);
        *s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&gmap) : "memory");
    }
    if (warp == 2) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(s_tmem)),
                     "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fence_proxy_async();           // basis stores -> visible to the tensor-core (async) proxy
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *s_tmem;

    if (warp == 0) {
        // ================================================================ TMA producer
        if (lane == 0) {
            uint32_t g = 0;
            bool stop = false;
            for (int64_t u = blockIdx.x; u < units && !stop; u += gridDim.x) {
                const int p = (int)(u / tiles), t = (int)(u - (int64_t)p * tiles);
                for (int ch = 0; ch < kChunks; ++ch, ++g) {
                    const uint32_t slot = g % kStages, use = g / kStages;
                    if (!mbar_wait(bar_empty0 + 8 * slot, (use & 1u) ^ 1u, abort_flag)) {
                        *abort_flag = 1;
                        stop = true;
                        break;
                    }
                    const uint32_t full = bar_full0 + 8 * slot;
                    mbar_expect_tx(full, kSlotBytes);
                    const uint32_t dst = smem_u32(s_ring + slot * kSlotBytes);
                    tma_load_4d(dst, &gmap, t * kRows, 0, p, ch * (kChunk / 2), full);
                    tma_load_4d(dst + kBoxBytes, &gmap, t * kRows + 64, 0, p, ch * (kChunk / 2), full);
                }
            }
            // the copies issued last must land before the CTA exits (they complete on their own)
            volatile int never = 0;
            const uint32_t n_issued = g;
            for (uint32_t i = 0; i < kStages && i < n_issued; ++i) {
                const uint32_t gg = n_issued - 1 - i, slot = gg % kStages, use = gg / kStages;
                mbar_wait(bar_full0 + 8 * slot, use & 1u, &never);
            }
        }
    } else if (warp == 1) {
        // ================================================================ MMA issuer
        if (lane == 0 && !c.stall) {
            const uint32_t idesc = idesc_bf16_amn(kRows, kN);
            const uint32_t ring0 = smem_u32(s_ring), basis0 = smem_u32(s_basis);
            uint32_t g = 0, tt = 0;
            bool stop = false, issued = false;
            uint32_t last_bar = 0, last_par = 0;
            for (int64_t u = blockIdx.x; u < units && !stop; u += gridDim.x, ++tt) {
                if (!mbar_wait(bar_acce, (tt & 1u) ^ 1u, abort_flag)) {
                    *abort_flag = 1;
                    break;
                }
                tc_fence_after();
                for (int ch = 0; ch < kChunks; ++ch, ++g) {
                    const uint32_t slot = g % kStages, use = g / kStages;
                    if (!mbar_wait(bar_full0 + 8 * slot, use & 1u, abort_flag)) {
                        *abort_flag = 1;
                        stop = true;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t d = tmem + (ch < kChunks / 2 ? 0u : (uint32_t)kN);
#pragma unroll
                    for (int ks = 0; ks < kChunk / 16; ++ks) {
                        const uint64_t a = sdesc_mnmajor(ring0 + slot * kSlotBytes + ks * 2048, kBoxBytes);
                        const uint64_t b = sdesc_kmajor(basis0 + ch * kBasisChunkBytes + ks * 32);
                        mma_bf16(d, a, b, idesc, (ch % (kChunks / 2) == 0 && ks == 0) ? 0u : 1u);
                    }
                    mma_commit(bar_empty0 + 8 * slot);
                    last_bar = bar_empty0 + 8 * slot;
                    last_par = use & 1u;
                    issued = true;
                }
                if (stop) break;
                mma_commit(bar_accf);
            }
            if (stop && issued) {
                // let the MMAs already issued finish before TMEM is released
                volatile int never = 0;
                mbar_wait(last_bar, last_par, &never);
            }
        }
    } else if (warp >= kEpiWarp0) {
        // ================================================================ epilogue (warps 4-11)
        const int ew = warp - kEpiWarp0;
        const int quad = warp & 3, half = ew >> 2;            // TMEM lanes 32 quad.., shift columns by half
        const int row = quad * 32 + lane;
        const int et = ew * 32 + lane;                         // epilogue thread index
        const uint32_t tbase = tmem + ((uint32_t)(quad * 32) << 16);
        constexpr int kBlocks = kN / 32 / 2;                   // 32-column blocks per half
        uint32_t tt = 0;
        for (int64_t u = blockIdx.x; u < units; u += gridDim.x, ++tt) {
            const int p = (int)(u / tiles), t = (int)(u - (int64_t)p * tiles);
            // one thread waits and publishes one decision (a word per unit parity, so the next
            // unit's write cannot overtake a slow reader of this one)
            if (et == 0) {
                const bool ok = mbar_wait(bar_accf, tt & 1u, abort_flag);
                if (!ok) *abort_flag = 1;
                s_epi_stop[tt & 1u] = (!ok || *abort_flag) ? 1 : 0;
            }
            named_bar(1, kEpiThreads);
            if (*(volatile int*)&s_epi_stop[tt & 1u]) break;
            tc_fence_after();
            float best = -FLT_MAX;
#pragma unroll 1
            for (int b = 0; b < kBlocks; ++b) {
                const int cb = half * kBlocks + b;
                float e[32], o[32];
                tmem_ld32(tbase + cb * 32, e);
                tmem_ld32(tbase + kN + cb * 32, o);
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    if (cb * 32 + j < H) best = fmaxf(best, e[j] + fabsf(o[j]));
            }
            tc_fence_before();
            mbar_arrive(bar_acce);
            s_part[half * kRows + row] = best;
            named_bar(2, kEpiThreads);
            const int k = t * kRows + row;
            if (half == 0 && k < c.K) {
                best = fmaxf(best, s_part[kRows + row]);
                const int64_t p_glob = c.p0 + p;
                bool keep = true;
                if (c.mask) keep = (c.mask[p_glob * c.words + (k >> 5)] >> (k & 31)) & 1u;
                c.pre[p_glob * c.K + k] = keep ? best : __int_as_float(0xFFFFFFFF);
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (*abort_flag && threadIdx.x == 0) atomicOr(c.error, 1u);
    if (warp == 2) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
    }
}

}  // namespace

size_t dense_smem_bytes() {
    return 1024 + (size_t)kChunks * kBasisChunkBytes + (size_t)kStages * kSlotBytes + (2 * kStages + 2) * 8 + 16 +
           2 * kRows * 4;
}

bool dense_supported(int n_theta) { return n_theta % 2 == 0 && n_theta >= 4 && n_theta / 2 <= kN && (n_theta / 2) / 2 + 1 <= kN / 2; }

int dense_basis_rows() { return kN; }
int dense_basis_cols() { return kKB; }
int dense_slots() { return kKB / 2; }

cudaError_t launch_dense(const void* tmap, const DenseCall& c, int num_sms, cudaStream_t st) {
    if (c.n <= 0 || c.K <= 0) return cudaSuccess;
    const size_t smem = dense_smem_bytes();
    const cudaError_t e = kernel_occupancy((const void*)dense_kernel, kThreads, smem, nullptr);
    if (e != cudaSuccess) return e;
    const int64_t units = c.n * (int64_t)((c.K + kRows - 1) / kRows);
    int64_t grid = num_sms;
    if (grid > units) grid = units;
    dense_kernel<<<(int)grid, kThreads, smem, st>>>(*(const CUtensorMap*)tmap, c);
    return cudaGetLastError();
}

}  // namespace tmgb
