// Angular DFT of the polar images for the BF16 tensor-core path.
//
// The paper notes (Section 2.2, complexity paragraph) that the azimuthal cross-correlation
// can be computed through an FFT along phi instead of sliding the template.  The tensor-core
// path uses the correlation theorem along theta: with X^[r, m] = sum_theta X[r, theta]
// e^{-2 pi i m theta / n}, the correlation of template k with pattern P at shift s is
//   C[k, s] = sum_{m=0}^{n/2} (w_m / n) Re( G[k, m] e^{2 pi i m s / n} ),
//   G[k, m] = sum_r conj(T^_k[r, m]) P^[r, m]                (w = 1 at m = 0, n/2; else 2).
// The DFT itself is a TF32 GEMM of the polar images with the DFT matrix (cuBLAS, a plain
// library GEMM); this file packs its result, P^ / |P| for the radii one library uses, as BF16
// in the layout of stage A's GEMM (G = T^ x P^ per frequency slot, real arithmetic):
//   out[j][p][0][2 a + {0, 1}] = ( Re P^[r_a, m],  Im P^[r_a, m])   -> Re G column,
//   out[j][p][1][2 a + {0, 1}] = ( Im P^[r_a, m], -Re P^[r_a, m])   -> Im G column,
// for slot j (m = 2 j for j < 96, m = 2 (j - 96) + 1 for j >= 96; slots with m > n/2 and the
// rows a >= n_rad up to the padded count R are zero), so that with T^ stored as
// (Re T^, Im T^) pairs, Re G = sum_a (Re T^ Re P^ + Im T^ Im P^) and
// Im G = sum_a (Re T^ Im P^ - Im T^ Re P^).
#include <cuda_bf16.h>

#include "tm_internal.h"

namespace tmgb {
namespace {

constexpr int kSlots = 192;

__device__ __forceinline__ int slot_freq(int j) { return j < kSlots / 2 ? 2 * j : 2 * (j - kSlots / 2) + 1; }

// Packs the angular DFT of a batch into stage A's operand layout.  dftc [192][2][nb][n_r] FP32
// holds, for slot j, sum_theta P[p, r, theta] (cos, -sin)(2 pi m_j theta / n) for every polar row
// (a TF32 GEMM of the polar images with the DFT matrix, columns past n/2 zero); this kernel keeps
// the library's radii, divides by |P| and writes out[j][p][c][2 a + {0, 1}] as BF16.  A thread
// takes one (slot, pattern, row a); rows are fastest, so the writes of a warp are contiguous.
__global__ void __launch_bounds__(256)
pack_kernel(const float* __restrict__ dftc, const float* __restrict__ pnorm, int64_t nb, int n_r,
            const int32_t* __restrict__ radii, int n_rad, int R, __nv_bfloat162* __restrict__ out) {
    const int64_t total = (int64_t)kSlots * nb * R;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int a = (int)(idx % R);
        const int64_t jp = idx / R;
        const int64_t p = jp % nb;
        const int j = (int)(jp / nb);
        float re = 0.0f, im = 0.0f;
        if (a < n_rad) {
            const float pn = __ldg(pnorm + p);
            const float inv = pn > 0.0f ? 1.0f / pn : 0.0f;
            const int r = __ldg(radii + a);
            re = __ldg(dftc + ((size_t)(2 * j) * nb + p) * n_r + r) * inv;
            im = __ldg(dftc + ((size_t)(2 * j + 1) * nb + p) * n_r + r) * inv;
        }
        __nv_bfloat162* o = out + ((size_t)j * nb + p) * 2 * R;
        o[a] = __floats2bfloat162_rn(re, im);
        o[R + a] = __floats2bfloat162_rn(im, -re);
    }
}

// Template spectra for stage A (built once per library): out[j][2 a + {0, 1}][k] =
// (Re, Im) of T^_k[r_a, m] / |T_k| = sum over the spots i of k at radius r_a of
// (I_i / |T_k|) e^{-2 pi i m t_i / n}, BF16, rows a >= n_rad and slots with m > n/2 zero.
// A block takes 128 templates of one slot j; each thread adds its template's spots into its own
// column of a shared [2 R][128] FP32 image, which the block then writes row by row.
__global__ void __launch_bounds__(128)
spectra_kernel(const int32_t* __restrict__ off, const int32_t* __restrict__ rt, const int2* __restrict__ spot,
               const float* __restrict__ norm, const int32_t* __restrict__ rowmap, int K, int K_pad, int R,
               int n_theta, const float2* __restrict__ twiddle, __nv_bfloat16* __restrict__ out) {
    extern __shared__ float acc[];                     // [2 R][128]
    const int j = blockIdx.y, k0 = blockIdx.x * 128, k = k0 + threadIdx.x;
    const int m = slot_freq(j), H = n_theta / 2;
    for (int i = threadIdx.x; i < 2 * R * 128; i += 128) acc[i] = 0.0f;
    __syncthreads();
    if (k < K && m <= H) {
        const float nk = norm[k];
        const float inv = nk > 0.0f ? 1.0f / nk : 0.0f;
        for (int i = off[k]; i < off[k + 1]; ++i) {
            const int v = rt[i];
            const int r = v & 0xffff, t = v >> 16;
            const int a = rowmap[r];
            const float I = __int_as_float(spot[i].y) * inv;
            const float2 w = twiddle[(int)(((int64_t)m * t) % n_theta)];
            acc[(2 * a) * 128 + threadIdx.x] += I * w.x;
            acc[(2 * a + 1) * 128 + threadIdx.x] -= I * w.y;
        }
    }
    __syncthreads();
    if (k < K_pad)
        for (int row = 0; row < 2 * R; ++row)
            out[((size_t)j * 2 * R + row) * K_pad + k] = __float2bfloat16_rn(acc[row * 128 + threadIdx.x]);
}

}  // namespace

cudaError_t launch_spectra(const int32_t* off, const int32_t* rt, const int2* spot, const float* norm,
                           const int32_t* rowmap, int K, int K_pad, int R, int n_theta, const float2* twiddle,
                           void* out, cudaStream_t st) {
    if (K <= 0) return cudaSuccess;
    const size_t smem = (size_t)2 * R * 128 * 4;
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    const cudaError_t e = kernel_occupancy((const void*)spectra_kernel, 128, smem, nullptr);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((K_pad + 127) / 128), (unsigned)kSlots);
    spectra_kernel<<<grid, 128, smem, st>>>(off, rt, spot, norm, rowmap, K, K_pad, R, n_theta, twiddle,
                                            (__nv_bfloat16*)out);
    return cudaGetLastError();
}

cudaError_t launch_pack(const float* dftc, const float* pnorm, int64_t nb, int n_r, const int32_t* radii, int n_rad,
                        int R, void* out, int num_sms, cudaStream_t st) {
    if (nb <= 0) return cudaSuccess;
    const int64_t total = (int64_t)kSlots * nb * R;
    int64_t grid = (total + 255) / 256;
    if (grid > (int64_t)num_sms * 16) grid = (int64_t)num_sms * 16;
    pack_kernel<<<(int)grid, 256, 0, st>>>(dftc, pnorm, nb, n_r, radii, n_rad, R, (__nv_bfloat162*)out);
    return cudaGetLastError();
}

}  // namespace tmgb
