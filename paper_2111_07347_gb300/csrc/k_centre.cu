// Direct-beam centring (arXiv 2111.07347 Section 3.1: the direct beam of every pattern was
// centred before the polar transform, whose origin must be the beam's centre, Section 2.2).
// Per pattern, the intensity-weighted centre of mass of the pixels within `radius` of the
// current estimate, repeated `iterations` times from the starting centre.
//
// One thread per pattern visits the disc's bounding box row by row in FP64 with explicitly
// rounded operations (no fused multiply-adds), so the sums, and hence the centres, are the
// same bit for bit as a plain double-precision loop in the same order.  The work is a few
// hundred pixels per pattern; the frames' other pixels are not read.
#include "tm_internal.h"

namespace tmgb {
namespace {

template <typename T>
__global__ void find_centres_kernel(const T* __restrict__ frames, int64_t n, int H, int W, double cx0, double cy0,
                                    double radius, int iterations, float2* __restrict__ out) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const T* f = frames + (size_t)p * H * W;
    const double r2 = __dmul_rn(radius, radius);
    double cx = cx0, cy = cy0;
    for (int it = 0; it < iterations; ++it) {
        const int y_lo = max(0, (int)ceil(__dsub_rn(cy, radius)));
        const int y_hi = min(H - 1, (int)floor(__dadd_rn(cy, radius)));
        const int x_lo = max(0, (int)ceil(__dsub_rn(cx, radius)));
        const int x_hi = min(W - 1, (int)floor(__dadd_rn(cx, radius)));
        double s0 = 0.0, sx = 0.0, sy = 0.0;
        for (int y = y_lo; y <= y_hi; ++y) {
            const double dy = __dsub_rn((double)y, cy);
            const double dy2 = __dmul_rn(dy, dy);
            for (int x = x_lo; x <= x_hi; ++x) {
                const double dx = __dsub_rn((double)x, cx);
                if (__dadd_rn(__dmul_rn(dx, dx), dy2) <= r2) {
                    const double v = (double)__ldg(f + (size_t)y * W + x);
                    s0 = __dadd_rn(s0, v);
                    sx = __dadd_rn(sx, __dmul_rn((double)x, v));
                    sy = __dadd_rn(sy, __dmul_rn((double)y, v));
                }
            }
        }
        if (s0 > 0.0) {
            cx = __ddiv_rn(sx, s0);
            cy = __ddiv_rn(sy, s0);
        }
    }
    out[p] = make_float2((float)cx, (float)cy);
}

}  // namespace

cudaError_t launch_find_centres(const void* frames, int dtype, int64_t n, int H, int W, double cx0, double cy0,
                                double radius, int iterations, float2* out, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int threads = 128;
    const int64_t grid = (n + threads - 1) / threads;
    if (dtype == TM_DTYPE_U16)
        find_centres_kernel<uint16_t><<<(unsigned)grid, threads, 0, st>>>((const uint16_t*)frames, n, H, W, cx0, cy0,
                                                                          radius, iterations, out);
    else
        find_centres_kernel<float><<<(unsigned)grid, threads, 0, st>>>((const float*)frames, n, H, W, cx0, cy0,
                                                                       radius, iterations, out);
    return cudaGetLastError();
}

}  // namespace tmgb
