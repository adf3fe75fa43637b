// Orientation maps (arXiv 2111.07347, Section 4.1: inverse pole figure maps along the sample
// axes) and the angular deviation between two maps (Eq. 2).
//
// orient_kernel: per pattern, the best hit's template b (its mirror copy reflects the beam
//   frame's y axis) and in-plane angle phi give the orientation O = Rz(phi) M R_b; the crystal
//   direction along the sample axis e is v = O^T e.  FP64 with each operation rounded in the
//   oracle's order (cos and sin of phi are the library functions).
// deviation_kernel: |acos(va . vb / (|va| |vb|))| in degrees, the cosine clipped to [-1, 1];
//   NaN where a vector is missing.
#include <math.h>

#include "tm_internal.h"

namespace tmgb {
namespace {

constexpr double kDegToRad = 3.14159265358979323846 / 180.0;
constexpr double kRadToDeg = 180.0 / 3.14159265358979323846;

__global__ void orient_kernel(const tm_hit* __restrict__ hits, int64_t n, int stride, const double* __restrict__ rot,
                              int64_t K0, double e0, double e1, double e2, double* __restrict__ v) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const tm_hit h = hits[p * stride];
        const int64_t k = h.template_index;
        if (k < 0 || k >= 2 * K0) {
            v[p * 3] = v[p * 3 + 1] = v[p * 3 + 2] = __longlong_as_double(0x7ff8000000000000ll);
            continue;
        }
        const bool mirror = k >= K0;
        const int64_t b = mirror ? k - K0 : k;
        const double phi = __dmul_rn((double)h.angle_deg, kDegToRad);
        const double c = cos(phi), s = sin(phi);
        const double u0 = __dadd_rn(__dmul_rn(c, e0), __dmul_rn(s, e1));
        double u1 = __dadd_rn(__dmul_rn(-s, e0), __dmul_rn(c, e1));
        const double u2 = e2;
        if (mirror) u1 = -u1;
        const double* R = rot + b * 9;
#pragma unroll
        for (int j = 0; j < 3; ++j)
            v[p * 3 + j] = __dadd_rn(__dadd_rn(__dmul_rn(R[j], u0), __dmul_rn(R[3 + j], u1)), __dmul_rn(R[6 + j], u2));
    }
}

__global__ void deviation_kernel(const double* __restrict__ va, const double* __restrict__ vb, int64_t n,
                                 double* __restrict__ deg) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const double a0 = va[p * 3], a1 = va[p * 3 + 1], a2 = va[p * 3 + 2];
        const double b0 = vb[p * 3], b1 = vb[p * 3 + 1], b2 = vb[p * 3 + 2];
        if (isnan(a0) || isnan(a1) || isnan(a2) || isnan(b0) || isnan(b1) || isnan(b2)) {
            deg[p] = __longlong_as_double(0x7ff8000000000000ll);
            continue;
        }
        const double dot = __dadd_rn(__dadd_rn(__dmul_rn(a0, b0), __dmul_rn(a1, b1)), __dmul_rn(a2, b2));
        const double na = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(a0, a0), __dmul_rn(a1, a1)), __dmul_rn(a2, a2)));
        const double nb = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(b0, b0), __dmul_rn(b1, b1)), __dmul_rn(b2, b2)));
        const double cosv = fmax(-1.0, fmin(1.0, __ddiv_rn(dot, __dmul_rn(na, nb))));
        deg[p] = fabs(__dmul_rn(acos(cosv), kRadToDeg));
    }
}

int grid1d(int64_t n) {
    const int64_t g = (n + 255) / 256, cap = (int64_t)device_sms() * 8;
    return (int)(g < 1 ? 1 : (g < cap ? g : cap));
}

}  // namespace

cudaError_t launch_orientation_vectors(const tm_hit* hits, int64_t n, int stride, const double* rot, int64_t K0,
                                       double e0, double e1, double e2, double* v, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    orient_kernel<<<grid1d(n), 256, 0, st>>>(hits, n, stride, rot, K0, e0, e1, e2, v);
    return cudaGetLastError();
}

cudaError_t launch_angular_deviation(const double* va, const double* vb, int64_t n, double* deg, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    deviation_kernel<<<grid1d(n), 256, 0, st>>>(va, vb, n, deg);
    return cudaGetLastError();
}

}  // namespace tmgb
