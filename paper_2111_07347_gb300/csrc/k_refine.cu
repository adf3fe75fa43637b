// Sub-step in-plane angle of the top-N hits (arXiv 2111.07347 Section 2.2: the resolution of
// phi_1 is the polar transform's angular step; Section 5 names a better phi_1 optimisation as
// future work).  For each hit (template k, best shift s) the correlation index Q of Eq. 1 is
// evaluated at s - 1, s and s + 1 (mod n_theta) and the angle is the vertex of the parabola
// through the three values: delta = (Q- - Q+) / (2 (Q- - 2 Q0 + Q+)) for a negative curvature
// (else 0), clipped to [-1/2, 1/2], angle = (s + delta) 360 / n_theta.
//
// One thread per hit.  Each sum runs over the template's spots in list order, the first
// product then fused multiply-adds -- the order and operations of the sparse kernel -- so Q0
// equals the hit's score.  The work is three spot sums per hit.
#include "tm_internal.h"

namespace tmgb {
namespace {

__device__ __forceinline__ float q_at(const float* P, int n_theta, const int32_t* rt, const int2* spot, int beg,
                                      int end, int s, float d) {
    float acc = 0.0f;
    for (int i = beg; i < end; ++i) {
        const int v = __ldg(rt + i);
        const int r = v & 0xffff, t = v >> 16;
        int col = t + s;
        col -= col >= n_theta ? n_theta : 0;
        col += col < 0 ? n_theta : 0;
        const float I = __int_as_float(__ldg(&spot[i].y));
        const float p = __ldg(P + (size_t)r * n_theta + col);
        acc = i == beg ? I * p : fmaf(I, p, acc);
    }
    return d > 0.0f ? __fdiv_rn(acc, d) : 0.0f;
}

__global__ void refine_kernel(const RefineCall c) {
    const int64_t total = (int64_t)c.n_libs * c.n * c.top_n;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int li = (int)(t / ((int64_t)c.n * c.top_n));
        const int64_t rest = t - (int64_t)li * c.n * c.top_n;
        const int64_t p = rest / c.top_n;
        const int j = (int)(rest - p * c.top_n);
        tm_hit* h = c.hits + (size_t)li * c.hits_lib_stride + (size_t)p * c.top_n + j;
        const int k = h->template_index;
        if (k < 0) continue;
        const int s = h->shift;
        const RefineLib& L = c.lib[li];
        const float d = __ldg(c.pnorm + p) * __ldg(L.norm + k);
        const float* P = c.polar + (size_t)p * c.n_r * c.n_theta;
        const int beg = __ldg(L.off + k), end = __ldg(L.off + k + 1);
        const int nt = c.n_theta;
        const float qm = q_at(P, nt, L.rt, L.spot, beg, end, s == 0 ? nt - 1 : s - 1, d);
        const float q0 = q_at(P, nt, L.rt, L.spot, beg, end, s, d);
        const float qp = q_at(P, nt, L.rt, L.spot, beg, end, s == nt - 1 ? 0 : s + 1, d);
        const float curv = (qm - q0) + (qp - q0);
        float delta = curv < 0.0f ? (qm - qp) / (2.0f * curv) : 0.0f;
        delta = fminf(0.5f, fmaxf(-0.5f, delta));
        h->angle_deg = ((float)s + delta) * (360.0f / (float)nt);
    }
}

}  // namespace

cudaError_t launch_refine(const RefineCall& c, int num_sms, cudaStream_t st) {
    const int64_t total = (int64_t)c.n_libs * c.n * c.top_n;
    if (total <= 0) return cudaSuccess;
    const int threads = 256;
    int64_t grid = (total + threads - 1) / threads;
    if (grid > (int64_t)num_sms * 8) grid = (int64_t)num_sms * 8;
    refine_kernel<<<(int)grid, threads, 0, st>>>(c);
    return cudaGetLastError();
}

}  // namespace tmgb
