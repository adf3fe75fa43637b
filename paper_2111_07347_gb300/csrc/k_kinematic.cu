// Template simulation over an orientation grid (arXiv 2111.07347, Section 2.1: for each
// orientation the reflections near the Ewald sphere are found from their excitation error,
// weighted by |F|^2 and a linear relrod shape, and projected onto the detector; the strongest
// are kept).  The step before the library is loaded (tm_load_library), so that libraries for
// parameter sweeps are made on the device.
//
// One warp per orientation: lanes take the reciprocal lattice points, compute the beam-frame
// components and the excitation error in double precision with every operation explicitly
// rounded (no fused multiply-add), in the order the oracle's plain loops use, so the kept set
// and the values are the same bit for bit; candidates are gathered in shared memory by a
// ballot and placed by rank (intensity descending, |g| ascending, point index ascending;
// the keys are distinct, so the order is total).
#include "tm_internal.h"

namespace tmgb {
namespace {

constexpr int kKinWarps = 4;

struct Cand {
    double x, y, inten, gn;
    int idx;
};

__device__ __forceinline__ bool before(const Cand& a, const Cand& b) {
    if (a.inten != b.inten) return a.inten > b.inten;
    if (a.gn != b.gn) return a.gn < b.gn;
    return a.idx < b.idx;
}

__global__ void __launch_bounds__(32 * kKinWarps)
kinematic_kernel(const double* __restrict__ g, const double* __restrict__ f2, const double* __restrict__ gnorm,
                 int64_t G, const double* __restrict__ rot, int64_t D, double k, double s_max, int max_spots,
                 int cand_max, int32_t* __restrict__ counts, double* __restrict__ spots) {
    extern __shared__ Cand cands[];                          // [kKinWarps][cand_max]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    Cand* c = cands + (size_t)warp * cand_max;
    for (int64_t d = (int64_t)blockIdx.x * kKinWarps + warp; d < D; d += (int64_t)gridDim.x * kKinWarps) {
        double R[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) R[i] = __ldg(rot + d * 9 + i);
        int n = 0;                                           // candidates so far (warp-uniform)
        for (int64_t i0 = 0; i0 < G; i0 += 32) {
            const int64_t i = i0 + lane;
            bool keep = false;
            Cand v;
            if (i < G) {
                const double g0 = __ldg(g + i * 3), g1 = __ldg(g + i * 3 + 1), g2 = __ldg(g + i * 3 + 2);
                double x[3];
#pragma unroll
                for (int j = 0; j < 3; ++j)
                    x[j] = __dadd_rn(__dadd_rn(__dmul_rn(R[3 * j], g0), __dmul_rn(R[3 * j + 1], g1)),
                                     __dmul_rn(R[3 * j + 2], g2));
                const double t = __dadd_rn(x[2], k);
                const double s = __dsub_rn(k, __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(x[0], x[0]), __dmul_rn(x[1], x[1])),
                                                                   __dmul_rn(t, t))));
                const double as = fabs(s);
                if (as <= s_max) {
                    const double inten = __dmul_rn(__ldg(f2 + i), __dsub_rn(1.0, __ddiv_rn(as, s_max)));
                    if (inten > 0.0) {
                        keep = true;
                        v.x = x[0];
                        v.y = x[1];
                        v.inten = inten;
                        v.gn = __ldg(gnorm + i);
                        v.idx = (int)i;
                    }
                }
            }
            const unsigned b = __ballot_sync(0xffffffffu, keep);
            const int at = n + __popc(b & ((1u << lane) - 1u));
            if (keep && at < cand_max) c[at] = v;
            n += __popc(b);
        }
        __syncwarp();
        if (n > cand_max) {                                  // more reflections than the buffer holds
            if (lane == 0) counts[d] = -1;
            __syncwarp();
            continue;
        }
        double* out = spots + (size_t)d * max_spots * 3;
        for (int a = lane; a < n; a += 32) {
            int r = 0;
            for (int b2 = 0; b2 < n; ++b2) r += before(c[b2], c[a]) ? 1 : 0;
            if (r < max_spots) {
                out[3 * r] = c[a].x;
                out[3 * r + 1] = c[a].y;
                out[3 * r + 2] = c[a].inten;
            }
        }
        if (lane == 0) counts[d] = n < max_spots ? n : max_spots;
        __syncwarp();
    }
}

}  // namespace

int kinematic_cand_max() { return 512; }

cudaError_t launch_kinematic(const double* g, const double* f2, const double* gnorm, int64_t G, const double* rot,
                             int64_t D, double wavelength, double s_max, int max_spots, int32_t* counts, double* spots,
                             cudaStream_t st) {
    if (D <= 0) return cudaSuccess;
    const int cand_max = kinematic_cand_max();
    const size_t smem = (size_t)kKinWarps * cand_max * sizeof(Cand);
    const cudaError_t e = kernel_occupancy((const void*)kinematic_kernel, 32 * kKinWarps, smem, nullptr);
    if (e != cudaSuccess) return e;
    const int64_t blocks = (D + kKinWarps - 1) / kKinWarps;
    const int64_t cap = (int64_t)device_sms() * 8;
    const int grid = (int)(blocks < cap ? blocks : cap);
    kinematic_kernel<<<grid, 32 * kKinWarps, smem, st>>>(g, f2, gnorm, G, rot, D, 1.0 / wavelength, s_max, max_spots,
                                                         cand_max, counts, spots);
    return cudaGetLastError();
}

}  // namespace tmgb
