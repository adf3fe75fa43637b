// Whole-path indexing (FP32 sparse path, one library) that allocates no device memory.
//
// Who needs this: callers that cannot call cudaMalloc while indexing -- an application
// whose device memory is owned by another allocator (a framework's caching allocator that
// must see every allocation), or an acquisition callback in instrument-control software
// that runs inside a fixed, pre-reserved device budget and must not block on the driver's
// allocator.  tm_index_patterns grows per-stream scratch buffers on first use; this entry
// point instead keeps its scratch (polar ray steps, polar images, image norms and the
// pattern counter) in one statically sized device array that every GPU which loads the
// library holds for the life of the process.
//
// Limits and rules:
// * The array holds kScratchBytes (64 MiB); a call whose scratch does not fit (for a
//   128 x 360 polar grid: about 360 patterns per call) is rejected with
//   TM_ERR_INVALID_ARG and a message giving the size it needed.
// * All calls share the one array and it keeps the previous call's contents; the call
//   rewrites every part it reads (the pattern counter is cleared on the stream first).
//   Calls whose work overlaps on the GPU (several streams, several host threads) race on
//   the array: serialise them on one stream.
// * The first call on a device looks up the array's device address
//   (cudaGetSymbolAddress) with that device current; make that first call before any
//   stream capture begins.
// * No cudaMalloc, cudaFree or other allocating call is made, on the device or the host:
//   the ray steps of the polar grid are computed in double precision into a static host
//   staging area and copied into the array on the caller's stream.
#include <math.h>
#include <stdio.h>

#include <mutex>

#include "tm_internal.h"

namespace {

constexpr size_t kScratchBytes = (size_t)64 << 20;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;                      // guards the lookups below and the host staging
longlong2 g_host_rays[4096];          // n_theta <= 4096
void* g_scratch_dev[128] = {};        // device address of g_scratch, per CUDA device

int fail(int code, const char* msg) {
    tmgb::set_last_error(msg);
    return code;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Device address of the scratch array on the current device (looked up once per device).
int scratch_for(int device, unsigned char** out) {
    if (device < 0 || device >= 128) return fail(TM_ERR_INVALID_ARG, "tm_index_patterns_noalloc: device id");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_dev[device]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            char buf[256];
            snprintf(buf, sizeof buf, "tm_index_patterns_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            cudaGetLastError();
            return fail(TM_ERR_CUDA, buf);
        }
        g_scratch_dev[device] = p;
    }
    *out = (unsigned char*)g_scratch_dev[device];
    return TM_OK;
}

}  // namespace

extern "C" int tm_index_patterns_noalloc(tm_ctx* ctx, const tm_index_params* params, const void* frames_dev,
                                         int32_t dtype, int64_t n, int32_t H, int32_t W, int32_t lib_id,
                                         tm_hit* out_dev, void* stream) {
    if (!ctx || !params) return fail(TM_ERR_INVALID_ARG, "tm_index_patterns_noalloc: NULL argument");
    if (!(params->gamma > 0.0 && isfinite(params->gamma)) || !isfinite(params->subtract) || isinf(params->cx) ||
        isinf(params->cy) || fabs(params->cx) >= 1048576.0 || fabs(params->cy) >= 1048576.0)
        return fail(TM_ERR_INVALID_ARG, "tm_index_patterns_noalloc: bad gamma, subtract or centre");
    if (params->path != TM_PATH_FP32_SPARSE || params->prefilter_fraction != 1.0)
        return fail(TM_ERR_INVALID_ARG, "tm_index_patterns_noalloc: only the FP32 sparse path without pre-filter");
    if (params->top_n < 1 || params->top_n > TM_MAX_TOPN)
        return fail(TM_ERR_INVALID_ARG, "tm_index_patterns_noalloc: top_n out of range");
    if (n < 0 || H < 1 || W < 1 || H > 32000 || W > 32000 || (dtype != TM_DTYPE_U16 && dtype != TM_DTYPE_F32))
        return fail(TM_ERR_INVALID_ARG, "tm_index_patterns_noalloc: bad frames");
    int device = 0, num_sms = 0, n_r = 0, n_theta = 0;
    double dr = 1.0;
    tmgb::SparseLib view;
    int rc = tmgb::library_view(ctx, lib_id, &device, &num_sms, &view, &n_r, &n_theta, &dr);
    if (rc) return rc;
    if (n == 0) return TM_OK;
    if (!frames_dev || !out_dev) return fail(TM_ERR_INVALID_ARG, "tm_index_patterns_noalloc: NULL buffer");
    const int N = params->top_n;
    if (!tmgb::sparse_smem_bytes(view.n_rad, n_theta, N))
        return fail(TM_ERR_UNSUPPORTED, "tm_index_patterns_noalloc: polar grid does not fit shared memory");

    // scratch layout: ray steps | polar images | image norms | counter
    const size_t m = (size_t)n_r * n_theta;
    if (n_theta > 4096) return fail(TM_ERR_INVALID_ARG, "tm_index_patterns_noalloc: n_theta > 4096");
    const size_t o_rays = 0;
    const size_t o_polar = align256(o_rays + (size_t)n_theta * sizeof(longlong2));
    const size_t o_norm = align256(o_polar + (size_t)n * m * 4);
    const size_t o_count = align256(o_norm + (size_t)n * 4);
    const size_t need = o_count + 256;
    if (need > kScratchBytes) {
        char buf[256];
        snprintf(buf, sizeof buf,
                 "tm_index_patterns_noalloc: %lld patterns on a %dx%d grid need %zu bytes of scratch; "
                 "the static scratch holds %zu (index fewer patterns per call)",
                 (long long)n, n_r, n_theta, need, kScratchBytes);
        return fail(TM_ERR_INVALID_ARG, buf);
    }

    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != device) cudaSetDevice(device);
    unsigned char* scratch = nullptr;
    rc = scratch_for(device, &scratch);
    cudaStream_t st = (cudaStream_t)stream;
    if (!rc) {
        // ray steps of this grid, in double precision on the host; the staging is reused
        // once the copy below has consumed it (a copy from pageable memory returns after
        // the data has been taken)
        std::lock_guard<std::mutex> lk(g_mu);
        const double cx = isnan(params->cx) ? (W - 1) / 2.0 : params->cx;
        const double cy = isnan(params->cy) ? (H - 1) / 2.0 : params->cy;
        tmgb::build_polar_rays(n_theta, dr, g_host_rays);
        cudaError_t e = cudaMemcpyAsync(scratch + o_rays, g_host_rays, (size_t)n_theta * sizeof(longlong2),
                                        cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) {
            const longlong2* rays = (const longlong2*)(scratch + o_rays);
            float* polar = (float*)(scratch + o_polar);
            float* pnorm = (float*)(scratch + o_norm);
            e = tmgb::launch_polar(frames_dev, dtype, n, H, W, rays, cx, cy, params->gamma, params->subtract, n_r,
                                   n_theta, polar, pnorm, nullptr, st, nullptr, nullptr, params->pixel_mask,
                                   params->threshold);
            if (e == cudaSuccess) {
                tmgb::SparseCall c{};
                c.polar = polar;
                c.pnorm = pnorm;
                c.n = n;
                c.n_r = n_r;
                c.n_theta = n_theta;
                c.pitch = 0;
                c.max_rad = view.n_rad;
                c.pattern_counter = (int*)(scratch + o_count);
                c.n_libs = 1;
                c.lib[0] = view;
                c.hits = out_dev;
                c.hits_lib_stride = n * N;
                c.top_n = N;
                e = tmgb::launch_sparse(c, num_sms, st);
            }
        }
        if (e != cudaSuccess) {
            char buf[256];
            snprintf(buf, sizeof buf, "tm_index_patterns_noalloc: %s", cudaGetErrorString(e));
            rc = fail(TM_ERR_CUDA, buf);
        }
    }
    if (prev >= 0 && prev != device) cudaSetDevice(prev);
    return rc;
}
