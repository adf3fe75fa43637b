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
// * The array holds kScratchBytes (64 MiB).  Its first kRayBytes hold the ray steps of up
//   to kRaySlots polar grids; a call needs n_r * n_theta * 4 + 4 bytes per frame (polar
//   image and norm) plus 512 bytes from the rest (for a 128 x 360 grid: 361 frames per
//   call).  A call whose scratch does not fit is rejected with TM_ERR_INVALID_ARG and a
//   message giving the size it needed.
// * All calls share the one array and it keeps the previous call's contents; the call
//   rewrites every part it reads (the pattern counter is cleared on the stream first).
//   Calls whose work overlaps on the GPU (several streams, several host threads) race on
//   the array: serialise them on one stream.
// * Set-up: the first call on a device looks up the array's device address
//   (cudaGetSymbolAddress) with that device current, and the first call for each polar
//   grid (n_theta, dr) on a device writes that grid's ray steps into the array with a
//   synchronous copy.  Make those first calls before any stream capture begins.
// * No cudaMalloc, cudaFree or other allocating call is made, on the device or the host.
#include <math.h>
#include <stdio.h>

#include <mutex>

#include "tm_internal.h"

namespace {

constexpr size_t kScratchBytes = (size_t)64 << 20;
constexpr int kMaxTheta = 4096;
constexpr int kRaySlots = 8;
constexpr size_t kRaySlotBytes = (size_t)kMaxTheta * sizeof(longlong2);   // 64 KiB
constexpr size_t kRayBytes = kRaySlots * kRaySlotBytes;                      // 512 KiB
constexpr int kMaxDevices = 128;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

struct RaySlot {
    int n_theta = 0;                  // 0: free
    double dr = 0.0;
};

std::mutex g_mu;                      // guards everything below
void* g_scratch_dev[kMaxDevices] = {};         // device address of g_scratch, per CUDA device
RaySlot g_rays[kMaxDevices][kRaySlots];        // grid held by each ray slot, per device
longlong2 g_host_rays[kMaxTheta];              // host staging of one grid's ray steps

int fail(int code, const char* msg) {
    tmgb::set_last_error(msg);
    return code;
}

int fail_cuda(const char* what, cudaError_t e) {
    char buf[256];
    snprintf(buf, sizeof buf, "tm_index_patterns_noalloc: %s: %s", what, cudaGetErrorString(e));
    cudaGetLastError();
    return fail(TM_ERR_CUDA, buf);
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Device address of the scratch array on `device`, which must be the current device (looked
// up once per device), and the ray slot holding the grid (n_theta, dr), written on first use.
int scratch_for(int device, int n_theta, double dr, unsigned char** out, const longlong2** rays) {
    if (device < 0 || device >= kMaxDevices) return fail(TM_ERR_INVALID_ARG, "tm_index_patterns_noalloc: device id");
    int cur = -1;
    const cudaError_t ge = cudaGetDevice(&cur);
    if (ge != cudaSuccess) return fail_cuda("cudaGetDevice", ge);
    if (cur != device) return fail(TM_ERR_CUDA, "tm_index_patterns_noalloc: the library's device is not current");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_dev[device]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) return fail_cuda("cudaGetSymbolAddress", e);
        g_scratch_dev[device] = p;
    }
    unsigned char* base = (unsigned char*)g_scratch_dev[device];
    int slot = -1;
    for (int i = 0; i < kRaySlots && slot < 0; ++i)
        if (g_rays[device][i].n_theta == n_theta && g_rays[device][i].dr == dr) slot = i;
    if (slot < 0) {
        for (int i = 0; i < kRaySlots && slot < 0; ++i)
            if (g_rays[device][i].n_theta == 0) slot = i;
        if (slot < 0)
            return fail(TM_ERR_UNSUPPORTED, "tm_index_patterns_noalloc: more than 8 polar grids on one device");
        // ray steps of this grid, in double precision on the host, copied once
        tmgb::build_polar_rays(n_theta, dr, g_host_rays);
        const cudaError_t e = cudaMemcpy(base + (size_t)slot * kRaySlotBytes, g_host_rays,
                                         (size_t)n_theta * sizeof(longlong2), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return fail_cuda("ray steps", e);
        g_rays[device][slot].n_theta = n_theta;
        g_rays[device][slot].dr = dr;
    }
    *out = base;
    *rays = (const longlong2*)(base + (size_t)slot * kRaySlotBytes);
    return TM_OK;
}

}  // namespace

extern "C" int tm_index_patterns_noalloc(tm_ctx* ctx, const tm_index_params* params, const void* frames_dev,
                                         int32_t dtype, int64_t n, int32_t H, int32_t W, int32_t lib_id,
                                         tm_hit* out_dev, void* stream) {
    int rc = tmgb::check_index_params(params);     // the same checks as tm_index_patterns
    if (rc) return rc;
    if (params->path != TM_PATH_FP32_SPARSE || params->prefilter_fraction != 1.0)
        return fail(TM_ERR_INVALID_ARG, "tm_index_patterns_noalloc: only the FP32 sparse path without pre-filter");
    if (!ctx) return fail(TM_ERR_INVALID_ARG, "tm_index_patterns_noalloc: ctx is NULL");
    if (n < 0 || H < 1 || W < 1 || H > 32000 || W > 32000 || (dtype != TM_DTYPE_U16 && dtype != TM_DTYPE_F32))
        return fail(TM_ERR_INVALID_ARG, "tm_index_patterns_noalloc: bad frames");
    int device = 0, num_sms = 0, n_r = 0, n_theta = 0;
    double dr = 1.0;
    tmgb::SparseLib view;
    rc = tmgb::library_view(ctx, lib_id, &device, &num_sms, &view, &n_r, &n_theta, &dr);
    if (rc) return rc;
    if (n == 0) return TM_OK;
    if (!frames_dev || !out_dev) return fail(TM_ERR_INVALID_ARG, "tm_index_patterns_noalloc: NULL buffer");
    const int N = params->top_n;
    if (!tmgb::sparse_smem_bytes(view.n_rad, n_theta, N))
        return fail(TM_ERR_UNSUPPORTED, "tm_index_patterns_noalloc: polar grid does not fit shared memory");
    if (n_theta > kMaxTheta) return fail(TM_ERR_INVALID_ARG, "tm_index_patterns_noalloc: n_theta > 4096");

    // per-call scratch after the ray slots: polar images | image norms | counter
    const size_t m = (size_t)n_r * n_theta;
    const size_t o_polar = kRayBytes;
    const size_t o_norm = align256(o_polar + (size_t)n * m * 4);
    const size_t o_count = align256(o_norm + (size_t)n * 4);
    const size_t need = o_count + 256;
    if (need > kScratchBytes) {
        char buf[320];
        snprintf(buf, sizeof buf,
                 "tm_index_patterns_noalloc: %lld patterns on a %dx%d grid need %zu bytes of scratch; "
                 "the static scratch holds %zu (n_r * n_theta * 4 + 4 bytes per pattern: index fewer "
                 "patterns per call)",
                 (long long)n, n_r, n_theta, need, kScratchBytes);
        return fail(TM_ERR_INVALID_ARG, buf);
    }

    int prev = -1;
    cudaError_t e = cudaGetDevice(&prev);
    if (e != cudaSuccess) return fail_cuda("cudaGetDevice", e);
    if (prev != device) {
        e = cudaSetDevice(device);
        if (e != cudaSuccess) return fail_cuda("cudaSetDevice", e);
    }
    unsigned char* scratch = nullptr;
    const longlong2* rays = nullptr;
    rc = scratch_for(device, n_theta, dr, &scratch, &rays);
    cudaStream_t st = (cudaStream_t)stream;
    if (!rc) {
        const double cx = isnan(params->cx) ? (W - 1) / 2.0 : params->cx;
        const double cy = isnan(params->cy) ? (H - 1) / 2.0 : params->cy;
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
        if (e != cudaSuccess) rc = fail_cuda("launch", e);
    }
    if (prev >= 0 && prev != device) cudaSetDevice(prev);
    return rc;
}
