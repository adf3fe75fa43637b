// Host side of libtmgb.so: the C ABI declared in include/tmgb.h.
//
// Library loading follows arXiv 2111.07347 Section 2.1 (templates are spot lists at
// in-plane angle zero) and Section 2.2 (spot coordinates rounded to the nearest polar
// pixel; mirror templates by reflecting across y = 0; norms of Eq. 1 precomputed);
// Section 4.3 gives the unit-intensity option.  All template geometry is done in double
// precision here; the device receives float intensities and packed integer addresses.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <tuple>
#include <unordered_map>
#include <vector>

#include <cublas_v2.h>
#include <cuda.h>
#include <cudaTypedefs.h>

#include "tm_internal.h"

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    return fail(TM_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

#define TM_CUDA(call, what)                                  \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_fail(e_, what);   \
    } while (0)

constexpr double kPi = 3.14159265358979323846;

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

struct Library {
    int64_t K = 0, K0 = 0;
    int mirror = 0, n_r = 0, n_theta = 0;
    double dr = 1.0;
    int64_t n_sym = 0, macs = 0;
    int max_spots = 0;
    int nonneg = 1;                // every intensity >= 0
    // host copies (exported for tests)
    std::vector<int64_t> off;
    std::vector<int32_t> r, t, order;
    std::vector<float> I, norm;
    // device
    int32_t* d_off = nullptr;
    int2* d_spot = nullptr;
    int2* d_spot2 = nullptr;       // per-spot offsets in the dual / wrap-free layouts
    int2* d_bspot = nullptr;       // per-spot pruning-window entries (null: none)
    int4* d_meta = nullptr;        // per template {first spot, spots | shifts << 16, norm bits, 0}
    int4* d_smeta = nullptr;       // d_meta in spot-count order, with the order and the bound entries
    int32_t* d_sperm = nullptr;    //   by word (sliced ELL, lanes adjacent): see tmgb::SparseLib
    int32_t* d_ellw = nullptr;
    int2* d_ell = nullptr;
    float* d_norm = nullptr;
    int32_t* d_nshift = nullptr;
    float* d_radial = nullptr;     // [K][n_rad rounded up to 4] radial profiles at the distinct radii
    float* d_rnorm = nullptr;
    int32_t* d_rt = nullptr;       // r | (t << 16) per spot (BF16 path, refinement)
    int32_t* d_radii = nullptr;    // distinct spot radii (sparse kernel rows)
    std::vector<int32_t> radii;    // distinct radii with spots
    size_t bytes = 0;
    // angular spectra of the templates for the tensor-core path, built on first use:
    // [192 slots][2 R][K_pad] BF16 (R = distinct radii rounded up to 8, K_pad = K rounded up to 64)
    void* d_that = nullptr;
    int32_t* d_rowmap = nullptr;   // [n_r] radius -> row among the distinct radii (-1: none)
    int R = 0, K_pad = 0;
    size_t that_bytes = 0;
};

struct Buffer {
    void* p = nullptr;
    size_t bytes = 0;
};


struct SpectralTables {            // per n_theta: DFT matrix, inverse-DFT basis and twiddles
    void* basis = nullptr;         // bf16 [rows][cols]
    float2* twiddle = nullptr;     // [n_theta]
    float* dftmat = nullptr;       // [2 x 192 columns][n_theta]: (cos, -sin)(2 pi m_j theta / n), 0 for m_j > n/2
};

struct RadiusMap {                 // per set of libraries: union of radii
    int32_t* radii = nullptr;      // [n_rad]
    int32_t* rmap = nullptr;       // [n_r]
    uint8_t* keep_row = nullptr;   // [n_r]  1 for the polar rows later stages read
    int n_rad = 0;
};

}  // namespace

namespace tmgb {
void set_last_error(const char* msg) { g_err = msg; }

namespace {
std::mutex g_launch_mu;
std::map<std::tuple<const void*, int, int, size_t>, int> g_occupancy;   // (fn, device, threads, smem)
std::map<std::pair<const void*, int>, size_t> g_smem_limit;              // (fn, device) -> limit set
std::map<int, int> g_sms;
}  // namespace

cudaError_t kernel_occupancy(const void* fn, int threads, size_t smem, int* per_sm) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_launch_mu);
    size_t& lim = g_smem_limit[std::make_pair(fn, dev)];
    if (smem > 48 * 1024 && smem > lim) {
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        lim = smem;
    }
    if (!per_sm) return cudaSuccess;
    const auto key = std::make_tuple(fn, dev, threads, smem);
    auto it = g_occupancy.find(key);
    if (it == g_occupancy.end()) {
        int b = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, threads, smem);
        if (e != cudaSuccess) return e;
        it = g_occupancy.emplace(key, b).first;
    }
    *per_sm = it->second;
    return cudaSuccess;
}

namespace {
thread_local int t_sm_cap = 0;      // persistent grids of this thread's calls use at most this many SMs
}

void set_sm_cap(int cap) { t_sm_cap = cap > 0 ? cap : 0; }

int device_sms() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    std::lock_guard<std::mutex> lk(g_launch_mu);
    auto it = g_sms.find(dev);
    if (it == g_sms.end()) {
        int sms = 1;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) sms = 1;
        it = g_sms.emplace(dev, sms).first;
    }
    return t_sm_cap ? std::min(t_sm_cap, it->second) : it->second;
}
}  // namespace tmgb

struct tm_ctx {
    int device = 0;
    size_t budget = 0, used = 0;
    int num_sms = 0;
    std::mutex mu;
    std::map<int, std::unique_ptr<Library>> libs;
    int next_id = 0;
    std::map<std::pair<int, double>, longlong2*> rays;   // polar ray steps per (n_theta, dr)
    std::map<std::string, Buffer> ws;
    cudaEvent_t ws_event = nullptr;
    unsigned* d_error = nullptr;   // device error word of the bounded waits
    unsigned long long* d_work = nullptr;   // sparse multiply-adds executed while profiling
    std::map<int, SpectralTables> spectral;
    cublasHandle_t cublas = nullptr;                     // stage A of the tensor-core path
    PFN_cuTensorMapEncodeTiled_v12000 encode_tiled = nullptr;
    std::map<std::string, RadiusMap> radius_maps;
    // CUDA graphs of whole-path calls (TM_INDEX_GRAPH)
    struct GraphEntry {
        cudaGraphExec_t exec = nullptr;
        uint64_t ws_gen = 0;
        bool seen = false;
        int64_t launches = 0, corr = 0, scored = 0;
    };
    std::map<std::string, GraphEntry> graphs;
    uint64_t ws_gen = 1;           // bumped whenever a workspace buffer is reallocated
    bool capturing = false;
    // autotuned sparse-kernel shape per library signature (tm_autotune): block size and
    // seeds per warp of its pruned top-N
    struct Tune { int threads = 0, seeds = 0, tile = 0; };
    std::map<std::string, Tune> tuned;
    Tune tune_override;
    std::string tune_file;
    // host-buffer entry point: two streams alternate over the chunks of a call
    cudaStream_t host_streams[2] = {nullptr, nullptr};
    std::mutex host_mu;            // one host-buffer call at a time per context
    // stage timing
    bool profiling = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::tuple<int, cudaEvent_t, cudaEvent_t>> ev_marks;
};

namespace {

int dev_alloc(tm_ctx* ctx, void** p, size_t bytes, const char* what) {
    if (bytes == 0) bytes = 16;
    if (ctx->budget && ctx->used + bytes > ctx->budget)
        return fail(TM_ERR_OOM, "%s: %zu bytes exceed the context budget (%zu of %zu used)", what, bytes,
                    ctx->used, ctx->budget);
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(TM_ERR_OOM, "%s: cudaMalloc(%zu) failed: %s", what, bytes, cudaGetErrorString(e));
    }
    ctx->used += bytes;
    return TM_OK;
}

void dev_free(tm_ctx* ctx, void* p, size_t bytes) {
    if (!p) return;
    cudaFree(p);
    ctx->used -= std::min(ctx->used, bytes ? bytes : 16);
}

// Workspace buffer `name` of at least `bytes` for work enqueued on stream `st`, grown on
// demand.  Each stream has its own buffers, so calls on different streams never share
// scratch memory and may overlap on the GPU; calls on one stream are ordered by it.
int workspace(tm_ctx* ctx, cudaStream_t st, const std::string& name, size_t bytes, void** out) {
    char key[64];
    snprintf(key, sizeof key, "@%llx", (unsigned long long)(uintptr_t)st);
    Buffer& b = ctx->ws[name + key];
    if (b.bytes < bytes) {
        if (ctx->capturing) return fail(TM_ERR_CUDA, "workspace growth during graph capture");
        ctx->ws_gen++;
        if (b.p) {
            cudaDeviceSynchronize();
            dev_free(ctx, b.p, b.bytes);
            b.p = nullptr;
            b.bytes = 0;
        }
        size_t want = bytes + bytes / 8;
        int rc = dev_alloc(ctx, &b.p, want, name.c_str());
        if (rc) return rc;
        b.bytes = want;
    }
    *out = b.p;
    return TM_OK;
}

// Stage timer: records an event pair around the launches of one stage when profiling.
struct StageTimer {
    tm_ctx* ctx;
    int stage;
    cudaStream_t st;
    cudaEvent_t a = nullptr, b = nullptr;
    static cudaEvent_t take(tm_ctx* c) {
        if (!c->ev_pool.empty()) {
            cudaEvent_t e = c->ev_pool.back();
            c->ev_pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        return e;
    }
    StageTimer(tm_ctx* c, int s, cudaStream_t stream) : ctx(c), stage(s), st(stream) {
        if (!ctx->profiling || ctx->capturing) return;
        a = take(ctx);
        b = take(ctx);
        if (a && b) cudaEventRecord(a, st);
    }
    ~StageTimer() {
        if (!a || !b) return;
        cudaEventRecord(b, st);
        ctx->ev_marks.emplace_back(stage, a, b);
    }
};

// ---------------------------------------------------------------- template geometry

struct Merged {
    std::vector<int32_t> r, t;
    std::vector<double> I;
};

// Nearest polar pixel of a spot (Section 2.2): r = floor(r_px / dr + 1/2),
// t = floor(theta' / (2 pi / n_theta) + 1/2) mod n_theta, theta' in [0, 2 pi).
inline void round_spot(double r_px, double theta, int n_theta, double dr, int64_t* ri, int64_t* ti) {
    double th = fmod(theta, 2.0 * kPi);
    if (th < 0.0) th += 2.0 * kPi;
    const double step = 2.0 * kPi / n_theta;
    int64_t t = (int64_t)floor(th / step + 0.5);
    t %= n_theta;
    *ti = t;
    *ri = (int64_t)floor(r_px / dr + 0.5);
}

// Largest n dividing n_theta such that the merged spot multiset is invariant under a
// rotation by n_theta / n columns (exact comparison of integer positions and intensities).
int rotational_order(const Merged& m, int n_theta) {
    const size_t s = m.r.size();
    if (s == 0) return n_theta;
    std::vector<std::tuple<int32_t, int32_t, double>> a(s), b(s);
    for (size_t i = 0; i < s; ++i) a[i] = std::make_tuple(m.r[i], m.t[i], m.I[i]);
    std::sort(a.begin(), a.end());
    for (int n = n_theta; n >= 2; --n) {
        if (n_theta % n) continue;
        const int sh = n_theta / n;
        for (size_t i = 0; i < s; ++i)
            b[i] = std::make_tuple(m.r[i], (int32_t)((m.t[i] + sh) % n_theta), m.I[i]);
        std::sort(b.begin(), b.end());
        if (a == b) return n;
    }
    return 1;
}

// Host half of library loading: validation, rounding, merging, mirrors, norms, orders.
struct Prepared {
    std::vector<int2> spot, spot2, bspot, ell;
    std::vector<int4> meta, smeta;
    std::vector<int32_t> sperm, ellw;
    std::vector<int32_t> nshift;
    std::vector<double> radial, rnorm;
};

int prepare_library(const tm_library_desc* d, Library* L, Prepared* P) {
    if (!d) return fail(TM_ERR_INVALID_ARG, "tm_load_library: desc is NULL");
    if (d->n_templates < 1 || d->n_templates > (1 << 24))
        return fail(TM_ERR_INVALID_ARG, "tm_load_library: n_templates=%lld out of range", (long long)d->n_templates);
    if (!d->spot_offsets) return fail(TM_ERR_INVALID_ARG, "tm_load_library: spot_offsets is NULL");
    if (d->coords != TM_COORDS_POLAR && d->coords != TM_COORDS_XY)
        return fail(TM_ERR_INVALID_ARG, "tm_load_library: coords=%d invalid", d->coords);
    if (d->coords == TM_COORDS_XY && !(d->px_per_unit > 0.0 && isfinite(d->px_per_unit)))
        return fail(TM_ERR_INVALID_ARG, "tm_load_library: px_per_unit must be > 0");
    if (d->n_r < 1 || d->n_r > 4096) return fail(TM_ERR_INVALID_ARG, "tm_load_library: n_r=%d", d->n_r);
    if (d->n_theta < 1 || d->n_theta > 1024) return fail(TM_ERR_INVALID_ARG, "tm_load_library: n_theta=%d", d->n_theta);
    if (!(d->dr > 0.0 && d->n_r * d->dr < 1048576.0))
        return fail(TM_ERR_INVALID_ARG, "tm_load_library: dr must be > 0 with n_r dr < 2^20");
    if (d->flags & ~(uint32_t)(TM_LIB_MIRROR | TM_LIB_UNIT_INTENSITY))
        return fail(TM_ERR_INVALID_ARG, "tm_load_library: unknown flags 0x%x", d->flags);
    const int64_t K0 = d->n_templates;
    if (d->spot_offsets[0] != 0) return fail(TM_ERR_INVALID_ARG, "tm_load_library: spot_offsets[0] != 0");
    for (int64_t k = 0; k < K0; ++k)
        if (d->spot_offsets[k + 1] < d->spot_offsets[k])
            return fail(TM_ERR_INVALID_ARG, "tm_load_library: spot_offsets decreasing at %lld", (long long)k);
    const int64_t S = d->spot_offsets[K0];
    const bool unit = (d->flags & TM_LIB_UNIT_INTENSITY) != 0;
    if (S > 0 && (!d->spot_a || !d->spot_b || (!unit && !d->intensity)))
        return fail(TM_ERR_INVALID_ARG, "tm_load_library: spot arrays are NULL");
    for (int64_t i = 0; i < S; ++i)
        if (!isfinite(d->spot_a[i]) || !isfinite(d->spot_b[i]) || (!unit && !isfinite(d->intensity[i])))
            return fail(TM_ERR_INVALID_ARG, "tm_load_library: spot %lld is not finite", (long long)i);

    const int n_r = d->n_r, n_theta = d->n_theta;
    if (n_r >= 8192 || n_theta >= 2048)
        return fail(TM_ERR_UNSUPPORTED, "tm_load_library: polar grid %dx%d too large for the sparse layout", n_r, n_theta);
    L->K0 = K0;
    L->mirror = (d->flags & TM_LIB_MIRROR) ? 1 : 0;
    L->K = K0 * (L->mirror ? 2 : 1);
    L->n_r = n_r;
    L->n_theta = n_theta;
    L->dr = d->dr;
    L->off.assign(1, 0);
    std::vector<double>& radial = P->radial;
    std::vector<double>& rnorm = P->rnorm;
    std::vector<int2>& spot = P->spot;
    std::vector<int32_t>& nshift = P->nshift;
    radial.assign((size_t)L->K * n_r, 0.0);
    rnorm.assign(L->K, 0.0);
    nshift.assign(L->K, 0);
    std::unordered_map<int64_t, int> slot;
    for (int copy = 0; copy < (L->mirror ? 2 : 1); ++copy) {
        for (int64_t k0 = 0; k0 < K0; ++k0) {
            const int64_t k = copy * K0 + k0;
            Merged m;
            slot.clear();
            for (int64_t i = d->spot_offsets[k0]; i < d->spot_offsets[k0 + 1]; ++i) {
                double r_px, th;
                if (d->coords == TM_COORDS_XY) {
                    const double x = d->spot_a[i] * d->px_per_unit;
                    double y = d->spot_b[i] * d->px_per_unit;
                    if (copy) y = -y;                       // mirror across y = 0
                    r_px = hypot(x, y);
                    th = atan2(y, x);
                } else {
                    r_px = d->spot_a[i];
                    th = copy ? -d->spot_b[i] : d->spot_b[i];
                }
                int64_t ri, ti;
                round_spot(r_px, th, n_theta, d->dr, &ri, &ti);
                if (ri < 0 || ri >= n_r) continue;           // outside the polar grid
                const double w = unit ? 1.0 : d->intensity[i];
                const int64_t key = ri * n_theta + ti;
                auto it = slot.find(key);
                if (it == slot.end()) {
                    slot.emplace(key, (int)m.r.size());
                    m.r.push_back((int32_t)ri);
                    m.t.push_back((int32_t)ti);
                    m.I.push_back(w);
                } else {
                    m.I[it->second] += w;
                }
            }
            double n2 = 0.0;
            for (size_t i = 0; i < m.r.size(); ++i) {
                n2 += m.I[i] * m.I[i];
                radial[(size_t)k * n_r + m.r[i]] += m.I[i];
                L->r.push_back(m.r[i]);
                L->t.push_back(m.t[i]);
                L->I.push_back((float)m.I[i]);
            }
            const int ord = rotational_order(m, n_theta);
            L->order.push_back(ord);
            nshift[k] = n_theta / ord;
            if (ord > 1) ++L->n_sym;
            L->macs += (int64_t)m.r.size() * (n_theta / ord);
            L->max_spots = std::max(L->max_spots, (int)m.r.size());
            L->norm.push_back((float)sqrt(n2));
            L->off.push_back((int64_t)L->r.size());
            double rn = 0.0;
            for (int j = 0; j < n_r; ++j) rn += radial[(size_t)k * n_r + j] * radial[(size_t)k * n_r + j];
            rnorm[k] = sqrt(rn);
        }
    }
    const int64_t ns = (int64_t)L->r.size();
    if (ns >= (int64_t)1 << 31) return fail(TM_ERR_UNSUPPORTED, "tm_load_library: too many spots");
    // distinct radii (rows of the sparse kernel's shared-memory image) and packed spots
    {
        std::vector<int32_t> rr(L->r);
        std::sort(rr.begin(), rr.end());
        rr.erase(std::unique(rr.begin(), rr.end()), rr.end());
        L->radii = rr;
    }
    std::vector<int32_t> row_of(n_r, -1);
    for (size_t i = 0; i < L->radii.size(); ++i) row_of[L->radii[i]] = (int32_t)i;
    spot.resize(ns);
    const int n_rows = (int)std::max<size_t>(1, L->radii.size());
    for (int64_t i = 0; i < ns; ++i) {
        const int row = row_of[L->r[i]];
        const int t = L->t[i];
        const int w = (n_theta - t + 31) / 32;
        if (row < 0 || row >= n_rows || row >= 8192 || t < 0 || t >= n_theta || t >= 2048 || w < 1 || w > 63)
            return fail(TM_ERR_INVALID_ARG, "tm_load_library: internal layout check failed for spot %lld",
                        (long long)i);
        spot[i].x = t | (row << 11) | (w << 24);
        memcpy(&spot[i].y, &L->I[i], 4);
    }
    for (float I : L->I)
        if (!(I >= 0.0f)) L->nonneg = 0;
    // offsets in the dual-copy and wrap-free row layouts (0 where a layout cannot be used)
    const int64_t pd = tmgb::sparse_pitch(n_theta, tmgb::TM_LAYOUT_DUAL);
    const int64_t pw = tmgb::sparse_pitch(n_theta, tmgb::TM_LAYOUT_WF);
    const bool dual_ok = 2 * n_rows * pd <= 65535, wf_ok = n_rows * pw <= 65535;
    P->spot2.resize(ns);
    for (int64_t i = 0; i < ns; ++i) {
        const int64_t row = row_of[L->r[i]], t = L->t[i];
        const int64_t od = dual_ok ? ((t & 1) ? n_rows + row : row) * pd + (t & ~(int64_t)1) : 0;
        const int64_t ow = wf_ok ? row * pw + t : 0;
        P->spot2[i].x = (int32_t)(uint32_t)(od | (ow << 16));
        P->spot2[i].y = spot[i].y;
    }
    // per spot, the sparse kernel's window-table entries for its pruning bound: row * nchw +
    // (t + h ww) / 32 for h = 0, 1, 2, as the first (16 bits) and two increments (8 bits each);
    // none when the table does not fit (the kernel then bounds by whole rows)
    {
        const int ww = tmgb::prune_ww(n_theta), nchw = tmgb::prune_nchw(n_theta);
        const bool win = nchw + tmgb::prune_ncov(n_theta) - 1 <= 32 && (int64_t)n_rows * nchw <= 65536 &&
                         (2 * ww) / 32 + 1 <= 255;
        if (win) {
            P->bspot.resize(ns);
            for (int64_t i = 0; i < ns; ++i) {
                const int64_t row = row_of[L->r[i]], t = L->t[i];
                const int64_t j0 = row * nchw + (t >> 5);
                const int64_t d1 = ((t + ww) >> 5) - (t >> 5), d2 = ((t + 2 * ww) >> 5) - (t >> 5);
                if (j0 > 65535 || d1 < 0 || d2 < d1 || d2 > 255 || j0 + d2 >= (int64_t)n_rows * nchw)
                    return fail(TM_ERR_INVALID_ARG, "tm_load_library: internal window-table check failed for spot %lld",
                                (long long)i);
                P->bspot[i].x = spot[i].y;
                P->bspot[i].y = (int32_t)(uint32_t)(j0 | (d1 << 16) | (d2 << 24));
            }
        }
    }
    P->meta.resize(L->K);
    for (int64_t k = 0; k < L->K; ++k) {
        const int64_t cnt = L->off[k + 1] - L->off[k];
        if (cnt > 65535) return fail(TM_ERR_UNSUPPORTED, "tm_load_library: template %lld has %lld spots (max 65535)",
                                     (long long)k, (long long)cnt);
        int32_t nb, sb;
        memcpy(&nb, &L->norm[k], 4);
        // sum of |intensities|, rounded up: bounds the rounding of the sparse kernel's sums
        double isum = 0.0;
        for (int64_t i = L->off[k]; i < L->off[k + 1]; ++i) isum += fabs((double)L->I[i]);
        float fs = (float)isum;
        if ((double)fs < isum) fs = nextafterf(fs, INFINITY);
        memcpy(&sb, &fs, 4);
        P->meta[k] = make_int4((int32_t)L->off[k], (int32_t)(cnt | ((int64_t)P->nshift[k] << 16)), nb, sb);
    }
    // the bound entries again, templates ordered by spot count (descending, stable: the words
    // taken last are the cheapest) and each word's entries stored spot-major with its 32 lanes
    // adjacent, so the bound loop of a warp neither diverges much nor scatters its loads;
    // padding positions hold empty templates
    if (!P->bspot.empty()) {
        const int64_t words = (L->K + 31) / 32;
        std::vector<int32_t> perm(L->K);
        for (int64_t k = 0; k < L->K; ++k) perm[k] = (int32_t)k;
        std::stable_sort(perm.begin(), perm.end(), [&](int32_t a, int32_t b) {
            return L->off[a + 1] - L->off[a] > L->off[b + 1] - L->off[b];
        });
        P->smeta.assign(words * 32, make_int4(0, 0, 0, 0));
        P->sperm.assign(words * 32, 0);
        P->ellw.resize(words);
        int64_t n_ell = 0;
        for (int64_t w = 0; w < words; ++w) {
            int64_t mc = 0;
            for (int64_t j = 32 * w; j < std::min<int64_t>(32 * w + 32, L->K); ++j)
                mc = std::max<int64_t>(mc, L->off[perm[j] + 1] - L->off[perm[j]]);
            if (n_ell > INT32_MAX - 32 * mc)
                return fail(TM_ERR_UNSUPPORTED, "tm_load_library: too many spots for the sorted bound entries");
            P->ellw[w] = (int32_t)n_ell;
            n_ell += 32 * mc;
        }
        P->ell.assign(n_ell, make_int2(0, 0));
        for (int64_t j = 0; j < L->K; ++j) {
            const int32_t k = perm[j];
            P->sperm[j] = k;
            P->smeta[j] = P->meta[k];
            const int64_t w = j >> 5, l = j & 31;
            for (int64_t i = 0; i < L->off[k + 1] - L->off[k]; ++i)
                P->ell[P->ellw[w] + 32 * i + l] = P->bspot[L->off[k] + i];
        }
    }
    return TM_OK;
}

int build_library(tm_ctx* ctx, const tm_library_desc* d, Library* L) {
    Prepared P;
    int rc = prepare_library(d, L, &P);
    if (rc) return rc;
    std::vector<int2>& spot = P.spot;
    std::vector<int32_t>& nshift = P.nshift;
    std::vector<double>& radial = P.radial;
    std::vector<double>& rnorm = P.rnorm;
    std::vector<int32_t> off32(L->K + 1);
    for (int64_t k = 0; k <= L->K; ++k) off32[k] = (int32_t)L->off[k];
    // radial profiles at the library's distinct radii only (zero elsewhere), [K][n_pad]
    // with n_pad = n_rad rounded up to 4 and zero padding
    const size_t n_rad = L->radii.size(), n_pad = (n_rad + 3) & ~(size_t)3;
    std::vector<float> radf(n_pad * (size_t)L->K, 0.0f), rnf(rnorm.begin(), rnorm.end());
    for (int64_t k = 0; k < L->K; ++k)
        for (size_t j = 0; j < n_rad; ++j)
            radf[(size_t)k * n_pad + j] = (float)radial[(size_t)k * L->n_r + L->radii[j]];
    std::vector<int32_t> rt(L->r.size());
    for (size_t i = 0; i < rt.size(); ++i) rt[i] = L->r[i] | (L->t[i] << 16);
    struct Up { void** dst; const void* src; size_t bytes; const char* what; };
    Up ups[] = {
        {(void**)&L->d_off, off32.data(), off32.size() * 4, "library offsets"},
        {(void**)&L->d_spot, spot.data(), spot.size() * 8, "library spots"},
        {(void**)&L->d_spot2, P.spot2.data(), P.spot2.size() * 8, "library spot offsets"},
        {(void**)&L->d_meta, P.meta.data(), P.meta.size() * 16, "library template metadata"},
        {(void**)&L->d_norm, L->norm.data(), L->norm.size() * 4, "library norms"},
        {(void**)&L->d_nshift, nshift.data(), nshift.size() * 4, "library shifts"},
        {(void**)&L->d_radial, radf.data(), radf.size() * 4, "library radial profiles"},
        {(void**)&L->d_rnorm, rnf.data(), rnf.size() * 4, "library radial norms"},
        {(void**)&L->d_rt, rt.data(), rt.size() * 4, "library spot positions"},
        {(void**)&L->d_radii, L->radii.data(), L->radii.size() * 4, "library radii"},
    };
    for (auto& u : ups) {
        rc = dev_alloc(ctx, u.dst, u.bytes, u.what);
        if (rc) return rc;
        L->bytes += u.bytes ? u.bytes : 16;
        if (u.bytes) TM_CUDA(cudaMemcpy(*u.dst, u.src, u.bytes, cudaMemcpyHostToDevice), u.what);
    }
    if (!P.bspot.empty()) {                        // absent (null) when the window table does not fit
        const size_t b = P.bspot.size() * 8;
        rc = dev_alloc(ctx, (void**)&L->d_bspot, b, "library spot bound entries");
        if (rc) return rc;
        L->bytes += b;
        TM_CUDA(cudaMemcpy(L->d_bspot, P.bspot.data(), b, cudaMemcpyHostToDevice), "library spot bound entries");
        Up sorted[] = {
            {(void**)&L->d_smeta, P.smeta.data(), P.smeta.size() * 16, "library sorted template metadata"},
            {(void**)&L->d_sperm, P.sperm.data(), P.sperm.size() * 4, "library sorted template order"},
            {(void**)&L->d_ellw, P.ellw.data(), P.ellw.size() * 4, "library sorted bound words"},
            {(void**)&L->d_ell, P.ell.data(), P.ell.size() * 8, "library sorted bound entries"},
        };
        for (auto& u : sorted) {
            rc = dev_alloc(ctx, u.dst, u.bytes ? u.bytes : 16, u.what);
            if (rc) return rc;
            L->bytes += u.bytes ? u.bytes : 16;
            if (u.bytes) TM_CUDA(cudaMemcpy(*u.dst, u.src, u.bytes, cudaMemcpyHostToDevice), u.what);
        }
    }
    return TM_OK;
}

void free_library(tm_ctx* ctx, Library* L) {
    void* ps[] = {L->d_off,    L->d_spot,  L->d_spot2, L->d_meta,  L->d_norm,   L->d_nshift, L->d_radial,
                  L->d_rnorm,  L->d_rt,    L->d_radii, L->d_bspot, L->d_that,   L->d_rowmap,
                  L->d_smeta,  L->d_sperm, L->d_ellw,  L->d_ell};
    for (void* p : ps)
        if (p) cudaFree(p);
    ctx->used -= std::min(ctx->used, L->bytes + L->that_bytes);
}

tmgb::SparseLib sparse_view(const Library* L) {
    tmgb::SparseLib v;
    v.off = L->d_off;
    v.spot = L->d_spot;
    v.spot2 = L->d_spot2;
    v.bspot = L->d_bspot;
    v.meta = L->d_meta;
    v.smeta = L->d_smeta;
    v.sperm = L->d_sperm;
    v.ellw = L->d_ellw;
    v.ell = L->d_ell;
    v.norm = L->d_norm;
    v.nshift = L->d_nshift;
    v.radii = L->d_radii;
    v.n_rad = (int32_t)std::max<size_t>(1, L->radii.size());
    v.K = (int32_t)L->K;
    v.K0 = (int32_t)L->K0;
    v.mirror = L->mirror;
    v.words = (int32_t)((L->K + 31) / 32);
    v.nonneg = L->nonneg;
    return v;
}

// Ray steps of the polar grid (fixed point, built in double precision), cached per grid.
int polar_rays(tm_ctx* ctx, int n_theta, double dr, const longlong2** out) {
    const auto key = std::make_pair(n_theta, dr);
    auto it = ctx->rays.find(key);
    if (it == ctx->rays.end()) {
        std::vector<longlong2> v(n_theta);
        tmgb::build_polar_rays(n_theta, dr, v.data());
        longlong2* d = nullptr;
        int rc = dev_alloc(ctx, (void**)&d, v.size() * sizeof(longlong2), "polar rays");
        if (rc) return rc;
        TM_CUDA(cudaMemcpy(d, v.data(), v.size() * sizeof(longlong2), cudaMemcpyHostToDevice), "polar rays");
        it = ctx->rays.emplace(key, d).first;
    }
    *out = it->second;
    return TM_OK;
}

uint16_t f32_to_bf16(float f) {
    uint32_t u;
    memcpy(&u, &f, 4);
    if ((u & 0x7fffffffu) > 0x7f800000u) return 0x7fc0;      // NaN
    u += 0x7fffu + ((u >> 16) & 1u);                           // round to nearest even
    return (uint16_t)(u >> 16);
}

// Inverse-DFT basis for the radix-2 split (rows: shift s < n/2; columns: even-m then odd-m
// (re, im) pairs) and the twiddle table, built in FP64 and cached per n_theta.
int spectral_tables(tm_ctx* ctx, int n_theta, SpectralTables* out) {
    auto it = ctx->spectral.find(n_theta);
    if (it == ctx->spectral.end()) {
        const int R = tmgb::dense_basis_rows(), C = tmgb::dense_basis_cols(), half = C / 2;
        const int H = n_theta / 2;
        std::vector<uint16_t> basis((size_t)R * C, 0);
        for (int s = 0; s < R && s < H; ++s) {
            for (int kk = 0; kk < C; ++kk) {
                const int part = kk / half, j = (kk % half) / 2, comp = kk % 2;
                const int m = 2 * j + part;
                if (m > H) continue;
                const double w = (m == 0 || m == H) ? 1.0 : 2.0;
                const double ang = 2.0 * kPi * (double)m * (double)s / n_theta;
                const double v = (w / n_theta) * (comp == 0 ? cos(ang) : -sin(ang));
                basis[(size_t)s * C + kk] = f32_to_bf16((float)v);
            }
        }
        std::vector<float2> tw(n_theta);
        for (int j = 0; j < n_theta; ++j) {
            const double ang = 2.0 * kPi * j / n_theta;
            tw[j] = make_float2((float)cos(ang), (float)sin(ang));
        }
        // forward DFT matrix, column-major [n_theta][2 x 192]: column 2 j + comp of slot j
        // (m = 2 j for j < 96, else 2 (j - 96) + 1)
        const int slots = tmgb::dense_slots();
        std::vector<float> dm((size_t)n_theta * 2 * slots, 0.0f);
        for (int j = 0; j < slots; ++j) {
            const int m = j < slots / 2 ? 2 * j : 2 * (j - slots / 2) + 1;
            if (m > H) continue;
            for (int th = 0; th < n_theta; ++th) {
                const double ang = 2.0 * kPi * (double)(((int64_t)m * th) % n_theta) / n_theta;
                dm[(size_t)(2 * j) * n_theta + th] = (float)cos(ang);
                dm[(size_t)(2 * j + 1) * n_theta + th] = (float)-sin(ang);
            }
        }
        SpectralTables t;
        int rc = dev_alloc(ctx, &t.basis, basis.size() * 2, "dft basis");
        if (!rc) rc = dev_alloc(ctx, (void**)&t.twiddle, tw.size() * 8, "twiddles");
        if (!rc) rc = dev_alloc(ctx, (void**)&t.dftmat, dm.size() * 4, "dft matrix");
        if (rc) return rc;
        TM_CUDA(cudaMemcpy(t.basis, basis.data(), basis.size() * 2, cudaMemcpyHostToDevice), "dft basis");
        TM_CUDA(cudaMemcpy(t.twiddle, tw.data(), tw.size() * 8, cudaMemcpyHostToDevice), "twiddles");
        TM_CUDA(cudaMemcpy(t.dftmat, dm.data(), dm.size() * 4, cudaMemcpyHostToDevice), "dft matrix");
        it = ctx->spectral.emplace(n_theta, t).first;
    }
    *out = it->second;
    return TM_OK;
}

// Union of the radii the libraries use, and the radius -> row map of the spectra.
int radius_map(tm_ctx* ctx, Library* const* libs, const int32_t* ids, int n_libs, int n_r, RadiusMap* out) {
    std::string key;
    for (int i = 0; i < n_libs; ++i) key += std::to_string(ids[i]) + ",";
    auto it = ctx->radius_maps.find(key);
    if (it == ctx->radius_maps.end()) {
        std::vector<int32_t> u;
        for (int i = 0; i < n_libs; ++i) u.insert(u.end(), libs[i]->radii.begin(), libs[i]->radii.end());
        std::sort(u.begin(), u.end());
        u.erase(std::unique(u.begin(), u.end()), u.end());
        if (u.empty()) u.push_back(0);
        std::vector<int32_t> rmap(n_r, -1);
        for (size_t i = 0; i < u.size(); ++i) rmap[u[i]] = (int32_t)i;
        std::vector<uint8_t> keep(n_r, 0);
        for (int32_t r : u) keep[r] = 1;
        RadiusMap m;
        m.n_rad = (int)u.size();
        int rc = dev_alloc(ctx, (void**)&m.radii, u.size() * 4, "radius list");
        if (!rc) rc = dev_alloc(ctx, (void**)&m.rmap, rmap.size() * 4, "radius map");
        if (!rc) rc = dev_alloc(ctx, (void**)&m.keep_row, keep.size(), "row mask");
        if (rc) return rc;
        TM_CUDA(cudaMemcpy(m.radii, u.data(), u.size() * 4, cudaMemcpyHostToDevice), "radius list");
        TM_CUDA(cudaMemcpy(m.rmap, rmap.data(), rmap.size() * 4, cudaMemcpyHostToDevice), "radius map");
        TM_CUDA(cudaMemcpy(m.keep_row, keep.data(), keep.size(), cudaMemcpyHostToDevice), "row mask");
        it = ctx->radius_maps.emplace(key, m).first;
    }
    *out = it->second;
    return TM_OK;
}

// ---------------------------------------------------------------- tensor-core path (A7)

// Batch of the tensor-core stages: patterns whose spectra P^ and products G are resident at
// once, sized so that G (768 B per pattern and padded template) stays within 4 GiB (or a
// quarter of the context's free budget).
struct TensorPlan {
    int64_t nb = 0;
    size_t dftc_per = 0, phat_per = 0, g_per = 0;   // bytes per pattern
    size_t bytes(int64_t m) const { return (size_t)m * (dftc_per + phat_per + g_per) + ((size_t)32 << 20); }
};
struct TensorBuffers {
    int64_t nb = 0;
    float* dftc = nullptr;
    void* phat = nullptr;
    void* g = nullptr;
    void* cublas_ws = nullptr;
    size_t cublas_ws_bytes = 0;
};

inline int lib_R(const Library* L) { return ((int)std::max<size_t>(1, L->radii.size()) + 7) & ~7; }
inline int lib_K_pad(const Library* L) { return (int)((L->K + 63) & ~(int64_t)63); }

int tensor_plan(tm_ctx* ctx, Library* const* libs, int n_libs, int n_theta, TensorPlan* tp) {
    int R = 8, K_pad = 64;
    for (int i = 0; i < n_libs; ++i) {
        R = std::max(R, lib_R(libs[i]));
        K_pad = std::max(K_pad, lib_K_pad(libs[i]));
    }
    const size_t slots = (size_t)tmgb::dense_slots();
    tp->dftc_per = slots * 2 * (size_t)libs[0]->n_r * 4;
    tp->phat_per = slots * 2 * 2 * R * 2;
    tp->g_per = slots * 2 * K_pad * 2;
    size_t cap = (size_t)4 << 30;
    if (ctx->budget) {
        const size_t freeb = ctx->budget > ctx->used ? ctx->budget - ctx->used : 0;
        cap = std::min(cap, freeb / 4);
    }
    tp->nb = (int64_t)std::max<size_t>(1, cap / (tp->dftc_per + tp->phat_per + tp->g_per));
    return TM_OK;
}

int tensor_buffers(tm_ctx* ctx, cudaStream_t st, const TensorPlan& tp, int64_t nb, TensorBuffers* tb) {
    tb->nb = nb;
    tb->cublas_ws_bytes = (size_t)32 << 20;
    int rc = workspace(ctx, st, "dftc", (size_t)nb * tp.dftc_per, (void**)&tb->dftc);
    if (!rc) rc = workspace(ctx, st, "phat", (size_t)nb * tp.phat_per, &tb->phat);
    if (!rc) rc = workspace(ctx, st, "gmat", (size_t)nb * tp.g_per, &tb->g);
    if (!rc) rc = workspace(ctx, st, "cublas_ws", tb->cublas_ws_bytes, &tb->cublas_ws);
    return rc;
}

// Angular spectra T^ of a library's templates (stage A's left operand), built on the device the
// first time the tensor-core path uses the library; the call waits for the build, so that work
// on other streams can use the spectra as soon as it returns.
int ensure_spectra(tm_ctx* ctx, Library* L, const SpectralTables& spec, cudaStream_t st) {
    if (L->d_that) return TM_OK;
    if (ctx->capturing) return fail(TM_ERR_CUDA, "library spectra built during graph capture");
    const int R = lib_R(L), K_pad = lib_K_pad(L);
    std::vector<int32_t> rowmap(L->n_r, -1);
    for (size_t i = 0; i < L->radii.size(); ++i) rowmap[L->radii[i]] = (int32_t)i;
    const size_t tb = (size_t)tmgb::dense_slots() * 2 * R * K_pad * 2;
    void* that = nullptr;
    void* rows = nullptr;
    int rc = dev_alloc(ctx, &that, tb, "library spectra");
    if (rc) return rc;
    rc = dev_alloc(ctx, &rows, rowmap.size() * 4, "library radius rows");
    if (rc) {
        dev_free(ctx, that, tb);
        return rc;
    }
    L->d_that = that;
    L->d_rowmap = (int32_t*)rows;
    L->R = R;
    L->K_pad = K_pad;
    L->that_bytes = tb + rowmap.size() * 4;
    TM_CUDA(cudaMemcpy(L->d_rowmap, rowmap.data(), rowmap.size() * 4, cudaMemcpyHostToDevice), "library radius rows");
    TM_CUDA(tmgb::launch_spectra(L->d_off, L->d_rt, L->d_spot, L->d_norm, L->d_rowmap, (int)L->K, K_pad, R, L->n_theta,
                                 spec.twiddle, L->d_that, st),
            "library spectra");
    TM_CUDA(cudaStreamSynchronize(st), "library spectra");
    return TM_OK;
}

// Tensor map of G [192][nb][2][K_pad] BF16 for stage B: 4-D (k, c, p, j), boxes of
// 64 templates x 2 x 1 pattern x 32 slots, 128-byte swizzle, zero fill past K.
int g_tensor_map(tm_ctx* ctx, void* g, int K, int K_pad, int64_t nb, CUtensorMap* out) {
    if (!ctx->encode_tiled) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        const cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) {
            cudaGetLastError();
            return fail(TM_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
        }
        ctx->encode_tiled = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    }
    const cuuint64_t dims[4] = {(cuuint64_t)K, 2, (cuuint64_t)nb, (cuuint64_t)tmgb::dense_slots()};
    const cuuint64_t strides[3] = {(cuuint64_t)K_pad * 2, (cuuint64_t)K_pad * 4, (cuuint64_t)nb * K_pad * 4};
    const cuuint32_t box[4] = {64, 2, 1, 32};
    const cuuint32_t es[4] = {1, 1, 1, 1};
    const CUresult r = ctx->encode_tiled(out, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, g, dims, strides, box, es,
                                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(TM_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return TM_OK;
}

// Stage A: for every frequency slot j, G_j [K_pad x 2 nb] = T^_j [K_pad x 2 R] x P^_j [2 R x 2 nb]
// (column-major, BF16 in and out, FP32 accumulation): one strided batched GEMM on the tensor
// cores through cuBLAS (a plain library GEMM).
int cublas_on(tm_ctx* ctx, cudaStream_t st, const TensorBuffers& tb) {
    cublasStatus_t s = CUBLAS_STATUS_SUCCESS;
    if (!ctx->cublas) {
        if (ctx->capturing) return fail(TM_ERR_CUDA, "cuBLAS handle created during graph capture");
        s = cublasCreate(&ctx->cublas);
        if (s != CUBLAS_STATUS_SUCCESS) {
            ctx->cublas = nullptr;
            return fail(TM_ERR_CUDA, "cublasCreate failed (%d)", (int)s);
        }
    }
    s = cublasSetStream(ctx->cublas, st);
    if (s == CUBLAS_STATUS_SUCCESS) s = cublasSetWorkspace(ctx->cublas, tb.cublas_ws, tb.cublas_ws_bytes);
    if (s != CUBLAS_STATUS_SUCCESS) return fail(TM_ERR_CUDA, "cuBLAS set-up failed (%d)", (int)s);
    return TM_OK;
}

// Angular DFT of a batch of polar images: dftc [2 x 192][nb n_r] = polar^T-rows x DFT matrix, i.e.
// for every pattern and polar row the (Re, Im) of P^ at each frequency slot, in TF32 with FP32
// accumulation (cuBLAS, a plain library GEMM).  Rows the polar stage did not store give values
// no later stage reads.
int dft_gemm(tm_ctx* ctx, cudaStream_t st, const SpectralTables& spec, const float* polar, int64_t nb, int n_r,
             int n_theta, const TensorBuffers& tb) {
    int rc = cublas_on(ctx, st, tb);
    if (rc) return rc;
    const float one = 1.0f, zero = 0.0f;
    const cublasStatus_t s = cublasGemmEx(ctx->cublas, CUBLAS_OP_T, CUBLAS_OP_N, (int)(nb * n_r),
                                          2 * tmgb::dense_slots(), n_theta, &one, polar, CUDA_R_32F, n_theta,
                                          spec.dftmat, CUDA_R_32F, n_theta, &zero, tb.dftc, CUDA_R_32F,
                                          (int)(nb * n_r), CUBLAS_COMPUTE_32F_FAST_TF32, CUBLAS_GEMM_DEFAULT);
    if (s != CUBLAS_STATUS_SUCCESS) return fail(TM_ERR_CUDA, "angular DFT GEMM failed (cuBLAS status %d)", (int)s);
    return TM_OK;
}

int stage_a(tm_ctx* ctx, cudaStream_t st, const Library* L, const TensorBuffers& tb, int64_t nb) {
    int rc = cublas_on(ctx, st, tb);
    if (rc) return rc;
    cublasStatus_t s = CUBLAS_STATUS_SUCCESS;
    const float one = 1.0f, zero = 0.0f;
    const int R2 = 2 * L->R;
    s = cublasGemmStridedBatchedEx(ctx->cublas, CUBLAS_OP_N, CUBLAS_OP_N, L->K_pad, (int)(2 * nb), R2, &one,
                                   L->d_that, CUDA_R_16BF, L->K_pad, (long long)R2 * L->K_pad, tb.phat, CUDA_R_16BF,
                                   R2, (long long)nb * 2 * R2, &zero, tb.g, CUDA_R_16BF, L->K_pad,
                                   (long long)2 * nb * L->K_pad, tmgb::dense_slots(), CUBLAS_COMPUTE_32F,
                                   CUBLAS_GEMM_DEFAULT);
    if (s != CUBLAS_STATUS_SUCCESS) return fail(TM_ERR_CUDA, "stage A GEMM failed (cuBLAS status %d)", (int)s);
    return TM_OK;
}

// Pre-scores of libraries libs[0..n_libs) for the call's rows [0, m): per batch of tb.nb patterns
// the angular DFT of the polar rows (once), then per library its P^ (packed), stage A (G) and
// stage B (inverse DFT and maximum over shifts on tcgen05).  masks[i] (nullable): templates to
// score per row; outs[i] [m][K_i] (-NaN where not scored).
int prescore_rows(tm_ctx* ctx, cudaStream_t st, Library* const* libs, int n_libs, const SpectralTables& spec,
                  const TensorBuffers& tb, const float* polar, const float* pnorm, int64_t m,
                  uint32_t* const* masks, float* const* outs, int stall, int64_t* launches) {
    const int n_r = libs[0]->n_r, n_theta = libs[0]->n_theta;
    for (int64_t b0 = 0; b0 < m; b0 += tb.nb) {
        const int64_t nb = std::min(tb.nb, m - b0);
        {
            StageTimer tmr(ctx, TM_STAGE_DFT, st);
            const int rc = dft_gemm(ctx, st, spec, polar + (size_t)b0 * n_r * n_theta, nb, n_r, n_theta, tb);
            if (rc) return rc;
        }
        for (int i = 0; i < n_libs; ++i) {
            const Library* L = libs[i];
            const int n_rad = (int)std::max<size_t>(1, L->radii.size());
            {
                StageTimer tmr(ctx, TM_STAGE_DFT, st);
                TM_CUDA(tmgb::launch_pack(tb.dftc, pnorm + b0, nb, n_r, L->d_radii, n_rad, L->R, tb.phat,
                                          tmgb::device_sms(), st),
                        "tensor path: pack");
            }
            {
                StageTimer tmr(ctx, TM_STAGE_GEMM, st);
                const int rc = stage_a(ctx, st, L, tb, nb);
                if (rc) return rc;
            }
            CUtensorMap map;
            const int rc = g_tensor_map(ctx, tb.g, (int)L->K, L->K_pad, nb, &map);
            if (rc) return rc;
            tmgb::DenseCall dc{};
            dc.n = nb;
            dc.p0 = b0;
            dc.n_theta = n_theta;
            dc.K = (int)L->K;
            dc.basis = spec.basis;
            dc.mask = masks ? masks[i] : nullptr;
            dc.words = (int)((L->K + 31) / 32);
            dc.pre = outs[i];
            dc.error = ctx->d_error;
            dc.stall = stall;
            {
                StageTimer tmr(ctx, TM_STAGE_DENSE, st);
                TM_CUDA(tmgb::launch_dense(&map, dc, tmgb::device_sms(), st), "tensor path: stage B");
            }
            *launches += 2;              // this library's kernels (the GEMMs are cuBLAS's)
        }
    }
    return TM_OK;
}

// Signature of a set of libraries for the autotuner: shapes, not ids, so that a tuning
// cache written by one process applies in the next.
std::string tune_key(Library* const* libs, int n_libs, int top_n) {
    std::string k = "sparse";
    for (int i = 0; i < n_libs; ++i) {
        k += "|" + std::to_string(libs[i]->K) + "/" + std::to_string(libs[i]->r.size()) + "/" +
             std::to_string(libs[i]->radii.size()) + "/" + std::to_string(libs[i]->n_theta);
    }
    return k + "|N" + std::to_string(top_n);
}

int check_params(const tm_index_params* p) {
    if (!p) return fail(TM_ERR_INVALID_ARG, "params is NULL");
    if (!(p->gamma > 0.0 && isfinite(p->gamma))) return fail(TM_ERR_INVALID_ARG, "gamma must be finite and > 0");
    if (!isfinite(p->subtract)) return fail(TM_ERR_INVALID_ARG, "subtract must be finite");
    if (isinf(p->cx) || isinf(p->cy) || fabs(p->cx) >= 1048576.0 || fabs(p->cy) >= 1048576.0)
        return fail(TM_ERR_INVALID_ARG, "centre must be NaN or finite with |c| < 2^20");
    if (!(p->prefilter_fraction > 0.0 && p->prefilter_fraction <= 1.0))
        return fail(TM_ERR_INVALID_ARG, "prefilter_fraction must be in (0, 1]");
    if (p->top_n < 1 || p->top_n > TM_MAX_TOPN) return fail(TM_ERR_INVALID_ARG, "top_n must be in [1, %d]", TM_MAX_TOPN);
    if (((uintptr_t)p->pixel_mask & 15) != 0) return fail(TM_ERR_INVALID_ARG, "pixel_mask must be 16-byte aligned");
    if (!(p->threshold >= 0.0 && isfinite(p->threshold)))
        return fail(TM_ERR_INVALID_ARG, "threshold must be finite and >= 0");
    return TM_OK;
}

}  // namespace

namespace tmgb {
int check_index_params(const tm_index_params* p) { return check_params(p); }
}  // namespace tmgb

namespace {

tmgb::RadialLib radial_lib(const Library* L) {
    return tmgb::RadialLib{L->d_radial, L->d_rnorm, L->d_radii, (int32_t)L->radii.size(), (int32_t)L->K};
}

int keep_count(double f, int64_t K) {
    if (f >= 1.0) return (int)K;
    int64_t k = (int64_t)ceil(f * (double)K);
    return (int)std::max<int64_t>(1, std::min<int64_t>(k, K));
}

Library* find_lib(tm_ctx* ctx, int id) {
    auto it = ctx->libs.find(id);
    return it == ctx->libs.end() ? nullptr : it->second.get();
}

}  // namespace

namespace tmgb {
int library_view(tm_ctx* ctx, int lib_id, int* device, int* num_sms, SparseLib* view, int* n_r, int* n_theta,
                 double* dr) {
    if (!ctx) return fail(TM_ERR_INVALID_ARG, "library_view: ctx is NULL");
    std::lock_guard<std::mutex> lk(ctx->mu);
    Library* L = find_lib(ctx, lib_id);
    if (!L) return fail(TM_ERR_NOT_FOUND, "no library %d", lib_id);
    *device = ctx->device;
    *num_sms = ctx->num_sms;
    *view = sparse_view(L);
    *n_r = L->n_r;
    *n_theta = L->n_theta;
    *dr = L->dr;
    return TM_OK;
}
}  // namespace tmgb

// ====================================================================== C ABI

extern "C" {

// Whole path from host buffers: chunks of the batch alternate between two streams, so the
// host->device copy of one chunk overlaps the kernels of the previous one.
int tm_index_patterns_host(tm_ctx* ctx, const tm_index_params* params, const void* frames_host, int32_t dtype,
                           int64_t n, int32_t H, int32_t W, const float* centres_host, const int32_t* lib_ids,
                           int32_t n_libs, tm_hit* out_host, int64_t chunk, tm_stats* stats) {
    if (!ctx) return fail(TM_ERR_INVALID_ARG, "tm_index_patterns_host: ctx is NULL");
    int rc = check_params(params);
    if (rc) return rc;
    if (n < 0 || H < 1 || W < 1 || H > 32000 || W > 32000)
        return fail(TM_ERR_INVALID_ARG, "tm_index_patterns_host: bad shape");
    if (dtype != TM_DTYPE_U16 && dtype != TM_DTYPE_F32) return fail(TM_ERR_INVALID_ARG, "tm_index_patterns_host: dtype");
    if (n_libs < 1 || n_libs > TM_MAX_LIBS || !lib_ids)
        return fail(TM_ERR_INVALID_ARG, "tm_index_patterns_host: n_libs must be in [1, %d]", TM_MAX_LIBS);
    if (chunk < 0) return fail(TM_ERR_INVALID_ARG, "tm_index_patterns_host: chunk must be >= 0");
    if (stats) memset(stats, 0, sizeof *stats);
    if (n == 0) return TM_OK;
    if (!frames_host || !out_host) return fail(TM_ERR_INVALID_ARG, "tm_index_patterns_host: NULL buffer");
    if (chunk == 0) chunk = 4096;
    if (chunk > n) chunk = n;
    std::lock_guard<std::mutex> hl(ctx->host_mu);
    DeviceGuard g(ctx->device);
    const size_t esz = dtype == TM_DTYPE_U16 ? 2 : 4;
    const size_t frame_bytes = (size_t)H * W * esz;
    const int N = params->top_n;
    const size_t hit_row = (size_t)N * sizeof(tm_hit);       // one pattern's hits for one library
    void* dfr[2];
    void* dcen[2] = {nullptr, nullptr};
    void* dhit[2];
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        for (int i = 0; i < 2; ++i) {
            if (!ctx->host_streams[i])
                TM_CUDA(cudaStreamCreateWithFlags(&ctx->host_streams[i], cudaStreamNonBlocking), "host streams");
            cudaStream_t hs = ctx->host_streams[i];
            rc = workspace(ctx, hs, "host_frames", (size_t)chunk * frame_bytes, &dfr[i]);
            if (!rc) rc = workspace(ctx, hs, "host_hits", (size_t)n_libs * chunk * hit_row, &dhit[i]);
            if (!rc && centres_host) rc = workspace(ctx, hs, "host_centres", (size_t)chunk * 8, &dcen[i]);
            if (rc) return rc;
        }
    }
    int slot = 0;
    for (int64_t p0 = 0; p0 < n; p0 += chunk, slot ^= 1) {
        const int64_t m = std::min<int64_t>(chunk, n - p0);
        cudaStream_t hs = ctx->host_streams[slot];
        cudaError_t e = cudaMemcpyAsync(dfr[slot], (const char*)frames_host + (size_t)p0 * frame_bytes,
                                        (size_t)m * frame_bytes, cudaMemcpyHostToDevice, hs);
        if (e == cudaSuccess && centres_host)
            e = cudaMemcpyAsync(dcen[slot], centres_host + 2 * p0, (size_t)m * 8, cudaMemcpyHostToDevice, hs);
        if (e != cudaSuccess) {
            cudaGetLastError();
            rc = fail(TM_ERR_CUDA, "tm_index_patterns_host: copy to the device: %s", cudaGetErrorString(e));
            break;
        }
        tm_stats cs;
        rc = tm_index_patterns(ctx, params, dfr[slot], dtype, m, H, W, centres_host ? (const float*)dcen[slot] : nullptr,
                               lib_ids, n_libs, (tm_hit*)dhit[slot], stats ? &cs : nullptr, hs);
        if (rc) break;
        // hits [n_libs][m][N] of the chunk -> rows p0.. of out_host [n_libs][n][N]
        e = cudaMemcpy2DAsync((char*)out_host + (size_t)p0 * hit_row, (size_t)n * hit_row, dhit[slot],
                              (size_t)m * hit_row, (size_t)m * hit_row, (size_t)n_libs, cudaMemcpyDeviceToHost, hs);
        if (e != cudaSuccess) {
            cudaGetLastError();
            rc = fail(TM_ERR_CUDA, "tm_index_patterns_host: copy to the host: %s", cudaGetErrorString(e));
            break;
        }
        if (stats) {
            stats->patterns += cs.patterns;
            stats->correlations += cs.correlations;
            stats->templates_scored += cs.templates_scored;
            stats->launches += cs.launches;
        }
    }
    for (cudaStream_t hs : ctx->host_streams) {
        cudaError_t e = cudaStreamSynchronize(hs);
        if (e != cudaSuccess && !rc) {
            cudaGetLastError();
            rc = fail(TM_ERR_CUDA, "tm_index_patterns_host: %s", cudaGetErrorString(e));
        }
    }
    return rc;
}

int tm_frame_sum(tm_ctx* ctx, const void* frames_dev, int32_t dtype, int64_t n, int32_t H, int32_t W,
                 int32_t accumulate, double* sum_dev, void* stream) {
    if (!ctx) return fail(TM_ERR_INVALID_ARG, "tm_frame_sum: ctx is NULL");
    if (n < 0 || H < 1 || W < 1 || H > 32000 || W > 32000) return fail(TM_ERR_INVALID_ARG, "tm_frame_sum: bad shape");
    if (dtype != TM_DTYPE_U16 && dtype != TM_DTYPE_F32) return fail(TM_ERR_INVALID_ARG, "tm_frame_sum: dtype");
    if (!sum_dev || (n > 0 && !frames_dev)) return fail(TM_ERR_INVALID_ARG, "tm_frame_sum: NULL buffer");
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (n == 0 && !accumulate) {
        TM_CUDA(cudaMemsetAsync(sum_dev, 0, (size_t)H * W * sizeof(double), st), "tm_frame_sum: memset");
        return TM_OK;
    }
    void* scratch = nullptr;
    const size_t sb = tmgb::frame_sum_scratch_bytes(dtype, n, H, W, ctx->num_sms);
    if (sb) {
        int rc = workspace(ctx, st, "frame_sum_partials", sb, &scratch);
        if (rc) return rc;
    }
    TM_CUDA(tmgb::launch_frame_sum(frames_dev, dtype, n, H, W, accumulate ? 1 : 0, sum_dev, (double*)scratch,
                                   ctx->num_sms, st),
            "tm_frame_sum: launch");
    return TM_OK;
}

int tm_matrix_mask(tm_ctx* ctx, const double* sum_dev, int64_t n_frames, int32_t H, int32_t W, double threshold,
                   int32_t n_open, int32_t n_dilate, uint8_t* mask_dev, void* stream) {
    if (!ctx) return fail(TM_ERR_INVALID_ARG, "tm_matrix_mask: ctx is NULL");
    if (n_frames < 1 || H < 1 || W < 1 || H > 32000 || W > 32000)
        return fail(TM_ERR_INVALID_ARG, "tm_matrix_mask: bad shape or frame count");
    if (!isfinite(threshold)) return fail(TM_ERR_INVALID_ARG, "tm_matrix_mask: threshold must be finite");
    if (n_open < 0 || n_dilate < 0 || n_open > 1000 || n_dilate > 1000)
        return fail(TM_ERR_INVALID_ARG, "tm_matrix_mask: n_open and n_dilate must be in [0, 1000]");
    if (!sum_dev || !mask_dev) return fail(TM_ERR_INVALID_ARG, "tm_matrix_mask: NULL buffer");
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    void* scratch = nullptr;
    int rc = workspace(ctx, st, "mask_scratch", (size_t)H * W, &scratch);
    if (rc) return rc;
    const double thr_n = threshold * (double)n_frames;       // the comparison of the oracle: sum > threshold * n
    TM_CUDA(tmgb::launch_matrix_mask(sum_dev, H, W, thr_n, n_open, n_dilate, mask_dev, (uint8_t*)scratch,
                                     ctx->num_sms, st),
            "tm_matrix_mask: launch");
    return TM_OK;
}

int tm_find_centres(tm_ctx* ctx, const void* frames_dev, int32_t dtype, int64_t n, int32_t H, int32_t W,
                    double cx0, double cy0, double radius, int32_t iterations, float* centres_dev, void* stream) {
    if (!ctx) return fail(TM_ERR_INVALID_ARG, "tm_find_centres: ctx is NULL");
    if (n < 0 || H < 1 || W < 1 || H > 32000 || W > 32000) return fail(TM_ERR_INVALID_ARG, "tm_find_centres: bad shape");
    if (dtype != TM_DTYPE_U16 && dtype != TM_DTYPE_F32) return fail(TM_ERR_INVALID_ARG, "tm_find_centres: dtype");
    if (!(radius > 0.0 && radius <= 1e4)) return fail(TM_ERR_INVALID_ARG, "tm_find_centres: radius must be in (0, 1e4]");
    if (iterations < 1 || iterations > 100) return fail(TM_ERR_INVALID_ARG, "tm_find_centres: iterations must be in [1, 100]");
    if (isinf(cx0) || isinf(cy0)) return fail(TM_ERR_INVALID_ARG, "tm_find_centres: centre must be finite or NaN");
    if (n == 0) return TM_OK;
    if (!frames_dev || !centres_dev) return fail(TM_ERR_INVALID_ARG, "tm_find_centres: NULL buffer");
    if (isnan(cx0)) cx0 = (W - 1) / 2.0;
    if (isnan(cy0)) cy0 = (H - 1) / 2.0;
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    TM_CUDA(tmgb::launch_find_centres(frames_dev, dtype, n, H, W, cx0, cy0, radius, iterations, (float2*)centres_dev,
                                      (cudaStream_t)stream),
            "tm_find_centres: launch");
    return TM_OK;
}

int tm_preprocess(tm_ctx* ctx, const tm_preprocess_params* pp, const void* frames_dev, int32_t dtype, int64_t n,
                  int32_t H, int32_t W, float* out_dev, void* stream) {
    if (!ctx || !pp) return fail(TM_ERR_INVALID_ARG, "tm_preprocess: NULL argument");
    if (n < 0 || H < 1 || W < 1 || H > 32000 || W > 32000) return fail(TM_ERR_INVALID_ARG, "tm_preprocess: bad shape");
    if (dtype != TM_DTYPE_U16 && dtype != TM_DTYPE_F32) return fail(TM_ERR_INVALID_ARG, "tm_preprocess: dtype");
    const bool dog = pp->dog_sigma_max > 0.0, blur = pp->blur_sigma > 0.0;
    const double tr = pp->truncate > 0.0 ? pp->truncate : 4.0;
    auto sigma_ok = [](double s) { return s >= 0.1 && s <= 64.0; };
    if ((dog && !(sigma_ok(pp->dog_sigma_min) && sigma_ok(pp->dog_sigma_max) && pp->dog_sigma_min < pp->dog_sigma_max)) ||
        (blur && !sigma_ok(pp->blur_sigma)) || !(tr <= 64.0) || isnan(pp->dog_sigma_max) || isnan(pp->blur_sigma))
        return fail(TM_ERR_INVALID_ARG, "tm_preprocess: sigmas must be in [0.1, 64] (dog_sigma_min < dog_sigma_max)");
    auto radius = [&](double s) { return (int)floor(tr * s + 0.5); };
    const int r_min = dog ? radius(pp->dog_sigma_min) : 0, r_max = dog ? radius(pp->dog_sigma_max) : 0;
    const int r_blur = blur ? radius(pp->blur_sigma) : 0;
    if (r_min > 256 || r_max > 256 || r_blur > 256) return fail(TM_ERR_INVALID_ARG, "tm_preprocess: radius above 256");
    if (tmgb::gauss_cols_smem(H, r_min, r_max, 1) > 232448)
        return fail(TM_ERR_UNSUPPORTED, "tm_preprocess: frames of %d rows do not fit the column pass", H);
    if (n == 0) return TM_OK;
    if (!frames_dev || !out_dev) return fail(TM_ERR_INVALID_ARG, "tm_preprocess: NULL buffer");
    // weights (double precision, normalised, rounded to float): [min | max | blur | identity]
    std::vector<float> w;
    auto add = [&](double s, int r) -> size_t {
        const size_t at = w.size();
        if (s <= 0.0) {
            w.push_back(1.0f);
        } else {
            std::vector<double> d(2 * r + 1);
            double sum = 0.0;
            for (int i = -r; i <= r; ++i) sum += (d[i + r] = exp(-0.5 * (i / s) * (i / s)));
            for (double v : d) w.push_back((float)(v / sum));
        }
        w.resize(at + tmgb::gauss_padded_taps(r), 0.0f);    // the kernels take taps four at a time
        return at;
    };
    const size_t o_min = add(dog ? pp->dog_sigma_min : 0.0, r_min), o_max = add(dog ? pp->dog_sigma_max : 0.0, r_max);
    const size_t o_blur = add(blur ? pp->blur_sigma : 0.0, r_blur);
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    float* dw;
    int rc = workspace(ctx, st, "pre_weights", w.size() * sizeof(float), (void**)&dw);
    const size_t img = (size_t)n * H * W * sizeof(float);
    float *t1 = nullptr, *t2 = nullptr;
    if (!rc) rc = workspace(ctx, st, "pre_t1", img, (void**)&t1);
    if (!rc && dog) rc = workspace(ctx, st, "pre_t2", img, (void**)&t2);
    if (rc) return rc;
    TM_CUDA(cudaMemcpyAsync(dw, w.data(), w.size() * sizeof(float), cudaMemcpyHostToDevice, st), "tm_preprocess: weights");
    const int64_t rows = n * (int64_t)H;
    if (dog) {
        TM_CUDA(tmgb::launch_gauss_rows(frames_dev, dtype, rows, W, dw + o_min, r_min, dw + o_max, r_max, t1, t2, st),
                "tm_preprocess: rows");
        TM_CUDA(tmgb::launch_gauss_cols(t1, t2, n, H, W, dw + o_min, r_min, dw + o_max, r_max, 1, out_dev, st),
                "tm_preprocess: columns");
    }
    if (blur) {
        TM_CUDA(tmgb::launch_gauss_rows(dog ? (const void*)out_dev : frames_dev, dog ? TM_DTYPE_F32 : dtype, rows, W,
                                        dw + o_blur, r_blur, nullptr, 0, t1, nullptr, st),
                "tm_preprocess: rows");
        TM_CUDA(tmgb::launch_gauss_cols(t1, nullptr, n, H, W, dw + o_blur, r_blur, nullptr, 0, 0, out_dev, st),
                "tm_preprocess: columns");
    }
    if (!dog && !blur)                                       // identity: the frames as floats
        TM_CUDA(tmgb::launch_gauss_rows(frames_dev, dtype, rows, W, dw + o_blur, 0, nullptr, 0, out_dev, nullptr, st),
                "tm_preprocess: copy");
    return TM_OK;
}

int tm_kinematic_spots(tm_ctx* ctx, const double* g_dev, const double* f2_dev, const double* gnorm_dev, int64_t G,
                       const double* rot_dev, int64_t D, double wavelength, double s_max, int32_t max_spots,
                       int32_t* counts_dev, double* spots_dev, void* stream) {
    if (!ctx) return fail(TM_ERR_INVALID_ARG, "tm_kinematic_spots: ctx is NULL");
    if (G < 0 || G > (1 << 24) || D < 0 || max_spots < 1 || max_spots > 65535)
        return fail(TM_ERR_INVALID_ARG, "tm_kinematic_spots: sizes out of range");
    if (!(wavelength > 0.0 && isfinite(wavelength)) || !(s_max > 0.0 && isfinite(s_max)))
        return fail(TM_ERR_INVALID_ARG, "tm_kinematic_spots: wavelength and s_max must be finite and > 0");
    if (D == 0) return TM_OK;
    if ((G > 0 && (!g_dev || !f2_dev || !gnorm_dev)) || !rot_dev || !counts_dev || !spots_dev)
        return fail(TM_ERR_INVALID_ARG, "tm_kinematic_spots: NULL buffer");
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    TM_CUDA(tmgb::launch_kinematic(g_dev, f2_dev, gnorm_dev, G, rot_dev, D, wavelength, s_max, max_spots, counts_dev,
                                   spots_dev, (cudaStream_t)stream),
            "tm_kinematic_spots: launch");
    return TM_OK;
}

int tm_orientation_vectors(tm_ctx* ctx, const tm_hit* hits_dev, int64_t n, int32_t stride, const double* rot_dev,
                           int64_t K0, double ex, double ey, double ez, double* v_dev, void* stream) {
    if (!ctx) return fail(TM_ERR_INVALID_ARG, "tm_orientation_vectors: ctx is NULL");
    if (n < 0 || stride < 1 || K0 < 1) return fail(TM_ERR_INVALID_ARG, "tm_orientation_vectors: bad sizes");
    if (!isfinite(ex) || !isfinite(ey) || !isfinite(ez)) return fail(TM_ERR_INVALID_ARG, "tm_orientation_vectors: axis");
    if (n == 0) return TM_OK;
    if (!hits_dev || !rot_dev || !v_dev) return fail(TM_ERR_INVALID_ARG, "tm_orientation_vectors: NULL buffer");
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    TM_CUDA(tmgb::launch_orientation_vectors(hits_dev, n, stride, rot_dev, K0, ex, ey, ez, v_dev, (cudaStream_t)stream),
            "tm_orientation_vectors: launch");
    return TM_OK;
}

int tm_angular_deviation(tm_ctx* ctx, const double* va_dev, const double* vb_dev, int64_t n, double* deg_dev,
                         void* stream) {
    if (!ctx) return fail(TM_ERR_INVALID_ARG, "tm_angular_deviation: ctx is NULL");
    if (n < 0) return fail(TM_ERR_INVALID_ARG, "tm_angular_deviation: n < 0");
    if (n == 0) return TM_OK;
    if (!va_dev || !vb_dev || !deg_dev) return fail(TM_ERR_INVALID_ARG, "tm_angular_deviation: NULL buffer");
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    TM_CUDA(tmgb::launch_angular_deviation(va_dev, vb_dev, n, deg_dev, (cudaStream_t)stream),
            "tm_angular_deviation: launch");
    return TM_OK;
}

void tm_index_params_default(tm_index_params* p) {
    if (!p) return;
    p->gamma = 0.5;
    p->subtract = 0.0;
    p->cx = NAN;
    p->cy = NAN;
    p->prefilter_fraction = 1.0;
    p->top_n = 5;
    p->path = TM_PATH_FP32_SPARSE;
    p->rescore_k = 256;
    p->reserved = 0;
    p->pixel_mask = nullptr;
    p->threshold = 0.0;
}

const char* tm_last_error(void) { return g_err.c_str(); }

int tm_create(int device, size_t hbm_budget_bytes, tm_ctx** out) {
    if (!out) return fail(TM_ERR_INVALID_ARG, "tm_create: out is NULL");
    *out = nullptr;
    int count = 0;
    TM_CUDA(cudaGetDeviceCount(&count), "tm_create: cudaGetDeviceCount");
    if (device < 0 || device >= count) return fail(TM_ERR_INVALID_ARG, "tm_create: device %d of %d", device, count);
    DeviceGuard g(device);
    cudaDeviceProp prop;
    TM_CUDA(cudaGetDeviceProperties(&prop, device), "tm_create: cudaGetDeviceProperties");
    if (prop.major * 10 + prop.minor != 103)
        return fail(TM_ERR_UNSUPPORTED, "tm_create: device is sm_%d%d; this library is built for sm_103a only",
                    prop.major, prop.minor);
    auto ctx = std::make_unique<tm_ctx>();
    ctx->device = device;
    ctx->budget = hbm_budget_bytes;
    ctx->num_sms = prop.multiProcessorCount;
    TM_CUDA(cudaEventCreateWithFlags(&ctx->ws_event, cudaEventDisableTiming), "tm_create: cudaEventCreate");
    TM_CUDA(cudaMalloc(&ctx->d_error, sizeof(unsigned)), "tm_create: error word");
    TM_CUDA(cudaMalloc(&ctx->d_work, sizeof(unsigned long long)), "tm_create: work counter");
    TM_CUDA(cudaMemset(ctx->d_work, 0, sizeof(unsigned long long)), "tm_create: work counter");
    if (const char* f = getenv("TMGB_TUNE_CACHE")) {
        ctx->tune_file = f;
        if (FILE* fh = fopen(f, "r")) {
            // lines "key threads seeds tile ms" (older lines without the tile: 1)
            char line[1024], key[512];
            while (fgets(line, sizeof line, fh)) {
                int threads = 0, seeds = 0, tile = 1;
                double ms = 0;
                const int got = sscanf(line, "%511s %d %d %d %lf", key, &threads, &seeds, &tile, &ms);
                if (got == 5) ctx->tuned[key] = {threads, seeds, tile};
                else if (got == 4) ctx->tuned[key] = {threads, seeds, 1};
            }
            fclose(fh);
        }
    }
    TM_CUDA(cudaMemset(ctx->d_error, 0, sizeof(unsigned)), "tm_create: error word");
    *out = ctx.release();
    g_err.clear();
    return TM_OK;
}

int tm_profile_enable(tm_ctx* ctx, int enable) {
    if (!ctx) return fail(TM_ERR_INVALID_ARG, "tm_profile_enable: ctx is NULL");
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    for (auto& m : ctx->ev_marks) {
        cudaEventSynchronize(std::get<2>(m));
        ctx->ev_pool.push_back(std::get<1>(m));
        ctx->ev_pool.push_back(std::get<2>(m));
    }
    ctx->ev_marks.clear();
    ctx->profiling = enable != 0;
    TM_CUDA(cudaMemset(ctx->d_work, 0, sizeof(unsigned long long)), "tm_profile_enable: reset");
    return TM_OK;
}

int tm_profile_read(tm_ctx* ctx, tm_profile* out) {
    if (!ctx || !out) return fail(TM_ERR_INVALID_ARG, "tm_profile_read: NULL argument");
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    memset(out, 0, sizeof *out);
    for (auto& m : ctx->ev_marks) {
        TM_CUDA(cudaEventSynchronize(std::get<2>(m)), "tm_profile_read: wait");
        float ms = 0.0f;
        TM_CUDA(cudaEventElapsedTime(&ms, std::get<1>(m), std::get<2>(m)), "tm_profile_read: elapsed");
        const int s = std::get<0>(m);
        out->ms[s] += ms;
        out->launches[s] += 1;
        ctx->ev_pool.push_back(std::get<1>(m));
        ctx->ev_pool.push_back(std::get<2>(m));
    }
    ctx->ev_marks.clear();
    unsigned long long w = 0;
    TM_CUDA(cudaMemcpy(&w, ctx->d_work, sizeof w, cudaMemcpyDeviceToHost), "tm_profile_read: work");
    TM_CUDA(cudaMemset(ctx->d_work, 0, sizeof w), "tm_profile_read: reset");
    out->sparse_macs = (int64_t)w;
    return TM_OK;
}

void tm_destroy(tm_ctx* ctx) {
    if (!ctx) return;
    {
        DeviceGuard g(ctx->device);
        cudaDeviceSynchronize();
        for (auto& m : ctx->ev_marks) {
            cudaEventDestroy(std::get<1>(m));
            cudaEventDestroy(std::get<2>(m));
        }
        for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
        for (auto& kv : ctx->libs) free_library(ctx, kv.second.get());
        for (auto& kv : ctx->rays) cudaFree(kv.second);
        for (auto& kv : ctx->ws)
            if (kv.second.p) cudaFree(kv.second.p);
        for (auto& kv : ctx->spectral) {
            cudaFree(kv.second.basis);
            cudaFree(kv.second.twiddle);
            cudaFree(kv.second.dftmat);
        }
        for (auto& kv : ctx->radius_maps) {
            cudaFree(kv.second.radii);
            cudaFree(kv.second.rmap);
            cudaFree(kv.second.keep_row);
        }
        if (ctx->cublas) cublasDestroy(ctx->cublas);
        if (ctx->d_error) cudaFree(ctx->d_error);
        if (ctx->d_work) cudaFree(ctx->d_work);
        for (cudaStream_t hs : ctx->host_streams)
            if (hs) cudaStreamDestroy(hs);
        for (auto& kv : ctx->graphs)
            if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        if (ctx->ws_event) cudaEventDestroy(ctx->ws_event);
    }
    delete ctx;
}

int tm_check(tm_ctx* ctx, void* stream) {
    if (!ctx) return fail(TM_ERR_INVALID_ARG, "tm_check: ctx is NULL");
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    TM_CUDA(cudaStreamSynchronize((cudaStream_t)stream), "tm_check: stream");
    unsigned err = 0;
    TM_CUDA(cudaMemcpy(&err, ctx->d_error, sizeof err, cudaMemcpyDeviceToHost), "tm_check: read");
    if (err) {
        TM_CUDA(cudaMemset(ctx->d_error, 0, sizeof err), "tm_check: reset");
        return fail(TM_ERR_TIMEOUT, "tm_check: a kernel's bounded wait ran out (error word 0x%x)", err);
    }
    return TM_OK;
}

int tm_load_library(tm_ctx* ctx, const tm_library_desc* desc, int* lib_id) {
    if (!ctx || !lib_id) return fail(TM_ERR_INVALID_ARG, "tm_load_library: NULL argument");
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    auto L = std::make_unique<Library>();
    int rc = build_library(ctx, desc, L.get());
    if (rc) {
        free_library(ctx, L.get());
        return rc;
    }
    const int id = ctx->next_id++;
    ctx->libs.emplace(id, std::move(L));
    *lib_id = id;
    return TM_OK;
}

int tm_unload_library(tm_ctx* ctx, int lib_id) {
    if (!ctx) return fail(TM_ERR_INVALID_ARG, "tm_unload_library: ctx is NULL");
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    auto it = ctx->libs.find(lib_id);
    if (it == ctx->libs.end()) return fail(TM_ERR_NOT_FOUND, "tm_unload_library: no library %d", lib_id);
    TM_CUDA(cudaDeviceSynchronize(), "tm_unload_library: wait for pending work");
    for (auto& kv : ctx->graphs)                       // graphs may reference the library
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    ctx->graphs.clear();
    free_library(ctx, it->second.get());
    ctx->libs.erase(it);
    return TM_OK;
}

static void fill_info(const Library* L, tm_library_info* out) {
    out->n_templates = L->K;
    out->n_base = L->K0;
    out->n_spots = (int64_t)L->r.size();
    out->max_spots = L->max_spots;
    out->mirror = L->mirror;
    out->n_r = L->n_r;
    out->n_theta = L->n_theta;
    out->dr = L->dr;
    out->n_symmetric = L->n_sym;
    out->macs_per_pattern = L->macs;
    out->device_bytes = (int64_t)L->bytes;
}

int tm_library_info_get(tm_ctx* ctx, int lib_id, tm_library_info* out) {
    if (!ctx || !out) return fail(TM_ERR_INVALID_ARG, "tm_library_info_get: NULL argument");
    std::lock_guard<std::mutex> lk(ctx->mu);
    Library* L = find_lib(ctx, lib_id);
    if (!L) return fail(TM_ERR_NOT_FOUND, "tm_library_info_get: no library %d", lib_id);
    fill_info(L, out);
    return TM_OK;
}

static void export_host(const Library* L, int64_t* offsets, int32_t* r, int32_t* t, float* intensity,
                        float* norm, int32_t* order) {
    if (offsets) memcpy(offsets, L->off.data(), L->off.size() * 8);
    if (r) memcpy(r, L->r.data(), L->r.size() * 4);
    if (t) memcpy(t, L->t.data(), L->t.size() * 4);
    if (intensity) memcpy(intensity, L->I.data(), L->I.size() * 4);
    if (norm) memcpy(norm, L->norm.data(), L->norm.size() * 4);
    if (order) memcpy(order, L->order.data(), L->order.size() * 4);
}

int tm_library_prepare_host(const tm_library_desc* desc, tm_library_info* info, int64_t* offsets, int32_t* r,
                            int32_t* t, float* intensity, float* norm, int32_t* order, int32_t* packed,
                            int32_t* packed2) {
    if (!info) return fail(TM_ERR_INVALID_ARG, "tm_library_prepare_host: info is NULL");
    Library L;
    Prepared P;
    int rc = prepare_library(desc, &L, &P);
    if (rc) return rc;
    fill_info(&L, info);
    export_host(&L, offsets, r, t, intensity, norm, order);
    if (packed)
        for (size_t i = 0; i < P.spot.size(); ++i) packed[i] = P.spot[i].x;
    if (packed2)
        for (size_t i = 0; i < P.spot2.size(); ++i) packed2[i] = P.spot2[i].x;
    return TM_OK;
}

int tm_library_bound_entries_host(const tm_library_desc* desc, int32_t* n_words, int64_t* n_entries,
                                  int32_t* order, int32_t* word_start, int32_t* entries) {
    if (!n_words || !n_entries) return fail(TM_ERR_INVALID_ARG, "tm_library_bound_entries_host: NULL size");
    Library L;
    Prepared P;
    int rc = prepare_library(desc, &L, &P);
    if (rc) return rc;
    if (P.ell.empty() && P.ellw.empty())
        return fail(TM_ERR_UNSUPPORTED, "tm_library_bound_entries_host: the library has no window table");
    *n_words = (int32_t)P.ellw.size();
    *n_entries = (int64_t)P.ell.size();
    if (order) memcpy(order, P.sperm.data(), P.sperm.size() * 4);
    if (word_start) memcpy(word_start, P.ellw.data(), P.ellw.size() * 4);
    if (entries) memcpy(entries, P.ell.data(), P.ell.size() * 8);
    return TM_OK;
}

int tm_library_export(tm_ctx* ctx, int lib_id, int64_t* offsets, int32_t* r, int32_t* t, float* intensity,
                      float* norm, int32_t* order) {
    if (!ctx) return fail(TM_ERR_INVALID_ARG, "tm_library_export: ctx is NULL");
    std::lock_guard<std::mutex> lk(ctx->mu);
    Library* L = find_lib(ctx, lib_id);
    if (!L) return fail(TM_ERR_NOT_FOUND, "tm_library_export: no library %d", lib_id);
    export_host(L, offsets, r, t, intensity, norm, order);
    return TM_OK;
}

int tm_polar_transform(tm_ctx* ctx, const tm_index_params* params, const void* frames_dev, int32_t dtype,
                       int64_t n, int32_t H, int32_t W, const float* centres_dev, int32_t n_r, int32_t n_theta,
                       double dr, float* polar_dev, float* norm_dev, float* radial_dev, void* stream) {
    if (!ctx) return fail(TM_ERR_INVALID_ARG, "tm_polar_transform: ctx is NULL");
    int rc = check_params(params);
    if (rc) return rc;
    if (n < 0 || H < 1 || W < 1 || H > 32000 || W > 32000) return fail(TM_ERR_INVALID_ARG, "tm_polar_transform: bad shape");
    if (dtype != TM_DTYPE_U16 && dtype != TM_DTYPE_F32) return fail(TM_ERR_INVALID_ARG, "tm_polar_transform: dtype");
    if (n_r < 1 || n_r > 4096 || n_theta < 1 || n_theta > 4096 || !(dr > 0.0 && n_r * dr < 1048576.0))
        return fail(TM_ERR_INVALID_ARG, "tm_polar_transform: bad polar grid");
    if (n == 0) return TM_OK;
    if (!frames_dev || !polar_dev) return fail(TM_ERR_INVALID_ARG, "tm_polar_transform: NULL buffer");
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    const double cx = isnan(params->cx) ? (W - 1) / 2.0 : params->cx;
    const double cy = isnan(params->cy) ? (H - 1) / 2.0 : params->cy;
    const longlong2* rays = nullptr;
    rc = polar_rays(ctx, n_theta, dr, &rays);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    TM_CUDA(tmgb::launch_polar(frames_dev, dtype, n, H, W, rays, cx, cy, params->gamma, params->subtract, n_r, n_theta,
                               polar_dev, norm_dev, radial_dev, st, nullptr, (const float2*)centres_dev,
                               params->pixel_mask, params->threshold, ctx->d_error),
            "tm_polar_transform: launch");
    return TM_OK;
}

int tm_prefilter(tm_ctx* ctx, int lib_id, const float* radial_dev, int64_t n, double fraction, uint32_t* mask_dev,
                 float* score_dev, void* stream) {
    if (!ctx) return fail(TM_ERR_INVALID_ARG, "tm_prefilter: ctx is NULL");
    if (!(fraction > 0.0 && fraction <= 1.0)) return fail(TM_ERR_INVALID_ARG, "tm_prefilter: fraction in (0, 1]");
    if (n < 0) return fail(TM_ERR_INVALID_ARG, "tm_prefilter: n < 0");
    if (n == 0) return TM_OK;
    if (!radial_dev || !mask_dev) return fail(TM_ERR_INVALID_ARG, "tm_prefilter: NULL buffer");
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    Library* L = find_lib(ctx, lib_id);
    if (!L) return fail(TM_ERR_NOT_FOUND, "tm_prefilter: no library %d", lib_id);
    cudaStream_t st = (cudaStream_t)stream;
    float* rn;
    int rc = workspace(ctx, st, "radial_norm", (size_t)n * 4, (void**)&rn);
    if (rc) return rc;
    TM_CUDA(tmgb::launch_radial_norm(radial_dev, n, L->n_r, rn, st), "tm_prefilter: radial norm");
    const int keep = keep_count(fraction, L->K);
    TM_CUDA(tmgb::launch_prefilter(radial_dev, rn, n, L->n_r, radial_lib(L), keep, mask_dev, score_dev, st),
            "tm_prefilter: scores and selection");
    return TM_OK;
}

int tm_correlate(tm_ctx* ctx, int lib_id, const float* polar_dev, const float* norm_dev, int64_t n,
                 const uint32_t* mask_dev, float* q_dev, int32_t* s_dev, void* stream) {
    if (!ctx) return fail(TM_ERR_INVALID_ARG, "tm_correlate: ctx is NULL");
    if (n < 0) return fail(TM_ERR_INVALID_ARG, "tm_correlate: n < 0");
    if (n == 0) return TM_OK;
    if (!polar_dev || !norm_dev || !q_dev || !s_dev) return fail(TM_ERR_INVALID_ARG, "tm_correlate: NULL buffer");
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    Library* L = find_lib(ctx, lib_id);
    if (!L) return fail(TM_ERR_NOT_FOUND, "tm_correlate: no library %d", lib_id);
    const int n_rad = (int)std::max<size_t>(1, L->radii.size());
    if (!tmgb::sparse_smem_bytes(n_rad, L->n_theta, 1))
        return fail(TM_ERR_UNSUPPORTED, "tm_correlate: %d radii x %d angles do not fit shared memory", n_rad, L->n_theta);
    cudaStream_t st = (cudaStream_t)stream;
    int* pc;
    int rc = workspace(ctx, st, "pattern_counter", sizeof(int), (void**)&pc);
    if (rc) return rc;
    tmgb::SparseCall c{};
    c.max_rad = n_rad;
    c.pattern_counter = pc;
    c.polar = polar_dev;
    c.pnorm = norm_dev;
    c.n = n;
    c.n_r = L->n_r;
    c.n_theta = L->n_theta;
    c.pitch = 0;
    c.n_libs = 1;
    c.lib[0] = sparse_view(L);
    c.mask[0] = mask_dev;
    c.q_out[0] = q_dev;
    c.s_out[0] = s_dev;
    c.bulk = L->n_theta % 4 == 0 && ((uintptr_t)polar_dev & 15) == 0;
    c.error = ctx->d_error;
    c.hits = nullptr;
    c.top_n = 1;
    TM_CUDA(tmgb::launch_sparse(c, ctx->num_sms, st), "tm_correlate: launch");
    return TM_OK;
}

int tm_index_patterns(tm_ctx* ctx, const tm_index_params* params, const void* frames_dev, int32_t dtype, int64_t n,
                      int32_t H, int32_t W, const float* centres_dev, const int32_t* lib_ids, int32_t n_libs,
                      tm_hit* out_dev, tm_stats* stats, void* stream) {
    return tmgb::index_patterns_ex(ctx, params, frames_dev, dtype, n, H, W, centres_dev, lib_ids, n_libs, out_dev, 0,
                                   stats, stream);
}

}  // extern "C"

int tmgb::index_patterns_ex(tm_ctx* ctx, const tm_index_params* params, const void* frames_dev, int32_t dtype,
                            int64_t n, int32_t H, int32_t W, const float* centres_dev, const int32_t* lib_ids,
                            int32_t n_libs, tm_hit* out_dev, int64_t lib_stride, tm_stats* stats, void* stream) {
    if (!ctx) return fail(TM_ERR_INVALID_ARG, "tm_index_patterns: ctx is NULL");
    int rc = check_params(params);
    if (rc) return rc;
    if (n < 0 || H < 1 || W < 1 || H > 32000 || W > 32000) return fail(TM_ERR_INVALID_ARG, "tm_index_patterns: bad shape");
    if (dtype != TM_DTYPE_U16 && dtype != TM_DTYPE_F32) return fail(TM_ERR_INVALID_ARG, "tm_index_patterns: dtype");
    if (n_libs < 1 || n_libs > TM_MAX_LIBS || !lib_ids)
        return fail(TM_ERR_INVALID_ARG, "tm_index_patterns: n_libs must be in [1, %d]", TM_MAX_LIBS);
    if (params->path != TM_PATH_FP32_SPARSE && params->path != TM_PATH_BF16_RESCORE)
        return fail(TM_ERR_INVALID_ARG, "tm_index_patterns: unknown path %d", params->path);
    const bool bf16 = params->path == TM_PATH_BF16_RESCORE;
    if (bf16 && params->rescore_k < 1)
        return fail(TM_ERR_INVALID_ARG, "tm_index_patterns: rescore_k must be >= 1");
    if (stats) memset(stats, 0, sizeof *stats);
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    Library* libs[TM_MAX_LIBS];
    for (int i = 0; i < n_libs; ++i) {
        libs[i] = find_lib(ctx, lib_ids[i]);
        if (!libs[i]) return fail(TM_ERR_NOT_FOUND, "tm_index_patterns: no library %d", lib_ids[i]);
        if (libs[i]->n_r != libs[0]->n_r || libs[i]->n_theta != libs[0]->n_theta || libs[i]->dr != libs[0]->dr)
            return fail(TM_ERR_INVALID_ARG, "tm_index_patterns: libraries are built for different polar grids");
    }
    if (n == 0) return TM_OK;
    if (!frames_dev || !out_dev) return fail(TM_ERR_INVALID_ARG, "tm_index_patterns: NULL buffer");
    const int n_r = libs[0]->n_r, n_theta = libs[0]->n_theta, N = params->top_n;
    if (lib_stride == 0) lib_stride = n * N;
    if (lib_stride < n * N) return fail(TM_ERR_INVALID_ARG, "tm_index_patterns: hits stride below n * top_n");
    const int sms = tmgb::device_sms();
    const double dr = libs[0]->dr;
    int max_rad = 1;
    for (int i = 0; i < n_libs; ++i) max_rad = std::max<int>(max_rad, (int)libs[i]->radii.size());
    if (!tmgb::sparse_smem_bytes(max_rad, n_theta, N))
        return fail(TM_ERR_UNSUPPORTED, "tm_index_patterns: %d radii x %d angles do not fit shared memory", max_rad,
                    n_theta);
    const double cx = isnan(params->cx) ? (W - 1) / 2.0 : params->cx;
    const double cy = isnan(params->cy) ? (H - 1) / 2.0 : params->cy;
    const longlong2* rays = nullptr;
    rc = polar_rays(ctx, n_theta, dr, &rays);
    if (rc) return rc;
    const bool pre = params->prefilter_fraction < 1.0;
    const int kc = params->rescore_k;
    SpectralTables spec;
    RadiusMap rmap;
    rc = radius_map(ctx, libs, lib_ids, n_libs, n_r, &rmap);
    if (rc) return rc;
    TensorPlan tp;
    if (bf16) {
        if (!tmgb::dense_supported(n_theta))
            return fail(TM_ERR_UNSUPPORTED, "tm_index_patterns: the BF16 path needs an even n_theta <= 376 (got %d)",
                        n_theta);
        rc = spectral_tables(ctx, n_theta, &spec);
        if (!rc) rc = tensor_plan(ctx, libs, n_libs, n_theta, &tp);
        if (rc) return rc;
    }
    int keep[TM_MAX_LIBS];
    for (int i = 0; i < n_libs; ++i) keep[i] = keep_count(params->prefilter_fraction, libs[i]->K);

    // chunk size from a per-pattern workspace estimate (<= 4 GiB of workspace)
    size_t per = (size_t)n_r * n_theta * 4 + 4 + (size_t)n_r * 4 + 4;
    for (int i = 0; i < n_libs; ++i)
        if (pre || bf16) per += (size_t)libs[i]->K * 4 + ((libs[i]->K + 31) / 32) * 4;
    size_t cap = (size_t)4 << 30;
    if (ctx->budget) {
        const size_t freeb = ctx->budget > ctx->used ? ctx->budget - ctx->used : 0;
        cap = std::min(cap, (freeb - std::min(freeb, tp.bytes(tp.nb))) / 2);
    }
    int64_t chunk = (int64_t)std::max<size_t>(1, cap / per);
    chunk = std::min<int64_t>(chunk, n);

    float *polar, *pnorm, *radial, *rn = nullptr;
    int* pcount = nullptr;
    rc = workspace(ctx, st, "pattern_counter", sizeof(int), (void**)&pcount);
    if (!rc) rc = workspace(ctx, st, "polar", (size_t)chunk * n_r * n_theta * 4, (void**)&polar);
    if (!rc) rc = workspace(ctx, st, "pnorm", (size_t)chunk * 4, (void**)&pnorm);
    if (!rc) rc = workspace(ctx, st, "radial", (size_t)chunk * n_r * 4, (void**)&radial);
    if (!rc && pre) rc = workspace(ctx, st, "radial_norm", (size_t)chunk * 4, (void**)&rn);
    // per-CTA words of the sparse kernel's seeded templates (pruned top-N)
    int max_words = 1;
    for (int i = 0; i < n_libs; ++i) max_words = std::max<int>(max_words, (int)((libs[i]->K + 31) / 32));
    uint32_t* seed_bits = nullptr;
    __half* seed_qub = nullptr;
    const int seed_ctas = tmgb::sparse_max_ctas(sms);
    const size_t seed_slots = (size_t)seed_ctas * tmgb::kSparseTile;   // one per pattern of a CTA's tile
    if (!rc) rc = workspace(ctx, st, "seed_bits", seed_slots * max_words * 4, (void**)&seed_bits);
    if (!rc) rc = workspace(ctx, st, "seed_qub", seed_slots * max_words * 32 * 2, (void**)&seed_qub);
    int32_t* seed_cand = nullptr;
    if (!rc) rc = workspace(ctx, st, "seed_cand", (size_t)seed_ctas * max_words * 32 * 4, (void**)&seed_cand);
    TensorBuffers tb;
    if (!rc && bf16) rc = tensor_buffers(ctx, st, tp, std::min<int64_t>(tp.nb, chunk), &tb);
    if (rc) return rc;
    float* score[TM_MAX_LIBS] = {};
    uint32_t* mask[TM_MAX_LIBS] = {};
    for (int i = 0; i < n_libs; ++i) {
        const std::string s = std::to_string(i);
        // mask: the pre-filter's keep-mask, on the BF16 path reused afterwards for the mask of
        // the candidates to rescore; score: the BF16 pre-scores
        if (bf16) rc = workspace(ctx, st, "score" + s, (size_t)chunk * libs[i]->K * 4, (void**)&score[i]);
        if (!rc && (pre || bf16))
            rc = workspace(ctx, st, "mask" + s, (size_t)chunk * ((libs[i]->K + 31) / 32) * 4, (void**)&mask[i]);
        if (rc) return rc;
    }
    if (bf16)
        for (int i = 0; i < n_libs; ++i) {
            rc = ensure_spectra(ctx, libs[i], spec, st);
            if (rc) return rc;
        }
    const size_t esz = dtype == TM_DTYPE_U16 ? 2 : 4;
    // the sparse kernel's block size: forced (autotuning), tuned for these libraries, or by
    // default 256 -- but 512 when the chunk has at most two patterns per SM, so that each
    // pattern is shared by twice the warps (the latency of small batches such as scan lines)
    int sparse_threads = ctx->tune_override.threads, sparse_seeds = ctx->tune_override.seeds;
    int sparse_tile = ctx->tune_override.tile;
    if (!sparse_threads) {
        auto tt = ctx->tuned.find(tune_key(libs, n_libs, N));
        if (tt != ctx->tuned.end()) {
            sparse_threads = tt->second.threads;
            sparse_seeds = tt->second.seeds;
            sparse_tile = tt->second.tile;
        }
    }
    if (!sparse_threads && std::min(chunk, n) <= 2 * (int64_t)sms) sparse_threads = 512;
    int64_t launches = 0, corr = 0, scored = 0;
    auto enqueue = [&]() -> int {
        for (int64_t c0 = 0; c0 < n; c0 += chunk) {
            const int64_t m = std::min(chunk, n - c0);
            const void* fr = (const char*)frames_dev + (size_t)c0 * H * W * esz;
            {
                StageTimer tmr(ctx, TM_STAGE_POLAR, st);
                TM_CUDA(tmgb::launch_polar(fr, dtype, m, H, W, rays, cx, cy, params->gamma, params->subtract, n_r,
                                           n_theta, polar, pnorm, radial, st, rmap.keep_row,
                                           centres_dev ? (const float2*)centres_dev + c0 : nullptr,
                                           params->pixel_mask, params->threshold, ctx->d_error),
                        "tm_index_patterns: polar");
            }
            ++launches;
            if (pre) {
                StageTimer tmr(ctx, TM_STAGE_PREFILTER, st);
                TM_CUDA(tmgb::launch_radial_norm(radial, m, n_r, rn, st), "tm_index_patterns: radial norm");
                ++launches;
                for (int i = 0; i < n_libs; ++i) {
                    TM_CUDA(tmgb::launch_prefilter(radial, rn, m, n_r, radial_lib(libs[i]), keep[i], mask[i], nullptr,
                                                   st),
                            "tm_index_patterns: pre-filter");
                    ++launches;
                }
            }
            tmgb::SparseCall c{};
            c.polar = polar;
            c.pnorm = pnorm;
            c.n = m;
            c.n_r = n_r;
            c.n_theta = n_theta;
            c.pitch = 0;
            c.max_rad = max_rad;
            c.pattern_counter = pcount;
            c.n_libs = n_libs;
            for (int i = 0; i < n_libs; ++i) {
                c.lib[i] = sparse_view(libs[i]);
                if (pre || bf16) c.mask[i] = mask[i];
            }
            c.hits = out_dev + (size_t)c0 * N;
            c.hits_lib_stride = lib_stride;
            c.top_n = N;
            c.threads = sparse_threads;
            c.work = ctx->profiling ? ctx->d_work : nullptr;
            c.seed_bits = seed_bits;
            c.seed_qub = seed_qub;
            c.seed_cand = seed_cand;
            c.seed_words = max_words;
            c.seed_ctas = seed_ctas;
            c.seeds_per_warp = sparse_seeds;
            c.tile = sparse_tile;
            c.bulk = n_theta % 4 == 0 && ((uintptr_t)polar & 15) == 0;
            c.error = ctx->d_error;
            c.test_stall = (params->reserved & TM_INDEX_TEST_STALL) ? 1 : 0;
            if (bf16) {
                int64_t nl = 0;
                const int rc2 = prescore_rows(ctx, st, libs, n_libs, spec, tb, polar, pnorm, m, pre ? mask : nullptr,
                                              score, (params->reserved & TM_INDEX_TEST_STALL) ? 1 : 0, &nl);
                if (rc2) return rc2;
                launches += nl;
                {
                    StageTimer tmr(ctx, TM_STAGE_SELECT, st);
                    for (int i = 0; i < n_libs; ++i) {
                        const int kci = std::min(kc, keep[i]);
                        TM_CUDA(tmgb::launch_prefilter_select(score[i], m, (int)libs[i]->K, kci, mask[i], st),
                                "tm_index_patterns: candidates");
                        ++launches;
                    }
                }
                {
                    StageTimer tmr(ctx, TM_STAGE_RESCORE, st);
                    TM_CUDA(tmgb::launch_sparse(c, sms, st), "tm_index_patterns: rescore");
                }
                ++launches;
                for (int i = 0; i < n_libs; ++i) {
                    corr += m * ((int64_t)keep[i] + std::min<int64_t>(kc, keep[i])) * n_theta;
                    scored += m * std::min<int64_t>(kc, keep[i]);
                }
            } else {
                {
                    StageTimer tmr(ctx, TM_STAGE_SPARSE, st);
                    TM_CUDA(tmgb::launch_sparse(c, sms, st), "tm_index_patterns: sparse");
                }
                ++launches;
                for (int i = 0; i < n_libs; ++i) {
                    corr += m * (int64_t)keep[i] * n_theta;
                    scored += m * keep[i];
                }
            }
            if (params->reserved & TM_INDEX_REFINE) {
                tmgb::RefineCall rc{};
                rc.polar = polar;
                rc.pnorm = pnorm;
                rc.n = m;
                rc.n_r = n_r;
                rc.n_theta = n_theta;
                rc.top_n = N;
                rc.n_libs = n_libs;
                for (int i = 0; i < n_libs; ++i)
                    rc.lib[i] = tmgb::RefineLib{libs[i]->d_off, libs[i]->d_rt, libs[i]->d_spot, libs[i]->d_norm};
                rc.hits = out_dev + (size_t)c0 * N;
                rc.hits_lib_stride = lib_stride;
                TM_CUDA(tmgb::launch_refine(rc, sms, st), "tm_index_patterns: refine");
                ++launches;
            }
        }
        return TM_OK;
    };
    auto report = [&]() {
        if (stats) {
            stats->patterns = n;
            stats->correlations = corr;
            stats->templates_scored = scored;
            stats->launches = launches;
        }
    };
    // CUDA graph: the second identical call on a created stream is captured, later ones replay
    if ((params->reserved & TM_INDEX_GRAPH) && st != nullptr && !ctx->profiling) {
        char key[512];
        int off = snprintf(key, sizeof key, "%p|%p|%p|%p|%p|%d|%lld|%d|%d|%.17g|%.17g|%.17g|%.17g|%.17g|%.17g|%d|%d|%d|",
                           st, frames_dev, (const void*)centres_dev, (void*)out_dev, (const void*)params->pixel_mask,
                           dtype, (long long)n, H, W, params->gamma, params->subtract, params->cx, params->cy,
                           params->prefilter_fraction, params->threshold, params->top_n, params->path,
                           params->rescore_k);
        off += snprintf(key + off, sizeof key - off, "r%d|t%d.%d|s%lld|m%d|", params->reserved & ~TM_INDEX_GRAPH,
                        sparse_threads, sparse_seeds, (long long)lib_stride, sms);
        for (int i = 0; i < n_libs && off < (int)sizeof key - 12; ++i) off += snprintf(key + off, sizeof key - off, "%d,", lib_ids[i]);
        tm_ctx::GraphEntry& ge = ctx->graphs[key];
        if (ge.exec && ge.ws_gen == ctx->ws_gen) {
            TM_CUDA(cudaGraphLaunch(ge.exec, st), "tm_index_patterns: graph launch");
            launches = ge.launches;
            corr = ge.corr;
            scored = ge.scored;
            report();
            return TM_OK;
        }
        if (ge.seen) {
            if (ge.exec) {
                cudaGraphExecDestroy(ge.exec);
                ge.exec = nullptr;
            }
            TM_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "tm_index_patterns: begin capture");
            ctx->capturing = true;
            const int rc2 = enqueue();
            ctx->capturing = false;
            cudaGraph_t graph = nullptr;
            const cudaError_t e = cudaStreamEndCapture(st, &graph);
            if (rc2 || e != cudaSuccess) {
                if (graph) cudaGraphDestroy(graph);
                return rc2 ? rc2 : cuda_fail(e, "tm_index_patterns: end capture");
            }
            const cudaError_t e2 = cudaGraphInstantiate(&ge.exec, graph, 0);
            cudaGraphDestroy(graph);
            if (e2 != cudaSuccess) {
                ge.exec = nullptr;
                return cuda_fail(e2, "tm_index_patterns: graph instantiate");
            }
            ge.ws_gen = ctx->ws_gen;
            ge.launches = launches;
            ge.corr = corr;
            ge.scored = scored;
            TM_CUDA(cudaGraphLaunch(ge.exec, st), "tm_index_patterns: graph launch");
            report();
            return TM_OK;
        }
        ge.seen = true;
    }
    rc = enqueue();
    if (rc) return rc;
    report();
    return TM_OK;
}

extern "C" {

int tm_autotune(tm_ctx* ctx, const tm_index_params* params, const void* frames_dev, int32_t dtype, int64_t n,
                int32_t H, int32_t W, const int32_t* lib_ids, int32_t n_libs, int32_t* best_threads, void* stream) {
    if (!ctx || !params || !lib_ids || n_libs < 1 || n_libs > TM_MAX_LIBS || n < 1)
        return fail(TM_ERR_INVALID_ARG, "tm_autotune: bad arguments");
    std::string key;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        Library* libs[TM_MAX_LIBS];
        for (int i = 0; i < n_libs; ++i) {
            libs[i] = find_lib(ctx, lib_ids[i]);
            if (!libs[i]) return fail(TM_ERR_NOT_FOUND, "tm_autotune: no library %d", lib_ids[i]);
        }
        key = tune_key(libs, n_libs, params->top_n);
    }
    // shapes on the first m frames; the tile (patterns bounded together) on up to m2, enough
    // tiles per CTA that the last ones do not decide the time
    const int64_t m = std::min<int64_t>(n, 2048), m2 = std::min<int64_t>(n, 16384);
    const int64_t N = params->top_n;
    tm_hit* out = nullptr;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        DeviceGuard g(ctx->device);
        int rc = workspace(ctx, (cudaStream_t)stream, "tune_out", (size_t)n_libs * m2 * N * sizeof(tm_hit), (void**)&out);
        if (rc) return rc;
    }
    tm_index_params p = *params;
    p.path = TM_PATH_FP32_SPARSE;
    p.reserved = 0;
    p.pixel_mask = nullptr;
    p.threshold = 0.0;
    // milliseconds of the sparse kernel per call of shape tc on the first mm frames (3 timed calls)
    auto time_shape = [&](const tm_ctx::Tune& tc, int64_t mm, double* ms) -> int {
        {
            std::lock_guard<std::mutex> lk(ctx->mu);
            ctx->tune_override = tc;
        }
        int rc = tm_index_patterns(ctx, &p, frames_dev, dtype, mm, H, W, nullptr, lib_ids, n_libs, out, nullptr, stream);
        if (!rc) rc = tm_profile_enable(ctx, 1);
        for (int r = 0; r < 3 && !rc; ++r)
            rc = tm_index_patterns(ctx, &p, frames_dev, dtype, mm, H, W, nullptr, lib_ids, n_libs, out, nullptr, stream);
        tm_profile prof;
        if (!rc) rc = tm_profile_read(ctx, &prof);
        tm_profile_enable(ctx, 0);
        {
            std::lock_guard<std::mutex> lk(ctx->mu);
            ctx->tune_override = tm_ctx::Tune{};
        }
        *ms = prof.ms[TM_STAGE_SPARSE] / 3.0;
        return rc;
    };
    // block sizes x seeds per warp (the templates of highest bound scored first, whose scores
    // set the top-N threshold the rest is pruned against), then the best block size with tiles
    // of 4 patterns bounded together and each seed count
    const int cand_t[3] = {128, 256, 512}, cand_s[3] = {4, 8, 16};
    tm_ctx::Tune best{256, 8, 1};
    double best_ms = 1e30;
    for (int ci = 0; ci < 9; ++ci) {
        const tm_ctx::Tune tc{cand_t[ci / 3], cand_s[ci % 3], 1};
        double ms = 0.0;
        const int rc = time_shape(tc, m, &ms);
        if (rc) return rc;
        if (ms < best_ms) {
            best_ms = ms;
            best = tc;
        }
    }
    {
        // on the larger sample: that shape, and tiles of 4 with each seed count
        double ms = 0.0;
        int rc = time_shape(best, m2, &ms);
        if (rc) return rc;
        double best2 = ms;
        for (int si = 0; si < 3; ++si) {
            const tm_ctx::Tune t4{best.threads, cand_s[si], tmgb::kSparseTile};
            rc = time_shape(t4, m2, &ms);
            if (rc) return rc;
            if (ms < best2) {
                best2 = ms;
                best = t4;
            }
        }
        best_ms = best2 * (double)m / (double)m2;
    }
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        ctx->tuned[key] = best;
        if (!ctx->tune_file.empty()) {
            if (FILE* fh = fopen(ctx->tune_file.c_str(), "a")) {
                fprintf(fh, "%s %d %d %d %.6f\n", key.c_str(), best.threads, best.seeds, best.tile, best_ms);
                fclose(fh);
            }
        }
    }
    if (best_threads) *best_threads = best.threads;
    return TM_OK;
}

int tm_prescore(tm_ctx* ctx, int lib_id, const float* polar_dev, const float* norm_dev, const float* radial_dev,
                int64_t n, double fraction, float* score_dev, void* stream) {
    if (!ctx) return fail(TM_ERR_INVALID_ARG, "tm_prescore: ctx is NULL");
    if (n < 0 || !(fraction > 0.0 && fraction <= 1.0)) return fail(TM_ERR_INVALID_ARG, "tm_prescore: bad n or fraction");
    if (n == 0) return TM_OK;
    if (!polar_dev || !norm_dev || !score_dev || (fraction < 1.0 && !radial_dev))
        return fail(TM_ERR_INVALID_ARG, "tm_prescore: NULL buffer");
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    Library* L = find_lib(ctx, lib_id);
    if (!L) return fail(TM_ERR_NOT_FOUND, "tm_prescore: no library %d", lib_id);
    const int n_r = L->n_r, n_theta = L->n_theta;
    if (!tmgb::dense_supported(n_theta))
        return fail(TM_ERR_UNSUPPORTED, "tm_prescore: needs an even n_theta <= 376 (got %d)", n_theta);
    SpectralTables spec;
    TensorPlan tp;
    Library* libs[1] = {L};
    int rc = spectral_tables(ctx, n_theta, &spec);
    if (!rc) rc = tensor_plan(ctx, libs, 1, n_theta, &tp);
    if (rc) return rc;
    const int keep = keep_count(fraction, L->K);
    cudaStream_t st = (cudaStream_t)stream;
    TensorBuffers tb;
    rc = tensor_buffers(ctx, st, tp, std::min<int64_t>(tp.nb, n), &tb);
    float* rn = nullptr;
    uint32_t* mask = nullptr;
    if (!rc && fraction < 1.0) {
        rc = workspace(ctx, st, "radial_norm", (size_t)n * 4, (void**)&rn);
        if (!rc) rc = workspace(ctx, st, "mask0", (size_t)n * ((L->K + 31) / 32) * 4, (void**)&mask);
    }
    if (!rc) rc = ensure_spectra(ctx, L, spec, st);
    if (rc) return rc;
    if (fraction < 1.0) {
        TM_CUDA(tmgb::launch_radial_norm(radial_dev, n, n_r, rn, st), "tm_prescore: radial norm");
        TM_CUDA(tmgb::launch_prefilter(radial_dev, rn, n, n_r, radial_lib(L), keep, mask, nullptr, st),
                "tm_prescore: pre-filter");
    }
    int64_t nl = 0;
    uint32_t* masks[1] = {mask};
    float* outs[1] = {score_dev};
    return prescore_rows(ctx, st, libs, 1, spec, tb, polar_dev, norm_dev, n, fraction < 1.0 ? masks : nullptr, outs, 0,
                         &nl);
}

}  // extern "C"
