// Serving loop: continuous batching of indexing requests (scan lines and whole maps) on
// one GPU, for on-line mapping during acquisition (arXiv 2111.07347, Section 5).
//
// A worker thread owns `slots` CUDA streams, each with device staging for one tile of
// frames.  Requests are split into tiles; whenever a slot is free the worker takes the next
// tile of the highest-priority request that still has tiles (ties: the earlier submission),
// copies its frames to the device (unless the request's frames are already on the device),
// runs the indexing path on the slot's stream with the hits written into the request's own
// device buffer, copies the tile's hits into the slot's pinned host staging, and records
// events.  Finished slots are detected by polling; the worker then copies the staged hits
// into the request's output (which may be pageable memory: a device-to-host copy into
// pageable memory would block the worker until the slot's kernels finish) and adds the
// tile's copy and kernel times (from the events) to the request's timeline.  So tiles of
// different requests overlap on the device (copies of one tile with the kernels of another).
// The last `priority_slots` slots take only requests of priority > 0 (scan lines), which
// therefore never wait for a slot held by a map's tile; tiles of such requests run on the
// slot's high-priority stream, and the persistent kernels of map tiles leave `reserve_sms`
// SMs free, so a line's kernels find SMs without waiting for a map's thread blocks to retire.
// Admission: the frame bytes of requests submitted and not finished stay within queue_bytes,
// and every admitted request holds its hits ([n_libs][n][top_n]) in a device arena of
// hbm_budget_bytes (first fit, freed when the request finishes).  Every wait is bounded by
// the caller's timeout.
#include <stdio.h>
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "tm_internal.h"

namespace {

struct Request {
    uint64_t ticket = 0;
    tm_request req{};
    std::vector<int32_t> libs;
    int64_t next = 0;            // first pattern not yet dispatched
    int64_t tiles_total = 0, tiles_done = 0, tiles_inflight = 0;
    int status = TM_OK;
    bool cancelled = false, finished = false;
    double t_submit = 0, t_admit = 0, t_first = -1, t_done = 0;
    double h2d_ms = 0, kernels_ms = 0, d2h_ms = 0;
    size_t bytes = 0;            // frame bytes (queue budget)
    size_t arena_off = 0, arena_bytes = 0;
    tm_hit* hits_dev = nullptr;  // [n_libs][n][top_n] in the arena
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaStream_t stream_hi = nullptr;   // high-priority stream for tiles of priority > 0
    bool lines_only = false;            // takes only requests of priority > 0
    cudaEvent_t ev[4] = {};             // before the frame copy, after it, after the kernels, after the hit copy
    void* frames = nullptr;      // device staging
    tm_hit* hits_host = nullptr; // pinned host staging [max_libs][tile][max_top_n]
    std::shared_ptr<Request> req;
    int64_t p0 = 0, m = 0;
    bool busy = false;
};

// First-fit allocator over the device arena (offsets; blocks aligned to 256 bytes).
struct Arena {
    void* base = nullptr;
    size_t size = 0;
    std::map<size_t, size_t> free_blocks;   // offset -> bytes

    bool alloc(size_t bytes, size_t* off) {
        bytes = (bytes + 255) & ~(size_t)255;
        for (auto it = free_blocks.begin(); it != free_blocks.end(); ++it) {
            if (it->second < bytes) continue;
            *off = it->first;
            const size_t rest = it->second - bytes;
            const size_t o = it->first + bytes;
            free_blocks.erase(it);
            if (rest) free_blocks[o] = rest;
            return true;
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = (bytes + 255) & ~(size_t)255;
        auto it = free_blocks.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_blocks.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_blocks.erase(nx);
        }
        if (it != free_blocks.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_blocks.erase(it);
            }
        }
    }
};

}  // namespace

struct tm_server {
    tm_ctx* ctx = nullptr;
    tm_server_params prm{};
    std::vector<Slot> slots;
    std::mutex mu;
    std::condition_variable cv_work, cv_done, cv_room;
    std::map<uint64_t, std::shared_ptr<Request>> reqs;
    std::deque<std::shared_ptr<Request>> pending;   // requests with tiles left to dispatch
    uint64_t next_ticket = 1;
    size_t bytes_in = 0;
    Arena arena;
    int map_sm_cap = 0;          // SM cap of map tiles' persistent kernels (0: none)
    bool stop = false, paused = false;
    std::thread worker;
    std::chrono::steady_clock::time_point t0;
    int device = 0;

    double now_ms() const {
        return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace {

int sfail(int code, const char* msg) {
    tmgb::set_last_error(msg);
    return code;
}

void finish_locked(tm_server* s, const std::shared_ptr<Request>& r) {
    r->finished = true;
    r->t_done = s->now_ms();
    s->bytes_in -= std::min(s->bytes_in, r->bytes);
    if (r->arena_bytes) {
        s->arena.release(r->arena_off, r->arena_bytes);
        r->arena_bytes = 0;
    }
    s->cv_done.notify_all();
    s->cv_room.notify_all();
}

// Pick the next tile: highest priority, then submission order; a slot reserved for scan
// lines takes only requests of priority > 0.
std::shared_ptr<Request> pick_locked(tm_server* s, bool lines_only) {
    std::shared_ptr<Request> best;
    for (auto& r : s->pending) {
        if (r->cancelled || r->next >= r->req.n || (lines_only && r->req.priority <= 0)) continue;
        if (!best || r->req.priority > best->req.priority) best = r;
    }
    return best;
}

float elapsed(cudaEvent_t a, cudaEvent_t b) {
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
        cudaGetLastError();
        return 0.0f;
    }
    return ms;
}

void worker_main(tm_server* s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        // 1. retire finished slots
        bool any_busy = false;
        for (auto& sl : s->slots) {
            if (!sl.busy) continue;
            const cudaError_t q = cudaEventQuery(sl.ev[3]);
            if (q == cudaErrorNotReady) { any_busy = true; continue; }
            auto r = sl.req;
            if (q != cudaSuccess && r->status == TM_OK) r->status = TM_ERR_CUDA;
            if (r->status == TM_OK) {
                const int N = r->req.params.top_n, L = r->req.n_libs;
                for (int li = 0; li < L; ++li)
                    memcpy(r->req.out_host + ((size_t)li * r->req.n + sl.p0) * N, sl.hits_host + (size_t)li * sl.m * N,
                           (size_t)sl.m * N * sizeof(tm_hit));
                r->h2d_ms += elapsed(sl.ev[0], sl.ev[1]);
                r->kernels_ms += elapsed(sl.ev[1], sl.ev[2]);
                r->d2h_ms += elapsed(sl.ev[2], sl.ev[3]);
            }
            sl.busy = false;
            sl.req.reset();
            r->tiles_inflight--;
            r->tiles_done++;
            const bool all_sent = r->next >= r->req.n || r->cancelled;
            if (all_sent && r->tiles_inflight == 0 && !r->finished) {
                if (r->cancelled && r->status == TM_OK) r->status = TM_ERR_CANCELLED;
                finish_locked(s, r);
            }
        }
        // drop fully dispatched or cancelled requests from the pending list
        for (auto it = s->pending.begin(); it != s->pending.end();) {
            auto& r = *it;
            if (r->cancelled && r->tiles_inflight == 0 && !r->finished) {
                r->status = TM_ERR_CANCELLED;
                finish_locked(s, r);
            }
            if (r->finished || r->next >= r->req.n || r->cancelled) it = s->pending.erase(it);
            else ++it;
        }
        if (s->stop && !any_busy) break;
        // 2. dispatch into free slots
        bool dispatched = false;
        if (!s->stop && !s->paused) {
            for (auto& sl : s->slots) {
                if (sl.busy) continue;
                auto r = pick_locked(s, sl.lines_only);
                if (!r) continue;
                const int64_t m = std::min<int64_t>(s->prm.tile_patterns, r->req.n - r->next);
                const size_t esz = r->req.dtype == TM_DTYPE_U16 ? 2 : 4;
                const size_t frame = (size_t)r->req.H * r->req.W * esz;
                sl.req = r;
                sl.p0 = r->next;
                sl.m = m;
                sl.busy = true;
                r->next += m;
                r->tiles_inflight++;
                if (r->t_first < 0) r->t_first = s->now_ms();
                int rc = TM_OK;
                const bool line = r->req.priority > 0;
                const cudaStream_t st = line ? sl.stream_hi : sl.stream;
                const int N = r->req.params.top_n, L = r->req.n_libs;
                const void* fr = nullptr;
                cudaEventRecord(sl.ev[0], st);
                if (r->req.frames_dev) {
                    fr = (const char*)r->req.frames_dev + (size_t)sl.p0 * frame;
                } else {
                    fr = sl.frames;
                    if (cudaMemcpyAsync(sl.frames, (const char*)r->req.frames_host + (size_t)sl.p0 * frame, m * frame,
                                        cudaMemcpyHostToDevice, st) != cudaSuccess)
                        rc = TM_ERR_CUDA;
                }
                cudaEventRecord(sl.ev[1], st);
                // hits of library li land at rows p0.. of the request's [n_libs][n][N] device buffer
                tm_hit* dst = r->hits_dev + (size_t)sl.p0 * N;
                if (rc == TM_OK) {
                    tmgb::set_sm_cap(line ? 0 : s->map_sm_cap);
                    rc = tmgb::index_patterns_ex(s->ctx, &r->req.params, fr, r->req.dtype, m, r->req.H, r->req.W,
                                                 nullptr, r->libs.data(), L, dst, r->req.n * N, nullptr, st);
                    tmgb::set_sm_cap(0);
                }
                cudaEventRecord(sl.ev[2], st);
                if (rc == TM_OK &&
                    cudaMemcpy2DAsync(sl.hits_host, (size_t)m * N * sizeof(tm_hit), dst,
                                      (size_t)r->req.n * N * sizeof(tm_hit), (size_t)m * N * sizeof(tm_hit), (size_t)L,
                                      cudaMemcpyDeviceToHost, st) != cudaSuccess)
                    rc = TM_ERR_CUDA;
                if (rc != TM_OK && r->status == TM_OK) r->status = rc;
                cudaEventRecord(sl.ev[3], st);
                dispatched = true;
            }
        }
        if (dispatched) continue;
        // 3. sleep briefly while tiles are in flight, else until work arrives
        if (any_busy) {
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(50));
            lk.lock();
        } else {
            s->cv_work.wait_for(lk, std::chrono::milliseconds(20));
        }
    }
}

void free_slots(std::vector<Slot>& slots) {
    for (auto& x : slots) {
        if (x.frames) cudaFree(x.frames);
        if (x.hits_host) cudaFreeHost(x.hits_host);
        for (cudaEvent_t e : x.ev)
            if (e) cudaEventDestroy(e);
        if (x.stream) cudaStreamDestroy(x.stream);
        if (x.stream_hi) cudaStreamDestroy(x.stream_hi);
    }
}

}  // namespace

extern "C" {

void tm_server_params_default(tm_server_params* p) {
    if (!p) return;
    memset(p, 0, sizeof *p);
    p->slots = 3;
    p->tile_patterns = 512;
    p->max_H = 256;
    p->max_W = 256;
    p->max_libs = 2;
    p->max_top_n = 5;
    p->queue_bytes = 0;
    p->blocking_submit = 1;
    p->priority_slots = 1;
    p->hbm_budget_bytes = 0;
    p->reserve_sms = -1;
}

int tm_server_create(tm_ctx* ctx, const tm_server_params* params, tm_server** out) {
    if (!ctx || !out) return sfail(TM_ERR_INVALID_ARG, "tm_server_create: NULL argument");
    tm_server_params p;
    if (params) p = *params;
    else tm_server_params_default(&p);
    if (p.slots < 1 || p.slots > 16 || p.tile_patterns < 1 || p.max_H < 1 || p.max_W < 1 || p.max_libs < 1 ||
        p.max_libs > TM_MAX_LIBS || p.max_top_n < 1 || p.max_top_n > TM_MAX_TOPN || p.priority_slots < 0 ||
        (p.priority_slots >= p.slots && p.slots > 1) || (p.slots == 1 && p.priority_slots > 0))
        return sfail(TM_ERR_INVALID_ARG, "tm_server_create: bad parameters");
    if (p.hbm_budget_bytes == 0) p.hbm_budget_bytes = (size_t)256 << 20;
    auto s = std::make_unique<tm_server>();
    s->ctx = ctx;
    s->prm = p;
    s->t0 = std::chrono::steady_clock::now();
    if (cudaGetDevice(&s->device) != cudaSuccess) return sfail(TM_ERR_CUDA, "tm_server_create: no device");
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device) != cudaSuccess)
        return sfail(TM_ERR_CUDA, "tm_server_create: no device");
    const int reserve = p.reserve_sms >= 0 ? p.reserve_sms : (p.priority_slots > 0 ? sms / 4 : 0);
    if (reserve >= sms) return sfail(TM_ERR_INVALID_ARG, "tm_server_create: reserve_sms leaves no SM for maps");
    s->map_sm_cap = reserve > 0 ? sms - reserve : 0;
    s->slots.resize(p.slots);
    int prio_lo = 0, prio_hi = 0;
    cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
    for (int i = 0; i < p.slots; ++i) s->slots[i].lines_only = i >= p.slots - p.priority_slots;
    bool ok = cudaMalloc(&s->arena.base, p.hbm_budget_bytes) == cudaSuccess;
    for (auto& sl : s->slots) {
        if (!ok) break;
        ok = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) == cudaSuccess &&
             cudaStreamCreateWithPriority(&sl.stream_hi, cudaStreamNonBlocking, prio_hi) == cudaSuccess &&
             cudaMalloc(&sl.frames, (size_t)p.tile_patterns * p.max_H * p.max_W * 4) == cudaSuccess &&
             cudaMallocHost(&sl.hits_host, (size_t)p.max_libs * p.tile_patterns * p.max_top_n * sizeof(tm_hit)) ==
                 cudaSuccess;
        for (int e = 0; e < 4 && ok; ++e) ok = cudaEventCreate(&sl.ev[e]) == cudaSuccess;
    }
    if (!ok) {
        cudaGetLastError();
        free_slots(s->slots);
        if (s->arena.base) cudaFree(s->arena.base);
        return sfail(TM_ERR_OOM, "tm_server_create: staging or arena allocation failed");
    }
    s->arena.size = p.hbm_budget_bytes;
    s->arena.free_blocks[0] = p.hbm_budget_bytes & ~(size_t)255;
    tm_server* raw = s.release();
    raw->worker = std::thread(worker_main, raw);
    *out = raw;
    return TM_OK;
}

int tm_server_submit(tm_server* s, const tm_request* req, uint64_t* ticket) {
    if (!s || !req || !ticket) return sfail(TM_ERR_INVALID_ARG, "tm_server_submit: NULL argument");
    if (req->n < 1 || (!req->frames_host == !req->frames_dev) || !req->out_host || req->H < 1 || req->W < 1 ||
        req->H > s->prm.max_H || req->W > s->prm.max_W || req->n_libs < 1 || req->n_libs > s->prm.max_libs ||
        !req->lib_ids || (req->dtype != TM_DTYPE_U16 && req->dtype != TM_DTYPE_F32) || req->params.top_n < 1 ||
        req->params.top_n > s->prm.max_top_n)
        return sfail(TM_ERR_INVALID_ARG, "tm_server_submit: request outside the server's limits");
    auto r = std::make_shared<Request>();
    r->req = *req;
    r->libs.assign(req->lib_ids, req->lib_ids + req->n_libs);
    r->req.lib_ids = r->libs.data();
    r->tiles_total = (req->n + s->prm.tile_patterns - 1) / s->prm.tile_patterns;
    r->bytes = req->frames_host ? (size_t)req->n * req->H * req->W * (req->dtype == TM_DTYPE_U16 ? 2 : 4) : 0;
    const size_t hb = (size_t)req->n_libs * req->n * req->params.top_n * sizeof(tm_hit);
    if (((hb + 255) & ~(size_t)255) > (s->arena.size & ~(size_t)255))
        return sfail(TM_ERR_INVALID_ARG, "tm_server_submit: the request's hits exceed the server's HBM budget");
    std::unique_lock<std::mutex> lk(s->mu);
    const double t_submit = s->now_ms();
    // admission: queued frame bytes, then room for the hits in the device arena
    bool got = false;
    auto room = [&] {
        if (s->stop) return true;
        if (s->prm.queue_bytes && s->bytes_in > 0 && s->bytes_in + r->bytes > s->prm.queue_bytes) return false;
        got = s->arena.alloc(hb, &r->arena_off);
        return got;
    };
    if (!room()) {
        if (!s->prm.blocking_submit) return sfail(TM_ERR_BUSY, "tm_server_submit: admission budget full");
        s->cv_room.wait(lk, room);
    }
    if (s->stop) {
        if (got) s->arena.release(r->arena_off, hb);
        return sfail(TM_ERR_CANCELLED, "tm_server_submit: server stopping");
    }
    r->arena_bytes = hb;
    r->hits_dev = (tm_hit*)((char*)s->arena.base + r->arena_off);
    r->ticket = s->next_ticket++;
    r->t_submit = t_submit;
    r->t_admit = s->now_ms();
    s->bytes_in += r->bytes;
    s->reqs[r->ticket] = r;
    s->pending.push_back(r);
    *ticket = r->ticket;
    s->cv_work.notify_all();
    return TM_OK;
}

int tm_server_wait(tm_server* s, uint64_t ticket, int32_t timeout_ms, tm_request_status* status) {
    if (!s) return sfail(TM_ERR_INVALID_ARG, "tm_server_wait: NULL server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return sfail(TM_ERR_NOT_FOUND, "tm_server_wait: unknown ticket");
    auto r = it->second;
    auto done = [&] { return r->finished; };
    if (timeout_ms < 0) s->cv_done.wait(lk, done);
    else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done))
        return sfail(TM_ERR_TIMEOUT, "tm_server_wait: request not finished in time");
    if (status) {
        status->status = r->status;
        status->tiles = (int32_t)r->tiles_done;
        status->submit_ms = r->t_submit;
        status->first_dispatch_ms = r->t_first;
        status->done_ms = r->t_done;
        status->admit_ms = r->t_admit;
        status->h2d_ms = r->h2d_ms;
        status->kernels_ms = r->kernels_ms;
        status->d2h_ms = r->d2h_ms;
    }
    s->reqs.erase(it);
    return TM_OK;
}

int tm_server_cancel(tm_server* s, uint64_t ticket) {
    if (!s) return sfail(TM_ERR_INVALID_ARG, "tm_server_cancel: NULL server");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return sfail(TM_ERR_NOT_FOUND, "tm_server_cancel: unknown ticket");
    it->second->cancelled = true;
    s->cv_work.notify_all();
    return TM_OK;
}

int tm_server_pause(tm_server* s, int32_t paused) {
    if (!s) return sfail(TM_ERR_INVALID_ARG, "tm_server_pause: NULL server");
    std::lock_guard<std::mutex> lk(s->mu);
    s->paused = paused != 0;
    s->cv_work.notify_all();
    return TM_OK;
}

void tm_server_destroy(tm_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        for (auto& kv : s->reqs) kv.second->cancelled = true;
        s->cv_work.notify_all();
        s->cv_room.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    for (auto& sl : s->slots) {
        cudaStreamSynchronize(sl.stream);
        cudaStreamSynchronize(sl.stream_hi);
    }
    free_slots(s->slots);
    if (s->arena.base) cudaFree(s->arena.base);
    delete s;
}

}  // extern "C"
