/*
 * tmgb -- GB300-native template-matching orientation mapping (indexing hot path).
 *
 * C ABI of libtmgb.so.  Plain pointers and sizes only.  Every function returns an int
 * status (TM_OK = 0); on failure tm_last_error() gives a message for the calling thread.
 * No function aborts, traps or falls back to the CPU: without a usable GPU the calls
 * fail with TM_ERR_CUDA.
 *
 * Method (arXiv 2111.07347, Section 2.2): every diffraction pattern P is compared with
 * every template T of a library by the correlation index of Eq. 1,
 *     Q = sum_i P(x_i) T(x_i) / ( sqrt(sum_i P(x_i)^2) sqrt(sum_i T(x_i)^2) ),
 * evaluated in polar coordinates about the direct beam, with the template slid along
 * the azimuthal axis with wraparound; the best Q and its in-plane angle are kept per
 * template and the top N templates are returned.
 *
 * Device pointers: arguments named *_dev are device memory owned by the caller (for
 * example torch.Tensor.data_ptr()).  Work is enqueued on the caller's CUDA stream
 * (`stream`, a cudaStream_t; NULL = legacy default stream) and is complete when that
 * stream is synchronised.  Host pointers are read before the call returns.
 *
 * Threading: one context may be used from several host threads; calls are serialised
 * on the host by the context.  Scratch memory is kept per CUDA stream handle: calls on
 * one stream are ordered by that stream, calls on different streams use separate
 * scratch buffers and may overlap on the GPU.  Do not destroy a stream while work of
 * this context is still pending on it.
 */
#ifndef TMGB_H
#define TMGB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status codes */
enum {
    TM_OK = 0,
    TM_ERR_INVALID_ARG = 1,  /* bad pointer, size, grid or parameter (NaN, out of range)   */
    TM_ERR_OOM = 2,          /* device allocation failed or the context's HBM budget is hit */
    TM_ERR_CUDA = 3,         /* a CUDA runtime call failed (message has the CUDA error)     */
    TM_ERR_TIMEOUT = 4,      /* a bounded wait ran out                                     */
    TM_ERR_BUSY = 5,         /* a non-blocking submit found no room                        */
    TM_ERR_CANCELLED = 6,    /* the request was cancelled                                  */
    TM_ERR_NOT_FOUND = 7,    /* unknown library id or ticket                               */
    TM_ERR_UNSUPPORTED = 8   /* valid request this build does not implement                */
};

enum { TM_DTYPE_U16 = 0, TM_DTYPE_F32 = 1 };             /* frame element type            */
enum { TM_COORDS_POLAR = 0, TM_COORDS_XY = 1 };          /* template spot coordinates     */
enum { TM_LIB_MIRROR = 1u, TM_LIB_UNIT_INTENSITY = 2u }; /* library flags                 */
enum { TM_PATH_FP32_SPARSE = 0, TM_PATH_BF16_RESCORE = 1 };

typedef struct tm_ctx tm_ctx;

/* ---------------------------------------------------------------- libraries
 * A template library (Section 2.1: each template is a list of reflections with
 * coordinates (kx, ky)_i and intensities I_i at in-plane angle zero).  At load time the
 * spots are put on the polar grid the library is built for (Section 2.2):
 *   r_i = floor(r / dr + 1/2),  t_i = floor(u + 1/2) mod n_theta,
 *   u = theta' / (2 pi / n_theta), theta' = theta reduced to [0, 2 pi),
 * computed in double precision; spots with r_i >= n_r are dropped; spots landing on the
 * same polar pixel are merged by summing intensity; with TM_LIB_MIRROR every template
 * gets a mirror copy made by reflecting its spots across y = 0 (theta -> -theta) before
 * rounding (Section 2.2, Fig. 2 caption), stored at index k + n_templates; with
 * TM_LIB_UNIT_INTENSITY every input spot has intensity 1 before merging (Section 4.3).
 * The template norm sqrt(sum I^2) of Eq. 1 is taken over the merged spots.  A template
 * whose merged spot set is invariant under a rotation by 2 pi / n (n dividing n_theta)
 * is only slid over n_theta / n shifts (its scores repeat exactly beyond).
 */
typedef struct tm_library_desc {
    int64_t n_templates;          /* K0 >= 1                                              */
    const int64_t* spot_offsets;  /* host [K0 + 1], CSR, offsets[0] = 0, non-decreasing   */
    const double* spot_a;         /* host [S]: r in pixels (POLAR) or kx (XY)             */
    const double* spot_b;         /* host [S]: theta in radians (POLAR) or ky (XY)        */
    const double* intensity;      /* host [S], finite (ignored with UNIT_INTENSITY)       */
    int32_t coords;               /* TM_COORDS_POLAR or TM_COORDS_XY                      */
    uint32_t flags;               /* TM_LIB_* bits                                        */
    double px_per_unit;           /* XY: detector pixels per unit of (kx, ky); > 0        */
    int32_t n_r;                  /* polar grid: radii r_j = j * dr, j in [0, n_r)        */
    int32_t n_theta;              /* polar grid: angles 2 pi k / n_theta, k in [0, n_theta) */
    double dr;                    /* radial step in pixels, > 0                           */
} tm_library_desc;

typedef struct tm_library_info {
    int64_t n_templates;          /* K, including mirror copies                          */
    int64_t n_base;               /* K0                                                  */
    int64_t n_spots;              /* merged spots over all K templates                   */
    int32_t max_spots;            /* largest merged spot count                           */
    int32_t mirror;               /* 1 if mirror copies were added                       */
    int32_t n_r, n_theta;
    double dr;
    int64_t n_symmetric;          /* templates with rotational order > 1                 */
    int64_t macs_per_pattern;     /* sum_k spots_k * n_theta / order_k (sparse work)     */
    int64_t device_bytes;         /* device memory held by the library                   */
} tm_library_info;

/* ---------------------------------------------------------------- indexing
 * Parameters of the per-pattern path (Section 2.2 and Section 4.1/4.3 preprocessing):
 * g = max(x, 0)^gamma - subtract per raw pixel, then bilinear polar resampling about
 * (cx, cy) (x = column, y = row; zero outside the frame), then [pre-filter], then Q. */
typedef struct tm_index_params {
    double gamma;                 /* > 0; 0.5 uses sqrt                                  */
    double subtract;              /* constant subtracted after gamma (0 = none)          */
    double cx, cy;                /* beam centre in pixels; NaN -> ((W-1)/2, (H-1)/2)    */
    double prefilter_fraction;    /* (0, 1]: keep ceil(f K) templates by radial cosine   */
    int32_t top_n;                /* N >= 1 results per pattern and library              */
    int32_t path;                 /* TM_PATH_FP32_SPARSE or TM_PATH_BF16_RESCORE         */
    int32_t rescore_k;            /* BF16 path: candidates rescored exactly (default 256) */
    int32_t reserved;             /* TM_INDEX_* flags                                     */
    const uint8_t* pixel_mask;    /* device [H][W] bytes, 16-byte aligned, or NULL: pixels
                                     whose byte is 0 read as 0 before gamma and subtraction
                                     (masked indexing, Section 4.3; see tm_matrix_mask)   */
    double threshold;             /* > 0: raw pixels below it read as 0 before gamma
                                     (Section 3.1: low-intensity pixels set to zero); 0 = off */
} tm_index_params;

/* tm_index_params.reserved flag: replay the call as a CUDA graph.  The first call with a
 * given set of arguments (pointers, sizes, parameters, libraries, stream) runs normally,
 * the second is captured into a graph on the caller's stream and launched, later identical
 * calls launch the graph.  Needs a created stream (not the legacy default stream, where
 * the call simply runs normally); a graph is rebuilt when the context's scratch buffers
 * were reallocated, and dropped when a library is unloaded.  Not used while stage timing
 * is on. */
#define TM_INDEX_GRAPH 1

/* tm_index_params.reserved flag for tests of the failure path: the BF16 tensor-core kernel's
 * MMA issuer issues nothing, so its producer and epilogue waits run out (about 1 s each);
 * the kernel records the timeout in the context's device error word, stops its roles,
 * frees its tensor memory and returns.  The FP32 sparse kernel's row staging (bulk copies,
 * for n_theta a multiple of 4 outside the dual row layout) expects 16 bytes more than its
 * copies bring, so its wait runs out (about 1 s, then 1 s more for the copies); it records
 * the timeout and returns.  tm_check then reports TM_ERR_TIMEOUT; the call's hits are
 * meaningless; the context stays usable. */
#define TM_INDEX_TEST_STALL 2

/* tm_index_params.reserved flag: in-plane angle below the polar step (Section 2.2: phi_1 is
 * resolved to the angular step of the polar grid; Section 5 names a better phi_1 optimisation
 * as future work).  Each hit's angle_deg becomes (shift + delta) 360 / n_theta, delta the
 * vertex of the parabola through Q at shift - 1, shift, shift + 1 (mod n_theta):
 * (Q- - Q+) / (2 (Q- - 2 Q0 + Q+)) for a negative curvature, else 0, clipped to [-1/2, 1/2].
 * The shift field keeps the integer best shift. */
#define TM_INDEX_REFINE 4

/* One result row.  Rows of a pattern are ordered by (score desc, template asc); when
 * fewer than N templates take part the tail rows have template_index = -1 and
 * score = -inf. */
typedef struct tm_hit {
    int32_t template_index;       /* expanded index k (mirror copies at k >= n_base)     */
    int32_t shift;                /* best azimuthal shift s (lowest among exact ties)    */
    float score;                  /* Q of Eq. 1                                          */
    float angle_deg;              /* in-plane angle phi1 = s * 360 / n_theta             */
    int32_t mirror;               /* 1 if the template is a mirror copy                  */
} tm_hit;

typedef struct tm_stats {
    int64_t patterns;             /* patterns indexed by the call                        */
    int64_t correlations;         /* (pattern, template, shift) triples evaluated        */
    int64_t templates_scored;     /* (pattern, template) pairs scored exactly            */
    int64_t launches;             /* this library's kernels launched by the call (the
                                     tensor-core path's stage A GEMM runs in cuBLAS and is
                                     not counted)                                         */
} tm_stats;

/* Create a context on CUDA device `device`.  hbm_budget_bytes caps the device memory
 * the context allocates (libraries + workspace); 0 = no cap.  The context owns every
 * library and workspace buffer it allocates; tm_destroy frees them. */
int tm_create(int device, size_t hbm_budget_bytes, tm_ctx** out);
void tm_destroy(tm_ctx* ctx);

/* Message of the last failed call on this thread ("" if none).  Valid until the next
 * call on this thread. */
const char* tm_last_error(void);

/* Copy a library to the device (see the library notes above).  *lib_id receives an id
 * >= 0.  Errors: TM_ERR_INVALID_ARG for a malformed descriptor, TM_ERR_OOM. */
int tm_load_library(tm_ctx* ctx, const tm_library_desc* desc, int* lib_id);
int tm_unload_library(tm_ctx* ctx, int lib_id);
int tm_library_info_get(tm_ctx* ctx, int lib_id, tm_library_info* out);

/* Copy the library's rounded, merged templates back to host buffers sized from
 * tm_library_info: offsets [K + 1], r [n_spots], t [n_spots], intensity [n_spots]
 * (float, as used on the device), norm [K] (float sqrt(sum I^2)), order [K] (rotational
 * order n_k).  Any pointer may be NULL to skip it.  Synchronous. */
int tm_library_export(tm_ctx* ctx, int lib_id, int64_t* offsets, int32_t* r, int32_t* t,
                      float* intensity, float* norm, int32_t* order);

/* The host half of tm_load_library without a device: validates the descriptor and puts
 * the templates on the polar grid exactly as tm_load_library does.  Call once with NULL
 * arrays to get the sizes in *info, then again with host buffers as for
 * tm_library_export.  The sparse kernel's spot words (both nullable, [n_spots]): packed
 * receives t | rho << 11 | w << 24 (t the angle column, rho the row of the spot's radius
 * among the library's distinct radii, w = ceil((n_theta - t) / 32) the first 32-wide shift
 * block that wraps), packed2 the spot's float offset in the kernel's dual-copy row layout
 * (bits 0..15: (t odd ? n_rad + rho : rho) * pitch_dual + (t & ~1)) and in its wrap-free
 * layout (bits 16..31: rho * pitch_wf + t), with pitch_dual = n_theta + 64 * NB2 rounded up
 * to even and pitch_wf = n_theta + 32 * NB, NB2 and NB the 64- and 32-wide block counts
 * ceil(n_theta / 64) and ceil(n_theta / 32) rounded up to 1, 2, 3, 4, 6, 8, 12, 16, 24 or
 * 32; a field is 0 when its layout would not fit 16 bits.  info->device_bytes is 0.  Needs
 * no GPU. */
int tm_library_prepare_host(const tm_library_desc* desc, tm_library_info* info, int64_t* offsets,
                            int32_t* r, int32_t* t, float* intensity, float* norm, int32_t* order,
                            int32_t* packed, int32_t* packed2);

/* The host half of tm_load_library, continued (no GPU): the sparse kernel's second copy of
 * its pruning-window entries, used by the unmasked top-N pass that bounds every template
 * (Eq. 1's numerator bounded over three windows of shifts, Section 2.2).  The templates are
 * in the order that pass visits them, by spot count, most first, ties by library index;
 * each 32-template word's entries are stored spot-major with its 32 lanes adjacent.
 * Call with NULL arrays to get *n_words (ceil(K / 32)) and *n_entries, then with host
 * buffers: order [n_words * 32] the library index at each position (padding 0);
 * word_start [n_words] the first entry of each word; entries [n_entries][2] int32 pairs,
 * entry word_start[w] + 32 i + l holding, for the template at position 32 w + l, its spot
 * i's {intensity (float bits), window entries j0 | d1 << 16 | d2 << 24} (j0 = rho * nchw +
 * t / 32 and the chunk increments of the second and third windows), zero where the
 * template has fewer spots.  TM_ERR_UNSUPPORTED when the library gets no window table
 * (the kernel then bounds by whole rows and keeps no second copy). */
int tm_library_bound_entries_host(const tm_library_desc* desc, int32_t* n_words, int64_t* n_entries,
                                  int32_t* order, int32_t* word_start, int32_t* entries);

/* Stage 1 (Section 2.2, Fig. 2 (a)-(c)): gamma/subtract and bilinear polar resampling.
 * frames_dev [n][H][W] (TM_DTYPE_U16 or TM_DTYPE_F32, row-major, contiguous);
 * centres_dev [n][2] float (cx, cy) per pattern, finite, or NULL to use params->cx/cy for
 * every pattern (the direct beam is the origin of the transform, Section 2.2);
 * polar_dev [n][n_r][n_theta] float; norm_dev [n] float = sqrt(sum over the polar image
 * of P^2) (nullable); radial_dev [n][n_r] float = sum over theta (nullable).
 * Uses params->gamma, subtract, cx, cy. */
int tm_polar_transform(tm_ctx* ctx, const tm_index_params* params, const void* frames_dev,
                       int32_t dtype, int64_t n, int32_t H, int32_t W, const float* centres_dev,
                       int32_t n_r, int32_t n_theta, double dr, float* polar_dev, float* norm_dev,
                       float* radial_dev, void* stream);

/* Stage 2 (Section 2.2, azimuthally integrated pre-filter, Fig. 3): score_k =
 * R_P . R_T,k / (|R_P| |R_T,k|) from radial_dev [n][n_r] (Stage 1 output); keeps the
 * ceil(fraction K) best per pattern, ties to the lower template index.  mask_dev
 * [n][ceil(K/32)] uint32 receives bit (k % 32) of word k / 32 set for kept templates;
 * score_dev [n][K] float (nullable). */
int tm_prefilter(tm_ctx* ctx, int lib_id, const float* radial_dev, int64_t n, double fraction,
                 uint32_t* mask_dev, float* score_dev, void* stream);

/* Stage 3 (Eq. 1 at every shift with wraparound, Section 2.2, Fig. 2 (e)): for each
 * pattern and template the best Q and the lowest shift attaining it, in FP32.
 * polar_dev / norm_dev from Stage 1; mask_dev from Stage 2 or NULL (all templates).
 * q_dev [n][K] float and s_dev [n][K] int32; masked-out templates get -inf and -1. */
int tm_correlate(tm_ctx* ctx, int lib_id, const float* polar_dev, const float* norm_dev,
                 int64_t n, const uint32_t* mask_dev, float* q_dev, int32_t* s_dev,
                 void* stream);

/* Stage A7 alone: the BF16 tensor-core pre-score.  The correlation along theta is taken
 * through the correlation theorem (Section 2.2 names the FFT cross-correlation as the
 * alternative to sliding): C[k, s] = sum_m (w_m / n) Re(G[k, m] e^{2 pi i m s / n}) with
 * G[k, m] = sum_r conj(T^_k[r, m]) P^[r, m] over the library's spot radii.  T^ (the templates'
 * angular spectra, divided by |T_k|) is built once per library on the device, the first time
 * the tensor-core path uses it; P^ (divided by |P|) is formed in FP32; both are rounded to BF16.
 * Stage A (G for every frequency, a batched GEMM over the radii) and stage B (the sum over
 * frequencies for every shift, with the maximum over shifts) run on the tensor cores with FP32
 * accumulation.  score_dev [n][K] float receives Q~ = max_s C / (|P| |T_k|) for every template
 * scored and -NaN for the others (the pre-filter's rejects when fraction < 1).  polar_dev /
 * norm_dev: Stage 1 outputs; radial_dev: Stage 1 azimuthal sums (used when fraction < 1).
 * n_theta must be even and <= 376, and the library's distinct radii must fit the DFT's shared
 * memory (about 150 at n_theta = 360), else TM_ERR_UNSUPPORTED. */
int tm_prescore(tm_ctx* ctx, int lib_id, const float* polar_dev, const float* norm_dev,
                const float* radial_dev, int64_t n, double fraction, float* score_dev, void* stream);

/* Autotune the FP32 sparse kernel for a set of libraries: time its shapes -- block size (128,
 * 256, 512 threads; default 256) x templates seeded per warp for the pruned top-N (4, 8, 16;
 * default 8: the templates of highest bound are scored first, so that the top-N threshold
 * the others are pruned against starts high) on the first min(n, 2048) frames, then the best
 * of these against its block size with 4 patterns per CTA bounded together (default 1) and
 * each seed count on the first min(n, 16384) -- with these parameters, keep the fastest for
 * later calls on libraries of the same shapes (template count, spot count, radii, n_theta)
 * and top_n, and, when the
 * environment variable TMGB_TUNE_CACHE names a file, append "key threads seeds tile ms" to
 * it (ms per 2048 frames); contexts created later read that file back (lines without the
 * tile: 1).  Synchronous.  *best_threads (nullable) receives the block size. */
int tm_autotune(tm_ctx* ctx, const tm_index_params* params, const void* frames_dev, int32_t dtype,
                int64_t n, int32_t H, int32_t W, const int32_t* lib_ids, int32_t n_libs,
                int32_t* best_threads, void* stream);

/* Wait for `stream`, then report whether a kernel of this context stopped on a bounded
 * wait since the last check (TM_ERR_TIMEOUT; the error word is cleared). */
int tm_check(tm_ctx* ctx, void* stream);

/* The whole path for a batch: frames -> polar -> [pre-filter] -> Q -> top-N, for each
 * of n_libs libraries (all built for the same polar grid).  path TM_PATH_FP32_SPARSE
 * scores every surviving template exactly in FP32 (Stage 3 with a fused top-N);
 * TM_PATH_BF16_RESCORE takes the rescore_k best by the Stage A7 pre-score (exact radix
 * select, ties to the lower index) and rescores them exactly in FP32 before the top-N.  out_dev [n_libs][n][top_n]
 * tm_hit.  centres_dev [n][2] float per-pattern beam centres (finite) or NULL for
 * params->cx/cy.  stats (host, nullable) receives counts for the call. */
int tm_index_patterns(tm_ctx* ctx, const tm_index_params* params, const void* frames_dev,
                      int32_t dtype, int64_t n, int32_t H, int32_t W, const float* centres_dev,
                      const int32_t* lib_ids, int32_t n_libs, tm_hit* out_dev,
                      tm_stats* stats, void* stream);

/* The whole path (as tm_index_patterns) for frames and results in HOST memory.  The paper's
 * GPU implementation moves each image to the device before indexing it (Section 2.2); here
 * the batch is cut into chunks of `chunk` patterns (0: 4096) that alternate between two
 * streams owned by the context, so the host->device copy of one chunk overlaps the kernels
 * of the previous one, and each chunk's hits are copied back as soon as they are ready.
 * frames_host [n][H][W] (dtype), centres_host [n][2] float or NULL, out_host
 * [n_libs][n][top_n] tm_hit.  Pass page-locked host memory for the overlap (pageable memory
 * works, with the copies serialised by the driver).  Synchronous: returns when out_host is
 * complete.  One host-buffer call at a time per context (later calls wait).  stats (nullable)
 * receives the totals.  Errors as tm_index_patterns. */
int tm_index_patterns_host(tm_ctx* ctx, const tm_index_params* params, const void* frames_host, int32_t dtype,
                           int64_t n, int32_t H, int32_t W, const float* centres_host, const int32_t* lib_ids,
                           int32_t n_libs, tm_hit* out_host, int64_t chunk, tm_stats* stats);

/* Per-stage device time, measured with CUDA events recorded on the stream each kernel
 * is launched on (around every launch of the stage). */
enum {
    TM_STAGE_POLAR = 0,       /* gamma + polar resampling                               */
    TM_STAGE_PREFILTER = 1,   /* radial norms, scores and selection                     */
    TM_STAGE_SPARSE = 2,      /* FP32 sparse correlation + top-N                        */
    TM_STAGE_DFT = 3,         /* angular DFT of the polar images (BF16 path)            */
    TM_STAGE_DENSE = 4,       /* BF16 tensor-core inverse DFT + max over shifts (stage B) */
    TM_STAGE_RESCORE = 5,     /* FP32 rescore of the candidates (BF16 path)             */
    TM_STAGE_GEMM = 6,        /* BF16 tensor-core contraction over radii (stage A)      */
    TM_STAGE_SELECT = 7,      /* exact selection of the candidates (BF16 path)          */
    TM_STAGE_COUNT = 8
};
typedef struct tm_profile {
    double ms[TM_STAGE_COUNT];        /* summed launch durations                        */
    int64_t launches[TM_STAGE_COUNT]; /* kernel launches timed                           */
    int64_t sparse_macs;              /* multiply-adds (spots x shifts of the templates
                                         scored) the FP32 sparse kernel executed; its bound
                                         pruning skips templates that cannot enter the top-N */
} tm_profile;

/* Enable (1) or disable (0) stage timing for later calls on ctx; resets the totals. */
int tm_profile_enable(tm_ctx* ctx, int enable);
/* Totals since the last enable/read; waits for the timed work to finish, then resets. */
int tm_profile_read(tm_ctx* ctx, tm_profile* out);

/* Whole path (FP32 sparse, one library, no pre-filter) without any allocation.  The paper
 * has no counterpart: this serves callers that cannot call cudaMalloc while they index --
 * an application whose device memory belongs to another allocator (a framework's caching
 * allocator that must see every allocation), or an acquisition callback that runs inside
 * a fixed, pre-reserved device budget and must not wait on the driver's allocator.
 * Scratch (polar ray steps, polar images, norms, counter) lives in one static 64 MiB device
 * array that every GPU loading this library keeps for the life of the process: 512 KiB hold
 * the ray steps of up to 8 polar grids, and a call needs n_r * n_theta * 4 + 4 bytes per
 * pattern plus 512 bytes of the rest (361 patterns per call on a 128 x 360 grid); a call
 * whose scratch would not fit fails with TM_ERR_INVALID_ARG and says how much it needed.
 * All calls share the array and find the previous call's data in it (each call rewrites
 * what it reads); calls that overlap on the GPU race, so issue them on one stream.  Set-up:
 * the first call on a device looks the array's address up (cudaGetSymbolAddress) with that
 * device current, and the first call for each polar grid (n_theta, dr) on a device writes
 * the grid's ray steps into the array with a synchronous copy; make those first calls
 * before any stream capture.  params are checked as for tm_index_patterns (pixel_mask
 * 16-byte aligned, threshold finite and >= 0, ...); params->path must be
 * TM_PATH_FP32_SPARSE and params->prefilter_fraction 1.  frames_dev [n][H][W], out_dev
 * [n][top_n] tm_hit.  Results equal tm_index_patterns'. */
int tm_index_patterns_noalloc(tm_ctx* ctx, const tm_index_params* params, const void* frames_dev,
                              int32_t dtype, int64_t n, int32_t H, int32_t W, int32_t lib_id,
                              tm_hit* out_dev, void* stream);

/* ---------------------------------------------------------------- two-stage indexing
 * Section 4.3: the intense matrix reflections are removed from every pattern with a mask
 * made from the average of all patterns, thresholded, then cleaned by erosions (noise-like
 * features) and dilations (tails of intense peaks); the masked patterns are indexed against
 * the precipitate library (tm_index_params.pixel_mask). */

/* Per-pixel sum over frames: sum_dev [H][W] double = (accumulate ? sum_dev : 0) + sum over
 * p of frames_dev[p] in frame order, in FP64 (exact for u16 frames; the fixed order makes
 * f32 results reproducible and chunked sums equal one pass).  Asynchronous on stream. */
int tm_frame_sum(tm_ctx* ctx, const void* frames_dev, int32_t dtype, int64_t n, int32_t H, int32_t W,
                 int32_t accumulate, double* sum_dev, void* stream);

/* Mask of the pixels to keep: mask_dev [H][W] bytes, 1 = keep.  Set pixels are those with
 * sum > threshold * n_frames (FP64; the mean exceeds threshold); then n_open erosions, n_open
 * dilations (an opening: removes features smaller than the 3 x 3 structuring element) and
 * n_dilate further dilations (cover the tails of the peaks); pixels outside the image count as
 * unset; the mask is the complement.  Asynchronous on stream. */
int tm_matrix_mask(tm_ctx* ctx, const double* sum_dev, int64_t n_frames, int32_t H, int32_t W, double threshold,
                   int32_t n_open, int32_t n_dilate, uint8_t* mask_dev, void* stream);

/* Direct-beam centring (Section 3.1: the beam of every pattern is centred; the polar
 * transform's origin is the beam's centre, Section 2.2).  centres_dev [n][2] float receives,
 * per pattern, the intensity-weighted centre of mass (x = column, y = row) of the raw pixels
 * within `radius` of the current estimate, recomputed `iterations` times starting from
 * (cx0, cy0) (NaN -> ((W-1)/2, (H-1)/2)); FP64 sums over the disc's bounding box row by row,
 * distances as dx*dx + dy*dy <= radius*radius; an empty disc keeps the estimate.  Pass the
 * result as tm_index_patterns' centres_dev.  radius in (0, 1e4], iterations in [1, 100].
 * Asynchronous on stream. */
int tm_find_centres(tm_ctx* ctx, const void* frames_dev, int32_t dtype, int64_t n, int32_t H, int32_t W,
                    double cx0, double cy0, double radius, int32_t iterations, float* centres_dev, void* stream);

/* Background removal and smoothing (Section 3.1: the diffuse background of every pattern was
 * removed with a difference of Gaussians and the result smoothed by a Gaussian blur; the
 * paper gives no parameters).  out_dev [n][H][W] float receives, per frame x (frames_dev
 * [n][H][W] u16 or f32): d = max(G(dog_sigma_min) * x - G(dog_sigma_max) * x, 0) when
 * dog_sigma_max > 0 (else d = x), then G(blur_sigma) * d when blur_sigma > 0.  G(s) is the
 * separable Gaussian of standard deviation s on the integer offsets |i| <= floor(truncate s
 * + 1/2) (truncate <= 0: 4), normalised to sum 1, applied along rows then along columns with
 * the edge pixel repeated outside the frame; FP32 sums in ascending offset order, weights
 * from double precision.  Radii up to 256; sigmas must be 0 or in [0.1, 64].  Index the
 * result as TM_DTYPE_F32 frames (gamma and the threshold then apply to it).  Uses context
 * workspace; asynchronous on stream. */
typedef struct tm_preprocess_params {
    double dog_sigma_min;    /* inner Gaussian of the difference (< dog_sigma_max)         */
    double dog_sigma_max;    /* outer Gaussian; <= 0: no background removal               */
    double blur_sigma;       /* smoothing after it; <= 0: none                            */
    double truncate;         /* kernel radius in sigmas (<= 0: 4)                         */
} tm_preprocess_params;
int tm_preprocess(tm_ctx* ctx, const tm_preprocess_params* params, const void* frames_dev, int32_t dtype, int64_t n,
                  int32_t H, int32_t W, float* out_dev, void* stream);

/* Template simulation over an orientation grid (Section 2.1: for each orientation the
 * reflections near the Ewald sphere, by their excitation error, weighted by |F|^2 and a
 * linear relrod shape, projected onto the detector; the strongest kept).  g_dev [G][3] are
 * reciprocal lattice points (1/Angstrom, crystal frame), f2_dev [G] their |F|^2 (unit
 * scattering factors or any table), gnorm_dev [G] their |g|; rot_dev [D][3][3] (row-major)
 * the orientations: row j is the beam-frame axis j in crystal coordinates, z along the beam.
 * Per orientation and point, in double precision with each operation rounded in this order:
 * x_j = (R_j0 g_0 + R_j1 g_1) + R_j2 g_2, t = x_2 + k with k = 1 / wavelength,
 * s = k - sqrt((x_0 x_0 + x_1 x_1) + t t); kept when |s| <= s_max and
 * I = |F|^2 (1 - |s| / s_max) > 0.  counts_dev [D] receives the number kept (at most
 * max_spots; -1 when more than 512 reflections of one orientation are within s_max: make
 * s_max or the point set smaller) and spots_dev [D][max_spots][3] the (x_0, x_1, I) of the
 * kept ones, I descending, ties by |g| ascending, then by point index.  Feed them to
 * tm_load_library as TM_COORDS_XY templates.  Asynchronous on stream. */
int tm_kinematic_spots(tm_ctx* ctx, const double* g_dev, const double* f2_dev, const double* gnorm_dev, int64_t G,
                       const double* rot_dev, int64_t D, double wavelength, double s_max, int32_t max_spots,
                       int32_t* counts_dev, double* spots_dev, void* stream);

/* Orientation maps (Section 4.1: inverse pole figure maps along the sample axes).  For each
 * pattern p, hit hits_dev[p * stride] (its best template b, mirror copies at b >= K0, and
 * in-plane angle phi = angle_deg) gives the orientation O = Rz(phi) M R_b, with rot_dev
 * [K0][3][3] the templates' orientation matrices (row-major; rows: the beam-frame axes in
 * crystal coordinates, as tm_kinematic_spots takes them) and M = diag(1, -1, 1) for a mirror
 * copy, else 1; v_dev [n][3] double receives v = O^T e, the crystal direction along the
 * sample axis e = (ex, ey, ez).  FP64, each operation rounded in a fixed order (cos and sin
 * from the math library); NaN for a missing hit (template index < 0).  Asynchronous. */
int tm_orientation_vectors(tm_ctx* ctx, const tm_hit* hits_dev, int64_t n, int32_t stride, const double* rot_dev,
                           int64_t K0, double ex, double ey, double ez, double* v_dev, void* stream);
/* Eq. 2: deg_dev [n] receives |acos(va . vb / (|va| |vb|))| in degrees (the cosine clipped to
 * [-1, 1]) for the vectors va_dev, vb_dev [n][3] of two maps; NaN where either is missing. */
int tm_angular_deviation(tm_ctx* ctx, const double* va_dev, const double* vb_dev, int64_t n, double* deg_dev,
                         void* stream);

/* Default parameters: gamma 0.5, subtract 0, centre NaN, prefilter 1, top_n 5,
 * FP32 sparse path, rescore_k 256, no pixel mask, no threshold. */
void tm_index_params_default(tm_index_params* p);

/* ---------------------------------------------------------------- serving loop
 * Continuous batching for on-line mapping (Section 5: indexing a pattern in a few to tens
 * of milliseconds, on the order of a detector's acquisition time, so indexing can run
 * beside acquisition).  A server owns a worker thread and `slots` CUDA streams, each
 * with device staging for one tile.  Requests (a scan line or a whole map) are split into
 * tiles of `tile_patterns`; tiles of different requests interleave on the device as
 * slots free up, higher-priority requests (scan lines) first, then submission order.
 * The libraries stay resident in the context, and every admitted request keeps its hits
 * ([n_libs][n][top_n] tm_hit, the partial top-N state as its tiles complete) in a device
 * arena of hbm_budget_bytes: a request is admitted when that arena has room for it (and
 * its frame bytes fit queue_bytes).  Tiles of maps leave reserve_sms SMs free, so a scan
 * line's kernels start without waiting for a map's.  Results of a pattern do not depend
 * on the other patterns of its tile, so a request's result is the same alone and in a mix.
 */
typedef struct tm_server tm_server;

typedef struct tm_server_params {
    int32_t slots;                /* tiles in flight (CUDA streams), >= 1; default 3      */
    int32_t tile_patterns;        /* patterns per tile, >= 1; default 512                 */
    int32_t max_H, max_W;         /* largest frame accepted (sizes the staging)           */
    int32_t max_libs;             /* largest n_libs of a request, in [1, 8]               */
    int32_t max_top_n;            /* largest top_n of a request                           */
    size_t queue_bytes;           /* admission budget: frame bytes of requests submitted
                                     and not finished; 0 = no limit                       */
    int32_t blocking_submit;      /* 1: submit waits for budget; 0: TM_ERR_BUSY           */
    int32_t priority_slots;       /* of the slots, how many take only requests of priority
                                     > 0 (scan lines), so that they never wait behind map
                                     tiles; such tiles also run on high-priority streams;
                                     default 1 (0 when slots == 1)                         */
    size_t hbm_budget_bytes;      /* device arena for the admitted requests' hits; 0: 256 MiB.
                                     A request needing more than the whole arena is refused
                                     (TM_ERR_INVALID_ARG)                                  */
    int32_t reserve_sms;          /* SMs the persistent kernels of map tiles leave free
                                     (< 0: a quarter of the SMs when priority_slots > 0,
                                     else none; default -1)                                */
} tm_server_params;

typedef struct tm_request {
    const void* frames_host;      /* [n][H][W] host memory (pinned for overlap), read until
                                     the request finishes; NULL when frames_dev is given   */
    int32_t dtype;                /* TM_DTYPE_U16 or TM_DTYPE_F32                          */
    int32_t H, W;
    int64_t n;                    /* patterns, >= 1                                        */
    const int32_t* lib_ids;       /* copied at submit                                      */
    int32_t n_libs;
    int32_t priority;             /* higher first: 1 = scan line, 0 = map                  */
    tm_index_params params;
    tm_hit* out_host;             /* [n_libs][n][top_n] host memory, complete when the
                                     request finishes                                      */
    const void* frames_dev;       /* [n][H][W] device memory of the context's device instead
                                     of frames_host (a map already resident on the GPU), or
                                     NULL; read until the request finishes                 */
} tm_request;

typedef struct tm_request_status {
    int32_t status;               /* TM_OK, TM_ERR_CANCELLED, or the error of a tile       */
    int32_t tiles;
    double submit_ms, first_dispatch_ms, done_ms;   /* server clock, ms since creation    */
    double admit_ms;              /* when its hits were given room in the device arena    */
    double h2d_ms, kernels_ms, d2h_ms;  /* device time of its tiles' frame copies, kernels
                                     and hit copies, summed over its tiles (CUDA events)   */
} tm_request_status;

void tm_server_params_default(tm_server_params* p);
int tm_server_create(tm_ctx* ctx, const tm_server_params* params, tm_server** out);
/* Queue a request; *ticket identifies it.  TM_ERR_BUSY when blocking_submit is 0 and
 * the admission budget is full.  TM_ERR_INVALID_ARG for requests beyond the server's
 * limits. */
int tm_server_submit(tm_server* s, const tm_request* req, uint64_t* ticket);
/* Wait up to timeout_ms (< 0: no limit) for the request.  TM_OK when it finished
 * (status->status tells how), TM_ERR_TIMEOUT when it did not finish in time,
 * TM_ERR_NOT_FOUND for an unknown or already collected ticket.  A finished request is
 * forgotten once waited for. */
int tm_server_wait(tm_server* s, uint64_t ticket, int32_t timeout_ms, tm_request_status* status);
/* Cancel: tiles not yet dispatched are dropped; the request finishes with
 * TM_ERR_CANCELLED once its dispatched tiles are done. */
int tm_server_cancel(tm_server* s, uint64_t ticket);
/* Stop (1) or resume (0) dispatching new tiles (tiles in flight complete). */
int tm_server_pause(tm_server* s, int32_t paused);
/* Finish dispatched tiles, drop the rest, stop the worker and free the staging. */
void tm_server_destroy(tm_server* s);

#ifdef __cplusplus
}
#endif
#endif /* TMGB_H */
