// Internal declarations shared by the host API and the kernels of libtmgb.so.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/tmgb.h"

#define TM_MAX_LIBS 8          // libraries indexed in one call
#define TM_MAX_TOPN 128        // largest N of the fused top-N

namespace tmgb {

// Message for tm_last_error() on the calling thread.
void set_last_error(const char* msg);


// ------------------------------------------------------------------ device library views
// Sparse templates in CSR.  The sparse kernel keeps only the library's distinct spot radii
// (radii[0..n_rad)) as rows of its shared-memory polar image, in one of three layouts
// (TM_LAYOUT_*, chosen per call by shared-memory size).
//   spot[i]  = {t | rho << 11 | w << 24, intensity bits}: t the angle column, rho the spot's row
//              in radii[], w = ceil((n_theta - t) / 32) the first 32-wide shift block whose
//              columns wrap past n_theta (wrapped layout);
//   spot2[i] = {off_dual | off_wf << 16, intensity bits}: the spot's float offset in the dual
//              layout ((t & 1 ? n_rad + rho : rho) * pitch_dual + (t & ~1)) and in the wrap-free
//              layout (rho * pitch_wf + t), each 0 when it does not fit 16 bits (the layout is
//              then never chosen);
//   meta[k]  = {first spot, spots | shifts << 16, norm bits, bits of sum_i |I_i| rounded up}.
enum { TM_LAYOUT_DUAL = 0, TM_LAYOUT_WF = 1, TM_LAYOUT_WRAP = 2 };

struct SparseLib {
    const int32_t* off;        // [K + 1]
    const int2* spot;          // [n_spots]
    const int2* spot2;         // [n_spots]
    const int4* meta;          // [K]
    const float* norm;         // [K]  sqrt(sum I^2)
    const int32_t* nshift;     // [K]  shifts to evaluate = n_theta / order_k
    const int32_t* radii;      // [n_rad]  distinct spot radii (polar rows), ascending
    int32_t n_rad;
    int32_t K;
    int32_t K0;
    int32_t mirror;
    int32_t words;             // ceil(K / 32)
    int32_t nonneg;            // every intensity >= 0 (the sparse kernel may then prune by bounds)
    const int2* bspot;         // [n_spots] {intensity, window-table entries} or null (no window bounds)
    // The same templates ordered by spot count, largest first (so the 32 templates of a word have
    // nearly equal counts), for the unmasked top-N pass that bounds every template; present with
    // bspot:
    const int4* smeta;         // [words * 32] meta of the template at each sorted position
    const int32_t* sperm;      // [words * 32] its library index
    const int32_t* ellw;       // [words] first entry of each sorted word in ell
    const int2* ell;           // bspot entries of sorted word w: spot i of lane l at ellw[w] + 32 i + l
};

// Windows of the shift range for the sparse kernel's pruning bound: three windows of
// ww = ceil(Nθ / 3) shifts; a spot at column t visits, over window h, the columns
// [t + h ww, t + h ww + ww) of its row, which the ncov 32-column chunks from chunk
// (t + h ww) / 32 on cover.  The kernel keeps, per library row, the maxima over the windows
// starting in each of the nchw chunks; one lane holds one chunk, so nchw + ncov - 1 <= 32.
__host__ __device__ inline int prune_ww(int n_theta) { return (n_theta + 2) / 3; }
__host__ __device__ inline int prune_ncov(int n_theta) { return (prune_ww(n_theta) + 31) / 32 + 1; }
__host__ __device__ inline int prune_nchw(int n_theta) { return ((n_theta - 1 + 2 * prune_ww(n_theta)) >> 5) + 1; }

struct RadialLib {
    const float* radc;         // [K][n_pad]  azimuthal sums of the templates at the library's radii
                               //             (n_pad = n_rad rounded up to 4, zero-padded)
    const float* rnorm;        // [K]         |R_T,k|
    const int32_t* radii;      // [n_rad]     ascending polar rows (every other row of R_T is 0)
    int32_t n_rad;
    int32_t K;
};

// ------------------------------------------------------------------ launch configuration
// Raises fn's dynamic shared-memory limit to smem (once per kernel, device and size) and
// returns its resident blocks per SM for `threads` threads (per_sm may be null).  Cached, so
// repeated launches make no driver queries.
cudaError_t kernel_occupancy(const void* fn, int threads, size_t smem, int* per_sm);
// Number of SMs of the current device (cached), or the calling thread's cap when one is set.
int device_sms();
// Caps the persistent grids of this thread's later calls at `cap` SMs (0 = no cap), so that work
// on other streams finds SMs free (the serving loop leaves SMs to scan lines this way).
void set_sm_cap(int cap);

// ------------------------------------------------------------------ launchers
// Host: the ray steps of the polar grid, (round(dr cos theta_k 2^32), round(dr sin theta_k
// 2^32)) for k < n_theta, in double precision: row j of ray k lies at (cx, cy) + j (step).
void build_polar_rays(int n_theta, double dr, longlong2* rays);

// rays [n_theta] from build_polar_rays; (cx, cy) the centre (|c| < 2^30, n_r dr < 2^30).
// keep_row [n_r] (nullable): rows whose polar values are stored; the norm and the row
// sums always cover every row.  centres [n] (nullable): per-pattern beam centres, used
// instead of (cx, cy).  err (nullable): device error word; when given, frames whose rows are
// whole 16-byte units (and no pixel mask) are staged by bulk copies, whose bounded wait sets
// bit 1 of err if it runs out.
cudaError_t launch_polar(const void* frames, int dtype, int64_t n, int H, int W, const longlong2* rays, double cx,
                         double cy, double gamma, double subtract, int n_r, int n_theta, float* polar, float* pnorm,
                         float* radial, cudaStream_t st, const uint8_t* keep_row = nullptr,
                         const float2* centres = nullptr, const uint8_t* pixel_mask = nullptr,
                         double threshold = 0.0, unsigned* err = nullptr);

// Sub-step in-plane angle of the top-N hits (parabola through Q at s - 1, s, s + 1).
struct RefineLib {
    const int32_t* off;        // [K + 1]
    const int32_t* rt;         // [n_spots]  r | t << 16
    const int2* spot;          // [n_spots]  .y = intensity bits
    const float* norm;         // [K]
};
struct RefineCall {
    const float* polar;        // [n][n_r][n_theta]  (rows of the libraries' radii)
    const float* pnorm;        // [n]
    int64_t n;
    int n_r, n_theta, top_n;
    int n_libs;
    RefineLib lib[TM_MAX_LIBS];
    tm_hit* hits;              // [n_libs][hits_lib_stride]: angle_deg rewritten in place
    int64_t hits_lib_stride;
};
cudaError_t launch_refine(const RefineCall& c, int num_sms, cudaStream_t st);

// Direct-beam centres: per pattern the centre of mass within `radius` of the estimate,
// `iterations` times from (cx0, cy0), FP64 in a fixed order; out [n] (cx, cy) floats.
// Separable Gaussian passes (k_preprocess.cu): rows of `rows` images rows x W (u16 / f32 /
// float input) filtered by w1 (and w2, nullable) into out1 (out2); columns of n frames H x W
// filtered by w1 (dog: and in2 by w2, out = max(a - b, 0)).  Weights [2 r + 1] on the device.
size_t gauss_cols_smem(int H, int r1, int r2, int dog);
int gauss_padded_taps(int r);               // weights per filter: 2 r + 1 rounded up, zero-padded
cudaError_t launch_gauss_rows(const void* in, int dtype, int64_t rows, int W, const float* w1, int r1, const float* w2,
                              int r2, float* out1, float* out2, cudaStream_t st);
cudaError_t launch_gauss_cols(const float* in1, const float* in2, int64_t n, int H, int W, const float* w1, int r1,
                              const float* w2, int r2, int dog, float* out, cudaStream_t st);

// Orientation maps and Eq. 2 (k_orient.cu).
cudaError_t launch_orientation_vectors(const tm_hit* hits, int64_t n, int stride, const double* rot, int64_t K0,
                                       double e0, double e1, double e2, double* v, cudaStream_t st);
cudaError_t launch_angular_deviation(const double* va, const double* vb, int64_t n, double* deg, cudaStream_t st);

// Template simulation (k_kinematic.cu): counts [D], spots [D][max_spots][3].
int kinematic_cand_max();
cudaError_t launch_kinematic(const double* g, const double* f2, const double* gnorm, int64_t G, const double* rot,
                             int64_t D, double wavelength, double s_max, int max_spots, int32_t* counts, double* spots,
                             cudaStream_t st);

cudaError_t launch_find_centres(const void* frames, int dtype, int64_t n, int H, int W, double cx0, double cy0,
                                double radius, int iterations, float2* out, cudaStream_t st);

// Two-stage indexing (Section 4.3): per-pixel FP64 sums over frames (accumulate: add onto
// out), and the mask of kept pixels from the sums (scratch: H * W bytes).
size_t frame_sum_scratch_bytes(int dtype, int64_t n, int H, int W, int num_sms);
cudaError_t launch_frame_sum(const void* frames, int dtype, int64_t n, int H, int W, int accumulate, double* out,
                             double* scratch, int num_sms, cudaStream_t st);
cudaError_t launch_matrix_mask(const double* sum, int H, int W, double thr_n, int n_open, int n_dilate,
                               uint8_t* mask, uint8_t* scratch, int num_sms, cudaStream_t st);

cudaError_t launch_radial_norm(const float* radial, int64_t n, int n_r, float* out,
                               cudaStream_t st);

// Scores and selection in one pass: mask [n][ceil(K/32)] of the keep best-correlated
// templates per pattern; score [n][K] (nullable) receives the scores.
cudaError_t launch_prefilter(const float* radial, const float* radial_norm, int64_t n, int n_r,
                             const RadialLib& lib, int keep, uint32_t* mask, float* score,
                             cudaStream_t st);

cudaError_t launch_prefilter_select(const float* score, int64_t n, int K, int keep,
                                    uint32_t* mask, cudaStream_t st);

struct SparseCall {
    const float* polar;        // [n][n_r][n_theta]
    const float* pnorm;        // [n]
    int64_t n;
    int n_r, n_theta;
    int pitch;                          // set by launch_sparse (layout row pitch)
    int max_rad;                        // largest n_rad of the libraries (shared-memory rows)
    int* pattern_counter;               // device int, zeroed by the launcher
    int n_libs;
    SparseLib lib[TM_MAX_LIBS];
    const uint32_t* mask[TM_MAX_LIBS];  // [n][words] or null
    float* q_out[TM_MAX_LIBS];          // [n][K] or null (stage output)
    int32_t* s_out[TM_MAX_LIBS];        // [n][K] or null
    tm_hit* hits;                       // [n_libs][hits_lib_stride] or null
    int64_t hits_lib_stride;            // elements between libraries (>= n * top_n)
    int top_n;
    int threads;                        // block size: 128, 256 or 512 (0 = 256)
    unsigned long long* work;           // nullable: += multiply-adds executed (per warp, at exit)
    // pruned top-N: per-CTA words marking the templates scored first (seeds),
    // [seed_ctas][kSparseTile][seed_words]; null (or a grid larger than seed_ctas) disables seeding
    uint32_t* seed_bits;
    __half* seed_qub;                   // [seed_ctas][kSparseTile][32 seed_words] bounds of the seeding pass
    int32_t* seed_cand;                 // [seed_ctas][32 seed_words] templates left after the seeds
    int seed_words;                     // >= the libraries' largest word count
    int seed_ctas;
    int seeds_per_warp;                 // 1..16 (0 = 8)
    int tile;                           // patterns bounded together by the unmasked top-N pass:
                                        // 1 (0) or up to kSparseTile
    int bulk;                           // stage the polar rows with bulk copies (n_theta a multiple
                                        // of 4, polar 16-byte aligned; not for the dual layout)
    unsigned* error;                    // device error word: bit 4 when a staging wait ran out
    int test_stall;                     // failure-path tests: the row staging expects 16 bytes more
                                        // than its copies bring, so its wait runs out
};
// Largest grid of the sparse kernel on a device with num_sms SMs (the seed words are per CTA),
// and the most patterns a CTA bounds together (seed words and stored bounds per pattern).
constexpr int kSparseTile = 4;
int sparse_max_ctas(int num_sms);

// Shared-memory bytes the sparse kernel needs (0 when unsupported), the layout it uses
// (wrap-free rows when they fit comfortably) and its row pitch.
size_t sparse_smem_bytes(int max_rad, int n_theta, int top_n, int* layout = nullptr, int* pitch = nullptr,
                         int tile = 1);
int sparse_pitch(int n_theta, int layout);
int sparse_rows(int n_rad, int layout);
cudaError_t launch_sparse(const SparseCall& c, int num_sms, cudaStream_t st);

// ------------------------------------------------------------------ BF16 tensor-core path
// Frequency slots of the angular spectra: slot j < 96 holds m = 2 j, slot j >= 96 holds
// m = 2 (j - 96) + 1 (even frequencies first, for the radix-2 split of stage B); slots whose
// frequency exceeds n_theta / 2 are zero.
//   T^ (per library, built once):  [192][2 R][K_pad] BF16, rows (Re, Im) of T^_k[r_a, m] / |T_k|
//   DFT of the polar rows:          [192][2][n][n_r]  FP32, (Re, Im) of P^[r, m] (a TF32 GEMM)
//   P^ (per call, per library):    [192][n][2][2 R]  BF16, (Re, Im) and (Im, -Re) of P^[r_a, m] / |P|
//   G  (stage A: G_j = T^_j P^_j): [192][n][2][K_pad] BF16, (Re, Im) of G[k, m]
// with R the library's distinct radii rounded up to 8 and K_pad its templates rounded up to 64.
struct DenseCall {
    int64_t n;                 // patterns of the G batch
    int64_t p0;                // first pattern of the batch in the call's rows (pre, mask)
    int n_theta;
    int K;                     // templates of the library
    const void* basis;         // [192][384] bf16, K-major (dense_basis_rows x dense_basis_cols)
    const uint32_t* mask;      // [rows][words] templates to score (pre-filter) or null (all)
    int words;
    float* pre;                // [rows][K] out: pre-score, -NaN where masked out
    unsigned* error;           // device word: bit 0 = a bounded wait timed out
    int stall;                 // test hook: the MMA issuer issues nothing
};

bool dense_supported(int n_theta);
int dense_basis_rows();
int dense_basis_cols();
int dense_slots();
size_t dense_smem_bytes();
// tmap: the CUtensorMap of G for this batch (4-D: k, c, p, j; box 64 x 2 x 1 x 32; 128-byte swizzle).
cudaError_t launch_dense(const void* tmap, const DenseCall& c, int num_sms, cudaStream_t st);
// dftc [192][2][nb][n_r] FP32 (the DFT GEMM's output for every polar row) -> P^ of one library
// [192][nb][2][2 R] BF16, divided by |P|.
cudaError_t launch_pack(const float* dftc, const float* pnorm, int64_t nb, int n_r, const int32_t* radii, int n_rad,
                        int R, void* out, int num_sms, cudaStream_t st);
cudaError_t launch_spectra(const int32_t* off, const int32_t* rt, const int2* spot, const float* norm,
                           const int32_t* rowmap, int K, int K_pad, int R, int n_theta, const float2* twiddle,
                           void* out, cudaStream_t st);

// tm_index_patterns with the hits of library i written at out_dev + i * lib_stride (0: n * top_n).
int index_patterns_ex(tm_ctx* ctx, const tm_index_params* params, const void* frames_dev, int32_t dtype, int64_t n,
                      int32_t H, int32_t W, const float* centres_dev, const int32_t* lib_ids, int32_t n_libs,
                      tm_hit* out_dev, int64_t lib_stride, tm_stats* stats, void* stream);

// Validation of tm_index_params shared by every whole-path entry point (finite gamma,
// subtraction and centre; pre-filter fraction; top_n; 16-byte aligned pixel mask; threshold).
// Returns a TM_* status and sets the thread's last error.
int check_index_params(const tm_index_params* p);

// Read-only view of a loaded library for entry points defined outside the host API file:
// device, SM count, the sparse view and the library's polar grid.  Returns a TM_* status.
int library_view(tm_ctx* ctx, int lib_id, int* device, int* num_sms, SparseLib* view, int* n_r,
                 int* n_theta, double* dr);

}  // namespace tmgb
