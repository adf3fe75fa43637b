/*
 * FP64 CPU oracle for the template-matching indexing path -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the package's smoke check and the benchmark's CPU-baseline leg may
 * load this library.  It shares no code with the CUDA path: plain loops, double
 * precision, written from the paper's definitions.
 *
 *   oracle_polar      -- gamma / constant subtraction of the raw frame (Section 2.2:
 *                        pixel values raised to a power < 1, then a constant
 *                        subtracted), then bilinear resampling onto the polar grid
 *                        about the direct beam (Section 2.2, Fig. 2 (a)-(c)):
 *                        r_j = j dr, theta_k = 2 pi k / n_theta.
 *   oracle_scores     -- correlation index Q of Eq. 1 for every template at every
 *                        azimuthal shift with wraparound (Section 2.2, Fig. 2 (e)),
 *                        keeping per template the maximum Q and the lowest shift
 *                        attaining it (within a relative window of 1e-12).
 *   oracle_scores_full-- the same, returning Q for every (template, shift).
 *
 * Readings (the paper is silent on these): bilinear interpolation with zero outside
 * the frame; gamma is applied to the raw frame before resampling; the image norm runs
 * over the whole polar image; a template or image with zero norm scores Q = 0.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_TIE_REL 1e-12
#define ORACLE_PI 3.14159265358979323846

static double pixel_value(const void* frame, int dtype, int H, int W, int x, int y,
                          double gamma, double subtract) {
    if (x < 0 || y < 0 || x >= W || y >= H) return 0.0;   /* zero outside the frame */
    double v;
    if (dtype == 0) v = (double)((const uint16_t*)frame)[(int64_t)y * W + x];
    else            v = (double)((const float*)frame)[(int64_t)y * W + x];
    if (v < 0.0) v = 0.0;
    double g = (gamma == 0.5) ? sqrt(v) : (gamma == 1.0 ? v : pow(v, gamma));
    return g - subtract;
}

/* frames: [n][H][W] (dtype 0 = uint16, 1 = float32); centres: [n][2] (cx, cy) or NULL
 * for (cx0, cy0); polar_out: [n][n_r][n_theta]. */
void oracle_polar(const void* frames, int dtype, int64_t n, int H, int W,
                  const double* centres, double cx0, double cy0,
                  double gamma, double subtract, int n_r, int n_theta, double dr,
                  double* polar_out) {
    const size_t esz = dtype == 0 ? 2 : 4;
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t p = 0; p < n; ++p) {
        const char* frame = (const char*)frames + (size_t)p * H * W * esz;
        double cx = centres ? centres[2 * p] : cx0;
        double cy = centres ? centres[2 * p + 1] : cy0;
        double* out = polar_out + (size_t)p * n_r * n_theta;
        for (int j = 0; j < n_r; ++j) {
            double r = j * dr;
            for (int k = 0; k < n_theta; ++k) {
                double th = 2.0 * ORACLE_PI * k / n_theta;
                double x = cx + r * cos(th);     /* column */
                double y = cy + r * sin(th);     /* row */
                double xf = floor(x), yf = floor(y);
                double fx = x - xf, fy = y - yf;
                int x0 = (int)xf, y0 = (int)yf;
                double v00 = pixel_value(frame, dtype, H, W, x0, y0, gamma, subtract);
                double v10 = pixel_value(frame, dtype, H, W, x0 + 1, y0, gamma, subtract);
                double v01 = pixel_value(frame, dtype, H, W, x0, y0 + 1, gamma, subtract);
                double v11 = pixel_value(frame, dtype, H, W, x0 + 1, y0 + 1, gamma, subtract);
                out[(size_t)j * n_theta + k] =
                    (1.0 - fx) * (1.0 - fy) * v00 + fx * (1.0 - fy) * v10 +
                    (1.0 - fx) * fy * v01 + fx * fy * v11;
            }
        }
    }
}

/* Q(k, s) for one pattern and one template into q[0..n_theta). */
static void template_q(const double* P, double normP, int n_theta,
                       const int64_t* off, const int32_t* ri, const int32_t* ti,
                       const double* I, const double* tnorm, int64_t k, double* q) {
    double denom = normP * tnorm[k];
    for (int s = 0; s < n_theta; ++s) {
        double acc = 0.0;
        for (int64_t i = off[k]; i < off[k + 1]; ++i) {
            int col = (ti[i] + s) % n_theta;                 /* wraparound along phi */
            acc += I[i] * P[(size_t)ri[i] * n_theta + col];
        }
        q[s] = denom > 0.0 ? acc / denom : 0.0;
    }
}

static double image_norm(const double* P, size_t m) {
    double s = 0.0;
    for (size_t i = 0; i < m; ++i) s += P[i] * P[i];
    return sqrt(s);
}

/* polar: [n][n_r][n_theta]; templates in CSR (merged, rounded spots: ri in [0, n_r),
 * ti in [0, n_theta)); tnorm[k] = sqrt(sum I^2); active: [n][K] bytes or NULL (all).
 * Outputs q_best[n][K], s_best[n][K]; inactive entries get -inf and -1. */
void oracle_scores(const double* polar, int64_t n, int n_r, int n_theta,
                   const int64_t* off, const int32_t* ri, const int32_t* ti, const double* I,
                   const double* tnorm, int64_t K, const uint8_t* active,
                   double* q_best, int32_t* s_best) {
    #pragma omp parallel
    {
        double* q = (double*)malloc(sizeof(double) * n_theta);
        #pragma omp for schedule(dynamic, 1)
        for (int64_t p = 0; p < n; ++p) {
            const double* P = polar + (size_t)p * n_r * n_theta;
            double normP = image_norm(P, (size_t)n_r * n_theta);
            for (int64_t k = 0; k < K; ++k) {
                size_t o = (size_t)p * K + k;
                if (active && !active[o]) { q_best[o] = -INFINITY; s_best[o] = -1; continue; }
                template_q(P, normP, n_theta, off, ri, ti, I, tnorm, k, q);
                double best = q[0];
                for (int s = 1; s < n_theta; ++s) if (q[s] > best) best = q[s];
                double thr = best - ORACLE_TIE_REL * fabs(best);
                int sb = 0;
                while (q[sb] < thr) ++sb;                      /* lowest shift attaining */
                q_best[o] = best;
                s_best[o] = sb;
            }
        }
        free(q);
    }
}

/* Q for every (pattern, template, shift): q_out[n][K][n_theta]. Small cases only. */
void oracle_scores_full(const double* polar, int64_t n, int n_r, int n_theta,
                        const int64_t* off, const int32_t* ri, const int32_t* ti, const double* I,
                        const double* tnorm, int64_t K, double* q_out) {
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t p = 0; p < n; ++p) {
        const double* P = polar + (size_t)p * n_r * n_theta;
        double normP = image_norm(P, (size_t)n_r * n_theta);
        for (int64_t k = 0; k < K; ++k)
            template_q(P, normP, n_theta, off, ri, ti, I, tnorm, k,
                       q_out + ((size_t)p * K + k) * n_theta);
    }
}

int oracle_num_threads(void) {
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
