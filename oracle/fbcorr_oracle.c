/*
 * fbcorr_oracle.c -- FP64 CPU oracle for multi-filter 3D filter-bank correlation.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  The GPU library
 * never links, includes or calls it, and it shares no code with the GPU path.
 *
 * What it computes (the plain definitions, written out as nested loops):
 *   The paper's vision case study (Sec. 6.2, "Computational Visual
 *   Neuroscience") names 3D filter-bank convolution -- a bank of filters
 *   applied across every channel of the previous layer -- as the key
 *   bottleneck of its models, and Table "Performance of RTCG auto-tuning on
 *   3D filter-bank convolutions" gives the shapes as an H x W x D input and an
 *   N x fh x fw x D bank.  The paper prints no formula; the reading used here
 *   is a 'valid' cross-correlation with no filter flip:
 *
 *     y[p][q][n] = sum_{i<fh} sum_{j<fw} sum_{d<D} x[p+i][q+j][d] * w[n][i][j][d]
 *
 *   for 0 <= p < H' = H-fh+1, 0 <= q < W' = W-fw+1, 0 <= n < N, optionally
 *   followed by a clamp y <- min(max(y, lo), hi) (a static non-linearity,
 *   Sec. 6.2).  The two gradients of L = <y, g> are the adjoints of that map:
 *
 *     dx[p][q][d]    = sum_n sum_i sum_j g~[p-i][q-j][n] * w[n][i][j][d]
 *                      (terms with p-i or q-j outside the output are zero)
 *     dw[n][i][j][d] = sum_p sum_q g~[p][q][n] * x[p+i][q+j][d]
 *
 *   where g~ = g, or g masked to lo < y < hi when the clamp is applied.
 *
 * Layouts: every array is row-major with the last index fastest:
 *   x [H][W][D], w [N][fh][fw][D], y and g [H'][W'][N].
 * Arithmetic: all inputs are FP64 (FP32 data is widened exactly by the caller);
 * every sum runs sequentially in FP64 in the loop order written below.  The
 * loops are parallelised only over independent output elements, so results do
 * not depend on the thread count.
 */
#include <stdint.h>
#include <stddef.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_EPI_NONE 0
#define ORACLE_EPI_CLAMP 1

static int g_threads = 0; /* 0: OpenMP default */

void oracle_set_threads(int n) { g_threads = n; }

int oracle_max_threads(void) {
#ifdef _OPENMP
    return g_threads > 0 ? g_threads : omp_get_max_threads();
#else
    return 1;
#endif
}

static int nthreads(void) { return oracle_max_threads(); }

static double clamp_d(double v, double lo, double hi) {
    if (v < lo) v = lo;
    if (v > hi) v = hi;
    return v;
}

/* One output element of the forward correlation, before any epilogue. */
static double corr_at(const double* x, int64_t W, int64_t D,
                      const double* w, int64_t fh, int64_t fw,
                      int64_t p, int64_t q, int64_t n) {
    double s = 0.0;
    for (int64_t i = 0; i < fh; ++i)
        for (int64_t j = 0; j < fw; ++j)
            for (int64_t d = 0; d < D; ++d)
                s += x[((p + i) * W + (q + j)) * D + d] *
                     w[((n * fh + i) * fw + j) * D + d];
    return s;
}

static int shape_ok(int64_t H, int64_t W, int64_t D, int64_t N, int64_t fh, int64_t fw) {
    return H > 0 && W > 0 && D > 0 && N > 0 && fh > 0 && fw > 0 && fh <= H && fw <= W;
}

/* Forward: y[H'][W'][N] = corr(x, w), then the optional clamp (applied to the
 * FP64 sum).  Returns 0 on success, -1 on a bad shape. */
int oracle_fbcorr_fwd(const double* x, int64_t H, int64_t W, int64_t D,
                      const double* w, int64_t N, int64_t fh, int64_t fw,
                      int epi_kind, double lo, double hi, double* y) {
    if (!shape_ok(H, W, D, N, fh, fw)) return -1;
    const int64_t Ho = H - fh + 1, Wo = W - fw + 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads())
    for (int64_t p = 0; p < Ho; ++p)
        for (int64_t q = 0; q < Wo; ++q)
            for (int64_t n = 0; n < N; ++n) {
                double s = corr_at(x, W, D, w, fh, fw, p, q, n);
                if (epi_kind == ORACLE_EPI_CLAMP) s = clamp_d(s, lo, hi);
                y[(p * Wo + q) * N + n] = s;
            }
    return 0;
}

/* Forward at selected output elements only: idx holds npts triples (p, q, n). */
int oracle_fbcorr_fwd_points(const double* x, int64_t H, int64_t W, int64_t D,
                             const double* w, int64_t N, int64_t fh, int64_t fw,
                             int epi_kind, double lo, double hi,
                             int64_t npts, const int64_t* idx, double* out) {
    if (!shape_ok(H, W, D, N, fh, fw)) return -1;
    const int64_t Ho = H - fh + 1, Wo = W - fw + 1;
    for (int64_t k = 0; k < npts; ++k) {
        const int64_t p = idx[3 * k], q = idx[3 * k + 1], n = idx[3 * k + 2];
        if (p < 0 || p >= Ho || q < 0 || q >= Wo || n < 0 || n >= N) return -2;
    }
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads())
    for (int64_t k = 0; k < npts; ++k) {
        const int64_t p = idx[3 * k], q = idx[3 * k + 1], n = idx[3 * k + 2];
        double s = corr_at(x, W, D, w, fh, fw, p, q, n);
        if (epi_kind == ORACLE_EPI_CLAMP) s = clamp_d(s, lo, hi);
        out[k] = s;
    }
    return 0;
}

/* The upstream gradient after the clamp's derivative: g where lo < y < hi
 * strictly, 0 elsewhere; g unchanged without an epilogue. */
static double g_eff(const double* g, const double* y, int64_t k,
                    int epi_kind, double lo, double hi) {
    if (epi_kind == ORACLE_EPI_CLAMP) {
        const double v = y[k];
        if (!(v > lo && v < hi)) return 0.0;
    }
    return g[k];
}

/* dL/dx: dx[H][W][D] by the gather formula.  y is required (the clamped
 * forward output) when epi_kind is CLAMP, ignored otherwise. */
int oracle_fbcorr_bwd_input(const double* g, const double* y,
                            int64_t H, int64_t W, int64_t D,
                            const double* w, int64_t N, int64_t fh, int64_t fw,
                            int epi_kind, double lo, double hi, double* dx) {
    if (!shape_ok(H, W, D, N, fh, fw)) return -1;
    if (epi_kind == ORACLE_EPI_CLAMP && !y) return -3;
    const int64_t Ho = H - fh + 1, Wo = W - fw + 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads())
    for (int64_t p = 0; p < H; ++p)
        for (int64_t q = 0; q < W; ++q)
            for (int64_t d = 0; d < D; ++d) {
                double s = 0.0;
                for (int64_t n = 0; n < N; ++n)
                    for (int64_t i = 0; i < fh; ++i) {
                        const int64_t po = p - i;
                        if (po < 0 || po >= Ho) continue;
                        for (int64_t j = 0; j < fw; ++j) {
                            const int64_t qo = q - j;
                            if (qo < 0 || qo >= Wo) continue;
                            s += g_eff(g, y, (po * Wo + qo) * N + n, epi_kind, lo, hi) *
                                 w[((n * fh + i) * fw + j) * D + d];
                        }
                    }
                dx[(p * W + q) * D + d] = s;
            }
    return 0;
}

/* dL/dw: dw[N][fh][fw][D], each a sum over the whole output plane. */
int oracle_fbcorr_bwd_filt(const double* x, const double* g, const double* y,
                           int64_t H, int64_t W, int64_t D,
                           int64_t N, int64_t fh, int64_t fw,
                           int epi_kind, double lo, double hi, double* dw) {
    if (!shape_ok(H, W, D, N, fh, fw)) return -1;
    if (epi_kind == ORACLE_EPI_CLAMP && !y) return -3;
    const int64_t Ho = H - fh + 1, Wo = W - fw + 1;
    const int64_t total = N * fh * fw * D;
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads())
    for (int64_t e = 0; e < total; ++e) {
        const int64_t d = e % D;
        const int64_t j = (e / D) % fw;
        const int64_t i = (e / (D * fw)) % fh;
        const int64_t n = e / (D * fw * fh);
        double s = 0.0;
        for (int64_t p = 0; p < Ho; ++p)
            for (int64_t q = 0; q < Wo; ++q)
                s += g_eff(g, y, (p * Wo + q) * N + n, epi_kind, lo, hi) *
                     x[((p + i) * W + (q + j)) * D + d];
        dw[e] = s;
    }
    return 0;
}

/* dL/dx at selected input elements (p, q, d) only. */
int oracle_fbcorr_bwd_input_points(const double* g, const double* y,
                                   int64_t H, int64_t W, int64_t D,
                                   const double* w, int64_t N, int64_t fh, int64_t fw,
                                   int epi_kind, double lo, double hi,
                                   int64_t npts, const int64_t* idx, double* out) {
    if (!shape_ok(H, W, D, N, fh, fw)) return -1;
    if (epi_kind == ORACLE_EPI_CLAMP && !y) return -3;
    const int64_t Ho = H - fh + 1, Wo = W - fw + 1;
    for (int64_t k = 0; k < npts; ++k) {
        const int64_t p = idx[3 * k], q = idx[3 * k + 1], d = idx[3 * k + 2];
        if (p < 0 || p >= H || q < 0 || q >= W || d < 0 || d >= D) return -2;
    }
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads())
    for (int64_t k = 0; k < npts; ++k) {
        const int64_t p = idx[3 * k], q = idx[3 * k + 1], d = idx[3 * k + 2];
        double s = 0.0;
        for (int64_t n = 0; n < N; ++n)
            for (int64_t i = 0; i < fh; ++i) {
                const int64_t po = p - i;
                if (po < 0 || po >= Ho) continue;
                for (int64_t j = 0; j < fw; ++j) {
                    const int64_t qo = q - j;
                    if (qo < 0 || qo >= Wo) continue;
                    s += g_eff(g, y, (po * Wo + qo) * N + n, epi_kind, lo, hi) *
                         w[((n * fh + i) * fw + j) * D + d];
                }
            }
        out[k] = s;
    }
    return 0;
}
