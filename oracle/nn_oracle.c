/*
 * nn_oracle.c -- FP64 CPU oracle for exact brute-force nearest-neighbour search.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite and the CPU-baseline leg of the
 * benchmark may load this library.  The GPU library never links, includes or
 * calls it, and it shares no code with the GPU path.
 *
 * What it computes (the plain definition, written out as loops): the paper's
 * natural-scene-statistics case study (Sec. 6.4, Table "NN-speedup") finds, for
 * every target patch (8x8 pixels, a 64-dimensional vector), its nearest
 * neighbour in Euclidean distance among a set of neighbour patches, by computing
 * the distance to every neighbour and taking the smallest (exact, exhaustive).
 * For target i:
 *
 *     d(i, j) = sum_{k<dim} (t[i][k] - n[j][k])^2
 *     idx[i]  = the smallest j with d(i, j) = min_j d(i, j)
 *     dist[i] = d(i, idx[i])
 *     dist2[i]= min over j != idx[i] of d(i, j)   (the runner-up; +inf if none)
 *
 * Layouts: t [nt][dim], n [nn][dim], row-major.  Arithmetic: FP64 inputs (FP32
 * data widened exactly by the caller), each d(i, j) summed sequentially over k,
 * the scan over j in increasing order with a strict '<' (so ties keep the lowest
 * index).  Parallelised only over independent targets.
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>
#ifdef _OPENMP
#include <omp.h>
#endif

extern int oracle_max_threads(void);

int oracle_nn(const double* t, int64_t nt, const double* n, int64_t nn, int64_t dim, int64_t* idx,
              double* dist, double* dist2) {
    if (!t || !n || !idx || !dist || !dist2 || nt < 0 || nn <= 0 || dim <= 0) return 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(oracle_max_threads())
    for (int64_t i = 0; i < nt; ++i) {
        const double* ti = t + i * dim;
        double best = INFINITY, second = INFINITY;
        int64_t bi = -1;
        for (int64_t j = 0; j < nn; ++j) {
            const double* nj = n + j * dim;
            double d = 0.0;
            for (int64_t k = 0; k < dim; ++k) {
                const double e = ti[k] - nj[k];
                d += e * e;
            }
            if (d < best) {
                second = best;
                best = d;
                bi = j;
            } else if (d < second) {
                second = d;
            }
        }
        idx[i] = bi;
        dist[i] = best;
        dist2[i] = second;
    }
    return 0;
}
