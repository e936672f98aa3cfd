/*
 * Plain CPU oracle for all-pairs binary mutual information (FP64).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file: only the tests, the smoke check and the benchmark's CPU
 * baseline leg do.  It shares no code with the CUDA library.
 *
 * What it computes (arXiv 2411.19702):
 *   For two binary variables X and Y observed on m samples,
 *     MI(X;Y) = sum_{x,y in {0,1}} p(x,y) * log2( p(x,y) / (p(x) p(y)) )      (Eq. 1, Sec. 1)
 *   written out as the four cells 11, 10, 01, 00                               (Eq. 2, Sec. 2 step 5)
 *   with p(x,y) = n_xy / m (Sec. 2 step 2: joint probability = count / #samples)
 *   and marginals p(x) = sum_y p(x,y), p(y) = sum_x p(x,y).
 *
 * It deliberately does NOT use the paper's Gram-matrix shortcut (Sec. 3,
 * Eq. 6-7): every cell count is obtained by walking all m samples of the pair,
 * which is the plain definition the shortcut must reproduce exactly.
 *
 * Readings of the paper taken here:
 *   - No epsilon (Sec. 2 step 5 mentions one without a value): a cell with
 *     n_xy = 0 contributes 0 (the limit 0*log 0 = 0).  When n_xy > 0 both of its
 *     marginals are > 0, so every logarithm taken is finite.
 *   - Logarithm base 2 (Eq. 1): results are in bits.
 *   - A sample value is "1" when its byte is non-zero (the data are binary).
 *   - The sum is taken in the fixed order 11, 10, 01, 00 (Eq. 2) and the value
 *     is not clamped: a rounding residue of either sign is reported as is.
 *
 * Layout convention of the inputs: X is m x n, row-major, rows = samples,
 * columns = variables (Sec. 2 step 1, with m = samples and n = variables).
 */
#include <stdint.h>
#include <stddef.h>
#include <math.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* Copy the columns of a row-major m x n byte matrix into rows of an n x m
 * matrix (a pure data-layout step: XT[j*m + r] = X[r*ldx + j]).  It lets the
 * counting loop read each variable contiguously. */
void oracle_transpose_u8(const uint8_t* X, int64_t m, int64_t n, int64_t ldx,
                         uint8_t* XT, int nthreads) {
    const int64_t B = 64;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic) if (nthreads != 1)
#endif
    for (int64_t jb = 0; jb < n; jb += B) {
        for (int64_t rb = 0; rb < m; rb += B) {
            int64_t je = jb + B < n ? jb + B : n;
            int64_t re = rb + B < m ? rb + B : m;
            for (int64_t j = jb; j < je; ++j)
                for (int64_t r = rb; r < re; ++r)
                    XT[j * m + r] = X[r * ldx + j];
        }
    }
}

/* Count the four cells of the 2x2 contingency table of two variables, each
 * given as m contiguous sample bytes.  cnt[0..3] = n11, n10, n01, n00 where
 * n_xy = #{ r : x_r = x, y_r = y } (Sec. 2 step 2: the counts behind P11,
 * P10, P01, P00). */
void oracle_cell_counts(const uint8_t* x, const uint8_t* y, int64_t m, int64_t cnt[4]) {
    int64_t c[2][2] = {{0, 0}, {0, 0}};
    for (int64_t r = 0; r < m; ++r) {
        int a = x[r] != 0;
        int b = y[r] != 0;
        c[a][b] += 1;
    }
    cnt[0] = c[1][1];
    cnt[1] = c[1][0];
    cnt[2] = c[0][1];
    cnt[3] = c[0][0];
}

/* Mutual information in bits from the four cell counts (Eq. 1 / Eq. 2).
 * Marginals are the row and column sums of the contingency table (Sec. 2
 * step 3: the marginal probability of a variable). */
double oracle_mi_from_counts(int64_t n11, int64_t n10, int64_t n01, int64_t n00) {
    const double m = (double)(n11 + n10 + n01 + n00);
    if (m <= 0.0) return 0.0;
    /* joint probabilities */
    const double p11 = (double)n11 / m, p10 = (double)n10 / m;
    const double p01 = (double)n01 / m, p00 = (double)n00 / m;
    /* marginals of X (first variable) and Y (second variable) */
    const double px1 = p11 + p10, px0 = p01 + p00;
    const double py1 = p11 + p01, py0 = p10 + p00;
    double mi = 0.0;
    if (n11 > 0) mi += p11 * log2(p11 / (px1 * py1));
    if (n10 > 0) mi += p10 * log2(p10 / (px1 * py0));
    if (n01 > 0) mi += p01 * log2(p01 / (px0 * py1));
    if (n00 > 0) mi += p00 * log2(p00 / (px0 * py0));
    return mi;
}

/* MI for an explicit list of pairs.  Variable pi[k] is row pi[k] of AT and
 * variable pj[k] is row pj[k] of BT, where AT (na x m) and BT (nb x m) hold one
 * variable per row (the transposed data; AT == BT for pairs within one
 * dataset).  counts (4 per pair, may be NULL) receives n11, n10, n01, n00 and
 * mi (may be NULL) the value in bits.  Returns 0, or -1 on a bad index. */
int oracle_mi_pairs(const uint8_t* AT, int64_t na, const uint8_t* BT, int64_t nb, int64_t m,
                    const int64_t* pi, const int64_t* pj, int64_t npairs,
                    int64_t* counts, double* mi, int nthreads) {
    for (int64_t k = 0; k < npairs; ++k)
        if (pi[k] < 0 || pi[k] >= na || pj[k] < 0 || pj[k] >= nb) return -1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16) if (nthreads != 1)
#endif
    for (int64_t k = 0; k < npairs; ++k) {
        int64_t c[4];
        oracle_cell_counts(AT + pi[k] * m, BT + pj[k] * m, m, c);
        if (counts) {
            counts[4 * k + 0] = c[0];
            counts[4 * k + 1] = c[1];
            counts[4 * k + 2] = c[2];
            counts[4 * k + 3] = c[3];
        }
        if (mi) mi[k] = oracle_mi_from_counts(c[0], c[1], c[2], c[3]);
    }
    return 0;
}

/* Full na x nb MI matrix between the variables of AT and BT (every ordered
 * pair computed on its own, diagonal included).  out is row-major na x nb;
 * n11 (may be NULL) receives the co-occurrence counts in the same layout. */
void oracle_mi_matrix(const uint8_t* AT, int64_t na, const uint8_t* BT, int64_t nb, int64_t m,
                      double* out, int64_t* n11, int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4) if (nthreads != 1)
#endif
    for (int64_t i = 0; i < na; ++i) {
        for (int64_t j = 0; j < nb; ++j) {
            int64_t c[4];
            oracle_cell_counts(AT + i * m, BT + j * m, m, c);
            out[i * nb + j] = oracle_mi_from_counts(c[0], c[1], c[2], c[3]);
            if (n11) n11[i * nb + j] = c[0];
        }
    }
}

/* Number of ones of each variable: v_j = #{ r : x_rj = 1 } (the marginal
 * count of Sec. 2 step 3), counted directly from the transposed data. */
void oracle_column_counts(const uint8_t* XT, int64_t n, int64_t m, int64_t* v, int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(static) if (nthreads != 1)
#endif
    for (int64_t j = 0; j < n; ++j) {
        int64_t s = 0;
        for (int64_t r = 0; r < m; ++r) s += XT[j * m + r] != 0;
        v[j] = s;
    }
}

int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
