// Per-pair mutual information from the co-occurrence count and the column
// counts, shared by every epilogue of the library (fused tensor-core kernel,
// popcount kernel, elementwise kernel of the plain path).
//
// Counts (Sec. 3.1, Eq. 6 and Eq. 7, with C_ij = v_j):
//   n10 = v_i - n11,  n01 = v_j - n11,  n00 = m - v_i - v_j + n11.
// MI (Eq. 1 / Eq. 2) in the determinant form: with det = n11*n00 - n10*n01,
// every cell satisfies n_c*m - a_c*b_c = s_c*det (a_c, b_c its marginal
// counts, s = +1 for 11/00 and -1 for 10/01), hence
//   MI = 1/(m ln 2) * sum_{c: n_c > 0} n_c * ln(1 + s_c*det/(a_c*b_c)).
// This has no cancellation near independence (det = 0 <=> MI = 0 exactly) and
// its error scales with the dependence.  Cells with n_c = 0 contribute 0
// (the 0*log 0 = 0 limit replaces the paper's epsilon).
//
// FP64 combine: for pairs whose FP32 value is below 1e-4 the value is
// recomputed from a table T[k] = k*log2(k) in FP64 (additions only):
//   m*MI = T[n11] + T[n10] + T[n01] + T[n00] - H_i - H_j + T[m],
//   H_i = T[v_i] + T[m - v_i],
// which follows from Eq. 1 by expanding the logarithm of the ratio.
//
// Both forms are symmetric in (i, j) to the last bit: exchanging the two
// variables swaps the 10 and 01 cells and the operands of commutative
// operations only, so MI(i, j) and MI(j, i) are the same float.
#pragma once

#include <cstdint>

namespace gbmi {

struct MiParams {
    int64_t m;           // samples
    float fm;            // (float)m
    float inv_m_ln2;     // 1 / (m ln 2)
    double inv_m;        // 1 / m
    int fixup;           // 1: FP64 combine for pairs whose FP32 value is below fixup_below
    float fixup_below;   // 1e-4
    const double* T;     // T[k] = k log2 k for k = 0..m, or nullptr: evaluate inline
};

// T[k] = k log2 k in FP64 (0 for k = 0, 1), from the table when there is one.
__device__ __forceinline__ double nlog2n(int64_t k, const MiParams& P) {
    if (P.T != nullptr) return P.T[k];
    const double x = static_cast<double>(k);
    return k > 1 ? x * log2(x) : 0.0;
}

// n_c * ln(n_c * m / (a * b)) for one cell with n_c > 0 (so a, b > 0), from
// the signed determinant sdet = s_c * det.
__device__ __forceinline__ float mi_cell(int64_t nc, float sdet, float a, float b, float fm) {
    const float ab = a * b;
    const float x = sdet / ab;
    float l;
    if (x > -0.5f) {
        l = log1pf(x);
    } else {
        // far below independence: the ratio itself is well conditioned
        l = logf((static_cast<float>(nc) * fm) / ab);
    }
    return static_cast<float>(nc) * l;
}

__device__ __forceinline__ float mi_pair(int64_t n11, int64_t vi, int64_t vj, double hi,
                                         double hj, const MiParams& P) {
    const int64_t m = P.m;
    const int64_t n10 = vi - n11;
    const int64_t n01 = vj - n11;
    const int64_t n00 = m - vi - vj + n11;
    const int64_t det = n11 * n00 - n10 * n01;
    if (det == 0) return 0.f;   // exact independence: every log ratio is 0
    const float fdet = static_cast<float>(det);
    const float ai = static_cast<float>(vi), a0 = static_cast<float>(m - vi);
    const float bj = static_cast<float>(vj), b0 = static_cast<float>(m - vj);
    float t11 = 0.f, t10 = 0.f, t01 = 0.f, t00 = 0.f;
    if (n11 > 0) t11 = mi_cell(n11, fdet, ai, bj, P.fm);
    if (n10 > 0) t10 = mi_cell(n10, -fdet, ai, b0, P.fm);
    if (n01 > 0) t01 = mi_cell(n01, -fdet, a0, bj, P.fm);
    if (n00 > 0) t00 = mi_cell(n00, fdet, a0, b0, P.fm);
    float mi = ((t11 + t00) + (t10 + t01)) * P.inv_m_ln2;
    if (P.fixup && mi < P.fixup_below) {
        const double s = (nlog2n(n11, P) + nlog2n(n00, P)) + (nlog2n(n10, P) + nlog2n(n01, P));
        const double r = (s + (nlog2n(m, P) - (hi + hj))) * P.inv_m;
        mi = static_cast<float>(r);
    }
    return fmaxf(mi, 0.f);
}

// H_j = T[v_j] + T[m - v_j] for the FP64 combine (0 when it is off).
__device__ __forceinline__ double mi_col_h(int64_t v, const MiParams& P) {
    if (!P.fixup) return 0.0;
    return nlog2n(v, P) + nlog2n(P.m - v, P);
}

}  // namespace gbmi
