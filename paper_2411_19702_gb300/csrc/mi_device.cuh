// Per-pair mutual information from the co-occurrence count and the column
// counts, shared by every epilogue of the library (fused tensor-core kernel,
// popcount kernel, elementwise kernel of the plain path).
//
// Counts (Sec. 3.1, Eq. 6 and Eq. 7, with C_ij = v_j):
//   n10 = v_i - n11,  n01 = v_j - n11,  n00 = m - v_i - v_j + n11.
// MI (Eq. 1 / Eq. 2).  With det = n11*n00 - n10*n01 every cell satisfies
// n_c*m - a_c*b_c = s_c*det (a_c, b_c its marginal counts, s = +1 for 11/00
// and -1 for 10/01), i.e. n_c = (a_c b_c / m)(1 + x_c) with
// x_c = s_c det / (a_c b_c).  Since sum_c s_c = 0, the linear terms cancel
// exactly and
//   m ln2 * MI = sum_c n_c ln(1 + x_c) = sum_c (a_c b_c / m) h(x_c),
//   h(x) = (1 + x) ln(1 + x) - x = x^2/2 - x^3/6 + x^4/12 - ...  (>= 0).
// Each cell is evaluated as
//   |x_c| < 1/4:   (a_c b_c / m) h(x_c) = (s_c det / m) x_c (h(x_c) / x_c^2), the
//                  series to x^12 (truncation about 3e-9 relative): no
//                  cancellation, no division, no log;
//   otherwise:     n_c ln(n_c m / (a_c b_c)) - s_c det / m, with 1 / (a_c b_c)
//                  from the per-variable reciprocals, and 0 * log 0 = 0 for an
//                  empty cell (the paper's epsilon).
// det = 0 <=> MI = 0 exactly.
//
// FP64 combine (optional, GBMI_OPT_FIXUP): pairs whose FP32 value is below
// 1e-4 are recomputed from a table T[k] = k*log2(k) in FP64 (additions only):
//   m*MI = T[n11] + T[n10] + T[n01] + T[n00] + K_i + K_j,
//   K_i = T[m] / 2 - T[v_i] - T[m - v_i]  (per variable, MiVar.h),
// which follows from Eq. 1 by expanding the logarithm of the ratio.  Pairs go
// there without the FP32 evaluation when the chi-square bound already places
// them below 1e-4: MI (nats) <= chi^2-divergence = det^2 / (v_i (m - v_i)
// v_j (m - v_j)) (KL <= chi^2).
//
// All forms are symmetric in (i, j) to the last bit: exchanging the two
// variables swaps the 10 and 01 cells and the operands of commutative
// operations only, so MI(i, j) and MI(j, i) are the same float.
#pragma once

#include <cstdint>

namespace gbmi {

struct MiParams {
    int32_t m;           // samples (< 2^31)
    float fm;            // (float)m
    float inv_m_ln2;     // 1 / (m ln 2)
    float inv_m;         // 1 / m
    int fixup;           // 1: FP64 combine for pairs whose FP32 value is below fixup_below
    float fixup_below;   // 1e-4
    float chi_below;     // chi-square bound (nats) under which a pair goes straight to FP64
    const double* T;     // T[k] = k log2 k for k = 0..m, or nullptr: evaluate inline
};

// Per-variable quantities of one side of a pair (32 bytes, so that the first
// four fields load as one 16-byte vector).
struct __align__(16) MiVar {
    int32_t v;     // ones of the variable
    float r1;      // 1 / v            (0 if v == 0)
    float r0;      // 1 / (m - v)      (0 if v == m)
    float rchi;    // 1 / (v (m - v))  (0 if either is 0)
    double h;      // T[m] / 2 - T[v] - T[m - v] for the FP64 combine (0 when it is off)
    double unused;
};

// The FP32 terms of a MiVar (its first 16 bytes): all the FP32 epilogue reads.
struct __align__(16) MiVarF {
    int32_t v;
    float r1, r0, rchi;
};

__device__ __forceinline__ MiVarF load_var_f(const MiVar* p) {
    const float4 f = __ldg(reinterpret_cast<const float4*>(p));
    return MiVarF{__float_as_int(f.x), f.y, f.z, f.w};
}

__device__ __forceinline__ MiVar load_var(const MiVar* p) {
    MiVar r;
    const float4 f = __ldg(reinterpret_cast<const float4*>(p));
    r.v = __float_as_int(f.x);
    r.r1 = f.y;
    r.r0 = f.z;
    r.rchi = f.w;
    r.h = __ldg(&p->h);
    r.unused = 0.0;
    return r;
}

// T[k] = k log2 k in FP64 (0 for k = 0, 1), from the table when there is one.
__device__ __forceinline__ double nlog2n(int64_t k, const MiParams& P) {
    if (P.T != nullptr) return P.T[k];
    const double x = static_cast<double>(k);
    return k > 1 ? x * log2(x) : 0.0;
}

__device__ __forceinline__ MiVar mi_var(int32_t v, const MiParams& P) {
    MiVar r;
    r.v = v;
    const float a1 = static_cast<float>(v), a0 = static_cast<float>(P.m - v);
    r.r1 = v > 0 ? 1.0f / a1 : 0.f;
    r.r0 = v < P.m ? 1.0f / a0 : 0.f;
    r.rchi = r.r1 * r.r0;
    r.h = P.fixup ? 0.5 * nlog2n(P.m, P) -
                        (nlog2n(v, P) + nlog2n(static_cast<int64_t>(P.m) - v, P))
                  : 0.0;
    r.unused = 0.0;
    return r;
}

// Contribution of one cell to m ln2 * MI (see the header comment), from
// x = s_c det / (a_c b_c), sdm = s_c det / m (so that (a_c b_c / m) x = sdm)
// and rab = 1 / (a_c b_c).
__device__ __forceinline__ float mi_cell(int32_t nc, float x, float sdm, float rab,
                                         const MiParams& P) {
    if (fabsf(x) < 0.25f) {
        // (a b / m) h(x) = sdm x (1/2 - x/6 + x^2/12 - ... + x^10/132): the
        // Taylor series of h (k-th term (-1)^k x^k / (k (k - 1))) truncated
        // after k = 12, about 3e-9 relative at |x| = 1/4
        float p = fmaf(x, 1.0f / 132.0f, -1.0f / 110.0f);
        p = fmaf(x, p, 1.0f / 90.0f);
        p = fmaf(x, p, -1.0f / 72.0f);
        p = fmaf(x, p, 1.0f / 56.0f);
        p = fmaf(x, p, -1.0f / 42.0f);
        p = fmaf(x, p, 1.0f / 30.0f);
        p = fmaf(x, p, -0.05f);
        p = fmaf(x, p, 1.0f / 12.0f);
        p = fmaf(x, p, -1.0f / 6.0f);
        p = fmaf(x, p, 0.5f);
        return (sdm * x) * p;
    }
    // n_c ln(n_c m / (a_c b_c)) - s_c det / m; an empty cell gives -sdm
    // (0 * log 0 = 0).  With |x| >= 1/4 the two terms cancel by a factor of
    // about 10 at most, so the ratio's few ulp of rounding stay far below the
    // result's tolerance.
    const float t = nc > 0 ? static_cast<float>(nc) * logf((static_cast<float>(nc) * P.fm) * rab)
                           : 0.f;
    return t - sdm;
}

struct MiCounts {
    int32_t n11, n10, n01, n00;
    int64_t det;
};

// The determinant as a float from the two exact 31-bit halves of its
// magnitude (both non-negative, so their sum does not cancel), within 1.5
// ulp: FP32 conversions and one FMA (a 64-bit integer conversion would run on
// the FP64 pipe, which is slow on this part).  |d| < 2^62.
__device__ __forceinline__ float det_to_float(int64_t d) {
    const uint64_t a = static_cast<uint64_t>(d < 0 ? -d : d);
    const uint32_t hi = static_cast<uint32_t>(a >> 31);
    const uint32_t lo = static_cast<uint32_t>(a) & 0x7FFFFFFFu;
    const float f = fmaf(static_cast<float>(hi), 2147483648.0f, static_cast<float>(lo));
    return d < 0 ? -f : f;
}

__device__ __forceinline__ MiCounts mi_counts(int32_t n11, int32_t vi, int32_t vj,
                                              const MiParams& P) {
    MiCounts c;
    c.n11 = n11;
    c.n10 = vi - n11;
    c.n01 = vj - n11;
    c.n00 = P.m - vi - vj + n11;
    c.det = static_cast<int64_t>(c.n11) * c.n00 - static_cast<int64_t>(c.n10) * c.n01;
    return c;
}

// True when the chi-square bound places the pair below the FP64 threshold.
template <class VA, class VB>
__device__ __forceinline__ bool mi_surely_small(float fdet, const VA& A, const VB& B,
                                                const MiParams& P) {
    return (fdet * fdet) * (A.rchi * B.rchi) < P.chi_below;
}

// FP32 MI in bits (det != 0); A and B are MiVar or MiVarF.
template <class VA, class VB>
__device__ __forceinline__ float mi_fp32(const MiCounts& c, float fdet, const VA& A,
                                         const VB& B, const MiParams& P) {
    const float sdm = fdet * P.inv_m;
    const float r11 = A.r1 * B.r1, r10 = A.r1 * B.r0, r01 = A.r0 * B.r1, r00 = A.r0 * B.r0;
    const float t11 = mi_cell(c.n11, fdet * r11, sdm, r11, P);
    const float t10 = mi_cell(c.n10, -fdet * r10, -sdm, r10, P);
    const float t01 = mi_cell(c.n01, -fdet * r01, -sdm, r01, P);
    const float t00 = mi_cell(c.n00, fdet * r00, sdm, r00, P);
    return ((t11 + t00) + (t10 + t01)) * P.inv_m_ln2;
}

// FP64 n*log2(n) combine in bits.
__device__ __forceinline__ float mi_fp64(const MiCounts& c, const MiVar& A, const MiVar& B,
                                         const MiParams& P) {
    const double s = (nlog2n(c.n11, P) + nlog2n(c.n00, P)) + (nlog2n(c.n10, P) + nlog2n(c.n01, P));
    const double r = s + (A.h + B.h);
    return static_cast<float>(r) * P.inv_m;
}

// MI of one pair from its co-occurrence count, the FP32 terms of both
// variables and (FP64 combine) their FP64 terms Ah, Bh (MiVar.h).
__device__ __forceinline__ float mi_pair_f(int32_t n11, const MiVarF& A, double Ah,
                                           const MiVarF& B, double Bh, const MiParams& P) {
    const MiCounts c = mi_counts(n11, A.v, B.v, P);
    if (c.det == 0) return 0.f;   // exact independence: every log ratio is 0
    const float fdet = det_to_float(c.det);
    bool need64 = P.fixup && mi_surely_small(fdet, A, B, P);
    float mi = 0.f;
    if (!need64) {
        mi = mi_fp32(c, fdet, A, B, P);
        need64 = P.fixup && mi < P.fixup_below;
    }
    if (need64) {
        const double s = (nlog2n(c.n11, P) + nlog2n(c.n00, P)) +
                         (nlog2n(c.n10, P) + nlog2n(c.n01, P));
        mi = static_cast<float>(s + (Ah + Bh)) * P.inv_m;
    }
    return fmaxf(mi, 0.f);
}

__device__ __forceinline__ float mi_pair(int32_t n11, const MiVar& A, const MiVar& B,
                                         const MiParams& P) {
    return mi_pair_f(n11, MiVarF{A.v, A.r1, A.r0, A.rchi}, A.h, MiVarF{B.v, B.r1, B.r0, B.rchi},
                     B.h, P);
}

}  // namespace gbmi
