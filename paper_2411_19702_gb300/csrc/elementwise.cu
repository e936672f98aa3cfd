// Elementwise kernels:
//   - zero fill,
//   - the n*log2(n) table T[k] = k log2 k (FP64) behind the FP64 combine,
//   - per-variable epilogue terms (MiVar: reciprocals of the marginal counts
//     and H_j = T[v_j] + T[m - v_j]),
//   - MI from a stored count matrix (second half of the plain, unfused path:
//     Eq. 6-7 counts and Eq. 1/Eq. 2 MI for every (i, j) of N11).
#include "internal.cuh"

namespace gbmi {

namespace {

__global__ void zero_kernel(uint32_t* p, int64_t words) {
    for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k < words;
         k += static_cast<int64_t>(gridDim.x) * blockDim.x)
        p[k] = 0u;
}

__global__ void nlogn_table_kernel(double* T, int64_t len) {
    for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k < len;
         k += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const double x = static_cast<double>(k);
        T[k] = k > 1 ? x * log2(x) : 0.0;
    }
}

__global__ void mi_vars_kernel(const int32_t* v, int64_t n, const MiParams P, MiVar* out) {
    for (int64_t j = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; j < n;
         j += static_cast<int64_t>(gridDim.x) * blockDim.x)
        out[j] = mi_var(v[j], P);
}

__global__ void mi_vars_grouped_kernel(const int32_t* v, const int64_t* var_begin, int njobs,
                                       int64_t total, const MiParams* params, MiVar* out) {
    for (int64_t x = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; x < total;
         x += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        int lo = 0, hi = njobs - 1;   // last job whose first variable <= x
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (var_begin[mid] <= x) lo = mid; else hi = mid - 1;
        }
        out[x] = mi_var(v[x], params[lo]);
    }
}

// Count at index idx of `slices` partial count matrices stride elements apart
// (the sample ranges of a split Gram); exact int32 sums.
__device__ __forceinline__ int32_t slice_sum(const int32_t* N11, int64_t idx, int slices,
                                             int64_t stride) {
    int32_t v = N11[idx];
    for (int k = 1; k < slices; ++k) v += N11[idx + k * stride];
    return v;
}

// One thread per output element; a CTA covers 256 consecutive j of one row
// block, so N11 reads and MI writes are coalesced and the row terms uniform.
__global__ void mi_from_counts_kernel(const int32_t* N11, int64_t ld_n11, const MiVar* va,
                                      const MiVar* vb, int64_t n1, int64_t n2, const MiParams P,
                                      float* out, int64_t ld_out, int slices, int64_t stride) {
    const int64_t j = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (j >= n2) return;
    const MiVar B = load_var(vb + j);
    for (int64_t i = blockIdx.y; i < n1; i += gridDim.y) {
        const MiVar A = load_var(va + i);
        out[i * ld_out + j] = mi_pair(slice_sum(N11, i * ld_n11 + j, slices, stride), A, B, P);
    }
}

// out[i][j] = sum over the slices of N11[i][j] (rows x cols, both row-major).
__global__ void slice_sum_kernel(const int32_t* N11, int64_t ld_n11, int slices, int64_t stride,
                                 int64_t rows, int64_t cols, int32_t* out, int64_t ld_out) {
    const int64_t total = rows * cols;
    for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t i = e / cols, j = e % cols;
        out[i * ld_out + j] = slice_sum(N11, i * ld_n11 + j, slices, stride);
    }
}

// Symmetric counts (all pairs of one matrix): only tiles with I <= J of 32 x 32
// pairs are evaluated; each value is written to (i, j) directly and to (j, i)
// through a shared-memory transpose, so both writes are coalesced rows.  A
// diagonal tile evaluates its 32 x 32 pairs itself.  The 32 row terms of a
// tile are staged in shared memory once, and each thread issues the count
// loads of its four pairs before any arithmetic, so the loads are in flight
// together (the kernel streams 4 bytes in and 8 bytes out per pair).
constexpr int kSymTile = 32;

template <bool kFix>
__global__ void __launch_bounds__(256)
mi_from_counts_sym_kernel(const int32_t* N11, int64_t ld_n11, const MiVar* vars, int64_t n,
                          const MiParams P, float* out, int64_t ld_out, int64_t tiles_per_side,
                          int upper_only, int slices, int64_t stride) {
    __shared__ float T[kSymTile][kSymTile + 1];
    __shared__ MiVarF As[kSymTile];
    __shared__ double Ah[kSymTile];
    // tile index -> (I, J) with I <= J, row-major over the upper triangle
    // first tile of row I: S(I) = I * tps - I (I - 1) / 2; take the largest I
    // with S(I) <= t (closed form, then exact integer correction)
    const int64_t t = blockIdx.x, tps = tiles_per_side;
    const double b = 2.0 * static_cast<double>(tps) + 1.0;
    int64_t I = static_cast<int64_t>((b - sqrt(b * b - 8.0 * static_cast<double>(t))) * 0.5);
    auto first = [tps](int64_t r) { return r * tps - r * (r - 1) / 2; };
    while (I > 0 && first(I) > t) --I;
    while (I + 1 < tps && first(I + 1) <= t) ++I;
    const int64_t J = I + (t - first(I));
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8 threads
    const int64_t j = J * kSymTile + tx;
    const bool jok = j < n;
    if (ty == 0) {
        const int64_t ia = I * kSymTile + tx;
        As[tx] = ia < n ? load_var_f(vars + ia) : MiVarF{0, 0.f, 0.f, 0.f};
        if (kFix) Ah[tx] = ia < n ? __ldg(&vars[ia].h) : 0.0;
    }
    const MiVarF B = jok ? load_var_f(vars + j) : MiVarF{0, 0.f, 0.f, 0.f};
    const double Bh = kFix && jok ? __ldg(&vars[j].h) : 0.0;
    int32_t cnt[kSymTile / 8];
#pragma unroll
    for (int k = 0; k < kSymTile / 8; ++k) {
        const int64_t i = I * kSymTile + ty + 8 * k;
        // upper_only: only N11[a][b], a <= b, is filled
        const int64_t lo = (upper_only && i > j) ? j : i, hi = (upper_only && i > j) ? i : j;
        cnt[k] = jok && i < n ? slice_sum(N11, lo * ld_n11 + hi, slices, stride) : 0;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kSymTile / 8; ++k) {
        const int r = ty + 8 * k;
        const int64_t i = I * kSymTile + r;
        float v = 0.f;
        if (jok && i < n) {
            v = mi_pair_f(cnt[k], As[r], kFix ? Ah[r] : 0.0, B, Bh, P);
            out[i * ld_out + j] = v;
        }
        T[r][tx] = v;
    }
    if (I == J) return;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kSymTile / 8; ++k) {
        const int c = ty + 8 * k;                 // column of the tile -> row of the mirror
        const int64_t jj = J * kSymTile + c;
        const int64_t ii = I * kSymTile + tx;
        if (jj < n && ii < n) out[jj * ld_out + ii] = T[tx][c];
    }
}

}  // namespace

cudaError_t launch_mi_from_counts_sym(const int32_t* N11, int64_t ld_n11, const MiVar* vars,
                                      int64_t n, const MiParams& P, float* out, int64_t ld_out,
                                      cudaStream_t s, int upper_only, int slices,
                                      int64_t slice_stride) {
    if (n <= 0) return cudaSuccess;
    if (slices < 1) return cudaErrorInvalidValue;
    const int64_t tps = (n + kSymTile - 1) / kSymTile;
    const int64_t tiles = tps * (tps + 1) / 2;
    if (tiles > 0x7FFFFFFF) return cudaErrorInvalidValue;
    if (P.fixup)
        mi_from_counts_sym_kernel<true><<<static_cast<unsigned>(tiles), 256, 0, s>>>(
            N11, ld_n11, vars, n, P, out, ld_out, tps, upper_only, slices, slice_stride);
    else
        mi_from_counts_sym_kernel<false><<<static_cast<unsigned>(tiles), 256, 0, s>>>(
            N11, ld_n11, vars, n, P, out, ld_out, tps, upper_only, slices, slice_stride);
    return cudaGetLastError();
}

cudaError_t launch_slice_sum(const int32_t* N11, int64_t ld_n11, int slices, int64_t slice_stride,
                             int64_t rows, int64_t cols, int32_t* out, int64_t ld_out,
                             cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    if (slices < 1) return cudaErrorInvalidValue;
    const int64_t blocks = (rows * cols + 255) / 256;
    slice_sum_kernel<<<static_cast<unsigned>(blocks < 8192 ? blocks : 8192), 256, 0, s>>>(
        N11, ld_n11, slices, slice_stride, rows, cols, out, ld_out);
    return cudaGetLastError();
}

cudaError_t launch_zero_u32(void* p, int64_t words, cudaStream_t s) {
    const int64_t blocks = (words + 255) / 256;
    zero_kernel<<<static_cast<unsigned>(blocks < 2048 ? (blocks > 0 ? blocks : 1) : 2048), 256, 0,
                  s>>>(static_cast<uint32_t*>(p), words);
    return cudaGetLastError();
}

cudaError_t launch_nlogn_table(double* T, int64_t len, cudaStream_t s) {
    nlogn_table_kernel<<<1024, 256, 0, s>>>(T, len);
    return cudaGetLastError();
}

cudaError_t launch_mi_vars(const int32_t* v, int64_t n, const MiParams& P, MiVar* out,
                           cudaStream_t s) {
    const int64_t blocks = (n + 255) / 256;
    mi_vars_kernel<<<static_cast<unsigned>(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(v, n, P,
                                                                                       out);
    return cudaGetLastError();
}

cudaError_t launch_mi_vars_grouped(const int32_t* v, const int64_t* var_begin, int njobs,
                                   int64_t total, const MiParams* params, MiVar* out,
                                   cudaStream_t s) {
    if (njobs <= 0 || total <= 0) return cudaSuccess;
    const int64_t blocks = (total + 255) / 256;
    mi_vars_grouped_kernel<<<static_cast<unsigned>(blocks < 8192 ? blocks : 8192), 256, 0, s>>>(
        v, var_begin, njobs, total, params, out);
    return cudaGetLastError();
}

cudaError_t launch_mi_from_counts(const int32_t* N11, int64_t ld_n11, const MiVar* va,
                                  const MiVar* vb, int64_t n1, int64_t n2, const MiParams& P,
                                  float* out, int64_t ld_out, cudaStream_t s, int slices,
                                  int64_t slice_stride) {
    if (slices < 1) return cudaErrorInvalidValue;
    const int64_t bx = (n2 + 255) / 256;
    if (bx > 0x7FFFFFFF) return cudaErrorInvalidValue;
    const int64_t by = n1 < 65535 ? n1 : 65535;
    dim3 grid(static_cast<unsigned>(bx), static_cast<unsigned>(by));
    mi_from_counts_kernel<<<grid, 256, 0, s>>>(N11, ld_n11, va, vb, n1, n2, P, out, ld_out,
                                               slices, slice_stride);
    return cudaGetLastError();
}

}  // namespace gbmi
