// Sparse input: co-occurrence counts from a CSR matrix (the paper's sparse
// variant, Sec. 4.2.3: a sparse-matrix Gram whose cost follows the number of
// ones instead of m * n^2).
//
// X is given by samples: row_ptr[m + 1], col_idx[nnz] = the variables that are
// 1 in each sample, strictly increasing.  A sample with k ones contributes 1
// to N11[a][b] for each of its k (k + 1) / 2 pairs a <= b (the diagonal gives
// the column counts).  One warp walks one sample's pairs, enumerated linearly
// so that short rows keep all lanes busy, and adds them to the upper triangle
// of N11 with atomic adds.  The kernel checks the CSR structure it reads (row
// bounds inside [0, nnz], indices inside [0, n) and strictly increasing); a
// malformed row is skipped and flagged in the error word, so no access leaves
// the caller's arrays.  Where the ones are not that sparse, the C ABI instead
// writes the dense 0/1 matrix (csr_densify_kernel) and runs the tensor-core
// path on it.
#include "internal.cuh"

namespace gbmi {

namespace {

constexpr int kCsrThreads = 256;

// (i, j), i <= j < k, of the p-th pair of the row-major upper triangle of k x k.
__device__ __forceinline__ void pair_of(int64_t p, int64_t k, int64_t& i, int64_t& j) {
    const float b = 2.f * static_cast<float>(k) + 1.f;
    int64_t r = static_cast<int64_t>((b - sqrtf(fmaxf(b * b - 8.f * static_cast<float>(p), 0.f))) *
                                     0.5f);
    auto first = [k](int64_t x) { return x * k - x * (x - 1) / 2; };
    r = r < 0 ? 0 : (r >= k ? k - 1 : r);
    while (r > 0 && first(r) > p) --r;
    while (r + 1 < k && first(r + 1) <= p) ++r;
    i = r;
    j = r + (p - first(r));
}

__global__ void __launch_bounds__(kCsrThreads)
csr_pair_counts_kernel(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                       int64_t m, int64_t n, int64_t nnz, int32_t* N11, unsigned int* err) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (static_cast<int64_t>(blockIdx.x) * kCsrThreads + threadIdx.x) >> 5;
    const int64_t nw = (static_cast<int64_t>(gridDim.x) * kCsrThreads) >> 5;
    for (int64_t r = w0; r < m; r += nw) {
        const int64_t b = row_ptr[r], e = row_ptr[r + 1];
        if (b < 0 || e < b || e > nnz) {
            if (lane == 0) atomicOr(err, kErrBadCsr);
            continue;
        }
        const int64_t k = e - b;
        bool bad = false;
        for (int64_t q = lane; q < k; q += 32) {
            const int32_t c = col[b + q];
            if (c < 0 || c >= n || (q > 0 && col[b + q - 1] >= c)) bad = true;
        }
        if (__any_sync(0xffffffffu, bad)) {
            if (lane == 0) atomicOr(err, kErrBadCsr);
            continue;
        }
        const int64_t pairs = k * (k + 1) / 2;
        for (int64_t p = lane; p < pairs; p += 32) {
            int64_t i, j;
            pair_of(p, k, i, j);
            const int64_t a = col[b + i], c = col[b + j];
            atomicAdd(N11 + a * n + c, 1);
        }
    }
}

// Dense form of a CSR matrix: X (m x n uint8, zeroed before) gets a 1 at
// every (sample, variable) listed, one warp per sample, with the same checks
// as the pair-count kernel (a malformed row writes nothing and is flagged).
__global__ void __launch_bounds__(kCsrThreads)
csr_densify_kernel(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                   int64_t m, int64_t n, int64_t nnz, uint8_t* X, unsigned int* err) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (static_cast<int64_t>(blockIdx.x) * kCsrThreads + threadIdx.x) >> 5;
    const int64_t nw = (static_cast<int64_t>(gridDim.x) * kCsrThreads) >> 5;
    for (int64_t r = w0; r < m; r += nw) {
        const int64_t b = row_ptr[r], e = row_ptr[r + 1];
        if (b < 0 || e < b || e > nnz) {
            if (lane == 0) atomicOr(err, kErrBadCsr);
            continue;
        }
        const int64_t k = e - b;
        bool bad = false;
        for (int64_t q = lane; q < k; q += 32) {
            const int32_t c = col[b + q];
            if (c < 0 || c >= n || (q > 0 && col[b + q - 1] >= c)) bad = true;
        }
        if (__any_sync(0xffffffffu, bad)) {
            if (lane == 0) atomicOr(err, kErrBadCsr);
            continue;
        }
        for (int64_t q = lane; q < k; q += 32) X[r * n + col[b + q]] = 1;
    }
}

// v[j] = N11[j][j] (the diagonal holds each variable's count of ones).
__global__ void diag_kernel(const int32_t* N11, int64_t n, int32_t* v) {
    for (int64_t j = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; j < n;
         j += static_cast<int64_t>(gridDim.x) * blockDim.x)
        v[j] = N11[j * n + j];
}

// Copy the upper triangle into the lower one, 32 x 32 tiles through shared memory.
__global__ void mirror_upper_kernel(int32_t* N11, int64_t n, int64_t tps) {
    __shared__ int32_t T[32][33];
    const int64_t I = blockIdx.y, J = blockIdx.x;
    if (J <= I) return;   // tile (I, J) with I < J is mirrored into (J, I); diagonal below
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int k = 0; k < 4; ++k) {
        const int r = ty + 8 * k;
        const int64_t i = I * 32 + r, j = J * 32 + tx;
        T[r][tx] = (i < n && j < n) ? N11[i * n + j] : 0;
    }
    __syncthreads();
    for (int k = 0; k < 4; ++k) {
        const int c = ty + 8 * k;
        const int64_t jj = J * 32 + c, ii = I * 32 + tx;
        if (jj < n && ii < n) N11[jj * n + ii] = T[tx][c];
    }
    (void)tps;
}

// Diagonal tiles: the strictly lower part of each from its upper part.
__global__ void mirror_diag_kernel(int32_t* N11, int64_t n) {
    const int64_t I = blockIdx.x;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int k = 0; k < 4; ++k) {
        const int r = ty + 8 * k;
        const int64_t i = I * 32 + r, j = I * 32 + tx;
        if (i < n && j < n && j < i) N11[i * n + j] = N11[j * n + i];
    }
}

}  // namespace

cudaError_t launch_csr_pair_counts(const int64_t* row_ptr, const int32_t* col, int64_t m,
                                   int64_t n, int64_t nnz, int32_t* N11, unsigned int* err,
                                   int sm_count, cudaStream_t s) {
    if (m <= 0) return cudaSuccess;
    const int64_t warps_max = static_cast<int64_t>(sm_count > 0 ? sm_count : 152) * 64;
    const int64_t warps = m < warps_max ? m : warps_max;
    const int64_t blocks = (warps * 32 + kCsrThreads - 1) / kCsrThreads;
    csr_pair_counts_kernel<<<static_cast<unsigned>(blocks), kCsrThreads, 0, s>>>(row_ptr, col, m,
                                                                                 n, nnz, N11, err);
    return cudaGetLastError();
}

cudaError_t launch_csr_densify(const int64_t* row_ptr, const int32_t* col, int64_t m, int64_t n,
                               int64_t nnz, uint8_t* X, unsigned int* err, int sm_count,
                               cudaStream_t s) {
    if (m <= 0) return cudaSuccess;
    const int64_t warps_max = static_cast<int64_t>(sm_count > 0 ? sm_count : 152) * 64;
    const int64_t warps = m < warps_max ? m : warps_max;
    const int64_t blocks = (warps * 32 + kCsrThreads - 1) / kCsrThreads;
    csr_densify_kernel<<<static_cast<unsigned>(blocks), kCsrThreads, 0, s>>>(row_ptr, col, m, n,
                                                                             nnz, X, err);
    return cudaGetLastError();
}

cudaError_t launch_diag(const int32_t* N11, int64_t n, int32_t* v, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int64_t blocks = (n + 255) / 256;
    diag_kernel<<<static_cast<unsigned>(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(N11, n, v);
    return cudaGetLastError();
}

cudaError_t launch_mirror_upper(int32_t* N11, int64_t n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int64_t tps = (n + 31) / 32;
    if (tps > 65535) return cudaErrorInvalidValue;
    mirror_upper_kernel<<<dim3(static_cast<unsigned>(tps), static_cast<unsigned>(tps)), 256, 0,
                          s>>>(N11, n, tps);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    mirror_diag_kernel<<<static_cast<unsigned>(tps), 256, 0, s>>>(N11, n);
    return cudaGetLastError();
}

}  // namespace gbmi
