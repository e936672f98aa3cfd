// Elementwise kernels:
//   - the n*log2(n) table T[k] = k log2 k (FP64) behind the FP64 combine,
//   - per-variable H_j = T[v_j] + T[m - v_j] (the marginal part of m*MI),
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

__global__ void col_h_kernel(const int32_t* v, int64_t n, const MiParams P, double* h) {
    for (int64_t j = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; j < n;
         j += static_cast<int64_t>(gridDim.x) * blockDim.x)
        h[j] = mi_col_h(v[j], P);
}

// One thread per output element, 2-D grid over (row block, column block):
// threadIdx.x runs along j for coalesced reads of N11 and writes of out.
__global__ void mi_from_counts_kernel(const int32_t* N11, int64_t ld_n11, const int32_t* va,
                                      const int32_t* vb, const double* ha, const double* hb,
                                      int64_t n1, int64_t n2, const MiParams P, float* out,
                                      int64_t ld_out) {
    const int64_t j = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (j >= n2) return;
    const int64_t vj = vb[j];
    const double hj = hb ? hb[j] : 0.0;
    for (int64_t i = blockIdx.y; i < n1; i += gridDim.y) {
        const double hi = ha ? ha[i] : 0.0;
        out[i * ld_out + j] = mi_pair(N11[i * ld_n11 + j], va[i], vj, hi, hj, P);
    }
}

}  // namespace

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

cudaError_t launch_col_h(const int32_t* v, int64_t n, const MiParams& P, double* h,
                         cudaStream_t s) {
    const int64_t blocks = (n + 255) / 256;
    col_h_kernel<<<static_cast<unsigned>(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(v, n, P,
                                                                                     h);
    return cudaGetLastError();
}

cudaError_t launch_mi_from_counts(const int32_t* N11, int64_t ld_n11, const int32_t* va,
                                  const int32_t* vb, const double* ha, const double* hb,
                                  int64_t n1, int64_t n2, const MiParams& P, float* out,
                                  int64_t ld_out, cudaStream_t s) {
    const int64_t bx = (n2 + 255) / 256;
    if (bx > 0x7FFFFFFF) return cudaErrorInvalidValue;
    const int64_t by = n1 < 65535 ? n1 : 65535;
    dim3 grid(static_cast<unsigned>(bx), static_cast<unsigned>(by));
    mi_from_counts_kernel<<<grid, 256, 0, s>>>(N11, ld_n11, va, vb, ha, hb, n1, n2, P, out,
                                               ld_out);
    return cudaGetLastError();
}

}  // namespace gbmi
