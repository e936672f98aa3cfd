// Bit-packed co-occurrence Gram: N11[i][j] = sum_w popc(Ba[i][w] & Bb[j][w]),
// the count of samples where both variables are 1 (G11 of Sec. 2 step 2),
// with integer ALU work only.  It is the exactness cross-check of the
// tensor-core Gram and the path for tiny shapes, where it also runs the MI
// epilogue (Eq. 6-7 counts, Eq. 1/Eq. 2 MI) in place.
//
// CTA tile 64 x 64 outputs, 256 threads with a 4 x 4 micro-tile each; the
// K loop stages 32 words (1024 samples) of 64 rows of each operand in shared
// memory (rows padded to 33 words: conflict-free column reads).
#include "internal.cuh"

namespace gbmi {

namespace {

constexpr int kPT = 64;       // outputs per tile side
constexpr int kKW = 32;       // words per K chunk
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads)
popcount_gram_kernel(const PopcArgs a) {
    const int I = blockIdx.y, J = blockIdx.x;
    if (a.symmetric && J < I) return;

    __shared__ uint32_t As[kPT][kKW + 1];
    __shared__ uint32_t Bs[kPT][kKW + 1];

    const int t = threadIdx.x;
    const int tx = t % 16, ty = t / 16;
    const int64_t ia = static_cast<int64_t>(I) * kPT;
    const int64_t jb = static_cast<int64_t>(J) * kPT;

    int acc[4][4];
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] = 0;

    const int lrow = t / 4;          // row loaded by this thread
    const int lw = (t % 4) * 8;      // first word loaded by this thread
    for (int64_t k0 = 0; k0 < a.wpr; k0 += kKW) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t w = k0 + lw + 4 * h;
            uint4 va = make_uint4(0, 0, 0, 0), vb = make_uint4(0, 0, 0, 0);
            if (w < a.wpr) {   // wpr is a multiple of 4: the uint4 is fully inside
                va = __ldg(reinterpret_cast<const uint4*>(a.Ba + (ia + lrow) * a.wpr + w));
                vb = __ldg(reinterpret_cast<const uint4*>(a.Bb + (jb + lrow) * a.wpr + w));
            }
            As[lrow][lw + 4 * h + 0] = va.x;
            As[lrow][lw + 4 * h + 1] = va.y;
            As[lrow][lw + 4 * h + 2] = va.z;
            As[lrow][lw + 4 * h + 3] = va.w;
            Bs[lrow][lw + 4 * h + 0] = vb.x;
            Bs[lrow][lw + 4 * h + 1] = vb.y;
            Bs[lrow][lw + 4 * h + 2] = vb.z;
            Bs[lrow][lw + 4 * h + 3] = vb.w;
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < kKW; ++k) {
            uint32_t av[4], bv[4];
#pragma unroll
            for (int x = 0; x < 4; ++x) av[x] = As[ty * 4 + x][k];
#pragma unroll
            for (int y = 0; y < 4; ++y) bv[y] = Bs[tx * 4 + y][k];
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) acc[x][y] += __popc(av[x] & bv[y]);
        }
        __syncthreads();
    }

#pragma unroll
    for (int x = 0; x < 4; ++x) {
        const int64_t i = ia + ty * 4 + x;
        if (i >= a.n_a) continue;
        MiVar A;
        if (a.out_f) A = load_var(a.va + i);
#pragma unroll
        for (int y = 0; y < 4; ++y) {
            const int64_t j = jb + tx * 4 + y;
            if (j >= a.n_b) continue;
            if (a.symmetric && j < i) continue;
            if (a.out_c != nullptr) {
                a.out_c[i * a.ld_out + j] = acc[x][y];
                if (a.symmetric && j != i) a.out_c[j * a.ld_out + i] = acc[x][y];
            }
            if (a.out_f != nullptr) {
                const float mi = mi_pair(acc[x][y], A, load_var(a.vb + j), a.mp);
                a.out_f[i * a.ld_out + j] = mi;
                if (a.symmetric && j != i) a.out_f[j * a.ld_out + i] = mi;
            }
        }
    }
}

}  // namespace

cudaError_t launch_popcount(const PopcArgs& a, cudaStream_t s) {
    if (a.wpr % 4 != 0) return cudaErrorInvalidValue;
    const int64_t ta = (a.n_a + kPT - 1) / kPT, tb = (a.n_b + kPT - 1) / kPT;
    if (ta > 65535 || tb > 0x7FFFFFFF) return cudaErrorInvalidValue;
    dim3 grid(static_cast<unsigned>(tb), static_cast<unsigned>(ta));
    popcount_gram_kernel<<<grid, kThreads, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace gbmi
