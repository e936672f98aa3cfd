// Tensor-core throughput of the MMA forms the Gram kernel issues, measured
// with operands resident in shared memory: no global-memory traffic, no TMA,
// no epilogue.  This is the denominator of the Gram kernel's roofline for
// the operand forms that have no library GEMM to time (block-scaled FP4), and
// a cross-check of the library figure for the others (FP8 E4M3).
//
// Every CTA (or CTA pair) fills its A and B tiles once with 0/1 values of the
// operand form (random bits, half of them ones), then one thread issues
// back-to-back tcgen05.mma of shape M x N x K (M = 128 on one SM, 256 on a
// pair; K = 32 bytes of the 128-byte swizzled rows: 32 FP8 or 64 FP4
// samples) into one TMEM accumulator, the same instruction descriptors and
// shared-memory descriptors as the Gram kernel.  MMAs are committed in
// batches of 16 with at most two batches outstanding; every wait is bounded.
#include <cstring>

#include "runtime.h"
#include "ptx.cuh"

namespace gbmi {
namespace {

constexpr int kPkBatch = 16;
constexpr int kPkAOff = 0;                       // 128 rows x 128 B
constexpr int kPkBOff = kTcBM * kTcBK;           // 256 rows x 128 B
constexpr int kPkBarOff = kPkBOff + kTcBNMax * kTcBK;
constexpr int kPkSmem = 1024 + kPkBarOff + 64;
constexpr int kPkSfa = 256;                      // scale-factor columns (all 1.0)
constexpr int kPkSfb = 288;

struct PeakArgs {
    int64_t mmas;          // MMAs issued by each issuing thread
    int n;                 // MMA N
    unsigned int* err;     // device error word
    uint64_t timeout_ns;
};

__device__ __forceinline__ uint32_t pk_hash(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352dU;
    x ^= x >> 15;
    x *= 0x846ca68bU;
    x ^= x >> 16;
    return x;
}

// kForm: 0 FP8 E4M3 (kind::f8f6f4), 1 FP4 E2M1 with UE8M0 scales per 32 (kind::mxf4),
// 2 FP4 E2M1 with UE4M3 scales per 16 (kind::mxf4nvf4, scale_vec::4X)
template <int kForm, bool kPair>
__global__ void __launch_bounds__(128, 1) mma_peak_kernel(const PeakArgs a) {
    constexpr bool kFp4 = kForm != 0;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                               ~static_cast<uintptr_t>(1023));
    uint64_t* bars = reinterpret_cast<uint64_t*>(base + kPkBarOff);   // 2 batch + drain
    uint32_t* holder = reinterpret_cast<uint32_t*>(base + kPkBarOff + 32);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(base + kPkBarOff + 40);
    const int warp = threadIdx.x >> 5;
    const uint32_t rank = kPair ? ptx::cluster_ctarank() : 0u;

    // operand tiles: every 32-bit word holds random 0/1 elements of the form
    // (FP4: nibbles 0x0 / 0x2, FP8: bytes 0x00 / 0x38)
    uint32_t* w = reinterpret_cast<uint32_t*>(base);
    for (int k = threadIdx.x; k < kPkBarOff / 4; k += blockDim.x) {
        const uint32_t r = pk_hash(static_cast<uint32_t>(k) * 2654435761u + blockIdx.x);
        uint32_t v = 0;
        if (kFp4) {
            for (int q = 0; q < 8; ++q) v |= ((r >> q) & 1u) ? (0x2u << (4 * q)) : 0u;
        } else {
            for (int q = 0; q < 4; ++q) v |= ((r >> q) & 1u) ? (0x38u << (8 * q)) : 0u;
        }
        w[k] = v;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // visible to the tensor core
    if (threadIdx.x == 0) {
        for (int b = 0; b < 3; ++b) ptx::mbar_init(ptx::smem_u32(bars + b), 1);
        *abort_flag = 0;
        ptx::fence_barrier_init();
    }
    if (warp == 1) {
        if constexpr (kPair) {
            ptx::tmem_alloc_pair(ptx::smem_u32(holder), 512);
            ptx::tmem_relinquish_pair();
        } else {
            ptx::tmem_alloc(ptx::smem_u32(holder), 512);
            ptx::tmem_relinquish();
        }
    }
    ptx::tc_fence_before();
    __syncthreads();
    if constexpr (kPair) ptx::cluster_sync();
    ptx::tc_fence_after();
    const uint32_t tmem = *holder;
    if (kFp4) {   // scale factors 1.0 (UE8M0 0x7F, UE4M3 0x38), one warp per lane quadrant
        const uint32_t lanes = static_cast<uint32_t>(warp * 32) << 16;
        const uint32_t one = kForm == 2 ? 0x38383838u : 0x7F7F7F7Fu;
        ptx::tmem_st_32x32b_x16_fill(tmem + lanes + kPkSfa, one);
        ptx::tmem_st_32x32b_x16_fill(tmem + lanes + kPkSfb, one);
        ptx::tmem_wait_st();
    }
    ptx::tc_fence_before();
    __syncthreads();
    if constexpr (kPair) ptx::cluster_sync();
    ptx::tc_fence_after();

    if (threadIdx.x == 0 && rank == 0) {
        const uint32_t M = kPair ? 2 * kTcBM : kTcBM;
        const uint32_t N = static_cast<uint32_t>(a.n);
        const uint32_t idesc = kForm == 2   ? ptx::idesc_nvf4_f32(M, N)
                               : kForm == 1 ? ptx::idesc_mxf4_f32(M, N)
                                            : ptx::idesc_e4m3_f32(M, N);
        const uint64_t adesc = ptx::smem_desc_kmajor_sw128(ptx::smem_u32(base + kPkAOff));
        const uint64_t bdesc = ptx::smem_desc_kmajor_sw128(ptx::smem_u32(base + kPkBOff));
        const int64_t batches = (a.mmas + kPkBatch - 1) / kPkBatch;
        bool ok = true;
        for (int64_t b = 0; b < batches && ok; ++b) {
#pragma unroll
            for (int kk = 0; kk < kPkBatch; ++kk) {
                const uint64_t off = static_cast<uint64_t>(((kk & 3) * 32) >> 4);
                const uint32_t acc = (b | kk) != 0 ? 1u : 0u;
                if constexpr (kForm == 2 && kPair)
                    ptx::mma_nvf4_pair(tmem, adesc + off, bdesc + off, idesc, tmem + kPkSfa,
                                       tmem + kPkSfb, acc);
                else if constexpr (kForm == 2)
                    ptx::mma_nvf4(tmem, adesc + off, bdesc + off, idesc, tmem + kPkSfa,
                                  tmem + kPkSfb, acc);
                else if constexpr (kFp4 && kPair)
                    ptx::mma_mxf4_pair(tmem, adesc + off, bdesc + off, idesc, tmem + kPkSfa,
                                       tmem + kPkSfb, acc);
                else if constexpr (kFp4)
                    ptx::mma_mxf4(tmem, adesc + off, bdesc + off, idesc, tmem + kPkSfa,
                                  tmem + kPkSfb, acc);
                else if constexpr (kPair)
                    ptx::mma_f8f6f4_pair(tmem, adesc + off, bdesc + off, idesc, acc);
                else
                    ptx::mma_f8f6f4(tmem, adesc + off, bdesc + off, idesc, acc);
            }
            const uint32_t bar = ptx::smem_u32(bars + (b & 1));
            if constexpr (kPair)
                ptx::mma_commit_pair(bar);
            else
                ptx::mma_commit(bar);
            if (b >= 1) {   // at most two batches outstanding
                const int64_t p = b - 1;
                if (!ptx::mbar_wait_bounded(ptx::smem_u32(bars + (p & 1)),
                                            static_cast<uint32_t>((p >> 1) & 1), a.timeout_ns,
                                            abort_flag)) {
                    atomicOr(a.err, kErrTimeoutMma);
                    ok = false;
                }
            }
        }
        // drain every MMA before the tensor memory is freed
        if constexpr (kPair)
            ptx::mma_commit_pair(ptx::smem_u32(bars + 2));
        else
            ptx::mma_commit(ptx::smem_u32(bars + 2));
        const uint64_t d2 = ptx::globaltimer_ns() + a.timeout_ns;
        while (!ptx::mbar_try_wait(ptx::smem_u32(bars + 2), 0)) {
            if (ptx::globaltimer_ns() > d2) {
                atomicOr(a.err, kErrTimeoutDrain);
                break;
            }
        }
    }
    ptx::tc_fence_before();
    __syncthreads();
    if constexpr (kPair) ptx::cluster_sync();
    if (warp == 1) {
        ptx::tc_fence_after();
        if constexpr (kPair)
            ptx::tmem_dealloc_pair(tmem, 512);
        else
            ptx::tmem_dealloc(tmem, 512);
    }
}

template <int kForm, bool kPair>
cudaError_t launch_peak(const PeakArgs& a, int grid, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(mma_peak_kernel<kForm, kPair>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kPkSmem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3(static_cast<unsigned>(grid), 1, 1);
    cfg.blockDim = dim3(128, 1, 1);
    cfg.dynamicSmemBytes = kPkSmem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kPair ? 2 : 1;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, mma_peak_kernel<kForm, kPair>, a);
}

}  // namespace
}  // namespace gbmi

using namespace gbmi;

extern "C" gbmi_status gbmi_mma_peak(int fp4, int pair, int n, int64_t mmas, double* flops_per_s,
                                     double* ms) {
    std::lock_guard<std::recursive_mutex> lk(rt::g_mu);
    if (flops_per_s == nullptr) return rt::fail(GBMI_ERR_ARG, "flops_per_s is null");
    if (mmas < 1 || mmas > (int64_t{1} << 32)) return rt::fail(GBMI_ERR_ARG, "mmas out of range");
    if (fp4 < 0 || fp4 > 2) return rt::fail(GBMI_ERR_ARG, "fp4 must be 0, 1 or 2");
    if (n < 16 || n > kTcBNMax || n % 16 != 0)
        return rt::fail(GBMI_ERR_ARG, "n must be a multiple of 16 in [16, 256]");
    rt::DeviceCtx* c = nullptr;
    GBMI_TRY(rt::get_ctx(&c));
    GBMI_TRY(rt::ensure(c->peak_err, 256, "error word"));
    cudaStream_t s = rt::g_stream;
    GBMI_CUDA(cudaMemsetAsync(c->peak_err.p, 0, 4, s), "memset");
    PeakArgs a;
    a.mmas = mmas;
    a.n = n;
    a.err = static_cast<unsigned int*>(c->peak_err.p);
    a.timeout_ns = rt::g_opt.timeout_ns;
    const int grid = pair ? (c->sm_count / 2) * 2 : c->sm_count;
    cudaEvent_t e0, e1;
    GBMI_CUDA(cudaEventCreate(&e0), "event");
    GBMI_CUDA(cudaEventCreate(&e1), "event");
    cudaEventRecord(e0, s);
    cudaError_t e;
    if (fp4 == 2)
        e = pair ? launch_peak<2, true>(a, grid, s) : launch_peak<2, false>(a, grid, s);
    else if (fp4)
        e = pair ? launch_peak<1, true>(a, grid, s) : launch_peak<1, false>(a, grid, s);
    else
        e = pair ? launch_peak<0, true>(a, grid, s) : launch_peak<0, false>(a, grid, s);
    if (e == cudaSuccess) rt::g_launches.fetch_add(1, std::memory_order_relaxed);
    cudaEventRecord(e1, s);
    cudaError_t e2 = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess && e2 == cudaSuccess) cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return rt::cuda_fail(e, "mma_peak");
    if (e2 != cudaSuccess) return rt::cuda_fail(e2, "mma_peak");
    unsigned int herr = 0;
    GBMI_CUDA(cudaMemcpyAsync(&herr, c->peak_err.p, 4, cudaMemcpyDeviceToHost, s), "copy");
    GBMI_CUDA(cudaStreamSynchronize(s), "sync");
    if (herr != 0) return rt::fail(GBMI_ERR_TIMEOUT, "a bounded device-side wait timed out");
    const double M = pair ? 2.0 * kTcBM : kTcBM, K = fp4 ? 64.0 : 32.0;
    const double issuers = pair ? grid / 2 : grid;
    const double flops = 2.0 * M * n * K * static_cast<double>((mmas + kPkBatch - 1) / kPkBatch *
                                                              kPkBatch) * issuers;
    *flops_per_s = t > 0.f ? flops / (static_cast<double>(t) * 1e-3) : 0.0;
    if (ms != nullptr) *ms = t;
    return GBMI_OK;
}
