// mi_all_pairs_noalloc: all-pairs MI for callers that cannot allocate device
// memory.
//
// Who needs this: code that runs where cudaMalloc/cudaFree are not allowed
// or not wanted.  Examples are a host framework that owns the whole device
// memory through its own pool and forbids stray allocations, a
// latency-critical loop where cudaFree's implicit device-wide
// synchronisation is unacceptable, and a process under a hard device-memory
// cap that must not grow.  The regular entry points keep a grow-only
// workspace and so may allocate on their first call or when sizes grow; this
// one never does.
//
// How: every buffer the fused tensor-core path needs besides the caller's
// input and output (the packed FP4 operand, the column counts, the
// per-variable epilogue terms, the tile list and the device error word)
// lives in one file-scope device array of kScratchBytes.  The array belongs
// to this library's module, so every GPU that loads the module holds it until
// the process exits.  Its device address is looked up once per device, with
// that device current, on the first call made on that device; that first call
// should therefore come before any stream capture.  Problems whose scratch
// need exceeds the array are rejected with GBMI_ERR_ARG.
//
// All calls share the array, and the array keeps the previous call's
// contents; this file clears what must start at zero (the column counts and
// the error word) on every call.  Two calls whose work overlaps on the GPU
// (other host threads, other streams) race on the array.  The call waits for
// its own work before returning, so sequential calls from one thread are safe.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "gbmi.h"
#include "internal.cuh"
#include "runtime.h"

namespace gbmi {
namespace {

constexpr size_t kScratchBytes = size_t{64} << 20;   // 64 MiB
constexpr int kMaxDev = 64;
constexpr int kTileN = kTcBNFp4;                     // tile width (FP4 operands: 240)
constexpr int kGroupCols = 8;

static __device__ __align__(256) uint8_t g_noalloc_scratch[kScratchBytes];

std::mutex g_na_mu;
bool g_na_ready[kMaxDev] = {};
uint8_t* g_na_ptr[kMaxDev] = {};
int g_na_sms[kMaxDev] = {};

// The message is readable through gbmi_last_error_string() on this thread.
gbmi_status na_fail(gbmi_status s, const std::string& msg) {
    set_last_error(msg.c_str());
    return s;
}

size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

// The fused kernel's upper-triangle tile order (groups of column blocks, all
// row blocks of a group before the next group), written by one thread.
__global__ void noalloc_tiles_kernel(GramTile* tiles, int TI, int TJ, int bn, int group) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    int k = 0;
    for (int g0 = 0; g0 < TJ; g0 += group) {
        const int g1 = min(TJ, g0 + group);
        for (int I = 0; I < TI; ++I)
            for (int J = g0; J < g1; ++J)
                if (I * kTcBM <= J * bn + bn - 1) tiles[k++] = GramTile{0, I, J, 0};
    }
}

gbmi_status na_setup(int* dev_out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return na_fail(GBMI_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDev) return na_fail(GBMI_ERR_UNSUPPORTED, "device ordinal too large");
    if (!g_na_ready[dev]) {
        int major = 0, minor = 0;
        cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
        if (major != 10 || minor != 3)
            return na_fail(GBMI_ERR_UNSUPPORTED, "needs a compute capability 10.3 GPU");
        e = cudaDeviceGetAttribute(&g_na_sms[dev], cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return na_fail(GBMI_ERR_CUDA, cudaGetErrorString(e));
        e = gram_tc_prepare();
        if (e != cudaSuccess) return na_fail(GBMI_ERR_CUDA, cudaGetErrorString(e));
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr)
            return na_fail(GBMI_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") +
                                              cudaGetErrorString(e));
        g_na_ptr[dev] = static_cast<uint8_t*>(p);
        g_na_ready[dev] = true;
    }
    *dev_out = dev;
    return GBMI_OK;
}

}  // namespace
}  // namespace gbmi

using namespace gbmi;

extern "C" gbmi_status mi_all_pairs_noalloc(const uint8_t* X, int64_t m, int64_t n, float* out) {
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (X == nullptr || out == nullptr) return na_fail(GBMI_ERR_ARG, "null pointer");
    if (m < 1 || m > (int64_t{1} << 24))
        return na_fail(GBMI_ERR_ARG, "mi_all_pairs_noalloc needs 1 <= m <= 2^24");
    if (n < 1 || n > (int64_t{1} << 20)) return na_fail(GBMI_ERR_ARG, "n out of range");

    // scratch layout: error word | v | per-variable terms | tile list | packed operand
    const int64_t rows_p = pack_rows(n), kb = pack_ld_of(m, true) / kKbSamplesFp4;
    const int TI = static_cast<int>((n + kTcBM - 1) / kTcBM);
    const int TJ = static_cast<int>((n + kTileN - 1) / kTileN);
    const int64_t ntiles = gram_tile_count(n, n, kTileN, true);
    const size_t off_err = 0;
    const size_t off_v = off_err + 256;
    const size_t off_var = off_v + align256(static_cast<size_t>(n) * 4);
    const size_t off_tiles = off_var + align256(static_cast<size_t>(n) * sizeof(MiVar));
    const size_t off_p = off_tiles + align256(static_cast<size_t>(ntiles) * sizeof(GramTile));
    const size_t need = off_p + static_cast<size_t>(kb * rows_p) * kTcBK;
    if (need > kScratchBytes)
        return na_fail(GBMI_ERR_ARG, "problem needs " + std::to_string(need) +
                                         " bytes of scratch; mi_all_pairs_noalloc holds " +
                                         std::to_string(kScratchBytes) + " (64 MiB)");
    const uintptr_t xa = reinterpret_cast<uintptr_t>(X), oa = reinterpret_cast<uintptr_t>(out);
    const size_t xb = static_cast<size_t>(m) * n, ob = static_cast<size_t>(n) * n * 4;
    if (xa < oa + ob && oa < xa + xb) return na_fail(GBMI_ERR_ARG, "out overlaps X");

    int dev = 0;
    gbmi_status st = na_setup(&dev);
    if (st != GBMI_OK) return st;
    uint8_t* base = g_na_ptr[dev];
    unsigned int* err = reinterpret_cast<unsigned int*>(base + off_err);
    int32_t* v = reinterpret_cast<int32_t*>(base + off_v);
    MiVar* vars = reinterpret_cast<MiVar*>(base + off_var);
    GramTile* tiles = reinterpret_cast<GramTile*>(base + off_tiles);
    uint8_t* P = base + off_p;
    cudaStream_t s = static_cast<cudaStream_t>(gbmi_get_stream());

    // what must start at zero: the error word and the column counts
    cudaError_t e = cudaMemsetAsync(base, 0, off_var, s);
    if (e != cudaSuccess) return na_fail(GBMI_ERR_CUDA, cudaGetErrorString(e));

    PackJob pj;
    std::memset(&pj, 0, sizeof(pj));
    pj.X = X;
    pj.m = m;
    pj.n = n;
    pj.ldx = n;
    pj.P = P;
    pj.v = v;
    pj.rows_p = rows_p;
    pj.ldp = kb * kKbSamplesFp4;
    pj.fp4 = 1;
    if ((e = launch_pack(pj, s)) != cudaSuccess) return na_fail(GBMI_ERR_CUDA, cudaGetErrorString(e));

    MiParams mp;
    mp.m = static_cast<int32_t>(m);
    mp.fm = static_cast<float>(m);
    mp.inv_m_ln2 = static_cast<float>(1.0 / (static_cast<double>(m) * std::log(2.0)));
    mp.inv_m = static_cast<float>(1.0 / static_cast<double>(m));
    mp.fixup = 0;   // FP32 epilogue only: the FP64 combine needs a table this call cannot hold
    mp.fixup_below = 1e-4f;
    mp.chi_below = 0.f;
    mp.T = nullptr;
    if ((e = launch_mi_vars(v, n, mp, vars, s)) != cudaSuccess)
        return na_fail(GBMI_ERR_CUDA, cudaGetErrorString(e));
    noalloc_tiles_kernel<<<1, 1, 0, s>>>(tiles, TI, TJ, kTileN, kGroupCols);
    if ((e = cudaGetLastError()) != cudaSuccess) return na_fail(GBMI_ERR_CUDA, cudaGetErrorString(e));

    OperandMaps maps;
    if (!make_operand_maps(&maps, P, kb * rows_p))
        return na_fail(GBMI_ERR_CUDA, "cuTensorMapEncodeTiled failed");
    GramLaunch L;
    std::memset(&L, 0, sizeof(L));
    GramJob& g = L.job0;
    g.rowA = 0;
    g.rowB = 0;
    g.strideA = rows_p;
    g.strideB = rows_p;
    g.k_begin = 0;
    g.k_blocks = static_cast<int32_t>(kb);
    g.n_a = static_cast<int32_t>(n);
    g.n_b = static_cast<int32_t>(n);
    g.symmetric = 1;
    g.bn = kTileN;
    g.va = vars;
    g.vb = vars;
    g.out_f = out;
    g.ld_out = n;
    g.mp = mp;
    L.jobs = nullptr;
    L.tiles = tiles;
    L.num_tiles = static_cast<int>(ntiles);
    L.mode = kTcModeMI;
    L.fp4 = 1;
    L.err = err;
    L.timeout_ns = rt::g_opt.timeout_ns;   // GBMI_OPT_TIMEOUT_NS, as for every other launch
    const int grid = static_cast<int>(std::min<int64_t>(g_na_sms[dev], ntiles));
    if ((e = launch_gram_tc(maps, L, grid, s)) != cudaSuccess)
        return na_fail(GBMI_ERR_CUDA, cudaGetErrorString(e));

    // the error word comes back on the library stream: one wait for this
    // call's own work, not for other streams of the device
    unsigned int host_err = 0;
    if ((e = cudaMemcpyAsync(&host_err, err, sizeof(host_err), cudaMemcpyDeviceToHost, s)) !=
        cudaSuccess)
        return na_fail(GBMI_ERR_CUDA, cudaGetErrorString(e));
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess)
        return na_fail(GBMI_ERR_CUDA, cudaGetErrorString(e));
    if (host_err != 0) return na_fail(GBMI_ERR_TIMEOUT, "a bounded device-side wait timed out");
    return GBMI_OK;
}
