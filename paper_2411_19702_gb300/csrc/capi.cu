// C ABI of libgbmi.so: argument checks, the grow-only device workspace, the
// tile list of the tensor-core Gram and the dispatch between the fused,
// plain and popcount paths.  Every computation step runs in this library's
// kernels; the host only validates, allocates, encodes TMA descriptors and
// launches.
#include <cudaTypedefs.h>

#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "gbmi.h"
#include "internal.cuh"

namespace gbmi {
namespace {

// Largest m whose n*log2(n) table is kept in device memory (1 GiB); beyond it
// the FP64 combine evaluates k*log2(k) inline.
constexpr int64_t kMaxTableM = int64_t{1} << 27;
// Samples accumulated by one Gram launch: FP32 holds every count exactly.
constexpr int64_t kExactChunk = int64_t{1} << 24;
// AUTO uses the popcount path when the Gram work is this small (m * n * n).
constexpr double kTinyWork = 6.0e7;

thread_local std::string t_last_error;
std::recursive_mutex g_mu;
std::atomic<uint64_t> g_launches{0};
cudaStream_t g_stream = nullptr;

struct Options {
    int fixup = 0;   // FP64 combine off: the FP32 h-form has no cancellation (see mi_device.cuh)
    uint64_t timeout_ns = 2000000000ull;
    int debug_flags = 0;
    int group_cols = 8;
    int max_ctas = 0;
} g_opt;

struct DevBuf {
    void* p = nullptr;
    size_t cap = 0;
};

struct DeviceCtx {
    bool ready = false;
    int sm_count = 0;
    DevBuf Pa, Pb, Ba, Bb, va, vb, ha, hb, counts, T, err, tiles, Xs, Ys, outs, flag;  // ha/hb: MiVar
    int64_t T_len = 0;
    // tile-list cache
    int64_t tl_na = -1, tl_nb = -1;
    int tl_sym = -1, tl_group = -1;
    std::vector<int2> tl_host;
};

constexpr int kMaxDevices = 64;
DeviceCtx g_dev[kMaxDevices];

gbmi_status fail(gbmi_status s, const std::string& msg) {
    t_last_error = msg;
    return s;
}

gbmi_status cuda_fail(cudaError_t e, const char* what) {
    t_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? GBMI_ERR_OOM : GBMI_ERR_CUDA;
}

#define GBMI_CUDA(call, what)                                 \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(e_, (what));  \
    } while (0)

// ---------------------------------------------------------------- profiler
// With GBMI_OPT_PROFILE on, every kernel launch is bracketed by two CUDA
// events on the library's stream; gbmi_profile_* sums their elapsed times per
// kernel name once the work has finished.
bool g_profile = false;
struct ProfPending {
    const char* name;
    cudaEvent_t a, b;
};
struct ProfAgg {
    std::string name;
    double ms = 0.0;
    int64_t launches = 0;
};
std::vector<ProfPending> g_prof_pending;
std::vector<ProfAgg> g_prof_agg;
std::vector<cudaEvent_t> g_event_pool;

cudaEvent_t take_event() {
    cudaEvent_t e = nullptr;
    if (!g_event_pool.empty()) {
        e = g_event_pool.back();
        g_event_pool.pop_back();
        return e;
    }
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

cudaEvent_t prof_begin() {
    if (!g_profile) return nullptr;
    cudaEvent_t e = take_event();
    if (e) cudaEventRecord(e, g_stream);
    return e;
}

void prof_end(const char* name, cudaEvent_t a) {
    if (!g_profile || a == nullptr) return;
    cudaEvent_t b = take_event();
    if (b == nullptr) return;
    cudaEventRecord(b, g_stream);
    g_prof_pending.push_back({name, a, b});
}

void prof_collect() {
    for (const ProfPending& p : g_prof_pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) ==
                                                              cudaSuccess) {
            ProfAgg* agg = nullptr;
            for (ProfAgg& x : g_prof_agg)
                if (x.name == p.name) agg = &x;
            if (agg == nullptr) {
                g_prof_agg.push_back(ProfAgg());
                agg = &g_prof_agg.back();
                agg->name = p.name;
            }
            agg->ms += ms;
            agg->launches += 1;
        } else {
            cudaGetLastError();
        }
        g_event_pool.push_back(p.a);
        g_event_pool.push_back(p.b);
    }
    g_prof_pending.clear();
}

#define GBMI_LAUNCH(call, what)                               \
    do {                                                      \
        cudaEvent_t ev0_ = prof_begin();                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(e_, (what));  \
        prof_end((what), ev0_);                               \
        g_launches.fetch_add(1, std::memory_order_relaxed);   \
    } while (0)

#define GBMI_TRY(expr)                       \
    do {                                     \
        gbmi_status s_ = (expr);             \
        if (s_ != GBMI_OK) return s_;        \
    } while (0)

gbmi_status ensure(DevBuf& b, size_t bytes, const char* what) {
    if (bytes == 0) bytes = 256;
    if (b.cap >= bytes) return GBMI_OK;
    if (b.p != nullptr) {
        cudaError_t e = cudaFree(b.p);   // implicitly waits for the device
        b.p = nullptr;
        b.cap = 0;
        if (e != cudaSuccess) return cuda_fail(e, "cudaFree");
    }
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        t_last_error = std::string("workspace allocation of ") + std::to_string(bytes) +
                       " bytes for " + what + " failed: " + cudaGetErrorString(e);
        return GBMI_ERR_OOM;
    }
    b.cap = bytes;
    return GBMI_OK;
}

void release(DevBuf& b) {
    if (b.p != nullptr) cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
}

gbmi_status get_ctx(DeviceCtx** out) {
    int dev = 0;
    GBMI_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(GBMI_ERR_UNSUPPORTED, "device ordinal too large");
    DeviceCtx& c = g_dev[dev];
    if (!c.ready) {
        int major = 0, minor = 0;
        GBMI_CUDA(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev),
                  "cudaDeviceGetAttribute");
        GBMI_CUDA(cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev),
                  "cudaDeviceGetAttribute");
        if (major != 10 || minor != 3)
            return fail(GBMI_ERR_UNSUPPORTED,
                        "libgbmi is built for sm_103a (compute capability 10.3); device has " +
                            std::to_string(major) + "." + std::to_string(minor));
        GBMI_CUDA(cudaDeviceGetAttribute(&c.sm_count, cudaDevAttrMultiProcessorCount, dev),
                  "cudaDeviceGetAttribute");
        GBMI_CUDA(gram_tc_prepare(), "cudaFuncSetAttribute");
        GBMI_TRY(ensure(c.err, 256, "error word"));
        GBMI_CUDA(cudaMemset(c.err.p, 0, 256), "cudaMemset");
        c.ready = true;
    }
    *out = &c;
    return GBMI_OK;
}

bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
    const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
    return x < y + nb && y < x + na;
}

gbmi_status check_sizes(int64_t m, int64_t n1, int64_t n2) {
    if (m < 1 || m > 0x7FFFFFFFLL) return fail(GBMI_ERR_ARG, "m must be in [1, 2^31 - 1]");
    if (n1 < 1 || n2 < 1) return fail(GBMI_ERR_ARG, "the number of variables must be >= 1");
    if (n1 > (int64_t{1} << 26) || n2 > (int64_t{1} << 26))
        return fail(GBMI_ERR_ARG, "the number of variables must be <= 2^26");
    return GBMI_OK;
}

// ------------------------------------------------------------------ pieces

gbmi_status pack(DeviceCtx& c, const uint8_t* X, int64_t m, int64_t n, DevBuf* P, DevBuf* B,
                 DevBuf& v) {
    const int64_t rows_p = pack_rows(n), ldp = pack_ld(m);
    GBMI_TRY(ensure(v, static_cast<size_t>(n) * 4, "column counts"));
    if (P) GBMI_TRY(ensure(*P, static_cast<size_t>(rows_p) * ldp, "FP8 operand"));
    if (B) GBMI_TRY(ensure(*B, static_cast<size_t>(rows_p) * (ldp / 8), "bit-packed operand"));
    GBMI_LAUNCH(launch_zero_u32(v.p, n, g_stream), "zero");
    PackArgs a;
    a.X = X;
    a.m = m;
    a.n = n;
    a.ldx = n;
    a.P = P ? static_cast<uint8_t*>(P->p) : nullptr;
    a.rows_p = rows_p;
    a.ldp = ldp;
    a.Bp = B ? static_cast<uint32_t*>(B->p) : nullptr;
    a.v = static_cast<int32_t*>(v.p);
    GBMI_LAUNCH(launch_pack(a, g_stream), "pack");
    return GBMI_OK;
}

gbmi_status mi_params(DeviceCtx& c, int64_t m, MiParams* P) {
    P->m = static_cast<int32_t>(m);
    P->fm = static_cast<float>(m);
    P->inv_m_ln2 = static_cast<float>(1.0 / (static_cast<double>(m) * std::log(2.0)));
    P->inv_m = static_cast<float>(1.0 / static_cast<double>(m));
    P->fixup = g_opt.fixup ? 1 : 0;
    P->fixup_below = 1e-4f;
    // chi^2-divergence bound under which MI (bits) is surely below 1e-4; the
    // factor keeps FP32 rounding of the bound on the safe side
    P->chi_below = static_cast<float>(1e-4 * std::log(2.0) * (1.0 - 1e-4));
    P->T = nullptr;
    if (P->fixup && m <= kMaxTableM) {
        if (c.T_len < m + 1) {
            int64_t len = std::max<int64_t>(m + 1, std::min<int64_t>(2 * c.T_len, kMaxTableM + 1));
            len = std::max<int64_t>(len, 1 << 16);
            GBMI_TRY(ensure(c.T, static_cast<size_t>(len) * 8, "n log n table"));
            GBMI_LAUNCH(launch_nlogn_table(static_cast<double*>(c.T.p), len, g_stream),
                        "nlogn_table");
            c.T_len = len;
        }
        P->T = static_cast<const double*>(c.T.p);
    }
    return GBMI_OK;
}

// Per-variable epilogue terms (MiVar) from the column counts v.
gbmi_status mi_vars(const int32_t* v, int64_t n, const MiParams& P, DevBuf& out,
                    const MiVar** res) {
    GBMI_TRY(ensure(out, static_cast<size_t>(n) * sizeof(MiVar), "per-variable terms"));
    GBMI_LAUNCH(launch_mi_vars(v, n, P, static_cast<MiVar*>(out.p), g_stream), "mi_vars");
    *res = static_cast<const MiVar*>(out.p);
    return GBMI_OK;
}

// Upper-triangle (symmetric) or full (cross) list of 128 x 256 tiles, in
// groups of group_cols column blocks: all rows of a group before the next.
gbmi_status tile_list(DeviceCtx& c, int64_t n_a, int64_t n_b, bool sym, int* count) {
    const int group = std::max(1, g_opt.group_cols);
    if (!(c.tl_na == n_a && c.tl_nb == n_b && c.tl_sym == (int)sym && c.tl_group == group)) {
        const int64_t TI = (n_a + kTcBM - 1) / kTcBM, TJ = (n_b + kTcBN - 1) / kTcBN;
        std::vector<int2> list;
        for (int64_t g0 = 0; g0 < TJ; g0 += group) {
            const int64_t g1 = std::min<int64_t>(TJ, g0 + group);
            const int64_t i_end = sym ? std::min<int64_t>(TI, 2 * g1) : TI;
            for (int64_t I = 0; I < i_end; ++I)
                for (int64_t J = g0; J < g1; ++J) {
                    if (sym && I > 2 * J + 1) continue;   // entirely below the diagonal
                    list.push_back(make_int2(static_cast<int>(I), static_cast<int>(J)));
                }
        }
        if (list.size() > 0x7FFFFFFF) return fail(GBMI_ERR_ARG, "too many tiles");
        GBMI_TRY(ensure(c.tiles, list.size() * sizeof(int2), "tile list"));
        c.tl_host.swap(list);
        GBMI_CUDA(cudaMemcpyAsync(c.tiles.p, c.tl_host.data(), c.tl_host.size() * sizeof(int2),
                                  cudaMemcpyHostToDevice, g_stream),
                  "tile list upload");
        c.tl_na = n_a;
        c.tl_nb = n_b;
        c.tl_sym = sym;
        c.tl_group = group;
    }
    *count = static_cast<int>(c.tl_host.size());
    return GBMI_OK;
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (fn == nullptr) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

int grid_for(const DeviceCtx& c, int tiles) {
    int g = c.sm_count;
    if (g_opt.max_ctas > 0) g = std::min(g, g_opt.max_ctas);
    return std::max(1, std::min(g, tiles));
}

// Run the tensor-core Gram over [0, m) in exact chunks.  mode MI needs one
// chunk (m <= 2^24); the counts modes add chunk results into out_c.
gbmi_status run_gram(DeviceCtx& c, const DevBuf& Pa, const DevBuf& Pb, int64_t m, int64_t n_a,
                     int64_t n_b, bool sym, int mode, const MiVar* va, const MiVar* vb,
                     const MiParams& mp, float* out_f, int32_t* out_c, int64_t ld_out) {
    const int64_t ldp = pack_ld(m);
    const int64_t rows_a = pack_rows(n_a), rows_b = pack_rows(n_b);
    CUtensorMap tmA, tmB;
    if (!make_operand_tmap(&tmA, static_cast<const uint8_t*>(Pa.p), rows_a, ldp, kTcBM) ||
        !make_operand_tmap(&tmB, static_cast<const uint8_t*>(Pb.p), rows_b, ldp, kTcBN))
        return fail(GBMI_ERR_CUDA, "cuTensorMapEncodeTiled failed");
    int tiles = 0;
    GBMI_TRY(tile_list(c, n_a, n_b, sym, &tiles));
    TcArgs a;
    a.tiles = static_cast<const int2*>(c.tiles.p);
    a.num_tiles = tiles;
    a.n_a = n_a;
    a.n_b = n_b;
    a.symmetric = sym ? 1 : 0;
    a.va = va;
    a.vb = vb;
    a.mp = mp;
    a.out_f = out_f;
    a.out_c = out_c;
    a.ld_out = ld_out;
    const uintptr_t base = reinterpret_cast<uintptr_t>(out_f ? static_cast<void*>(out_f)
                                                             : static_cast<void*>(out_c));
    a.vec_store = (ld_out % 4 == 0 && base % 16 == 0) ? 1 : 0;
    a.err = static_cast<unsigned int*>(c.err.p);
    a.timeout_ns = g_opt.timeout_ns;
    a.debug_flags = g_opt.debug_flags;
    const int64_t kb_total = ldp / kTcBK;
    const int64_t kb_chunk = kExactChunk / kTcBK;
    if (mode == kTcModeMI && kb_total > kb_chunk)
        return fail(GBMI_ERR_ARG, "fused path needs m <= 2^24");
    const int grid = grid_for(c, tiles);
    for (int64_t k0 = 0; k0 < kb_total; k0 += kb_chunk) {
        a.k_begin = static_cast<int>(k0);
        a.k_blocks = static_cast<int>(std::min(kb_chunk, kb_total - k0));
        a.mode = (mode == kTcModeMI) ? kTcModeMI : (k0 == 0 ? kTcModeCounts : kTcModeCountsAdd);
        GBMI_LAUNCH(launch_gram_tc(tmA, tmB, a, grid, g_stream),
                    a.mode == kTcModeMI ? "gram_tc_fused_mi" : "gram_tc_counts");
    }
    return GBMI_OK;
}

int choose_path(int path, int64_t m, int64_t n1, int64_t n2) {
    if (path != GBMI_PATH_AUTO) return path;
    if (static_cast<double>(m) * n1 * n2 <= kTinyWork) return GBMI_PATH_POPCOUNT;
    if (m > kExactChunk) return GBMI_PATH_PLAIN;
    return GBMI_PATH_FUSED;
}

// MI between the variables of X (n1) and Y (n2, or X itself when sym).
gbmi_status mi_impl(const uint8_t* X, const uint8_t* Y, int64_t m, int64_t n1, int64_t n2,
                    float* out, int path, bool sym) {
    if (X == nullptr || out == nullptr || (!sym && Y == nullptr))
        return fail(GBMI_ERR_ARG, "null pointer");
    GBMI_TRY(check_sizes(m, n1, n2));
    const size_t out_bytes = static_cast<size_t>(n1) * n2 * 4;
    if (overlaps(X, static_cast<size_t>(m) * n1, out, out_bytes) ||
        (!sym && overlaps(Y, static_cast<size_t>(m) * n2, out, out_bytes)))
        return fail(GBMI_ERR_ARG, "out overlaps an input");
    if (path < GBMI_PATH_AUTO || path > GBMI_PATH_POPCOUNT) return fail(GBMI_ERR_ARG, "bad path");
    DeviceCtx* cp = nullptr;
    GBMI_TRY(get_ctx(&cp));
    DeviceCtx& c = *cp;
    path = choose_path(path, m, n1, n2);
    if (path == GBMI_PATH_FUSED && m > kExactChunk)
        return fail(GBMI_ERR_ARG, "the fused path needs m <= 2^24; use the plain path");

    const bool popc = path == GBMI_PATH_POPCOUNT;
    GBMI_TRY(pack(c, X, m, n1, popc ? nullptr : &c.Pa, popc ? &c.Ba : nullptr, c.va));
    if (!sym) GBMI_TRY(pack(c, Y, m, n2, popc ? nullptr : &c.Pb, popc ? &c.Bb : nullptr, c.vb));
    MiParams mp;
    GBMI_TRY(mi_params(c, m, &mp));
    const MiVar *va = nullptr, *vbp = nullptr;
    GBMI_TRY(mi_vars(static_cast<const int32_t*>(c.va.p), n1, mp, c.ha, &va));
    if (sym)
        vbp = va;
    else
        GBMI_TRY(mi_vars(static_cast<const int32_t*>(c.vb.p), n2, mp, c.hb, &vbp));

    if (popc) {
        PopcArgs a;
        a.Ba = static_cast<const uint32_t*>(c.Ba.p);
        a.Bb = static_cast<const uint32_t*>(sym ? c.Ba.p : c.Bb.p);
        a.wpr = pack_ld(m) / 32;
        a.n_a = n1;
        a.n_b = n2;
        a.symmetric = sym ? 1 : 0;
        a.va = va;
        a.vb = vbp;
        a.mp = mp;
        a.out_f = out;
        a.out_c = nullptr;
        a.ld_out = n2;
        GBMI_LAUNCH(launch_popcount(a, g_stream), "popcount_gram");
        return GBMI_OK;
    }
    const DevBuf& Pb = sym ? c.Pa : c.Pb;
    if (path == GBMI_PATH_FUSED)
        return run_gram(c, c.Pa, Pb, m, n1, n2, sym, kTcModeMI, va, vbp, mp, out, nullptr, n2);
    // plain: exact counts to HBM, then the elementwise MI kernel
    GBMI_TRY(ensure(c.counts, static_cast<size_t>(n1) * n2 * 4, "count matrix"));
    int32_t* N11 = static_cast<int32_t*>(c.counts.p);
    GBMI_TRY(run_gram(c, c.Pa, Pb, m, n1, n2, sym, kTcModeCounts, va, vbp, mp, nullptr, N11,
                      n2));
    GBMI_LAUNCH(launch_mi_from_counts(N11, n2, va, vbp, n1, n2, mp, out, n2, g_stream),
                "mi_from_counts");
    return GBMI_OK;
}

gbmi_status counts_impl(const uint8_t* X, const uint8_t* Y, int64_t m, int64_t n1, int64_t n2,
                        int32_t* n11, int path, bool sym) {
    if (X == nullptr || n11 == nullptr || (!sym && Y == nullptr))
        return fail(GBMI_ERR_ARG, "null pointer");
    GBMI_TRY(check_sizes(m, n1, n2));
    const size_t out_bytes = static_cast<size_t>(n1) * n2 * 4;
    if (overlaps(X, static_cast<size_t>(m) * n1, n11, out_bytes) ||
        (!sym && overlaps(Y, static_cast<size_t>(m) * n2, n11, out_bytes)))
        return fail(GBMI_ERR_ARG, "output overlaps an input");
    if (path == GBMI_PATH_AUTO || path == GBMI_PATH_FUSED) path = GBMI_PATH_PLAIN;
    if (path != GBMI_PATH_PLAIN && path != GBMI_PATH_POPCOUNT)
        return fail(GBMI_ERR_ARG, "bad path");
    DeviceCtx* cp = nullptr;
    GBMI_TRY(get_ctx(&cp));
    DeviceCtx& c = *cp;
    const bool popc = path == GBMI_PATH_POPCOUNT;
    GBMI_TRY(pack(c, X, m, n1, popc ? nullptr : &c.Pa, popc ? &c.Ba : nullptr, c.va));
    if (!sym) GBMI_TRY(pack(c, Y, m, n2, popc ? nullptr : &c.Pb, popc ? &c.Bb : nullptr, c.vb));
    MiParams mp;
    std::memset(&mp, 0, sizeof(mp));
    mp.m = m;
    if (popc) {
        PopcArgs a;
        std::memset(&a, 0, sizeof(a));
        a.Ba = static_cast<const uint32_t*>(c.Ba.p);
        a.Bb = static_cast<const uint32_t*>(sym ? c.Ba.p : c.Bb.p);
        a.wpr = pack_ld(m) / 32;
        a.n_a = n1;
        a.n_b = n2;
        a.symmetric = sym ? 1 : 0;
        a.mp = mp;
        a.out_c = n11;
        a.ld_out = n2;
        GBMI_LAUNCH(launch_popcount(a, g_stream), "popcount_gram");
        return GBMI_OK;
    }
    return run_gram(c, c.Pa, sym ? c.Pa : c.Pb, m, n1, n2, sym, kTcModeCounts, nullptr, nullptr,
                    mp, nullptr, n11, n2);
}

gbmi_status host_impl(const uint8_t* X, const uint8_t* Y, int64_t m, int64_t n1, int64_t n2,
                      float* out, bool sym) {
    if (X == nullptr || out == nullptr || (!sym && Y == nullptr))
        return fail(GBMI_ERR_ARG, "null pointer");
    GBMI_TRY(check_sizes(m, n1, n2));
    DeviceCtx* cp = nullptr;
    GBMI_TRY(get_ctx(&cp));
    DeviceCtx& c = *cp;
    const size_t xb = static_cast<size_t>(m) * n1, yb = static_cast<size_t>(m) * n2;
    const size_t ob = static_cast<size_t>(n1) * n2 * 4;
    GBMI_TRY(ensure(c.Xs, xb, "input staging"));
    if (!sym) GBMI_TRY(ensure(c.Ys, yb, "input staging"));
    GBMI_TRY(ensure(c.outs, ob, "output staging"));
    GBMI_CUDA(cudaMemcpyAsync(c.Xs.p, X, xb, cudaMemcpyHostToDevice, g_stream), "copy X in");
    if (!sym)
        GBMI_CUDA(cudaMemcpyAsync(c.Ys.p, Y, yb, cudaMemcpyHostToDevice, g_stream), "copy Y in");
    GBMI_TRY(mi_impl(static_cast<const uint8_t*>(c.Xs.p),
                     sym ? nullptr : static_cast<const uint8_t*>(c.Ys.p), m, n1, n2,
                     static_cast<float*>(c.outs.p), GBMI_PATH_AUTO, sym));
    GBMI_CUDA(cudaMemcpyAsync(out, c.outs.p, ob, cudaMemcpyDeviceToHost, g_stream), "copy out");
    GBMI_CUDA(cudaStreamSynchronize(g_stream), "cudaStreamSynchronize");
    unsigned int err = 0;
    GBMI_CUDA(cudaMemcpy(&err, c.err.p, sizeof(err), cudaMemcpyDeviceToHost), "read error word");
    if (err != 0) {
        cudaMemset(c.err.p, 0, sizeof(err));
        return fail(GBMI_ERR_TIMEOUT, "a bounded device-side wait timed out");
    }
    return GBMI_OK;
}

}  // namespace

void set_last_error(const char* msg) { t_last_error = msg; }

bool make_operand_tmap(CUtensorMap* tm, const uint8_t* P, int64_t rows_p, int64_t ldp,
                       int box_rows) {
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (fn == nullptr) return false;
    cuuint64_t dims[2] = {static_cast<cuuint64_t>(ldp), static_cast<cuuint64_t>(rows_p)};
    cuuint64_t strides[1] = {static_cast<cuuint64_t>(ldp)};
    cuuint32_t box[2] = {static_cast<cuuint32_t>(kTcBK), static_cast<cuuint32_t>(box_rows)};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(tm, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<uint8_t*>(P), dims, strides,
                    box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

}  // namespace gbmi

using namespace gbmi;

extern "C" {

gbmi_status mi_all_pairs(const uint8_t* X, int64_t m, int64_t n, float* out) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    return mi_impl(X, nullptr, m, n, n, out, GBMI_PATH_AUTO, true);
}

gbmi_status mi_cross(const uint8_t* X, const uint8_t* Y, int64_t m, int64_t n1, int64_t n2,
                     float* out) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    return mi_impl(X, Y, m, n1, n2, out, GBMI_PATH_AUTO, false);
}

gbmi_status gbmi_mi_all_pairs_path(const uint8_t* X, int64_t m, int64_t n, float* out,
                                   int path) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    return mi_impl(X, nullptr, m, n, n, out, path, true);
}

gbmi_status gbmi_mi_cross_path(const uint8_t* X, const uint8_t* Y, int64_t m, int64_t n1,
                               int64_t n2, float* out, int path) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    return mi_impl(X, Y, m, n1, n2, out, path, false);
}

gbmi_status mi_all_pairs_host(const uint8_t* X, int64_t m, int64_t n, float* out) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    return host_impl(X, nullptr, m, n, n, out, true);
}

gbmi_status mi_cross_host(const uint8_t* X, const uint8_t* Y, int64_t m, int64_t n1, int64_t n2,
                          float* out) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    return host_impl(X, Y, m, n1, n2, out, false);
}

gbmi_status gbmi_counts_all_pairs(const uint8_t* X, int64_t m, int64_t n, int32_t* n11,
                                  int path) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    return counts_impl(X, nullptr, m, n, n, n11, path, true);
}

gbmi_status gbmi_counts_cross(const uint8_t* X, const uint8_t* Y, int64_t m, int64_t n1,
                              int64_t n2, int32_t* n11, int path) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    return counts_impl(X, Y, m, n1, n2, n11, path, false);
}

gbmi_status gbmi_column_counts(const uint8_t* X, int64_t m, int64_t n, int32_t* v) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    if (X == nullptr || v == nullptr) return fail(GBMI_ERR_ARG, "null pointer");
    GBMI_TRY(check_sizes(m, n, n));
    DeviceCtx* cp = nullptr;
    GBMI_TRY(get_ctx(&cp));
    GBMI_LAUNCH(launch_zero_u32(v, n, g_stream), "zero");
    PackArgs a;
    std::memset(&a, 0, sizeof(a));
    a.X = X;
    a.m = m;
    a.n = n;
    a.ldx = n;
    a.rows_p = pack_rows(n);
    a.ldp = pack_ld(m);
    a.v = v;
    GBMI_LAUNCH(launch_pack(a, g_stream), "pack");
    return GBMI_OK;
}

gbmi_status gbmi_mi_from_counts(const int32_t* N11, const int32_t* va, const int32_t* vb,
                                int64_t m, int64_t n1, int64_t n2, float* out) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    if (N11 == nullptr || va == nullptr || vb == nullptr || out == nullptr)
        return fail(GBMI_ERR_ARG, "null pointer");
    GBMI_TRY(check_sizes(m, n1, n2));
    DeviceCtx* cp = nullptr;
    GBMI_TRY(get_ctx(&cp));
    DeviceCtx& c = *cp;
    MiParams mp;
    GBMI_TRY(mi_params(c, m, &mp));
    const MiVar *A = nullptr, *B = nullptr;
    GBMI_TRY(mi_vars(va, n1, mp, c.ha, &A));
    GBMI_TRY(mi_vars(vb, n2, mp, c.hb, &B));
    GBMI_LAUNCH(launch_mi_from_counts(N11, n2, A, B, n1, n2, mp, out, n2, g_stream),
                "mi_from_counts");
    return GBMI_OK;
}

gbmi_status gbmi_validate_binary(const uint8_t* X, int64_t m, int64_t n) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    if (X == nullptr) return fail(GBMI_ERR_ARG, "null pointer");
    GBMI_TRY(check_sizes(m, n, n));
    DeviceCtx* cp = nullptr;
    GBMI_TRY(get_ctx(&cp));
    DeviceCtx& c = *cp;
    GBMI_TRY(ensure(c.flag, 256, "flag"));
    GBMI_LAUNCH(launch_zero_u32(c.flag.p, 1, g_stream), "zero");
    GBMI_LAUNCH(launch_validate(X, m, n, n, static_cast<unsigned int*>(c.flag.p), g_stream),
                "validate");
    unsigned int f = 0;
    GBMI_CUDA(cudaMemcpyAsync(&f, c.flag.p, sizeof(f), cudaMemcpyDeviceToHost, g_stream),
              "read flag");
    GBMI_CUDA(cudaStreamSynchronize(g_stream), "cudaStreamSynchronize");
    return f ? fail(GBMI_ERR_NOT_BINARY, "X has an entry other than 0 or 1") : GBMI_OK;
}

gbmi_status gbmi_set_stream(void* stream) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    g_stream = static_cast<cudaStream_t>(stream);
    return GBMI_OK;
}

void* gbmi_get_stream(void) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    return static_cast<void*>(g_stream);
}

gbmi_status gbmi_set_option(int option, int64_t value) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    switch (option) {
        case GBMI_OPT_FIXUP:
            g_opt.fixup = value != 0;
            return GBMI_OK;
        case GBMI_OPT_TIMEOUT_NS:
            if (value <= 0) return fail(GBMI_ERR_ARG, "timeout must be positive");
            g_opt.timeout_ns = static_cast<uint64_t>(value);
            return GBMI_OK;
        case GBMI_OPT_DEBUG_FLAGS:
            g_opt.debug_flags = static_cast<int>(value);
            return GBMI_OK;
        case GBMI_OPT_GROUP_COLS:
            if (value < 1 || value > 1 << 20) return fail(GBMI_ERR_ARG, "group width out of range");
            g_opt.group_cols = static_cast<int>(value);
            return GBMI_OK;
        case GBMI_OPT_MAX_CTAS:
            if (value < 0) return fail(GBMI_ERR_ARG, "max CTAs must be >= 0");
            g_opt.max_ctas = static_cast<int>(value);
            return GBMI_OK;
        case GBMI_OPT_PROFILE:
            g_profile = value != 0;
            return GBMI_OK;
        default:
            return fail(GBMI_ERR_ARG, "unknown option");
    }
}

gbmi_status gbmi_sync(void) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    GBMI_CUDA(cudaStreamSynchronize(g_stream), "cudaStreamSynchronize");
    int dev = 0;
    GBMI_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices || !g_dev[dev].ready) return GBMI_OK;
    unsigned int err = 0;
    GBMI_CUDA(cudaMemcpy(&err, g_dev[dev].err.p, sizeof(err), cudaMemcpyDeviceToHost),
              "read error word");
    if (err != 0) {
        GBMI_CUDA(cudaMemset(g_dev[dev].err.p, 0, sizeof(err)), "clear error word");
        return fail(GBMI_ERR_TIMEOUT, "a bounded device-side wait timed out (code " +
                                          std::to_string(err) + ")");
    }
    return GBMI_OK;
}

const char* gbmi_last_error_string(void) { return t_last_error.c_str(); }

uint64_t gbmi_launch_count(void) { return g_launches.load(); }

gbmi_status gbmi_shutdown(void) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    int cur = 0;
    if (cudaGetDevice(&cur) != cudaSuccess) return GBMI_OK;
    for (int d = 0; d < kMaxDevices; ++d) {
        DeviceCtx& c = g_dev[d];
        if (!c.ready) continue;
        cudaSetDevice(d);
        cudaDeviceSynchronize();
        for (DevBuf* b : {&c.Pa, &c.Pb, &c.Ba, &c.Bb, &c.va, &c.vb, &c.ha, &c.hb, &c.counts, &c.T,
                          &c.err, &c.tiles, &c.Xs, &c.Ys, &c.outs, &c.flag})
            release(*b);
        c = DeviceCtx();
    }
    cudaSetDevice(cur);
    return GBMI_OK;
}

int gbmi_profile_entries(void) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    prof_collect();
    return static_cast<int>(g_prof_agg.size());
}

const char* gbmi_profile_name(int k) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    if (k < 0 || k >= static_cast<int>(g_prof_agg.size())) return "";
    return g_prof_agg[k].name.c_str();
}

double gbmi_profile_ms(int k) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    if (k < 0 || k >= static_cast<int>(g_prof_agg.size())) return 0.0;
    return g_prof_agg[k].ms;
}

int64_t gbmi_profile_launches(int k) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    if (k < 0 || k >= static_cast<int>(g_prof_agg.size())) return 0;
    return g_prof_agg[k].launches;
}

gbmi_status gbmi_profile_reset(void) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    prof_collect();
    g_prof_agg.clear();
    return GBMI_OK;
}

int gbmi_version(void) { return 100; }

}  // extern "C"
