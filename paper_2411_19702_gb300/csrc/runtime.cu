// Host runtime shared by the C-ABI translation units (see runtime.h).
#include <cstdio>
#include <cstdlib>
#include "runtime.h"

#include <algorithm>
#include <cmath>
#include <map>

namespace gbmi {

namespace {
thread_local std::string t_last_error;
}  // namespace

void set_last_error(const char* msg) { t_last_error = msg; }

namespace rt {

std::recursive_mutex g_mu;
Options g_opt;

namespace {
// GBMI_LOG=1: every error text is also written to stderr.
bool log_errors() {
    static const bool on = [] {
        const char* e = std::getenv("GBMI_LOG");
        return e != nullptr && std::atoi(e) > 0;
    }();
    return on;
}

// Option defaults from the environment (GBMI_FIXUP, GBMI_TILE_N, GBMI_PAIR,
// GBMI_DIRECT, GBMI_FP4, GBMI_TIMEOUT_NS, GBMI_GROUP_COLS, GBMI_MAX_CTAS,
// GBMI_TAIL_SPLIT), read once
// when the library loads; values out of range are ignored.
struct EnvOptions {
    EnvOptions() {
        auto num = [](const char* name, long long lo, long long hi, long long* out) {
            const char* e = std::getenv(name);
            if (e == nullptr || *e == '\0') return false;
            char* end = nullptr;
            const long long v = std::strtoll(e, &end, 10);
            if (end == e || *end != '\0' || v < lo || v > hi) {
                if (log_errors()) std::fprintf(stderr, "gbmi: ignoring %s=%s\n", name, e);
                return false;
            }
            *out = v;
            return true;
        };
        long long v = 0;
        if (num("GBMI_FIXUP", 0, 1, &v)) g_opt.fixup = static_cast<int>(v);
        if (num("GBMI_TILE_N", 0, 256, &v) && (v == 0 || v == 64 || v == 128 || v == 256))
            g_opt.tile_n = static_cast<int>(v);
        if (num("GBMI_PAIR", 0, 2, &v)) g_opt.pair = static_cast<int>(v);
        if (num("GBMI_DIRECT", 0, 1, &v)) g_opt.direct = static_cast<int>(v);
        if (num("GBMI_FP4", 0, 1, &v)) g_opt.fp4 = static_cast<int>(v);
        if (num("GBMI_TIMEOUT_NS", 1000, 600000000000LL, &v))
            g_opt.timeout_ns = static_cast<uint64_t>(v);
        if (num("GBMI_GROUP_COLS", 1, 1 << 20, &v)) g_opt.group_cols = static_cast<int>(v);
        if (num("GBMI_MAX_CTAS", 0, 1 << 20, &v)) g_opt.max_ctas = static_cast<int>(v);
        if (num("GBMI_TAIL_SPLIT", 0, 15, &v)) g_opt.tail_split = static_cast<int>(v);
        if (num("GBMI_TAIL_COLS", 0, 4, &v)) g_opt.tail_cols = static_cast<int>(v);
    }
};
EnvOptions g_env_options;
}  // namespace
cudaStream_t g_stream = nullptr;
std::atomic<uint64_t> g_launches{0};

namespace {

constexpr int kMaxDevices = 64;
DeviceCtx g_dev[kMaxDevices];
// Largest m whose n*log2(n) table is kept in device memory (1 GiB); beyond it
// the FP64 combine evaluates k*log2(k) inline.
constexpr int64_t kMaxTableM = int64_t{1} << 27;

// ---------------------------------------------------------------- profiler
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

// ---------------------------------------------------------------- tuner table
// per (m, n) bucket: the single-CTA tile width (0: not tuned), the kernel
// (-1: the built-in rule, 0: single-CTA tiles, 1: CTA pairs) and the sample
// split of a Gram with fewer tiles than concurrent slots (0: the cost model,
// 1: no split, S >= 2: S sample ranges where feasible)
struct TunerEntry {
    int bn = 0;
    int pair = -1;
    int split = 0;
};
std::map<std::pair<int, int>, TunerEntry> g_tuner;

std::pair<int, int> bucket(int64_t m, int64_t n) {
    const int mb = static_cast<int>(std::floor(std::log2(static_cast<double>(std::max<int64_t>(m, 1)))));
    const int nb = static_cast<int>(
        std::floor(2.0 * std::log2(static_cast<double>(std::max<int64_t>(n, 1)))));
    return {mb, nb};
}

}  // namespace

gbmi_status fail(gbmi_status s, const std::string& msg) {
    t_last_error = msg;
    if (log_errors()) std::fprintf(stderr, "gbmi: %s\n", msg.c_str());
    return s;
}

gbmi_status cuda_fail(cudaError_t e, const char* what) {
    return fail(e == cudaErrorMemoryAllocation ? GBMI_ERR_OOM : GBMI_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

gbmi_status ensure(DevBuf& b, size_t bytes, const char* what) {
    if (bytes == 0) bytes = 256;
    if (b.cap >= bytes) return GBMI_OK;
    if (g_opt.debug_flags & 2)   // test hook: every new workspace allocation fails
        return fail(GBMI_ERR_OOM, std::string("device allocation of ") + std::to_string(bytes) +
                                      " bytes for " + what + " refused (injected failure)");
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
        return fail(GBMI_ERR_OOM, std::string("device allocation of ") + std::to_string(bytes) +
                                      " bytes for " + what + " failed: " + cudaGetErrorString(e));
    }
    b.cap = bytes;
    return GBMI_OK;
}

void release(DevBuf& b) {
    if (b.p != nullptr) cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
}

DeviceCtx* ctx_of(int dev) {
    if (dev < 0 || dev >= kMaxDevices) return nullptr;
    return &g_dev[dev];
}

gbmi_status get_ctx(DeviceCtx** out) {
    int dev = 0;
    GBMI_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices)
        return fail(GBMI_ERR_UNSUPPORTED, "device ordinal too large");
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
        c.pair_clusters = gram_tc_pair_clusters();
        GBMI_TRY(ensure(c.err, 256, "error word"));
        GBMI_CUDA(cudaMemset(c.err.p, 0, 256), "cudaMemset");
        c.ready = true;
    }
    *out = &c;
    return GBMI_OK;
}

cudaEvent_t prof_begin(cudaStream_t s) {
    if (!g_profile) return nullptr;
    cudaEvent_t e = take_event();
    if (e) cudaEventRecord(e, s);
    return e;
}

void prof_end(const char* name, cudaEvent_t a, cudaStream_t s) {
    if (!g_profile || a == nullptr) return;
    cudaEvent_t b = take_event();
    if (b == nullptr) return;
    cudaEventRecord(b, s);
    g_prof_pending.push_back({name, a, b});
}

void prof_set(bool on) { g_profile = on; }

void prof_collect() {
    for (const ProfPending& p : g_prof_pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(p.b) == cudaSuccess &&
            cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
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

int prof_entries() { return static_cast<int>(g_prof_agg.size()); }
const char* prof_name(int k) {
    return (k >= 0 && k < prof_entries()) ? g_prof_agg[k].name.c_str() : "";
}
double prof_ms(int k) { return (k >= 0 && k < prof_entries()) ? g_prof_agg[k].ms : 0.0; }
int64_t prof_launches(int k) {
    return (k >= 0 && k < prof_entries()) ? g_prof_agg[k].launches : 0;
}
void prof_reset() {
    prof_collect();
    g_prof_agg.clear();
}

MiParams mi_params_plain(int64_t m, int fixup, const double* T) {
    MiParams P;
    P.m = static_cast<int32_t>(m);
    P.fm = static_cast<float>(m);
    P.inv_m_ln2 = static_cast<float>(1.0 / (static_cast<double>(m) * std::log(2.0)));
    P.inv_m = static_cast<float>(1.0 / static_cast<double>(m));
    P.fixup = fixup ? 1 : 0;
    P.fixup_below = 1e-4f;
    // chi^2-divergence bound under which MI (bits) is surely below 1e-4; the
    // factor keeps FP32 rounding of the bound on the safe side
    P.chi_below = static_cast<float>(1e-4 * std::log(2.0) * (1.0 - 1e-4));
    P.T = T;
    return P;
}

gbmi_status mi_params(DeviceCtx& c, int64_t m, MiParams* P) {
    *P = mi_params_plain(m, g_opt.fixup, nullptr);
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

int choose_bn(int64_t m, int64_t n_a, int64_t n_b, bool symmetric) {
    if (g_opt.tile_n == 64 || g_opt.tile_n == 128 || g_opt.tile_n == 256) return g_opt.tile_n;
    const auto it = g_tuner.find(bucket(m, std::max(n_a, n_b)));
    if (it != g_tuner.end() && it->second.bn != 0) return it->second.bn;
    // operand traffic: every tile streams 128 + bn rows for each sample block
    int best = 256;
    double best_cost = -1.0;
    for (int bn : {256, 128, 64}) {
        const double cost =
            static_cast<double>(gram_tile_count(n_a, n_b, bn, symmetric)) * (kTcBM + bn);
        if (best_cost < 0.0 || cost < best_cost * 0.97) {   // prefer wide tiles on near-ties
            best = bn;
            best_cost = cost;
        }
    }
    return best;
}

void tuner_set(int64_t m, int64_t n, int bn) { g_tuner[bucket(m, n)].bn = bn; }
void tuner_set_pair(int64_t m, int64_t n, int pair) { g_tuner[bucket(m, n)].pair = pair; }
int tuner_pair(int64_t m, int64_t n) {
    const auto it = g_tuner.find(bucket(m, n));
    return it != g_tuner.end() ? it->second.pair : -1;
}
void tuner_set_split(int64_t m, int64_t n, int parts) { g_tuner[bucket(m, n)].split = parts; }
int tuner_split(int64_t m, int64_t n) {
    const auto it = g_tuner.find(bucket(m, n));
    return it != g_tuner.end() ? it->second.split : 0;
}
void tuner_clear() { g_tuner.clear(); }
int tuner_size() { return static_cast<int>(g_tuner.size()); }

int grid_for(const DeviceCtx& c, int64_t tiles) {
    int64_t g = c.sm_count;
    if (g_opt.max_ctas > 0) g = std::min<int64_t>(g, g_opt.max_ctas);
    return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(g, tiles)));
}

}  // namespace rt

namespace {
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

bool encode_box(CUtensorMap* tm, const uint8_t* P, int64_t total_rows, int box_rows) {
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (fn == nullptr) return false;
    cuuint64_t dims[2] = {static_cast<cuuint64_t>(kTcBK), static_cast<cuuint64_t>(total_rows)};
    cuuint64_t strides[1] = {static_cast<cuuint64_t>(kTcBK)};
    cuuint32_t box[2] = {static_cast<cuuint32_t>(kTcBK), static_cast<cuuint32_t>(box_rows)};
    cuuint32_t estr[2] = {1, 1};
    return fn(tm, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<uint8_t*>(P), dims, strides, box,
              estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}
// A row-major m x n uint8 matrix as a 2-D tensor (x = variable, y = sample)
// with boxes of 128 variables x 128 samples.
bool encode_direct(CUtensorMap* tm, const uint8_t* X, int64_t m, int64_t n) {
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (fn == nullptr || n % 16 != 0 || (reinterpret_cast<uintptr_t>(X) & 15u) != 0) return false;
    cuuint64_t dims[2] = {static_cast<cuuint64_t>(n), static_cast<cuuint64_t>(m)};
    cuuint64_t strides[1] = {static_cast<cuuint64_t>(n)};
    cuuint32_t box[2] = {static_cast<cuuint32_t>(kTcBM), static_cast<cuuint32_t>(kTcBK)};
    cuuint32_t estr[2] = {1, 1};
    return fn(tm, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<uint8_t*>(X), dims, strides, box,
              estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}
}  // namespace

const char* last_error_text() { return t_last_error.c_str(); }

bool make_direct_maps(OperandMaps* maps, const uint8_t* X, int64_t m, int64_t n1,
                      const uint8_t* Y, int64_t n2) {
    if (m <= 0 || m >= (int64_t{1} << 31)) return false;
    return encode_direct(&maps->xa, X, m, n1) && encode_direct(&maps->xb, Y, m, n2);
}

bool make_operand_maps(OperandMaps* maps, const uint8_t* P, int64_t total_rows) {
    if (total_rows <= 0 || total_rows >= (int64_t{1} << 31)) return false;
    return encode_box(&maps->box64, P, total_rows, 64) &&
           encode_box(&maps->box120, P, total_rows, 120) &&
           encode_box(&maps->box128, P, total_rows, 128) &&
           encode_box(&maps->box256, P, total_rows, 256);
}

}  // namespace gbmi

extern "C" const char* gbmi_last_error_string(void) { return gbmi::last_error_text(); }
