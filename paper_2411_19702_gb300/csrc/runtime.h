// Host runtime shared by the C-ABI translation units: per-device workspace,
// options, the current stream, error text, the launch profiler and counter,
// the tile-width choice (tuner table or cost model) and TMA descriptors.
#pragma once

#include <cudaTypedefs.h>
#include <nvtx3/nvToolsExt.h>

#include <atomic>
#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include "gbmi.h"
#include "internal.cuh"

namespace gbmi {
namespace rt {

struct DevBuf {
    void* p = nullptr;
    size_t cap = 0;
};

struct Options {
    int fixup = 0;                       // FP64 combine off: the FP32 h-form has no cancellation
    uint64_t timeout_ns = 2000000000ull;
    int debug_flags = 0;
    int group_cols = 8;
    int max_ctas = 0;
    int tile_n = 0;                      // 0: tuner table / cost model; else forced 64/128/256
    int direct = 0;                      // 1: no pack where X's rows are 16-byte multiples
    int pair = 1;                        // 1: CTA-pair (cta_group::2) Gram where it fills the GPU
    int csr_path = 0;                    // CSR input: 0 cost model, 1 pair enumeration, 2 dense
    int split_k = 0;                     // sample split of few-tile Grams: 0 auto, 1 off, 2 forced
    int fp4 = 1;                         // tensor-core operands in the FP4 form (block-scaled MMA)
    int tail_split = 0;                  // fused MI launch: last tiles in K-share units (off)
    int tail_cols = 1;                   // last partial wave in column shares (automatic)
};

struct DeviceCtx {
    bool ready = false;
    int sm_count = 0;
    DevBuf P, Ba, Bb, va, vb, ha, hb, counts, T, err, tiles, Xs, Ys, outs, flag;
    DevBuf peak_err;   // error word of the tensor-core throughput probe
    DevBuf sched;   // tile counter of the Gram launches (zeroed before each launch)
    // split Gram (sample ranges as jobs): job table and tile list, host copies kept
    // alive for the asynchronous uploads
    DevBuf split_jobs, split_tiles, split_part;   // split_part: the parts' count slices
    std::vector<GramJob> split_jobs_host;
    std::vector<GramTile> split_tiles_host;
    int64_t T_len = 0;
    // tile-list cache of the single-dataset path
    int64_t tl_na = -1, tl_nb = -1;
    int tl_sym = -1, tl_group = -1, tl_bn = -1, tl_bm = -1;
    int pair_clusters = 0;   // CTA pairs of the pair Gram kernel resident at once
    // host-buffer pipeline: copy stream, chunk events, panel counters / targets
    // and mapped host flags of panel completion
    cudaStream_t copy_stream = nullptr;
    std::vector<cudaEvent_t> events;
    DevBuf panel;
    unsigned int* hflags = nullptr;   // mapped pinned host memory
    unsigned int* dflags = nullptr;   // its device address
    int hflags_cap = 0;
    std::vector<GramTile> tl_host;
    int64_t tl_gen = 0;   // bumped whenever tl_host is rebuilt
    // split tile list of the fused MI launch (the cached list with its last
    // tiles as K-share units), keyed by the cached list's generation and the split
    DevBuf tail_tiles, part_counts, part_arrive;
    std::vector<GramTile> ts_host;
    int64_t ts_key_gen = -1;
    int ts_key_s = -1, ts_key_p = -1;
    // the cached list with its last tiles as column shares, keyed likewise
    DevBuf col_tiles;
    std::vector<GramTile> tc_host;
    int64_t tc_key_gen = -1;
    int tc_key_s = -1, tc_key_p = -1;
};

extern std::recursive_mutex g_mu;
extern Options g_opt;
extern cudaStream_t g_stream;
extern std::atomic<uint64_t> g_launches;

gbmi_status fail(gbmi_status s, const std::string& msg);
gbmi_status cuda_fail(cudaError_t e, const char* what);
gbmi_status ensure(DevBuf& b, size_t bytes, const char* what);
void release(DevBuf& b);
gbmi_status get_ctx(DeviceCtx** out);
DeviceCtx* ctx_of(int dev);

// profiler hooks around each kernel launch (active with GBMI_OPT_PROFILE)
cudaEvent_t prof_begin(cudaStream_t s);
void prof_end(const char* name, cudaEvent_t a, cudaStream_t s);
void prof_set(bool on);
void prof_collect();
int prof_entries();
const char* prof_name(int k);
double prof_ms(int k);
int64_t prof_launches(int k);
void prof_reset();

// MI parameters of m samples (allocates / extends the n log n table when the
// FP64 combine is on).
gbmi_status mi_params(DeviceCtx& c, int64_t m, MiParams* P);
MiParams mi_params_plain(int64_t m, int fixup, const double* T);

// Tile width (B rows per tile, 64/128/256) for a problem: GBMI_OPT_TILE_N if
// set, else a tuner-table entry for (m, n), else the operand-traffic cost model.
int choose_bn(int64_t m, int64_t n_a, int64_t n_b, bool symmetric);
void tuner_set(int64_t m, int64_t n, int bn);
// Kernel choice of the bucket of (m, n): -1 the built-in rule (untuned), 0
// single-CTA tiles, 1 CTA pairs.
void tuner_set_pair(int64_t m, int64_t n, int pair);
int tuner_pair(int64_t m, int64_t n);
// Sample split of the bucket of (m, n): 0 the cost model (untuned), 1 no
// split, S >= 2 sample ranges.
void tuner_set_split(int64_t m, int64_t n, int parts);
int tuner_split(int64_t m, int64_t n);
void tuner_clear();
int tuner_size();

int grid_for(const DeviceCtx& c, int64_t tiles);

}  // namespace rt
}  // namespace gbmi

#define GBMI_CUDA(call, what)                                         \
    do {                                                              \
        cudaError_t e_ = (call);                                      \
        if (e_ != cudaSuccess) return ::gbmi::rt::cuda_fail(e_, (what)); \
    } while (0)

// One kernel launch: an NVTX range around the enqueue (visible to profilers
// that collect NVTX), the optional event profiler, the launch counter.
#define GBMI_LAUNCH_ON(stream, call, what)                            \
    do {                                                              \
        nvtxRangePushA(what);                                         \
        cudaEvent_t ev0_ = ::gbmi::rt::prof_begin(stream);            \
        cudaError_t e_ = (call);                                      \
        nvtxRangePop();                                               \
        if (e_ != cudaSuccess) return ::gbmi::rt::cuda_fail(e_, (what)); \
        ::gbmi::rt::prof_end((what), ev0_, stream);                   \
        ::gbmi::rt::g_launches.fetch_add(1, std::memory_order_relaxed); \
    } while (0)

#define GBMI_LAUNCH(call, what) GBMI_LAUNCH_ON(::gbmi::rt::g_stream, call, what)

#define GBMI_TRY(expr)                       \
    do {                                     \
        gbmi_status s_ = (expr);             \
        if (s_ != GBMI_OK) return s_;        \
    } while (0)
