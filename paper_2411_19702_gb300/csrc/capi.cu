// C ABI of libgbmi.so, single-problem calls: argument checks, packing into
// the device workspace, the tile list and the dispatch between the fused,
// plain and popcount paths.  Every computation step runs in this library's
// kernels; the host only validates, allocates, encodes TMA descriptors and
// launches.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>

#include "runtime.h"

namespace gbmi {
namespace {

using rt::DevBuf;
using rt::DeviceCtx;
using rt::ensure;
using rt::fail;
using rt::g_opt;
using rt::g_stream;

// Samples accumulated by one Gram launch: FP32 holds every count exactly.
constexpr int64_t kExactChunk = int64_t{1} << 24;
// AUTO uses the popcount path when the Gram work is this small (m * n * n).
constexpr double kTinyWork = 6.0e7;

// Status for a non-zero device error word.
gbmi_status error_word_status(unsigned int err) {
    if (err & kErrBadCsr)
        return fail(GBMI_ERR_ARG,
                    "malformed CSR input: a row outside [0, nnz], an index outside [0, n) or "
                    "indices not strictly increasing (those rows were skipped)");
    if (err & kErrBadOperand)
        return fail(GBMI_ERR_ARG, "a direct operand copy was not 16-byte aligned (skipped)");
    if ((err & ~static_cast<unsigned int>(kErrNotBinary)) != 0)
        return fail(GBMI_ERR_TIMEOUT, "a bounded device-side wait timed out (code " +
                                          std::to_string(err) + ")");
    return fail(GBMI_ERR_NOT_BINARY,
                "the direct operand path met a byte other than 0 / 1 (the result is unspecified)");
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

// Pack one operand: the FP8 (fp4: FP4) operand into P (at row p_row of the
// K-block-major buffer) and/or the bit-packed operand into B, and the column
// counts into v.
gbmi_status pack(const uint8_t* X, int64_t m, int64_t n, uint8_t* P, uint32_t* B, int32_t* v,
                 bool fp4 = false) {
    GBMI_LAUNCH(launch_zero_u32(v, n, g_stream), "zero");
    PackJob j;
    std::memset(&j, 0, sizeof(j));
    j.X = X;
    j.m = m;
    j.n = n;
    j.ldx = n;
    j.P = P;
    j.Bp = B;
    j.v = v;
    j.rows_p = pack_rows(n);
    j.ldp = pack_ld_of(m, fp4);
    j.fp4 = fp4 ? 1 : 0;
    GBMI_LAUNCH(launch_pack(j, g_stream), "pack");
    return GBMI_OK;
}

gbmi_status mi_vars(const int32_t* v, int64_t n, const MiParams& P, DevBuf& out,
                    const MiVar** res) {
    GBMI_TRY(ensure(out, static_cast<size_t>(n) * sizeof(MiVar), "per-variable terms"));
    GBMI_LAUNCH(launch_mi_vars(v, n, P, static_cast<MiVar*>(out.p), g_stream), "mi_vars");
    *res = static_cast<const MiVar*>(out.p);
    return GBMI_OK;
}

// Tile list of one job (cached per shape), uploaded to the workspace.
gbmi_status tile_list(DeviceCtx& c, int64_t n_a, int64_t n_b, bool sym, int bn, int* count,
                      int bm = kTcBM) {
    const int group = std::max(1, g_opt.group_cols);
    if (!(c.tl_na == n_a && c.tl_nb == n_b && c.tl_sym == (int)sym && c.tl_group == group &&
          c.tl_bn == bn && c.tl_bm == bm)) {
        const int64_t k = gram_tile_count(n_a, n_b, bn, sym, bm);
        if (k > 0x7FFFFFFF) return fail(GBMI_ERR_ARG, "too many tiles");
        std::vector<GramTile> list(static_cast<size_t>(k));
        gram_tiles(0, n_a, n_b, bn, sym, group, list.data(), bm);
        GBMI_TRY(ensure(c.tiles, list.size() * sizeof(GramTile), "tile list"));
        c.tl_host.swap(list);
        GBMI_CUDA(cudaMemcpyAsync(c.tiles.p, c.tl_host.data(),
                                  c.tl_host.size() * sizeof(GramTile), cudaMemcpyHostToDevice,
                                  g_stream),
                  "tile list upload");
        c.tl_na = n_a;
        c.tl_nb = n_b;
        c.tl_sym = sym;
        c.tl_group = group;
        c.tl_bn = bn;
        c.tl_bm = bm;
        ++c.tl_gen;
    }
    *count = static_cast<int>(c.tl_host.size());
    return GBMI_OK;
}

// Tail split of the fused MI launch: a persistent launch of T tiles on U
// concurrent tile slots ends with a partial wave of T mod U tiles while the
// other slots idle.  The last (T mod U) + U tiles are instead run as `parts`
// units each accumulating 1 / parts of the samples, so the launch ends in
// pieces half as long (GBMI_OPT_TAIL_SPLIT: 0 off, 1 on, k >= 2 every tile in
// k parts).  Returns the number of split tiles (0: none).
int tail_split_plan(int tiles, int units, int64_t k_blocks, int* parts) {
    *parts = 0;
    if (g_opt.tail_split == 0 || tiles <= 0 || units <= 0) return 0;
    int S = 0, P = 2;
    if (g_opt.tail_split >= 2) {
        S = tiles;
        P = g_opt.tail_split;
    } else if (tiles >= units && tiles % units != 0) {
        S = std::min(tiles, tiles % units + units);
    }
    if (S <= 0 || k_blocks < P) return 0;
    *parts = P;
    return S;
}

// The split tile list (the cached list c.tl_host with its last S tiles as
// `parts` units each), uploaded to c.tail_tiles; part buffers sized.
gbmi_status tail_split_list(DeviceCtx& c, int S, int parts, int* count) {
    const int T = static_cast<int>(c.tl_host.size());
    const int n = T - S + S * parts;
    if (!(c.ts_key_gen == c.tl_gen && c.ts_key_s == S && c.ts_key_p == parts)) {
        c.ts_host.assign(c.tl_host.begin(), c.tl_host.begin() + (T - S));
        for (int s = 0; s < S; ++s)
            for (int p = 0; p < parts; ++p) {
                GramTile g = c.tl_host[static_cast<size_t>(T - S + s)];
                g.split = gram_split_code(s, p, parts);
                c.ts_host.push_back(g);
            }
        GBMI_TRY(ensure(c.tail_tiles, c.ts_host.size() * sizeof(GramTile), "split tile list"));
        GBMI_CUDA(cudaMemcpyAsync(c.tail_tiles.p, c.ts_host.data(),
                                  c.ts_host.size() * sizeof(GramTile), cudaMemcpyHostToDevice,
                                  g_stream),
                  "split tile list upload");
        c.ts_key_gen = c.tl_gen;
        c.ts_key_s = S;
        c.ts_key_p = parts;
    }
    GBMI_TRY(ensure(c.part_counts,
                    static_cast<size_t>(S) * (parts - 1) * gram_part_slot_ints() * sizeof(int32_t),
                    "split tile counts"));
    GBMI_TRY(ensure(c.part_arrive,
                    static_cast<size_t>(S) * gram_part_slot_counters() * sizeof(unsigned int),
                    "split tile counters"));
    *count = n;
    return GBMI_OK;
}

// Column shares of the tail (GBMI_OPT_TAIL_COLS): a persistent launch of T
// whole tiles on U concurrent tile slots ends with a partial wave of r = T mod
// U tiles while the other slots idle.  Those r tiles instead run as `parts`
// column shares each, every share an MMA as wide as its columns over all
// samples, so no share waits for another; parts (2..4) is the count whose
// shares fill the fewest part-length waves, ceil(parts r / U) / parts, the
// smallest first on ties (wider MMAs).  1 = automatic, k in 2..4 = every tile
// in k shares (tests), 0 = off.  Returns the number of tiles at the end of the
// list to split (0: none).
int tail_cols_plan(int tiles, int units, int* parts) {
    *parts = 0;
    if (g_opt.tail_cols == 0 || tiles <= 0 || units <= 0) return 0;
    if (g_opt.tail_cols >= 2) {
        *parts = g_opt.tail_cols;
        return tiles;
    }
    const int r = tiles % units;
    if (tiles < units || r == 0) return 0;
    int best = 0;
    double best_len = 1.0;   // a share plan must end before one whole-tile wave
    for (int p = 2; p <= 4; ++p) {
        const double len = static_cast<double>((p * r + units - 1) / units) / p;
        if (len < best_len - 1e-9) {
            best_len = len;
            best = p;
        }
    }
    if (best == 0) return 0;
    *parts = best;
    return r;
}

// The cached list c.tl_host with each of its last S tiles as `parts` column
// shares (tiles whose column window is narrower than 32 * parts stay whole),
// uploaded to c.col_tiles.
gbmi_status tail_cols_list(DeviceCtx& c, int S, int parts, int64_t n_b, bool sym, int bn,
                           int bm, int* count) {
    const int T = static_cast<int>(c.tl_host.size());
    if (!(c.tc_key_gen == c.tl_gen && c.tc_key_s == S && c.tc_key_p == parts)) {
        c.tc_host.assign(c.tl_host.begin(), c.tl_host.begin() + (T - S));
        for (int s = T - S; s < T; ++s) {
            GramTile g = c.tl_host[static_cast<size_t>(s)];
            const ColWindow w = gram_tile_window(n_b, sym, bn, g, bm, false);
            if (w.hi - w.lo < 32 * parts) {
                c.tc_host.push_back(g);
                continue;
            }
            for (int p = 0; p < parts; ++p) {
                g.split = gram_cols_code(p, parts);
                c.tc_host.push_back(g);
            }
        }
        GBMI_TRY(ensure(c.col_tiles, c.tc_host.size() * sizeof(GramTile), "column-share tiles"));
        GBMI_CUDA(cudaMemcpyAsync(c.col_tiles.p, c.tc_host.data(),
                                  c.tc_host.size() * sizeof(GramTile), cudaMemcpyHostToDevice,
                                  g_stream),
                  "column-share tile upload");
        c.tc_key_gen = c.tl_gen;
        c.tc_key_s = S;
        c.tc_key_p = parts;
    }
    *count = static_cast<int>(c.tc_host.size());
    return GBMI_OK;
}

// The CTA-pair kernel streams half the operand bytes per SM per MMA, so it is
// taken whenever its launch keeps at least as many SMs busy as the single-CTA
// launch of the same problem would (small problems keep the finer tiles).
// bn_max: the pair's tile width (256; 240 for FP4 operands).
bool use_pair(const DeviceCtx& c, int64_t m, int64_t n_a, int64_t n_b, bool sym, int bn,
              int bn_max = kTcBNMax) {
    if (g_opt.pair == 0 || c.pair_clusters <= 0) return false;
    if (g_opt.pair == 2) return true;   // forced (tests)
    if (g_opt.tile_n != 0) return false;   // a forced tile width names a single-CTA tile
    const int tuned = rt::tuner_pair(m, std::max(n_a, n_b));   // a tuned bucket decides
    if (tuned >= 0) return tuned == 1;
    const int64_t pair_tiles = gram_tile_count(n_a, n_b, bn_max, sym, 2 * kTcBM);
    const int64_t single_tiles = gram_tile_count(n_a, n_b, bn, sym, kTcBM);
    const int64_t pair_sms = 2 * std::min<int64_t>(pair_tiles, c.pair_clusters);
    return pair_sms >= std::min<int64_t>(single_tiles, c.sm_count);
}

// Run the tensor-core Gram of one job over [0, m) in exact chunks of at most
// 2^24 samples.  The counts modes add chunk results into out_c.  Mode MI with
// several chunks accumulates the earlier chunks' exact int32 counts in the
// workspace (counts, then counts-add) and runs the MI epilogue on the last
// chunk with those counts added to its accumulator.
// direct: the operands are the caller's matrices through *dmaps (no pack).
// Shard `shard` of `num_shards` runs only that contiguous share of the tile
// list (the same list and order as the whole problem), so the shards' writes
// together are the whole result.
// Sample split of a Gram with too few tiles to fill the GPU (few variables,
// many samples): the sample range is cut into S parts and every (part, tile)
// is a unit of one grouped launch (single-CTA or CTA-pair tiles), each part a
// job writing exact int32 counts into its own slice of the workspace; a final
// kernel adds the slices and evaluates MI (or writes the counts).  Returns S
// (1: no split).
// units: the launch's concurrent tile slots (SMs, or CTA pairs).  S is chosen
// by a model: the makespan of ceil(S * tiles / units) waves of units 1/S as
// long, plus the slices' traffic (written by the Gram, read by the final
// kernel: about 3 x S x n_a x n_b x 4 bytes at HBM rate); a split is taken
// only when the model gains at least 10% over one part.  spk: samples per K
// block (128 FP8, 256 FP4).
// tuned: the bucket's part count from the tuner table (0: none; 1: no split;
// S >= 2: S parts, taken where the limits below allow it, else the model).
int split_parts(int units, int tiles, int64_t kb_total, int64_t n_a, int64_t n_b,
                int64_t spk = kKbSamplesFp8, int tuned = 0) {
    const int64_t kMinPartKb = std::max<int64_t>(1, 2048 / spk);   // 2048 samples per part
    constexpr int64_t kMaxParts = 128;
    constexpr int64_t kMaxSliceBytes = int64_t{2} << 30;
    // one K block of one tile unit (FP8: 128 samples; FP4: 256 samples at
    // about twice the rate)
    constexpr double kBlockSeconds = 0.29e-6;
    constexpr double kHbmBytesPerSecond = 6.0e12;
    const int64_t kb_chunk = kExactChunk / spk;
    if (g_opt.split_k == 1 || tiles <= 0 || units <= 0) return 1;
    if (g_opt.split_k != 2 && tiles >= units) return 1;
    const int64_t exact = (kb_total + kb_chunk - 1) / kb_chunk;   // parts of at most 2^24
    const double slice = static_cast<double>(n_a) * n_b * 4.0;
    int64_t s_max = std::min(kMaxParts, kb_total / kMinPartKb);
    while (s_max > 1 && s_max * slice > kMaxSliceBytes) --s_max;
    if (g_opt.split_k != 2 && tuned == 1) return 1;
    if (g_opt.split_k != 2 && tuned >= 2 && tuned >= exact && tuned <= s_max) {
        const int64_t kb_s = (kb_total + tuned - 1) / tuned;
        return static_cast<int>((kb_total + kb_s - 1) / kb_s);
    }
    if (s_max < std::max<int64_t>(2, exact)) return 1;
    const double t_tile = kBlockSeconds * static_cast<double>(kb_total);
    auto cost = [&](int64_t S) {
        const int64_t waves = (S * tiles + units - 1) / units;
        return static_cast<double>(waves) / S * t_tile + 3.0 * S * slice / kHbmBytesPerSecond;
    };
    int64_t best = 0;
    double best_cost = 0.0;
    for (int64_t S = std::max<int64_t>(2, exact); S <= s_max; ++S) {
        const double c = cost(S);
        if (best == 0 || c < best_cost) {
            best = S;
            best_cost = c;
        }
    }
    if (best == 0) return 1;
    if (g_opt.split_k != 2 && exact <= 1 && best_cost > 0.9 * cost(1)) return 1;
    // equal parts of ceil(kb_total / S) K blocks; drop the parts that would be empty
    const int64_t kb_s = (kb_total + best - 1) / best;
    return static_cast<int>((kb_total + kb_s - 1) / kb_s);
}

gbmi_status run_gram_split(DeviceCtx& c, const OperandMaps& maps, const GramJob& proto, int bn,
                           bool pair, int tiles, int64_t kb_total, int S, int mode, bool fp4) {
    const int64_t slice = static_cast<int64_t>(proto.n_a) * proto.n_b;
    // its own buffer: the caller's counts may live in the workspace's count matrix
    GBMI_TRY(ensure(c.split_part, static_cast<size_t>(S) * slice * 4, "split partial counts"));
    int32_t* part = static_cast<int32_t*>(c.split_part.p);
    const int64_t kb_s = (kb_total + S - 1) / S;   // every part non-empty (split_parts)
    if ((S - 1) * kb_s >= kb_total || kb_s > kExactChunk / kb_samples(fp4))
        return fail(GBMI_ERR_ARG, "internal: bad sample split");
    c.split_jobs_host.assign(static_cast<size_t>(S), proto);
    for (int s = 0; s < S; ++s) {
        GramJob& j = c.split_jobs_host[static_cast<size_t>(s)];
        j.bn = bn;
        j.k_begin = static_cast<int32_t>(s * kb_s);
        j.k_blocks = static_cast<int32_t>(std::min(kb_s, kb_total - s * kb_s));
        j.out_f = nullptr;
        j.out_t = nullptr;
        j.out_c = part + s * slice;
        j.ld_out = proto.n_b;
    }
    // parts outer, tiles inner: the units in flight share a sample range
    c.split_tiles_host.resize(static_cast<size_t>(S) * tiles);
    for (int s = 0; s < S; ++s)
        for (int t = 0; t < tiles; ++t) {
            GramTile g = c.tl_host[static_cast<size_t>(t)];
            g.job = s;
            c.split_tiles_host[static_cast<size_t>(s) * tiles + t] = g;
        }
    GBMI_TRY(ensure(c.split_jobs, c.split_jobs_host.size() * sizeof(GramJob), "split job table"));
    GBMI_TRY(ensure(c.split_tiles, c.split_tiles_host.size() * sizeof(GramTile), "split tiles"));
    GBMI_CUDA(cudaMemcpyAsync(c.split_jobs.p, c.split_jobs_host.data(),
                              c.split_jobs_host.size() * sizeof(GramJob), cudaMemcpyHostToDevice,
                              g_stream),
              "split job table upload");
    GBMI_CUDA(cudaMemcpyAsync(c.split_tiles.p, c.split_tiles_host.data(),
                              c.split_tiles_host.size() * sizeof(GramTile),
                              cudaMemcpyHostToDevice, g_stream),
              "split tile upload");
    GramLaunch L;
    std::memset(&L, 0, sizeof(L));
    L.jobs = static_cast<const GramJob*>(c.split_jobs.p);
    L.job0 = c.split_jobs_host[0];
    L.tiles = static_cast<const GramTile*>(c.split_tiles.p);
    L.num_tiles = S * tiles;
    L.pair = pair ? 1 : 0;
    L.fp4 = fp4 ? 1 : 0;
    L.mode = kTcModeCounts;
    L.err = static_cast<unsigned int*>(c.err.p);
    L.timeout_ns = g_opt.timeout_ns;
    L.debug_flags = g_opt.debug_flags;
    GBMI_TRY(ensure(c.sched, 256, "tile counter"));
    L.counter = static_cast<unsigned int*>(c.sched.p);
    GBMI_CUDA(cudaMemsetAsync(L.counter, 0, sizeof(unsigned int), g_stream), "tile counter");
    const int grid = pair ? 2 * static_cast<int>(std::min<int64_t>(c.pair_clusters, L.num_tiles))
                          : rt::grid_for(c, L.num_tiles);
    GBMI_LAUNCH(launch_gram_tc(maps, L, grid, g_stream), "gram_tc_split_counts");
    if (mode != kTcModeMI) {   // counts: the sum of the slices into the caller's matrix
        GBMI_LAUNCH(launch_slice_sum(part, proto.n_b, S, slice, proto.n_a, proto.n_b, proto.out_c,
                                     proto.ld_out, g_stream),
                    "slice_sum");
        return GBMI_OK;
    }
    if (proto.symmetric)
        GBMI_LAUNCH(launch_mi_from_counts_sym(part, proto.n_b, proto.va, proto.n_a, proto.mp,
                                              proto.out_f, proto.ld_out, g_stream, 0, S, slice),
                    "mi_from_counts");
    else
        GBMI_LAUNCH(launch_mi_from_counts(part, proto.n_b, proto.va, proto.vb, proto.n_a,
                                          proto.n_b, proto.mp, proto.out_f, proto.ld_out,
                                          g_stream, S, slice),
                    "mi_from_counts");
    return GBMI_OK;
}

gbmi_status run_gram(DeviceCtx& c, int64_t total_rows, const GramJob& proto, int64_t m,
                     int mode, const OperandMaps* dmaps = nullptr, int shard = 0,
                     int num_shards = 1, bool fp4 = false) {
    OperandMaps maps;
    if (dmaps != nullptr)
        maps = *dmaps;
    else if (!make_operand_maps(&maps, static_cast<const uint8_t*>(c.P.p), total_rows))
        return fail(GBMI_ERR_CUDA, "cuTensorMapEncodeTiled failed");
    // CTA pairs: 256 x 256 tiles (256 x 240 for FP4 operands) on clusters of
    // two SMs (packed operands only)
    const int bn_max = fp4 ? kTcBNFp4 : kTcBNMax;
    const bool pair = dmaps == nullptr &&
                      use_pair(c, m, proto.n_a, proto.n_b, proto.symmetric != 0, proto.bn, bn_max);
    const int64_t spk = kb_samples(fp4);
    const int64_t kb_all = pack_ld_of(m, fp4) / spk;
    const int bn = pair ? bn_max : std::min(proto.bn, bn_max);
    const int bm = pair ? 2 * kTcBM : kTcBM;
    int tiles = 0;
    GBMI_TRY(tile_list(c, proto.n_a, proto.n_b, proto.symmetric != 0, bn, &tiles, bm));
    if (dmaps == nullptr && num_shards == 1 && proto.out_t == nullptr &&
        (mode == kTcModeMI || mode == kTcModeCounts)) {
        const int S = split_parts(pair ? c.pair_clusters : c.sm_count, tiles, kb_all,
                                  proto.n_a, proto.n_b, spk,
                                  rt::tuner_split(m, std::max(proto.n_a, proto.n_b)));
        if (S > 1)
            return run_gram_split(c, maps, proto, bn, pair, tiles, kb_all, S, mode, fp4);
    }
    GramLaunch L;
    std::memset(&L, 0, sizeof(L));
    L.jobs = nullptr;
    L.job0 = proto;
    L.job0.bn = bn;
    L.pair = pair ? 1 : 0;
    L.fp4 = fp4 ? 1 : 0;
    L.fixup = proto.mp.fixup;
    const int64_t t0 = static_cast<int64_t>(tiles) * shard / num_shards;
    const int64_t t1 = static_cast<int64_t>(tiles) * (shard + 1) / num_shards;
    L.tiles = static_cast<const GramTile*>(c.tiles.p) + t0;
    L.num_tiles = static_cast<int>(t1 - t0);
    tiles = L.num_tiles;
    L.err = static_cast<unsigned int*>(c.err.p);
    L.timeout_ns = g_opt.timeout_ns;
    L.debug_flags = g_opt.debug_flags;
    L.direct = dmaps != nullptr ? 1 : 0;
    GBMI_TRY(ensure(c.sched, 256, "tile counter"));
    L.counter = static_cast<unsigned int*>(c.sched.p);
    const int64_t kb_total = kb_all;
    const int64_t kb_chunk = kExactChunk / spk;
    int32_t* prefix = nullptr;   // MI over several chunks: counts of the earlier ones
    if (mode == kTcModeMI && kb_total > kb_chunk) {
        GBMI_TRY(ensure(c.counts, static_cast<size_t>(proto.n_a) * proto.n_b * 4,
                        "count matrix"));
        prefix = static_cast<int32_t*>(c.counts.p);
    }
    const int grid = pair ? 2 * static_cast<int>(std::min<int64_t>(c.pair_clusters, tiles))
                          : rt::grid_for(c, tiles);
    // The MI launch (the last sample chunk) may split its last tiles into
    // K-share units (tail_split): its own tile list, grid and part buffers.
    const GramTile* const plain_tiles = L.tiles;
    const int plain_num = L.num_tiles;
    const GramTile* mi_tiles = plain_tiles;
    int mi_num = plain_num, mi_grid = grid, split_slots = 0;
    if (mode == kTcModeMI && !proto.mp.fixup && num_shards == 1 && dmaps == nullptr &&
        proto.out_t == nullptr) {
        const int64_t kb_last = kb_total - (kb_total - 1) / kb_chunk * kb_chunk;
        const int units = pair ? static_cast<int>(std::min<int64_t>(c.pair_clusters, tiles))
                               : grid;
        int parts = 0;
        split_slots = tail_split_plan(tiles, units, kb_last, &parts);
        if (split_slots > 0) {
            GBMI_TRY(tail_split_list(c, split_slots, parts, &mi_num));
            mi_tiles = static_cast<const GramTile*>(c.tail_tiles.p);
            mi_grid = pair ? 2 * static_cast<int>(std::min<int64_t>(c.pair_clusters, mi_num))
                           : rt::grid_for(c, mi_num);
            L.part_counts = static_cast<int32_t*>(c.part_counts.p);
            L.part_arrive = static_cast<unsigned int*>(c.part_arrive.p);
        }
    }
    // Otherwise every launch may run the tail's tiles as column shares.
    const GramTile* all_tiles = plain_tiles;
    int all_num = plain_num;
    if (split_slots == 0 && num_shards == 1 && dmaps == nullptr) {
        const int units = pair ? static_cast<int>(std::min<int64_t>(c.pair_clusters, tiles))
                               : grid;
        int parts = 0;
        const int S = tail_cols_plan(tiles, units, &parts);
        if (S > 0) {
            GBMI_TRY(tail_cols_list(c, S, parts, proto.n_b, proto.symmetric != 0, bn, bm,
                                    &all_num));
            all_tiles = static_cast<const GramTile*>(c.col_tiles.p);
            mi_tiles = all_tiles;
            mi_num = all_num;
        }
    }
    const int all_grid = pair ? 2 * static_cast<int>(std::min<int64_t>(c.pair_clusters, all_num))
                              : rt::grid_for(c, all_num);
    for (int64_t k0 = 0; k0 < kb_total; k0 += kb_chunk) {
        L.job0.k_begin = static_cast<int32_t>(k0);
        L.job0.k_blocks = static_cast<int32_t>(std::min(kb_chunk, kb_total - k0));
        if (mode == kTcModeMI) {
            const bool last = k0 + kb_chunk >= kb_total;
            L.mode = last ? kTcModeMI : (k0 == 0 ? kTcModeCounts : kTcModeCountsAdd);
            L.job0.out_f = last ? proto.out_f : nullptr;
            L.job0.out_c = prefix;   // counts target, then the MI epilogue's prefix
        } else {
            L.mode = k0 == 0 ? kTcModeCounts : kTcModeCountsAdd;
        }
        const bool split = L.mode == kTcModeMI && split_slots > 0;
        L.tiles = split ? mi_tiles : all_tiles;
        L.num_tiles = split ? mi_num : all_num;
        if (split)
            GBMI_CUDA(cudaMemsetAsync(L.part_arrive, 0,
                                      static_cast<size_t>(split_slots) *
                                          gram_part_slot_counters() * sizeof(unsigned int),
                                      g_stream),
                      "split tile counters");
        GBMI_CUDA(cudaMemsetAsync(L.counter, 0, sizeof(unsigned int), g_stream), "tile counter");
        GBMI_LAUNCH(launch_gram_tc(maps, L, split ? mi_grid : all_grid, g_stream),
                    L.mode == kTcModeMI ? "gram_tc_fused_mi" : "gram_tc_counts");
    }
    return GBMI_OK;
}

int choose_path(int path, int64_t m, int64_t n1, int64_t n2) {
    if (path != GBMI_PATH_AUTO) return path;
    if (static_cast<double>(m) * n1 * n2 <= kTinyWork) return GBMI_PATH_POPCOUNT;
    return GBMI_PATH_FUSED;
}

// Workspace layout of the tensor-core path: X's operand rows, then Y's; or,
// for the direct path, the tensor maps over X and Y themselves.
// fp4: the packed operands are the FP4 form (kb counts 256-sample blocks).
struct TcLayout {
    int64_t kb = 0, rows_a = 0, rows_b = 0, total_rows = 0;
    bool direct = false;
    bool fp4 = false;
    OperandMaps maps;
};

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// The direct path (no pack: the tensor cores read X and Y as MN-major E4M3)
// applies when it is enabled and the rows of X and Y are 16-byte multiples.
bool direct_ok(const uint8_t* X, const uint8_t* Y, int64_t n1, int64_t n2, bool sym) {
    return g_opt.direct != 0 && n1 % 16 == 0 && aligned16(X) &&
           (sym || (n2 % 16 == 0 && aligned16(Y)));
}

gbmi_status tc_prepare(DeviceCtx& c, const uint8_t* X, const uint8_t* Y, int64_t m, int64_t n1,
                       int64_t n2, bool sym, TcLayout* L) {
    L->direct = direct_ok(X, Y, n1, n2, sym);
    if (L->direct) {
        L->kb = pack_ld(m) / kTcBK;
        L->rows_a = L->rows_b = L->total_rows = 0;
        if (!make_direct_maps(&L->maps, X, m, n1, sym ? X : Y, sym ? n1 : n2))
            return fail(GBMI_ERR_CUDA, "cuTensorMapEncodeTiled failed");
        unsigned int* err = static_cast<unsigned int*>(c.err.p);
        GBMI_TRY(ensure(c.va, static_cast<size_t>(n1) * 4, "column counts"));
        GBMI_LAUNCH(launch_zero_u32(c.va.p, n1, g_stream), "zero");
        GBMI_LAUNCH(launch_colsum_direct(X, m, n1, static_cast<int32_t*>(c.va.p), err,
                                         c.sm_count, g_stream),
                    "colsum_direct");
        if (!sym) {
            GBMI_TRY(ensure(c.vb, static_cast<size_t>(n2) * 4, "column counts"));
            GBMI_LAUNCH(launch_zero_u32(c.vb.p, n2, g_stream), "zero");
            GBMI_LAUNCH(launch_colsum_direct(Y, m, n2, static_cast<int32_t*>(c.vb.p), err,
                                             c.sm_count, g_stream),
                        "colsum_direct");
        }
        return GBMI_OK;
    }
    L->fp4 = g_opt.fp4 != 0;
    L->kb = pack_ld_of(m, L->fp4) / kb_samples(L->fp4);
    L->rows_a = pack_rows(n1);
    L->rows_b = sym ? 0 : pack_rows(n2);
    L->total_rows = L->kb * (L->rows_a + L->rows_b);
    if (L->total_rows >= (int64_t{1} << 31))
        return fail(GBMI_ERR_ARG, "packed operands exceed 2^31 rows of 128 bytes");
    GBMI_TRY(ensure(c.P, static_cast<size_t>(L->total_rows) * kTcBK, "packed operand"));
    GBMI_TRY(ensure(c.va, static_cast<size_t>(n1) * 4, "column counts"));
    uint8_t* P = static_cast<uint8_t*>(c.P.p);
    GBMI_TRY(pack(X, m, n1, P, nullptr, static_cast<int32_t*>(c.va.p), L->fp4));
    if (!sym) {
        GBMI_TRY(ensure(c.vb, static_cast<size_t>(n2) * 4, "column counts"));
        GBMI_TRY(pack(Y, m, n2, P + L->kb * L->rows_a * kTcBK, nullptr,
                      static_cast<int32_t*>(c.vb.p), L->fp4));
    }
    return GBMI_OK;
}

GramJob tc_job(const TcLayout& L, int64_t m, int64_t n1, int64_t n2, bool sym, int bn,
               const MiVar* va, const MiVar* vb, const MiParams& mp, float* out_f,
               int32_t* out_c) {
    GramJob g;
    std::memset(&g, 0, sizeof(g));
    g.rowA = 0;
    g.strideA = L.rows_a;
    g.rowB = sym ? 0 : L.kb * L.rows_a;
    g.strideB = sym ? L.rows_a : L.rows_b;
    if (L.direct) {   // first variables of X and Y; tiles 128 or 256 wide
        g.rowA = g.rowB = 0;
        g.strideA = g.strideB = 0;
        bn = bn < kTcBM ? kTcBM : bn;
    }
    g.k_begin = 0;
    g.k_blocks = static_cast<int32_t>(L.kb);
    g.n_a = static_cast<int32_t>(n1);
    g.n_b = static_cast<int32_t>(n2);
    g.symmetric = sym ? 1 : 0;
    g.bn = bn;
    g.va = va;
    g.vb = vb;
    g.out_f = out_f;
    g.out_c = out_c;
    g.ld_out = n2;
    g.mp = mp;
    (void)m;
    return g;
}

// MI between the variables of X (n1) and Y (n2, or X itself when sym).
// num_shards > 1 (fused path only): just shard `shard` of the Gram's tiles.
gbmi_status mi_impl(const uint8_t* X, const uint8_t* Y, int64_t m, int64_t n1, int64_t n2,
                    float* out, int path, bool sym, int shard = 0, int num_shards = 1) {
    if (X == nullptr || out == nullptr || (!sym && Y == nullptr))
        return fail(GBMI_ERR_ARG, "null pointer");
    GBMI_TRY(check_sizes(m, n1, n2));
    const size_t out_bytes = static_cast<size_t>(n1) * n2 * 4;
    if (overlaps(X, static_cast<size_t>(m) * n1, out, out_bytes) ||
        (!sym && overlaps(Y, static_cast<size_t>(m) * n2, out, out_bytes)))
        return fail(GBMI_ERR_ARG, "out overlaps an input");
    if (path < GBMI_PATH_AUTO || path > GBMI_PATH_POPCOUNT) return fail(GBMI_ERR_ARG, "bad path");
    DeviceCtx* cp = nullptr;
    GBMI_TRY(rt::get_ctx(&cp));
    DeviceCtx& c = *cp;
    path = choose_path(path, m, n1, n2);
    if (num_shards < 1 || shard < 0 || shard >= num_shards)
        return fail(GBMI_ERR_ARG, "shard must be in [0, num_shards)");
    if (num_shards > 1) path = GBMI_PATH_FUSED;

    if (path == GBMI_PATH_POPCOUNT) {
        const int64_t ldp = pack_ld(m);
        GBMI_TRY(ensure(c.Ba, static_cast<size_t>(pack_rows(n1)) * (ldp / 8), "bit operand"));
        GBMI_TRY(ensure(c.va, static_cast<size_t>(n1) * 4, "column counts"));
        GBMI_TRY(pack(X, m, n1, nullptr, static_cast<uint32_t*>(c.Ba.p),
                      static_cast<int32_t*>(c.va.p)));
        if (!sym) {
            GBMI_TRY(ensure(c.Bb, static_cast<size_t>(pack_rows(n2)) * (ldp / 8), "bit operand"));
            GBMI_TRY(ensure(c.vb, static_cast<size_t>(n2) * 4, "column counts"));
            GBMI_TRY(pack(Y, m, n2, nullptr, static_cast<uint32_t*>(c.Bb.p),
                          static_cast<int32_t*>(c.vb.p)));
        }
    } else {
        TcLayout L;
        GBMI_TRY(tc_prepare(c, X, Y, m, n1, n2, sym, &L));
        MiParams mp;
        GBMI_TRY(rt::mi_params(c, m, &mp));
        const MiVar *va = nullptr, *vb = nullptr;
        GBMI_TRY(mi_vars(static_cast<const int32_t*>(c.va.p), n1, mp, c.ha, &va));
        if (sym)
            vb = va;
        else
            GBMI_TRY(mi_vars(static_cast<const int32_t*>(c.vb.p), n2, mp, c.hb, &vb));
        const int bn = rt::choose_bn(m, n1, n2, sym);
        if (path == GBMI_PATH_FUSED)
            return run_gram(c, L.total_rows, tc_job(L, m, n1, n2, sym, bn, va, vb, mp, out, nullptr),
                            m, kTcModeMI, L.direct ? &L.maps : nullptr, shard, num_shards,
                            L.fp4);
        // plain: exact counts to HBM, then the elementwise MI kernel
        GBMI_TRY(ensure(c.counts, static_cast<size_t>(n1) * n2 * 4, "count matrix"));
        int32_t* N11 = static_cast<int32_t*>(c.counts.p);
        GBMI_TRY(run_gram(c, L.total_rows,
                          tc_job(L, m, n1, n2, sym, bn, va, vb, mp, nullptr, N11), m,
                          kTcModeCounts, L.direct ? &L.maps : nullptr, 0, 1, L.fp4));
        if (sym)
            GBMI_LAUNCH(launch_mi_from_counts_sym(N11, n2, va, n1, mp, out, n2, g_stream),
                        "mi_from_counts");
        else
            GBMI_LAUNCH(launch_mi_from_counts(N11, n2, va, vb, n1, n2, mp, out, n2, g_stream),
                        "mi_from_counts");
        return GBMI_OK;
    }
    // popcount: Gram and MI epilogue in one kernel
    MiParams mp;
    GBMI_TRY(rt::mi_params(c, m, &mp));
    const MiVar *va = nullptr, *vb = nullptr;
    GBMI_TRY(mi_vars(static_cast<const int32_t*>(c.va.p), n1, mp, c.ha, &va));
    if (sym)
        vb = va;
    else
        GBMI_TRY(mi_vars(static_cast<const int32_t*>(c.vb.p), n2, mp, c.hb, &vb));
    PopcArgs a;
    std::memset(&a, 0, sizeof(a));
    a.Ba = static_cast<const uint32_t*>(c.Ba.p);
    a.Bb = static_cast<const uint32_t*>(sym ? c.Ba.p : c.Bb.p);
    a.wpr = pack_ld(m) / 32;
    a.n_a = n1;
    a.n_b = n2;
    a.symmetric = sym ? 1 : 0;
    a.va = va;
    a.vb = vb;
    a.mp = mp;
    a.out_f = out;
    a.out_c = nullptr;
    a.ld_out = n2;
    GBMI_LAUNCH(launch_popcount(a, g_stream), "popcount_gram");
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
    GBMI_TRY(rt::get_ctx(&cp));
    DeviceCtx& c = *cp;
    if (path == GBMI_PATH_POPCOUNT) {
        const int64_t ldp = pack_ld(m);
        GBMI_TRY(ensure(c.Ba, static_cast<size_t>(pack_rows(n1)) * (ldp / 8), "bit operand"));
        GBMI_TRY(ensure(c.va, static_cast<size_t>(n1) * 4, "column counts"));
        GBMI_TRY(pack(X, m, n1, nullptr, static_cast<uint32_t*>(c.Ba.p),
                      static_cast<int32_t*>(c.va.p)));
        if (!sym) {
            GBMI_TRY(ensure(c.Bb, static_cast<size_t>(pack_rows(n2)) * (ldp / 8), "bit operand"));
            GBMI_TRY(ensure(c.vb, static_cast<size_t>(n2) * 4, "column counts"));
            GBMI_TRY(pack(Y, m, n2, nullptr, static_cast<uint32_t*>(c.Bb.p),
                          static_cast<int32_t*>(c.vb.p)));
        }
        PopcArgs a;
        std::memset(&a, 0, sizeof(a));
        a.Ba = static_cast<const uint32_t*>(c.Ba.p);
        a.Bb = static_cast<const uint32_t*>(sym ? c.Ba.p : c.Bb.p);
        a.wpr = pack_ld(m) / 32;
        a.n_a = n1;
        a.n_b = n2;
        a.symmetric = sym ? 1 : 0;
        a.mp = rt::mi_params_plain(m, 0, nullptr);
        a.out_c = n11;
        a.ld_out = n2;
        GBMI_LAUNCH(launch_popcount(a, g_stream), "popcount_gram");
        return GBMI_OK;
    }
    TcLayout L;
    GBMI_TRY(tc_prepare(c, X, Y, m, n1, n2, sym, &L));
    const MiParams mp = rt::mi_params_plain(m, 0, nullptr);
    const int bn = rt::choose_bn(m, n1, n2, sym);
    return run_gram(c, L.total_rows, tc_job(L, m, n1, n2, sym, bn, nullptr, nullptr, mp, nullptr, n11),
                    m, kTcModeCounts, L.direct ? &L.maps : nullptr, 0, 1, L.fp4);
}

// Resources of the host-buffer pipeline (created once per device context).
gbmi_status pipeline_resources(DeviceCtx& c, int events, int panels) {
    if (c.copy_stream == nullptr)
        GBMI_CUDA(cudaStreamCreateWithFlags(&c.copy_stream, cudaStreamNonBlocking), "copy stream");
    while (static_cast<int>(c.events.size()) < events) {
        cudaEvent_t e;
        GBMI_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event");
        c.events.push_back(e);
    }
    if (c.hflags_cap < panels) {
        if (c.hflags != nullptr) cudaFreeHost(c.hflags);
        c.hflags = nullptr;
        c.hflags_cap = 0;
        void* h = nullptr;
        GBMI_CUDA(cudaHostAlloc(&h, static_cast<size_t>(panels) * 4, cudaHostAllocMapped),
                  "mapped panel flags");
        c.hflags = static_cast<unsigned int*>(h);
        void* d = nullptr;
        GBMI_CUDA(cudaHostGetDevicePointer(&d, h, 0), "cudaHostGetDevicePointer");
        c.dflags = static_cast<unsigned int*>(d);
        c.hflags_cap = panels;
    }
    return ensure(c.panel, static_cast<size_t>(panels) * 8, "panel counters");
}

// Host buffers, fused tensor-core path, pipelined:
//   X (and Y) go up in row chunks on a copy stream, each chunk packed as soon
//   as it lands;
//   the Gram runs over the samples in kGramChunks chunks: each of the first
//   ones accumulates exact int32 counts in HBM (counts / counts-add launches)
//   while later chunks are still uploading, and the last one runs the fused
//   MI epilogue with those counts added to its accumulator;
//   that last launch takes its tiles in panel-major order (row panels of
//   panel_blocks tile rows), and the epilogue flags each finished panel in
//   mapped host memory; the host copies a panel's rows down as soon as it and
//   every earlier panel are flagged (rows of panel p are written only by
//   tiles of panels <= p), so the download overlaps the rest of the Gram.
constexpr int kUploadChunks = 8;
constexpr int kGramChunks = 4;

gbmi_status host_pipelined(DeviceCtx& c, const uint8_t* X, const uint8_t* Y, int64_t m,
                           int64_t n1, int64_t n2, float* out, bool sym) {
    TcLayout L;
    L.direct = false;
    L.fp4 = g_opt.fp4 != 0;
    const int64_t spk = kb_samples(L.fp4);
    L.kb = pack_ld_of(m, L.fp4) / spk;
    L.rows_a = pack_rows(n1);
    L.rows_b = sym ? 0 : pack_rows(n2);
    L.total_rows = L.kb * (L.rows_a + L.rows_b);
    if (L.total_rows >= (int64_t{1} << 31))
        return fail(GBMI_ERR_ARG, "packed operands exceed 2^31 rows of 128 bytes");
    const size_t ob = static_cast<size_t>(n1) * n2 * 4;
    GBMI_TRY(ensure(c.P, static_cast<size_t>(L.total_rows) * kTcBK, "packed operand"));
    GBMI_TRY(ensure(c.Xs, static_cast<size_t>(m) * n1, "input staging"));
    GBMI_TRY(ensure(c.va, static_cast<size_t>(n1) * 4, "column counts"));
    if (!sym) {
        GBMI_TRY(ensure(c.Ys, static_cast<size_t>(m) * n2, "input staging"));
        GBMI_TRY(ensure(c.vb, static_cast<size_t>(n2) * 4, "column counts"));
    }
    GBMI_TRY(ensure(c.outs, ob, "output staging"));
    MiParams mp;
    GBMI_TRY(rt::mi_params(c, m, &mp));

    // upload chunks (rows, whole K blocks) and Gram chunks (groups of them)
    const int64_t R = std::max<int64_t>(spk * 64, round_up((m + kUploadChunks - 1) / kUploadChunks,
                                                            spk));
    const int uchunks = static_cast<int>((m + R - 1) / R);
    // the FP64-combine kernel variant has no prefix input: one Gram launch then
    const int gchunks = mp.fixup ? 1 : std::min(kGramChunks, uchunks);
    if (gchunks > 1) GBMI_TRY(ensure(c.counts, ob, "count matrix"));

    // tiles in panel-major order
    const int bn_max = L.fp4 ? kTcBNFp4 : kTcBNMax;
    const int bn_single = std::min(rt::choose_bn(m, n1, n2, sym), bn_max);
    const bool pair = use_pair(c, m, n1, n2, sym, bn_single, bn_max);
    const int bm = pair ? 2 * kTcBM : kTcBM;
    const int bn = pair ? bn_max : bn_single;
    const int64_t TI = (n1 + bm - 1) / bm, TJ = (n2 + bn - 1) / bn;
    const int64_t pblocks = std::max<int64_t>(1, (TI + 7) / 8);   // about eight panels
    const int64_t panels = (TI + pblocks - 1) / pblocks;
    const int group = std::max(1, g_opt.group_cols);
    const unsigned int epi = static_cast<unsigned int>(
        gram_tc_epilogue_warps(kTcModeMI, mp.fixup) * (pair ? 2 : 1));
    std::vector<GramTile> tiles;
    std::vector<unsigned int> target(static_cast<size_t>(panels), 0);
    for (int64_t p = 0; p < panels; ++p) {
        const int64_t I0 = p * pblocks, I1 = std::min(TI, I0 + pblocks);
        for (int64_t g0 = 0; g0 < TJ; g0 += group)
            for (int64_t I = I0; I < I1; ++I)
                for (int64_t J = g0; J < std::min<int64_t>(TJ, g0 + group); ++J) {
                    if (sym && I * bm > J * bn + bn - 1) continue;
                    tiles.push_back(GramTile{0, static_cast<int32_t>(I), static_cast<int32_t>(J), 0});
                    target[static_cast<size_t>(p)] += epi;   // epilogue warps per tile
                }
    }
    if (tiles.size() > 0x7FFFFFFFu) return fail(GBMI_ERR_ARG, "too many tiles");
    GBMI_TRY(pipeline_resources(c, uchunks * (sym ? 1 : 2), static_cast<int>(panels)));
    GBMI_TRY(ensure(c.tiles, tiles.size() * sizeof(GramTile), "tile list"));
    c.tl_na = -1;   // the single-call tile cache no longer holds this buffer's contents
    cudaStream_t cs = c.copy_stream;
    unsigned int* counters = static_cast<unsigned int*>(c.panel.p);
    unsigned int* targets = counters + panels;
    std::memset(c.hflags, 0, static_cast<size_t>(panels) * 4);
    GBMI_CUDA(cudaMemcpyAsync(c.tiles.p, tiles.data(), tiles.size() * sizeof(GramTile),
                              cudaMemcpyHostToDevice, g_stream),
              "tile list upload");
    GBMI_CUDA(cudaMemcpyAsync(targets, target.data(), static_cast<size_t>(panels) * 4,
                              cudaMemcpyHostToDevice, g_stream),
              "panel targets");
    GBMI_CUDA(cudaMemsetAsync(counters, 0, static_cast<size_t>(panels) * 4, g_stream),
              "panel counters");

    uint8_t* P = static_cast<uint8_t*>(c.P.p);
    int ev = 0;
    // upload row chunk u of one operand and pack it as soon as it lands
    auto upload_pack = [&](int u, const uint8_t* src, uint8_t* stage, int64_t n, uint8_t* Pop,
                           int64_t rows_p, int32_t* v) -> gbmi_status {
        const int64_t r0 = u * R, rows = std::min(R, m - r0);
        GBMI_CUDA(cudaMemcpyAsync(stage + r0 * n, src + r0 * n, static_cast<size_t>(rows) * n,
                                  cudaMemcpyHostToDevice, cs),
                  "copy in");
        GBMI_CUDA(cudaEventRecord(c.events[ev], cs), "event");
        GBMI_CUDA(cudaStreamWaitEvent(g_stream, c.events[ev], 0), "wait chunk");
        ++ev;
        PackJob j;
        std::memset(&j, 0, sizeof(j));
        j.X = stage + r0 * n;
        j.m = rows;
        j.n = n;
        j.ldx = n;
        j.P = Pop + (r0 / spk) * rows_p * kTcBK;
        j.v = v;
        j.rows_p = rows_p;
        j.ldp = pack_ld_of(rows, L.fp4);
        j.fp4 = L.fp4 ? 1 : 0;
        GBMI_LAUNCH(launch_pack(j, g_stream), "pack");
        return GBMI_OK;
    };
    GBMI_LAUNCH(launch_zero_u32(c.va.p, n1, g_stream), "zero");
    if (!sym) GBMI_LAUNCH(launch_zero_u32(c.vb.p, n2, g_stream), "zero");

    OperandMaps maps;
    if (!make_operand_maps(&maps, P, L.total_rows))
        return fail(GBMI_ERR_CUDA, "cuTensorMapEncodeTiled failed");
    GBMI_TRY(ensure(c.sched, 256, "tile counter"));
    GramLaunch G;
    std::memset(&G, 0, sizeof(G));
    G.job0 = tc_job(L, m, n1, n2, sym, bn, nullptr, nullptr, mp, nullptr, nullptr);
    G.job0.bn = bn;
    G.tiles = static_cast<const GramTile*>(c.tiles.p);
    G.num_tiles = static_cast<int>(tiles.size());
    G.err = static_cast<unsigned int*>(c.err.p);
    G.timeout_ns = g_opt.timeout_ns;
    G.debug_flags = g_opt.debug_flags;
    G.pair = pair ? 1 : 0;
    G.fp4 = L.fp4 ? 1 : 0;
    G.fixup = mp.fixup;
    G.counter = static_cast<unsigned int*>(c.sched.p);
    const int grid = pair ? 2 * static_cast<int>(std::min<int64_t>(c.pair_clusters, G.num_tiles))
                          : rt::grid_for(c, G.num_tiles);
    int32_t* const counts = static_cast<int32_t*>(c.counts.p);
    for (int g = 0; g < gchunks; ++g) {
        const int u0 = g * uchunks / gchunks, u1 = (g + 1) * uchunks / gchunks;
        for (int u = u0; u < u1; ++u) {
            GBMI_TRY(upload_pack(u, X, static_cast<uint8_t*>(c.Xs.p), n1, P, L.rows_a,
                                 static_cast<int32_t*>(c.va.p)));
            if (!sym)
                GBMI_TRY(upload_pack(u, Y, static_cast<uint8_t*>(c.Ys.p), n2,
                                     P + L.kb * L.rows_a * kTcBK, L.rows_b,
                                     static_cast<int32_t*>(c.vb.p)));
        }
        const int64_t kb0 = (u0 * R) / spk;
        const int64_t kb1 = g + 1 < gchunks ? (u1 * R) / spk : L.kb;
        G.job0.k_begin = static_cast<int32_t>(kb0);
        G.job0.k_blocks = static_cast<int32_t>(kb1 - kb0);
        if (g + 1 < gchunks) {   // counts of this sample chunk, kept in HBM
            G.mode = g == 0 ? kTcModeCounts : kTcModeCountsAdd;
            G.job0.out_f = nullptr;
            G.job0.out_c = counts;
            GBMI_CUDA(cudaMemsetAsync(G.counter, 0, sizeof(unsigned int), g_stream),
                      "tile counter");
            GBMI_LAUNCH(launch_gram_tc(maps, G, grid, g_stream),
                        g == 0 ? "gram_tc_counts" : "gram_tc_counts_add");
            continue;
        }
        // last chunk: the fused MI epilogue, earlier chunks' counts added
        const MiVar *va = nullptr, *vb = nullptr;
        GBMI_TRY(mi_vars(static_cast<const int32_t*>(c.va.p), n1, mp, c.ha, &va));
        if (sym)
            vb = va;
        else
            GBMI_TRY(mi_vars(static_cast<const int32_t*>(c.vb.p), n2, mp, c.hb, &vb));
        G.mode = kTcModeMI;
        G.job0.va = va;
        G.job0.vb = vb;
        G.job0.out_f = static_cast<float*>(c.outs.p);
        G.job0.out_c = gchunks > 1 ? counts : nullptr;
        G.panel_done = counters;
        G.panel_target = targets;
        G.host_flags = c.dflags;
        G.panel_blocks = static_cast<int>(pblocks);
        GBMI_CUDA(cudaMemsetAsync(G.counter, 0, sizeof(unsigned int), g_stream), "tile counter");
        GBMI_LAUNCH(launch_gram_tc(maps, G, grid, g_stream), "gram_tc_fused_mi");
    }

    // download each panel once it and every earlier panel are complete; if
    // the launch ends first (or fails), the rest follows it on the stream
    const volatile unsigned int* flags = c.hflags;
    const float* outs = static_cast<const float*>(c.outs.p);
    bool launch_over = false, ordered = false;
    for (int64_t p = 0; p < panels; ++p) {
        const int64_t r0 = p * pblocks * bm;
        const int64_t r1 = std::min(n1, (p + 1) * pblocks * bm);
        for (uint64_t it = 0; !launch_over && flags[p] == 0u; ++it) {
            if ((it & 1023u) == 1023u) {
                const cudaError_t q = cudaStreamQuery(g_stream);
                if (q != cudaErrorNotReady) launch_over = true;   // done, or failed
            }
        }
        if (launch_over && !ordered) {   // the remaining copies follow the launch
            GBMI_CUDA(cudaEventRecord(c.events[0], g_stream), "event");
            GBMI_CUDA(cudaStreamWaitEvent(cs, c.events[0], 0), "wait launch");
            ordered = true;
        }
        GBMI_CUDA(cudaMemcpyAsync(out + r0 * n2, outs + r0 * n2,
                                  static_cast<size_t>(r1 - r0) * n2 * 4, cudaMemcpyDeviceToHost,
                                  cs),
                  "copy out");
    }
    GBMI_CUDA(cudaStreamSynchronize(cs), "cudaStreamSynchronize");
    GBMI_CUDA(cudaStreamSynchronize(g_stream), "cudaStreamSynchronize");
    unsigned int err = 0;
    GBMI_CUDA(cudaMemcpy(&err, c.err.p, sizeof(err), cudaMemcpyDeviceToHost), "read error word");
    if (err != 0) {
        cudaMemset(c.err.p, 0, sizeof(err));
        return error_word_status(err);
    }
    return GBMI_OK;
}

gbmi_status host_impl(const uint8_t* X, const uint8_t* Y, int64_t m, int64_t n1, int64_t n2,
                      float* out, bool sym) {
    if (X == nullptr || out == nullptr || (!sym && Y == nullptr))
        return fail(GBMI_ERR_ARG, "null pointer");
    GBMI_TRY(check_sizes(m, n1, n2));
    DeviceCtx* cp = nullptr;
    GBMI_TRY(rt::get_ctx(&cp));
    DeviceCtx& c = *cp;
    // the pipelined form splits the Gram at upload-chunk boundaries: one
    // exact chunk of at most 2^24 samples per launch is guaranteed only below it
    if (choose_path(GBMI_PATH_AUTO, m, n1, n2) == GBMI_PATH_FUSED && !g_opt.direct &&
        m <= kExactChunk)
        return host_pipelined(c, X, Y, m, n1, n2, out, sym);
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
        return error_word_status(err);
    }
    return GBMI_OK;
}

// Device staging of the out-of-core path (both slots, panel and mirror).
constexpr int64_t kStagingBytes = int64_t{4} << 30;

// Out-of-core output: the MI matrix in row panels, each computed into one of
// two device staging slots by the fused Gram and copied to host memory on a
// second stream while the next panel computes.  All pairs: panel [i0, i1)
// computes the block rows [i0, i1) x columns [i0, n) once and also writes its
// mirror (columns [i0, i1) of rows [i1, n)), so the host receives the full
// symmetric matrix with no pair computed twice off the diagonal blocks.
gbmi_status blocked_impl(const uint8_t* X, const uint8_t* Y, int64_t m, int64_t n1, int64_t n2,
                         float* host_out, int64_t panel, bool sym) {
    if (X == nullptr || host_out == nullptr || (!sym && Y == nullptr))
        return fail(GBMI_ERR_ARG, "null pointer");
    GBMI_TRY(check_sizes(m, n1, n2));
    if (m > kExactChunk) return fail(GBMI_ERR_ARG, "the out-of-core path needs m <= 2^24");
    if (panel < 0) return fail(GBMI_ERR_ARG, "panel_rows must be >= 0");
    DeviceCtx* cp = nullptr;
    GBMI_TRY(rt::get_ctx(&cp));
    DeviceCtx& c = *cp;
    if (panel == 0) {
        const int64_t per_row = (sym ? 2 : 1) * n2 * 4;          // staging bytes per panel row
        panel = std::max<int64_t>(1, kStagingBytes / 2 / per_row);
        if (panel >= kTcBM) panel = panel / kTcBM * kTcBM;
        // at least about eight panels, so that copies overlap the computation
        const int64_t eighth = (n1 + 8 * kTcBM - 1) / (8 * kTcBM) * kTcBM;
        panel = std::min(panel, std::max<int64_t>(kTcBM, eighth));
    }
    panel = std::min(panel, n1);
    // direct operands: a panel's first variable is a TMA x coordinate, which
    // must be a multiple of 16 bytes
    if (direct_ok(X, Y, n1, n2, sym) && panel % 16 != 0)
        panel = std::max<int64_t>(16, panel / 16 * 16);
    const int64_t panels = (n1 + panel - 1) / panel;

    TcLayout L;
    GBMI_TRY(tc_prepare(c, X, Y, m, n1, n2, sym, &L));
    MiParams mp;
    GBMI_TRY(rt::mi_params(c, m, &mp));
    const MiVar *va = nullptr, *vb = nullptr;
    GBMI_TRY(mi_vars(static_cast<const int32_t*>(c.va.p), n1, mp, c.ha, &va));
    if (sym)
        vb = va;
    else
        GBMI_TRY(mi_vars(static_cast<const int32_t*>(c.vb.p), n2, mp, c.hb, &vb));

    // every panel's job and tile list, uploaded once
    const int group = std::max(1, g_opt.group_cols);
    std::vector<GramJob> jobs(static_cast<size_t>(panels));
    std::vector<int64_t> first(static_cast<size_t>(panels) + 1, 0);
    std::vector<char> pair_panel(static_cast<size_t>(panels), 0);
    for (int64_t p = 0; p < panels; ++p) {
        const int64_t i0 = p * panel, rows = std::min(panel, n1 - i0);
        const int64_t j0 = sym ? i0 : 0, w = n2 - j0;
        GramJob& g = jobs[static_cast<size_t>(p)];
        std::memset(&g, 0, sizeof(g));
        g.rowA = i0;
        g.strideA = L.rows_a;
        g.rowB = sym ? i0 : (L.direct ? 0 : L.kb * L.rows_a);
        g.strideB = sym ? L.rows_a : L.rows_b;
        g.k_begin = 0;
        g.k_blocks = static_cast<int32_t>(L.kb);
        g.n_a = static_cast<int32_t>(rows);
        g.n_b = static_cast<int32_t>(w);
        g.symmetric = 0;
        const int bn_max = L.fp4 ? kTcBNFp4 : kTcBNMax;
        g.bn = std::min(rt::choose_bn(m, rows, w, false), bn_max);
        if (L.direct && g.bn < kTcBM) g.bn = kTcBM;
        if (!L.direct && use_pair(c, m, rows, w, false, g.bn, bn_max)) {
            g.bn = bn_max;
            pair_panel[static_cast<size_t>(p)] = 1;
        }
        g.va = va + i0;
        g.vb = vb + j0;
        g.ld_out = w;
        g.ld_t = rows;
        g.mp = mp;
        first[static_cast<size_t>(p) + 1] =
            first[static_cast<size_t>(p)] +
            gram_tile_count(rows, w, g.bn, false, pair_panel[p] ? 2 * kTcBM : kTcBM);
    }
    const int64_t total_tiles = first.back();
    std::vector<GramTile> tiles(static_cast<size_t>(total_tiles));
    for (int64_t p = 0; p < panels; ++p) {
        const GramJob& g = jobs[static_cast<size_t>(p)];
        if (first[p + 1] - first[p] > 0x7FFFFFFF) return fail(GBMI_ERR_ARG, "too many tiles");
        gram_tiles(0, g.n_a, g.n_b, g.bn, false, group, tiles.data() + first[p],
                   pair_panel[p] ? 2 * kTcBM : kTcBM);
    }

    const size_t up_bytes = static_cast<size_t>(panel) * n2 * 4;
    const size_t lo_bytes = sym ? static_cast<size_t>(n2) * panel * 4 : 0;
    DevBuf up[2], lo[2], tl;
    cudaStream_t cs = nullptr;
    cudaEvent_t computed[2] = {nullptr, nullptr}, copied[2] = {nullptr, nullptr};
    auto cleanup = [&]() {
        if (cs) cudaStreamSynchronize(cs);
        cudaStreamSynchronize(g_stream);
        for (int s = 0; s < 2; ++s) {
            if (computed[s]) cudaEventDestroy(computed[s]);
            if (copied[s]) cudaEventDestroy(copied[s]);
            rt::release(up[s]);
            rt::release(lo[s]);
        }
        rt::release(tl);
        if (cs) cudaStreamDestroy(cs);
    };
    gbmi_status st = [&]() -> gbmi_status {
        for (int s = 0; s < 2 && s < panels; ++s) {
            GBMI_TRY(ensure(up[s], up_bytes, "panel staging"));
            if (sym) GBMI_TRY(ensure(lo[s], lo_bytes, "mirror staging"));
            GBMI_CUDA(cudaEventCreateWithFlags(&computed[s], cudaEventDisableTiming), "event");
            GBMI_CUDA(cudaEventCreateWithFlags(&copied[s], cudaEventDisableTiming), "event");
        }
        GBMI_TRY(ensure(tl, tiles.size() * sizeof(GramTile), "tile list"));
        GBMI_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "copy stream");
        GBMI_CUDA(cudaMemcpyAsync(tl.p, tiles.data(), tiles.size() * sizeof(GramTile),
                                  cudaMemcpyHostToDevice, g_stream),
                  "tile list upload");
        OperandMaps maps;
        if (L.direct)
            maps = L.maps;
        else if (!make_operand_maps(&maps, static_cast<const uint8_t*>(c.P.p), L.total_rows))
            return fail(GBMI_ERR_CUDA, "cuTensorMapEncodeTiled failed");
        GBMI_TRY(ensure(c.sched, 256, "tile counter"));
        for (int64_t p = 0; p < panels; ++p) {
            const int s = static_cast<int>(p & 1);
            const int64_t i0 = p * panel, rows = std::min(panel, n1 - i0);
            const int64_t j0 = sym ? i0 : 0, w = n2 - j0;
            if (p >= 2) GBMI_CUDA(cudaStreamWaitEvent(g_stream, copied[s], 0), "wait copy");
            GramLaunch G;
            std::memset(&G, 0, sizeof(G));
            G.job0 = jobs[static_cast<size_t>(p)];
            G.job0.out_f = static_cast<float*>(up[s].p);
            G.job0.out_t = sym ? static_cast<float*>(lo[s].p) : nullptr;
            G.tiles = static_cast<const GramTile*>(tl.p) + first[p];
            G.num_tiles = static_cast<int>(first[p + 1] - first[p]);
            G.mode = kTcModeMI;
            G.err = static_cast<unsigned int*>(c.err.p);
            G.timeout_ns = g_opt.timeout_ns;
            G.debug_flags = g_opt.debug_flags;
            G.direct = L.direct ? 1 : 0;
            G.fp4 = L.fp4 ? 1 : 0;
            G.pair = pair_panel[p];
            G.fixup = mp.fixup;
            G.counter = static_cast<unsigned int*>(c.sched.p);
            const int grid =
                G.pair ? 2 * static_cast<int>(std::min<int64_t>(c.pair_clusters, G.num_tiles))
                       : rt::grid_for(c, G.num_tiles);
            GBMI_CUDA(cudaMemsetAsync(G.counter, 0, sizeof(unsigned int), g_stream), "tile counter");
            GBMI_LAUNCH(launch_gram_tc(maps, G, grid, g_stream), "gram_tc_fused_mi");
            GBMI_CUDA(cudaEventRecord(computed[s], g_stream), "event");
            GBMI_CUDA(cudaStreamWaitEvent(cs, computed[s], 0), "wait panel");
            if (sym) {
                GBMI_CUDA(cudaMemcpy2DAsync(host_out + i0 * n2 + i0, n2 * 4, up[s].p, w * 4, w * 4,
                                            rows, cudaMemcpyDeviceToHost, cs),
                          "panel copy");
                if (w > rows)
                    GBMI_CUDA(cudaMemcpy2DAsync(host_out + (i0 + rows) * n2 + i0, n2 * 4,
                                                static_cast<float*>(lo[s].p) + rows * rows,
                                                rows * 4, rows * 4, w - rows,
                                                cudaMemcpyDeviceToHost, cs),
                              "mirror copy");
            } else {
                GBMI_CUDA(cudaMemcpyAsync(host_out + i0 * n2, up[s].p,
                                          static_cast<size_t>(rows) * n2 * 4,
                                          cudaMemcpyDeviceToHost, cs),
                          "panel copy");
            }
            GBMI_CUDA(cudaEventRecord(copied[s], cs), "event");
        }
        GBMI_CUDA(cudaStreamSynchronize(cs), "cudaStreamSynchronize");
        GBMI_CUDA(cudaStreamSynchronize(g_stream), "cudaStreamSynchronize");
        unsigned int err = 0;
        GBMI_CUDA(cudaMemcpy(&err, c.err.p, sizeof(err), cudaMemcpyDeviceToHost),
                  "read error word");
        if (err != 0) {
            cudaMemset(c.err.p, 0, sizeof(err));
            return error_word_status(err);
        }
        return GBMI_OK;
    }();
    cleanup();
    return st;
}

// Sparse input: which form is cheaper, by a model of GB300 rates measured on
// this build (pair enumeration: about 4e10 atomic increments/s, plus the
// elementwise MI; dense: zero + scatter + pack of m*n bytes at HBM rate, plus
// the tensor-core Gram at about 6.4e15 flops/s with FP4 operands, 3.8e15 with
// FP8).  The increments are
// estimated from nnz alone (equal row lengths: sum k(k+1)/2 >= nnz^2/(2m) +
// nnz/2), so the call stays asynchronous; skewed rows only make the
// enumeration look cheaper than it is.
bool csr_dense_is_cheaper(int64_t m, int64_t n, int64_t nnz) {
    const double dm = static_cast<double>(m), dn = static_cast<double>(n);
    const double incr = static_cast<double>(nnz) * nnz / (2.0 * dm) + 0.5 * nnz;
    const double t_enum = incr / 4.0e10 + dn * dn * 8.0 / 6.0e12;
    const double gram_flops = g_opt.fp4 != 0 ? 6.4e15 : 3.8e15;
    const double t_dense = dm * dn * 3.0 / 6.0e12 + dm * dn * dn / gram_flops;
    return t_dense < t_enum;
}

// Sparse input (CSR by samples): pair counts into the upper triangle of N11,
// then either the symmetric count matrix or the MI of every pair; or, when
// the ones are not sparse enough for that to pay, the dense 0/1 matrix in the
// workspace and the tensor-core path on it.
gbmi_status csr_impl(const int64_t* row_ptr, const int32_t* col, int64_t m, int64_t n,
                     int64_t nnz, float* out, int32_t* n11) {
    if (row_ptr == nullptr || (col == nullptr && nnz > 0) || (out == nullptr && n11 == nullptr))
        return fail(GBMI_ERR_ARG, "null pointer");
    GBMI_TRY(check_sizes(m, n, n));
    if (nnz < 0) return fail(GBMI_ERR_ARG, "nnz must be >= 0");
    if (nnz > m * n) return fail(GBMI_ERR_ARG, "nnz exceeds m * n");
    DeviceCtx* cp = nullptr;
    GBMI_TRY(rt::get_ctx(&cp));
    DeviceCtx& c = *cp;
    const bool dense = g_opt.csr_path == 2 ||
                       (g_opt.csr_path == 0 && csr_dense_is_cheaper(m, n, nnz));
    if (dense) {
        GBMI_TRY(ensure(c.Xs, static_cast<size_t>(m) * n, "dense input"));
        uint8_t* Xd = static_cast<uint8_t*>(c.Xs.p);
        GBMI_CUDA(cudaMemsetAsync(Xd, 0, static_cast<size_t>(m) * n, g_stream), "zero dense input");
        GBMI_LAUNCH(launch_csr_densify(row_ptr, col, m, n, nnz, Xd,
                                       static_cast<unsigned int*>(c.err.p), c.sm_count, g_stream),
                    "csr_densify");
        if (n11 != nullptr) return counts_impl(Xd, nullptr, m, n, n, n11, GBMI_PATH_AUTO, true);
        return mi_impl(Xd, nullptr, m, n, n, out, GBMI_PATH_AUTO, true);
    }
    const size_t cbytes = static_cast<size_t>(n) * n * 4;
    int32_t* N11 = n11;
    if (N11 == nullptr) {
        GBMI_TRY(ensure(c.counts, cbytes, "count matrix"));
        N11 = static_cast<int32_t*>(c.counts.p);
    }
    GBMI_CUDA(cudaMemsetAsync(N11, 0, cbytes, g_stream), "zero counts");
    GBMI_LAUNCH(launch_csr_pair_counts(row_ptr, col, m, n, nnz, N11,
                                       static_cast<unsigned int*>(c.err.p), c.sm_count, g_stream),
                "csr_pair_counts");
    if (n11 != nullptr) {
        GBMI_LAUNCH(launch_mirror_upper(N11, n, g_stream), "mirror_upper");
        return GBMI_OK;
    }
    GBMI_TRY(ensure(c.va, static_cast<size_t>(n) * 4, "column counts"));
    GBMI_LAUNCH(launch_diag(N11, n, static_cast<int32_t*>(c.va.p), g_stream), "diag");
    MiParams mp;
    GBMI_TRY(rt::mi_params(c, m, &mp));
    const MiVar* vars = nullptr;
    GBMI_TRY(mi_vars(static_cast<const int32_t*>(c.va.p), n, mp, c.ha, &vars));
    GBMI_LAUNCH(launch_mi_from_counts_sym(N11, n, vars, n, mp, out, n, g_stream, 1),
                "mi_from_counts");
    return GBMI_OK;
}

}  // namespace
}  // namespace gbmi

using namespace gbmi;
using gbmi::rt::g_mu;

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

gbmi_status gbmi_mi_all_pairs_shard(const uint8_t* X, int64_t m, int64_t n, float* out,
                                    int shard, int num_shards) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    return mi_impl(X, nullptr, m, n, n, out, GBMI_PATH_FUSED, true, shard, num_shards);
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

gbmi_status gbmi_mi_all_pairs_to_host(const uint8_t* X, int64_t m, int64_t n, float* host_out,
                                      int64_t panel_rows) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    return blocked_impl(X, nullptr, m, n, n, host_out, panel_rows, true);
}

gbmi_status gbmi_mi_cross_to_host(const uint8_t* X, const uint8_t* Y, int64_t m, int64_t n1,
                                  int64_t n2, float* host_out, int64_t panel_rows) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    return blocked_impl(X, Y, m, n1, n2, host_out, panel_rows, false);
}

gbmi_status gbmi_mi_all_pairs_csr(const int64_t* row_ptr, const int32_t* col_idx, int64_t m,
                                  int64_t n, int64_t nnz, float* out) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    return csr_impl(row_ptr, col_idx, m, n, nnz, out, nullptr);
}

gbmi_status gbmi_counts_all_pairs_csr(const int64_t* row_ptr, const int32_t* col_idx, int64_t m,
                                      int64_t n, int64_t nnz, int32_t* n11) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    return csr_impl(row_ptr, col_idx, m, n, nnz, nullptr, n11);
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
    GBMI_TRY(rt::get_ctx(&cp));
    return pack(X, m, n, nullptr, nullptr, v);
}

gbmi_status gbmi_mi_from_counts(const int32_t* N11, const int32_t* va, const int32_t* vb,
                                int64_t m, int64_t n1, int64_t n2, float* out) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    if (N11 == nullptr || va == nullptr || vb == nullptr || out == nullptr)
        return fail(GBMI_ERR_ARG, "null pointer");
    GBMI_TRY(check_sizes(m, n1, n2));
    DeviceCtx* cp = nullptr;
    GBMI_TRY(rt::get_ctx(&cp));
    DeviceCtx& c = *cp;
    MiParams mp;
    GBMI_TRY(rt::mi_params(c, m, &mp));
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
    GBMI_TRY(rt::get_ctx(&cp));
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
    rt::g_stream = static_cast<cudaStream_t>(stream);
    return GBMI_OK;
}

void* gbmi_get_stream(void) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    return static_cast<void*>(rt::g_stream);
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
            rt::prof_set(value != 0);
            return GBMI_OK;
        case GBMI_OPT_DIRECT:
            g_opt.direct = value != 0 ? 1 : 0;
            return GBMI_OK;
        case GBMI_OPT_PAIR:
            if (value < 0 || value > 2) return fail(GBMI_ERR_ARG, "pair mode must be 0, 1 or 2");
            g_opt.pair = static_cast<int>(value);
            return GBMI_OK;
        case GBMI_OPT_SPLIT_K:
            if (value < 0 || value > 2) return fail(GBMI_ERR_ARG, "split mode must be 0, 1 or 2");
            g_opt.split_k = static_cast<int>(value);
            return GBMI_OK;
        case GBMI_OPT_FP4:
            g_opt.fp4 = value != 0 ? 1 : 0;
            return GBMI_OK;
        case GBMI_OPT_TAIL_SPLIT:
            if (value < 0 || value > 15) return fail(GBMI_ERR_ARG, "tail split must be in [0, 15]");
            g_opt.tail_split = static_cast<int>(value);
            return GBMI_OK;
        case GBMI_OPT_TAIL_COLS:
            if (value < 0 || value > 4) return fail(GBMI_ERR_ARG, "tail columns must be in [0, 4]");
            g_opt.tail_cols = static_cast<int>(value);
            return GBMI_OK;
        case GBMI_OPT_CSR_PATH:
            if (value < 0 || value > 2) return fail(GBMI_ERR_ARG, "CSR path must be 0, 1 or 2");
            g_opt.csr_path = static_cast<int>(value);
            return GBMI_OK;
        case GBMI_OPT_TILE_N:
            if (value != 0 && value != 64 && value != 128 && value != 256)
                return fail(GBMI_ERR_ARG, "tile width must be 0 (automatic), 64, 128 or 256");
            g_opt.tile_n = static_cast<int>(value);
            return GBMI_OK;
        default:
            return fail(GBMI_ERR_ARG, "unknown option");
    }
}

gbmi_status gbmi_sync(void) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    GBMI_CUDA(cudaStreamSynchronize(rt::g_stream), "cudaStreamSynchronize");
    int dev = 0;
    GBMI_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    DeviceCtx* c = rt::ctx_of(dev);
    if (c == nullptr || !c->ready) return GBMI_OK;
    unsigned int err = 0;
    GBMI_CUDA(cudaMemcpy(&err, c->err.p, sizeof(err), cudaMemcpyDeviceToHost),
              "read error word");
    if (err != 0) {
        GBMI_CUDA(cudaMemset(c->err.p, 0, sizeof(err)), "clear error word");
        return error_word_status(err);
    }
    return GBMI_OK;
}

gbmi_status gbmi_tuner_set(int64_t m, int64_t n, int tile_n) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    if (m < 1 || n < 1) return fail(GBMI_ERR_ARG, "m and n must be >= 1");
    if (tile_n != 64 && tile_n != 128 && tile_n != 256)
        return fail(GBMI_ERR_ARG, "tile width must be 64, 128 or 256");
    rt::tuner_set(m, n, tile_n);
    return GBMI_OK;
}

gbmi_status gbmi_tuner_clear(void) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    rt::tuner_clear();
    return GBMI_OK;
}

gbmi_status gbmi_tuner_set_pair(int64_t m, int64_t n, int pair) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    if (m < 1 || n < 1) return fail(GBMI_ERR_ARG, "m and n must be >= 1");
    if (pair < -1 || pair > 1) return fail(GBMI_ERR_ARG, "pair must be -1, 0 or 1");
    rt::tuner_set_pair(m, n, pair);
    return GBMI_OK;
}

int gbmi_tuner_pair(int64_t m, int64_t n) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    if (m < 1 || n < 1) return -1;
    return rt::tuner_pair(m, n);
}

gbmi_status gbmi_tuner_set_split(int64_t m, int64_t n, int parts) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    if (m < 1 || n < 1) return fail(GBMI_ERR_ARG, "m and n must be >= 1");
    if (parts < 0 || parts > 128) return fail(GBMI_ERR_ARG, "parts must be in [0, 128]");
    rt::tuner_set_split(m, n, parts);
    return GBMI_OK;
}

int gbmi_tuner_split(int64_t m, int64_t n) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    if (m < 1 || n < 1) return 0;
    return rt::tuner_split(m, n);
}

int gbmi_tail_cols_plan(int tiles, int units, int* parts) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    int p = 0;
    const int S = tail_cols_plan(tiles, units, &p);
    if (parts != nullptr) *parts = p;
    return S;
}

int gbmi_tile_n(int64_t m, int64_t n) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    if (m < 1 || n < 1) return 0;
    return rt::choose_bn(m, n, n, true);
}

uint64_t gbmi_launch_count(void) { return rt::g_launches.load(); }

gbmi_status gbmi_shutdown(void) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    int cur = 0;
    if (cudaGetDevice(&cur) != cudaSuccess) return GBMI_OK;
    for (int d = 0; d < 64; ++d) {
        DeviceCtx* c = rt::ctx_of(d);
        if (c == nullptr || !c->ready) continue;
        cudaSetDevice(d);
        cudaDeviceSynchronize();
        rt::release(c->sched);
        rt::release(c->split_jobs);
        rt::release(c->split_tiles);
        rt::release(c->split_part);
        rt::release(c->tail_tiles);
        rt::release(c->col_tiles);
        rt::release(c->part_counts);
        rt::release(c->part_arrive);
        rt::release(c->peak_err);
        for (DevBuf* b : {&c->P, &c->Ba, &c->Bb, &c->va, &c->vb, &c->ha, &c->hb, &c->counts,
                          &c->T, &c->err, &c->tiles, &c->Xs, &c->Ys, &c->outs, &c->flag,
                          &c->panel})
            rt::release(*b);
        for (cudaEvent_t e : c->events) cudaEventDestroy(e);
        if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
        if (c->hflags) cudaFreeHost(c->hflags);
        *c = DeviceCtx();
    }
    cudaSetDevice(cur);
    return GBMI_OK;
}

int gbmi_profile_entries(void) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    rt::prof_collect();
    return rt::prof_entries();
}

const char* gbmi_profile_name(int k) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    return rt::prof_name(k);
}

double gbmi_profile_ms(int k) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    return rt::prof_ms(k);
}

int64_t gbmi_profile_launches(int k) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    return rt::prof_launches(k);
}

gbmi_status gbmi_profile_reset(void) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    rt::prof_reset();
    return GBMI_OK;
}

int gbmi_version(void) { return 200; }

}  // extern "C"
