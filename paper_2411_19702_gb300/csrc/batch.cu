// Batched runs: many independent all-pairs / cross problems in one grouped
// pipeline captured in a CUDA graph (see gbmi_batch_* in gbmi.h).
//
// Plan layout in one workspace:
//   P      every job's K-block-major operand(s), FP4 (the default) or FP8 as
//          GBMI_OPT_FP4 was when the plan was made, one after another, so one
//          set of TMA descriptors reaches all of them;
//   v      every operand's column counts, one after another;
//   vars   the per-variable epilogue terms, same indexing as v;
//   tables PackJob[] (one per operand), variable ranges and MiParams per
//          operand, GramJob[] (one per job) and the flat GramTile[] list.
// The graph runs: zero(v) -> grouped pack -> grouped mi_vars -> the
// persistent Gram over all tiles: large jobs on CTA pairs in one launch, the
// rest on single-CTA tiles in a second (each in descending per-tile cost, so
// the persistent CTAs end with the small tiles).
#include <algorithm>
#include <cstring>
#include <numeric>
#include <vector>

#include "runtime.h"

struct gbmi_batch {
    int device = -1;
    int k = 0;
    std::vector<gbmi_job> jobs;
    gbmi::rt::DevBuf P, v, vars, packjobs, ctajob, varbegin, params, gramjobs, tiles, sched;
    std::vector<gbmi::PackJob> hpack;
    std::vector<int64_t> hvarbegin;
    std::vector<gbmi::MiParams> hparams;
    std::vector<gbmi::GramJob> hgram;
    std::vector<int> pack_of_x, pack_of_y;   // pack-job index of each job's X and Y
    int64_t total_rows = 0, total_vars = 0, total_ctas = 0;
    int64_t num_tiles = 0;
    int64_t pair_tiles = 0;   // tiles [0, pair_tiles) run on CTA pairs (256 x 256 or 240)
    bool fp4 = false;         // operands in the FP4 form
    int grid = 0, pair_grid = 0;
    gbmi::OperandMaps maps;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace gbmi {
namespace {

using rt::ensure;
using rt::fail;

constexpr int64_t kMaxM = int64_t{1} << 24;

gbmi_status check_job(const gbmi_job& j, int idx) {
    const std::string at = " (job " + std::to_string(idx) + ")";
    if (j.X == nullptr || j.out == nullptr) return fail(GBMI_ERR_ARG, "null pointer" + at);
    if (j.m < 1 || j.m > kMaxM) return fail(GBMI_ERR_ARG, "batch jobs need 1 <= m <= 2^24" + at);
    if (j.n < 1 || j.n > (int64_t{1} << 20)) return fail(GBMI_ERR_ARG, "n out of range" + at);
    if (j.Y != nullptr && (j.n2 < 1 || j.n2 > (int64_t{1} << 20)))
        return fail(GBMI_ERR_ARG, "n2 out of range" + at);
    return GBMI_OK;
}

void set_pack_pointers(PackJob& pj, const uint8_t* X) {
    pj.X = X;
    pj.vec = (pj.ldx % 16 == 0) && (pj.n % 16 == 0) && (reinterpret_cast<uintptr_t>(X) % 16 == 0);
}

void set_gram_output(GramJob& g, float* out) {
    g.out_f = out;
}

gbmi_status upload(rt::DevBuf& b, const void* host, size_t bytes, const char* what) {
    GBMI_TRY(ensure(b, bytes, what));
    GBMI_CUDA(cudaMemcpy(b.p, host, bytes, cudaMemcpyHostToDevice), what);
    return GBMI_OK;
}

void release_plan(gbmi_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap) cudaStreamDestroy(b->cap);
    for (rt::DevBuf* d : {&b->P, &b->v, &b->vars, &b->packjobs, &b->ctajob, &b->varbegin, &b->params,
                          &b->gramjobs, &b->tiles, &b->sched})
        rt::release(*d);
}

gbmi_status enqueue(gbmi_batch* b, cudaStream_t s, unsigned int* err) {
    GBMI_CUDA(launch_zero_u32(b->v.p, b->total_vars, s), "batch zero");
    GBMI_CUDA(launch_pack_grouped(static_cast<const PackJob*>(b->packjobs.p),
                                  static_cast<int>(b->hpack.size()), b->total_ctas,
                                  static_cast<const int32_t*>(b->ctajob.p), s),
              "batch pack");
    GBMI_CUDA(launch_mi_vars_grouped(static_cast<const int32_t*>(b->v.p),
                                     static_cast<const int64_t*>(b->varbegin.p),
                                     static_cast<int>(b->hpack.size()), b->total_vars,
                                     static_cast<const MiParams*>(b->params.p),
                                     static_cast<MiVar*>(b->vars.p), s),
              "batch mi_vars");
    GramLaunch L;
    std::memset(&L, 0, sizeof(L));
    L.jobs = static_cast<const GramJob*>(b->gramjobs.p);
    L.mode = kTcModeMI;
    L.fixup = b->hgram.empty() ? 0 : b->hgram[0].mp.fixup;   // one setting for every job
    L.fp4 = b->fp4 ? 1 : 0;
    L.err = err;
    L.timeout_ns = rt::g_opt.timeout_ns;
    L.debug_flags = rt::g_opt.debug_flags;
    if (b->pair_tiles > 0) {   // the large jobs, on CTA pairs
        GramLaunch P = L;
        P.tiles = static_cast<const GramTile*>(b->tiles.p);
        P.num_tiles = static_cast<int>(b->pair_tiles);
        P.pair = 1;
        P.counter = static_cast<unsigned int*>(b->sched.p);
        GBMI_CUDA(cudaMemsetAsync(b->sched.p, 0, sizeof(unsigned int), s), "batch tile counter");
        GBMI_CUDA(launch_gram_tc(b->maps, P, b->pair_grid, s), "batch gram (pairs)");
    }
    if (b->num_tiles > b->pair_tiles) {
        L.tiles = static_cast<const GramTile*>(b->tiles.p) + b->pair_tiles;
        L.num_tiles = static_cast<int>(b->num_tiles - b->pair_tiles);
        L.counter = static_cast<unsigned int*>(b->sched.p);
        GBMI_CUDA(cudaMemsetAsync(b->sched.p, 0, sizeof(unsigned int), s), "batch tile counter");
        GBMI_CUDA(launch_gram_tc(b->maps, L, b->grid, s), "batch gram");
    }
    return GBMI_OK;
}

gbmi_status create(const gbmi_job* jobs, int k, gbmi_batch** out) {
    if (jobs == nullptr || out == nullptr || k < 1) return fail(GBMI_ERR_ARG, "empty batch");
    for (int i = 0; i < k; ++i) GBMI_TRY(check_job(jobs[i], i));
    rt::DeviceCtx* cp = nullptr;
    GBMI_TRY(rt::get_ctx(&cp));
    rt::DeviceCtx& c = *cp;
    gbmi_batch* b = new gbmi_batch();
    b->k = k;
    b->jobs.assign(jobs, jobs + k);
    GBMI_CUDA(cudaGetDevice(&b->device), "cudaGetDevice");

    // MI parameters: one n log n table for the largest m when the FP64 combine is on
    int64_t m_max = 0;
    for (const gbmi_job& j : b->jobs) m_max = std::max(m_max, j.m);
    MiParams pmax;
    gbmi_status st = rt::mi_params(c, m_max, &pmax);
    if (st != GBMI_OK) {
        delete b;
        return st;
    }

    // ---- layout
    const bool fp4 = rt::g_opt.fp4 != 0;
    const int bn_max = fp4 ? kTcBNFp4 : kTcBNMax;
    b->fp4 = fp4;
    int64_t rows = 0, vars = 0;
    auto add_operand = [&](const uint8_t* X, int64_t m, int64_t n, const MiParams& mp) {
        PackJob pj;
        std::memset(&pj, 0, sizeof(pj));
        pj.m = m;
        pj.n = n;
        pj.ldx = n;
        pj.rows_p = pack_rows(n);
        pj.ldp = pack_ld_of(m, fp4);
        pj.fp4 = fp4 ? 1 : 0;
        set_pack_pointers(pj, X);
        pj.P = reinterpret_cast<uint8_t*>(rows * kTcBK);        // offset; rebased below
        pj.v = reinterpret_cast<int32_t*>(vars * 4);            // offset; rebased below
        b->hpack.push_back(pj);
        b->hvarbegin.push_back(vars);
        b->hparams.push_back(mp);
        const int64_t row0 = rows, var0 = vars;
        rows += (pj.ldp / kb_samples(fp4)) * pj.rows_p;
        vars += n;
        return std::make_pair(row0, var0);
    };
    for (int i = 0; i < k; ++i) {
        const gbmi_job& j = b->jobs[i];
        const bool sym = j.Y == nullptr;
        const MiParams mp = rt::mi_params_plain(j.m, pmax.fixup, pmax.T);
        const auto xa = add_operand(j.X, j.m, j.n, mp);
        b->pack_of_x.push_back(static_cast<int>(b->hpack.size()) - 1);
        std::pair<int64_t, int64_t> yb = xa;
        if (!sym) {
            yb = add_operand(j.Y, j.m, j.n2, mp);
            b->pack_of_y.push_back(static_cast<int>(b->hpack.size()) - 1);
        } else {
            b->pack_of_y.push_back(-1);
        }
        const int64_t nb = sym ? j.n : j.n2;
        GramJob g;
        std::memset(&g, 0, sizeof(g));
        g.rowA = xa.first;
        g.rowB = yb.first;
        g.strideA = pack_rows(j.n);
        g.strideB = pack_rows(nb);
        g.k_begin = 0;
        g.k_blocks = static_cast<int32_t>(pack_ld_of(j.m, fp4) / kb_samples(fp4));
        g.n_a = static_cast<int32_t>(j.n);
        g.n_b = static_cast<int32_t>(nb);
        g.symmetric = sym ? 1 : 0;
        g.bn = std::min(rt::choose_bn(j.m, j.n, nb, sym), bn_max);
        g.va = reinterpret_cast<const MiVar*>(xa.second * sizeof(MiVar));   // rebased below
        g.vb = reinterpret_cast<const MiVar*>(yb.second * sizeof(MiVar));
        g.ld_out = nb;
        set_gram_output(g, j.out);
        g.mp = mp;
        b->hgram.push_back(g);
    }
    b->total_rows = rows;
    b->total_vars = vars;
    b->hvarbegin.push_back(vars);
    if (rows >= (int64_t{1} << 31)) {
        delete b;
        return fail(GBMI_ERR_ARG, "batch operands exceed 2^31 rows of 128 bytes");
    }

    // ---- device buffers, with the offsets above turned into pointers
    st = ensure(b->P, static_cast<size_t>(rows) * kTcBK, "batch operands");
    if (st == GBMI_OK) st = ensure(b->v, static_cast<size_t>(vars) * 4, "batch column counts");
    if (st == GBMI_OK) st = ensure(b->vars, static_cast<size_t>(vars) * sizeof(MiVar), "batch terms");
    if (st == GBMI_OK) st = ensure(b->sched, 256, "batch tile counter");
    if (st != GBMI_OK) {
        release_plan(b);
        delete b;
        return st;
    }
    uint8_t* Pb = static_cast<uint8_t*>(b->P.p);
    int32_t* vb = static_cast<int32_t*>(b->v.p);
    MiVar* varsb = static_cast<MiVar*>(b->vars.p);
    int64_t ctas = 0;
    for (PackJob& pj : b->hpack) {
        pj.P = Pb + reinterpret_cast<uintptr_t>(pj.P);
        pj.v = vb + reinterpret_cast<uintptr_t>(pj.v) / 4;
        pj.cta_begin = ctas;
        ctas += pack_job_ctas(pj, true);
    }
    b->total_ctas = ctas;
    // CTA -> pack job table of the grouped pack
    std::vector<int32_t> cta_job(static_cast<size_t>(ctas));
    for (size_t q = 0; q < b->hpack.size(); ++q) {
        const int64_t e = q + 1 < b->hpack.size() ? b->hpack[q + 1].cta_begin : ctas;
        std::fill(cta_job.begin() + b->hpack[q].cta_begin, cta_job.begin() + e,
                  static_cast<int32_t>(q));
    }
    for (GramJob& g : b->hgram) {
        g.va = varsb + reinterpret_cast<uintptr_t>(g.va) / sizeof(MiVar);
        g.vb = varsb + reinterpret_cast<uintptr_t>(g.vb) / sizeof(MiVar);
    }

    // ---- tiles.  Jobs whose both sides span at least kPairMinN variables run
    // on CTA pairs (256 x 256 tiles, 256 x 240 for FP4; half the operand bytes
    // per SM per MMA) in
    // a first launch; the rest on single-CTA tiles of their own width in a
    // second.  Within each launch, jobs by descending per-tile cost, each job
    // in its own order.
    constexpr int64_t kPairMinN = 768;
    std::vector<char> pair_job(static_cast<size_t>(k), 0);
    const bool pairs_ok = rt::g_opt.pair != 0 && c.pair_clusters > 0 && rt::g_opt.tile_n == 0;
    for (int i = 0; i < k; ++i) {
        GramJob& g = b->hgram[i];
        // a tuned bucket decides; else the size rule
        const int tuned = rt::tuner_pair(g.mp.m, std::max<int64_t>(g.n_a, g.n_b));
        const bool rule = g.n_a >= kPairMinN && g.n_b >= kPairMinN;
        if (pairs_ok && (rt::g_opt.pair == 2 || (tuned >= 0 ? tuned == 1 : rule))) {
            pair_job[i] = 1;
            g.bn = bn_max;
        }
    }
    auto tile_m = [&](int i) { return pair_job[i] ? 2 * kTcBM : kTcBM; };
    std::vector<int> order(k);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        if (pair_job[x] != pair_job[y]) return pair_job[x] > pair_job[y];
        const GramJob& a = b->hgram[x];
        const GramJob& c2 = b->hgram[y];
        return static_cast<int64_t>(a.k_blocks) * (tile_m(x) + a.bn) >
               static_cast<int64_t>(c2.k_blocks) * (tile_m(y) + c2.bn);
    });
    int64_t ntiles = 0, npair = 0;
    for (int i = 0; i < k; ++i) {
        const GramJob& g = b->hgram[i];
        const int64_t t = gram_tile_count(g.n_a, g.n_b, g.bn, g.symmetric != 0, tile_m(i));
        ntiles += t;
        if (pair_job[i]) npair += t;
    }
    if (ntiles > 0x7FFFFFFF) {
        release_plan(b);
        delete b;
        return fail(GBMI_ERR_ARG, "too many tiles in one batch");
    }
    std::vector<GramTile> tiles(static_cast<size_t>(ntiles));
    int64_t pos = 0;
    for (int i : order) {
        const GramJob& g = b->hgram[i];
        gram_tiles(i, g.n_a, g.n_b, g.bn, g.symmetric != 0, rt::g_opt.group_cols,
                   tiles.data() + pos, tile_m(i));
        pos += gram_tile_count(g.n_a, g.n_b, g.bn, g.symmetric != 0, tile_m(i));
    }
    b->num_tiles = ntiles;
    b->pair_tiles = npair;
    b->grid = rt::grid_for(c, ntiles - npair);
    b->pair_grid = 2 * static_cast<int>(std::min<int64_t>(c.pair_clusters, npair));

    st = upload(b->packjobs, b->hpack.data(), b->hpack.size() * sizeof(PackJob), "batch pack table");
    if (st == GBMI_OK && ctas > 0)
        st = upload(b->ctajob, cta_job.data(), cta_job.size() * sizeof(int32_t),
                    "batch pack CTA table");
    if (st == GBMI_OK)
        st = upload(b->varbegin, b->hvarbegin.data(), b->hvarbegin.size() * sizeof(int64_t),
                    "batch variable ranges");
    if (st == GBMI_OK)
        st = upload(b->params, b->hparams.data(), b->hparams.size() * sizeof(MiParams),
                    "batch parameters");
    if (st == GBMI_OK)
        st = upload(b->gramjobs, b->hgram.data(), b->hgram.size() * sizeof(GramJob),
                    "batch job table");
    if (st == GBMI_OK)
        st = upload(b->tiles, tiles.data(), tiles.size() * sizeof(GramTile), "batch tile list");
    if (st == GBMI_OK && !make_operand_maps(&b->maps, Pb, rows))
        st = fail(GBMI_ERR_CUDA, "cuTensorMapEncodeTiled failed");
    if (st != GBMI_OK) {
        release_plan(b);
        delete b;
        return st;
    }

    // ---- capture the pipeline once
    cudaError_t e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        release_plan(b);
        delete b;
        return rt::cuda_fail(e, "batch graph capture");
    }
    st = enqueue(b, b->cap, static_cast<unsigned int*>(c.err.p));
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(b->cap, &graph);
    b->graph = graph;
    if (st == GBMI_OK && e != cudaSuccess) st = rt::cuda_fail(e, "batch graph capture");
    if (st == GBMI_OK) {
        e = cudaGraphInstantiate(&b->exec, b->graph, 0);
        if (e != cudaSuccess) st = rt::cuda_fail(e, "batch graph instantiate");
    }
    if (st != GBMI_OK) {
        release_plan(b);
        delete b;
        return st;
    }
    *out = b;
    return GBMI_OK;
}

// Kernels in the plan's graph: zero, grouped pack, grouped per-variable
// terms, and one or two Gram launches.
uint64_t launches_per_run(const gbmi_batch* b) {
    return 3u + (b->pair_tiles > 0 ? 1u : 0u) + (b->num_tiles > b->pair_tiles ? 1u : 0u);
}

gbmi_status run(gbmi_batch* b) {
    int dev = 0;
    GBMI_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev != b->device) return fail(GBMI_ERR_ARG, "batch plan belongs to another device");
    cudaEvent_t ev0 = rt::prof_begin(rt::g_stream);
    GBMI_CUDA(cudaGraphLaunch(b->exec, rt::g_stream), "cudaGraphLaunch");
    rt::prof_end("batch_graph", ev0, rt::g_stream);
    rt::g_launches.fetch_add(launches_per_run(b), std::memory_order_relaxed);
    return GBMI_OK;
}

}  // namespace
}  // namespace gbmi

using namespace gbmi;
using gbmi::rt::g_mu;

extern "C" {

gbmi_status gbmi_batch_create(const gbmi_job* jobs, int k, gbmi_batch** plan) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    if (plan == nullptr) return rt::fail(GBMI_ERR_ARG, "null plan pointer");
    *plan = nullptr;
    return create(jobs, k, plan);
}

gbmi_status gbmi_batch_run(gbmi_batch* plan) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    if (plan == nullptr) return rt::fail(GBMI_ERR_ARG, "null plan");
    return run(plan);
}

gbmi_status gbmi_batch_set_io(gbmi_batch* plan, const gbmi_job* jobs, int k) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    if (plan == nullptr || jobs == nullptr) return rt::fail(GBMI_ERR_ARG, "null pointer");
    if (k != plan->k) return rt::fail(GBMI_ERR_ARG, "job count differs from the plan's");
    for (int i = 0; i < k; ++i) {
        const gbmi_job& a = plan->jobs[i];
        const gbmi_job& j = jobs[i];
        if (j.m != a.m || j.n != a.n || (j.Y == nullptr) != (a.Y == nullptr) ||
            (j.Y != nullptr && j.n2 != a.n2))
            return rt::fail(GBMI_ERR_ARG, "job " + std::to_string(i) + " changes shape");
        if (j.X == nullptr || j.out == nullptr || (a.Y != nullptr && j.Y == nullptr))
            return rt::fail(GBMI_ERR_ARG, "null pointer (job " + std::to_string(i) + ")");
    }
    for (int i = 0; i < k; ++i) {
        plan->jobs[i] = jobs[i];
        set_pack_pointers(plan->hpack[plan->pack_of_x[i]], jobs[i].X);
        if (plan->pack_of_y[i] >= 0) set_pack_pointers(plan->hpack[plan->pack_of_y[i]], jobs[i].Y);
        set_gram_output(plan->hgram[i], jobs[i].out);
    }
    GBMI_CUDA(cudaMemcpyAsync(plan->packjobs.p, plan->hpack.data(),
                              plan->hpack.size() * sizeof(PackJob), cudaMemcpyHostToDevice,
                              rt::g_stream),
              "batch pack table");
    GBMI_CUDA(cudaMemcpyAsync(plan->gramjobs.p, plan->hgram.data(),
                              plan->hgram.size() * sizeof(GramJob), cudaMemcpyHostToDevice,
                              rt::g_stream),
              "batch job table");
    return GBMI_OK;
}

gbmi_status gbmi_batch_destroy(gbmi_batch* plan) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    if (plan == nullptr) return GBMI_OK;
    cudaDeviceSynchronize();
    release_plan(plan);
    delete plan;
    return GBMI_OK;
}

gbmi_status gbmi_mi_batch(const gbmi_job* jobs, int k) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    gbmi_batch* plan = nullptr;
    GBMI_TRY(create(jobs, k, &plan));
    gbmi_status st = run(plan);
    if (st == GBMI_OK) {
        cudaError_t e = cudaStreamSynchronize(rt::g_stream);
        if (e != cudaSuccess) st = rt::cuda_fail(e, "cudaStreamSynchronize");
    }
    cudaDeviceSynchronize();
    release_plan(plan);
    delete plan;
    return st;
}

int64_t gbmi_batch_tiles(const gbmi_batch* plan) { return plan ? plan->num_tiles : 0; }

}  // extern "C"
