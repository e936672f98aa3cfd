// Serving: a request loop with continuous batching over resident datasets
// (see gbmi_server_* in gbmi.h).
//
// Memory: one device arena of the budget, sub-allocated first-fit in 256-byte
// units.  A dataset owns a packed-operand region (K-block-major rows of 128
// bytes, FP4 or FP8 as GBMI_OPT_FP4 was when the server was created, so the
// arena's TMA descriptors reach every dataset) and a
// region for its column counts and per-variable terms; a request owns its
// output.  Admission is by memory: a queued request is admitted when its
// output, and the regions of any dataset it needs that is not yet resident,
// can be allocated.
//
// Worker thread: completes the batches whose event has fired (results become
// visible to waiters), then, while a stream slot is free (two slots), admits
// queued requests in arrival order (those that do not fit yet wait; later
// ones may pass them) up to max_batch and launches them as one batch on the
// slot's stream: zero + grouped pack + per-variable terms for the datasets
// not yet resident, then one persistent Gram launch over the tiles of all
// admitted requests, then the batch's error word is copied to pinned memory
// and an event recorded.  A batch that reads a dataset packed by the batch on
// the other slot waits for that batch's "packed" event first.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <numeric>
#include <thread>
#include <vector>

#include "runtime.h"

namespace gbmi {
namespace {

using Clock = std::chrono::steady_clock;

class Arena {
   public:
    void init(size_t bytes) {
        free_.clear();
        free_[0] = bytes;
        size_ = bytes;
        used_ = 0;
    }
    static size_t round(size_t b) { return (b + 255) & ~static_cast<size_t>(255); }
    int64_t alloc(size_t bytes) {
        bytes = round(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                const int64_t off = it->first;
                const size_t rem = it->second - bytes;
                free_.erase(it);
                if (rem > 0) free_[off + static_cast<int64_t>(bytes)] = rem;
                used_ += bytes;
                return off;
            }
        }
        return -1;
    }
    void release(int64_t off, size_t bytes) {
        if (off < 0) return;
        bytes = round(bytes);
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto next = std::next(it);
        if (next != free_.end() && it->first + static_cast<int64_t>(it->second) == next->first) {
            it->second += next->second;
            free_.erase(next);
        }
        if (it != free_.begin()) {
            auto prev = std::prev(it);
            if (prev->first + static_cast<int64_t>(prev->second) == it->first) {
                prev->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t size() const { return size_; }
    size_t used() const { return used_; }

   private:
    std::map<int64_t, size_t> free_;
    size_t size_ = 0, used_ = 0;
};

struct Dataset {
    const uint8_t* X = nullptr;
    int64_t m = 0, n = 0, kb = 0, rows_p = 0;
    int64_t off_p = -1, off_v = -1;   // arena offsets (-1: not resident)
    size_t bytes_p = 0, bytes_v = 0;
    int pack_slot = -1;               // slot whose batch packs it, until that batch is done
    int users = 0;                    // queued or running requests that read it
    bool removed = false;
};

struct Request {
    int64_t a = -1, b = -1;
    int64_t n_a = 0, n_b = 0, m = 0;
    int64_t off_out = -1;
    size_t bytes_out = 0;
    int state = 0;                    // 0 queued, 1 running, 2 done, 3 failed or cancelled
    gbmi_status err = GBMI_OK;
    Clock::time_point t_submit, t_done;
    int64_t pairs = 0;
};

struct Slot {
    cudaStream_t s = nullptr;
    cudaEvent_t done = nullptr, packed = nullptr;
    bool busy = false;
    std::vector<int64_t> tickets;
    std::vector<int64_t> packs;       // datasets packed by this batch
    rt::DevBuf dpack, djobs, dtiles;
    void* pin = nullptr;
    size_t pin_cap = 0;
    unsigned int* pin_err = nullptr;
    int64_t off_ctrl = -1;            // arena: tile counter, error word, pair tile counter
};

}  // namespace
}  // namespace gbmi

struct gbmi_server {
    int device = 0;
    int sm_count = 0;
    int pair_clusters = 0;
    int max_batch = 64;
    bool fp4 = false;   // datasets packed in the FP4 form (GBMI_OPT_FP4 at creation)
    gbmi::rt::DevBuf mem;
    gbmi::Arena arena;
    gbmi::OperandMaps maps;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::map<int64_t, gbmi::Dataset> datasets;
    std::map<int64_t, gbmi::Request> reqs;
    std::deque<int64_t> queue;
    int64_t next_ds = 0, next_ticket = 0;
    gbmi::Slot slots[2];
    std::thread worker;
    bool stop = false;
    // statistics
    std::vector<double> lat_ms;
    int64_t pairs_done = 0, batches = 0, batched = 0;
    bool started = false;
    gbmi::Clock::time_point t_first, t_last;
};

namespace gbmi {
namespace {

uint8_t* at(gbmi_server* S, int64_t off) { return static_cast<uint8_t*>(S->mem.p) + off; }

// Allocate the regions of a dataset that is not resident.  false: no room.
bool make_resident(gbmi_server* S, Dataset& d) {
    if (d.off_p >= 0) return true;
    d.bytes_p = static_cast<size_t>(d.kb * d.rows_p) * kTcBK;
    d.bytes_v = Arena::round(static_cast<size_t>(d.n) * 4) + static_cast<size_t>(d.n) * sizeof(MiVar);
    const int64_t p = S->arena.alloc(d.bytes_p);
    if (p < 0) return false;
    const int64_t v = S->arena.alloc(d.bytes_v);
    if (v < 0) {
        S->arena.release(p, d.bytes_p);
        return false;
    }
    d.off_p = p;
    d.off_v = v;
    return true;
}

void drop_dataset_if_done(gbmi_server* S, int64_t id) {
    auto it = S->datasets.find(id);
    if (it == S->datasets.end()) return;
    Dataset& d = it->second;
    if (!d.removed || d.users > 0 || d.pack_slot >= 0) return;
    S->arena.release(d.off_p, d.bytes_p);
    S->arena.release(d.off_v, d.bytes_v);
    S->datasets.erase(it);
}

int32_t* v_of(gbmi_server* S, const Dataset& d) {
    return reinterpret_cast<int32_t*>(at(S, d.off_v));
}
MiVar* vars_of(gbmi_server* S, const Dataset& d) {
    return reinterpret_cast<MiVar*>(at(S, d.off_v) + Arena::round(static_cast<size_t>(d.n) * 4));
}

cudaError_t stage_upload(Slot& sl, rt::DevBuf& dst, const void* src, size_t bytes, size_t pin_off) {
    std::memcpy(static_cast<uint8_t*>(sl.pin) + pin_off, src, bytes);
    return cudaMemcpyAsync(dst.p, static_cast<uint8_t*>(sl.pin) + pin_off, bytes,
                           cudaMemcpyHostToDevice, sl.s);
}

// Launch the admitted requests as one batch on slot k (called with S->mu held).
gbmi_status launch_batch(gbmi_server* S, int k, const std::vector<int64_t>& tickets) {
    Slot& sl = S->slots[k];
    const Slot& other = S->slots[1 - k];
    sl.tickets = tickets;
    sl.packs.clear();
    bool wait_other = false;
    for (int64_t t : tickets) {
        const Request& r = S->reqs[t];
        for (int64_t id : {r.a, r.b}) {
            if (id < 0) continue;
            Dataset& d = S->datasets[id];
            if (d.pack_slot < 0 && std::find(sl.packs.begin(), sl.packs.end(), id) == sl.packs.end() &&
                d.X != nullptr) {
                sl.packs.push_back(id);
            } else if (d.pack_slot == 1 - k && other.busy) {
                wait_other = true;
            }
        }
    }
    for (int64_t id : sl.packs) S->datasets[id].pack_slot = k;
    if (wait_other) GBMI_CUDA(cudaStreamWaitEvent(sl.s, other.packed, 0), "serve wait");

    // host tables
    std::vector<PackJob> pj;
    int64_t ctas = 0;
    for (int64_t id : sl.packs) {
        Dataset& d = S->datasets[id];
        GBMI_CUDA(cudaMemsetAsync(v_of(S, d), 0, static_cast<size_t>(d.n) * 4, sl.s), "serve zero");
        PackJob j;
        std::memset(&j, 0, sizeof(j));
        j.X = d.X;
        j.m = d.m;
        j.n = d.n;
        j.ldx = d.n;
        j.P = at(S, d.off_p);
        j.v = v_of(S, d);
        j.rows_p = d.rows_p;
        j.ldp = d.kb * kb_samples(S->fp4);
        j.fp4 = S->fp4 ? 1 : 0;
        j.cta_begin = ctas;
        ctas += pack_job_ctas(j);
        pj.push_back(j);
    }
    std::vector<GramJob> gj;
    std::vector<char> pair_job;
    std::vector<int64_t> order(tickets.size());
    std::iota(order.begin(), order.end(), 0);
    int64_t ntiles = 0, npair = 0;
    // requests whose both sides span at least 768 variables run on CTA pairs
    constexpr int64_t kPairMinN = 768;
    const bool pairs_ok = rt::g_opt.pair != 0 && S->pair_clusters > 0 && rt::g_opt.tile_n == 0;
    const int bn_max = S->fp4 ? kTcBNFp4 : kTcBNMax;
    for (int64_t t : tickets) {
        const Request& r = S->reqs[t];
        const Dataset& da = S->datasets[r.a];
        const Dataset& db = S->datasets[r.b >= 0 ? r.b : r.a];
        const bool sym = r.b < 0;
        GramJob g;
        std::memset(&g, 0, sizeof(g));
        g.rowA = da.off_p / kTcBK;
        g.rowB = db.off_p / kTcBK;
        g.strideA = da.rows_p;
        g.strideB = db.rows_p;
        g.k_begin = 0;
        g.k_blocks = static_cast<int32_t>(da.kb);
        g.n_a = static_cast<int32_t>(r.n_a);
        g.n_b = static_cast<int32_t>(r.n_b);
        g.symmetric = sym ? 1 : 0;
        {
            std::lock_guard<std::recursive_mutex> lk(rt::g_mu);
            g.bn = std::min(rt::choose_bn(r.m, r.n_a, r.n_b, sym), bn_max);
        }
        g.va = vars_of(S, da);
        g.vb = vars_of(S, db);
        g.out_f = reinterpret_cast<float*>(at(S, r.off_out));
        g.ld_out = r.n_b;
        g.mp = rt::mi_params_plain(r.m, 0, nullptr);
        const bool pj =
            pairs_ok && (rt::g_opt.pair == 2 || (r.n_a >= kPairMinN && r.n_b >= kPairMinN));
        if (pj) g.bn = bn_max;
        gj.push_back(g);
        pair_job.push_back(pj ? 1 : 0);
        const int64_t nt = gram_tile_count(r.n_a, r.n_b, g.bn, sym, pj ? 2 * kTcBM : kTcBM);
        ntiles += nt;
        if (pj) npair += nt;
    }
    auto tile_m = [&](int64_t i) { return pair_job[i] ? 2 * kTcBM : kTcBM; };
    std::stable_sort(order.begin(), order.end(), [&](int64_t x, int64_t y) {
        if (pair_job[x] != pair_job[y]) return pair_job[x] > pair_job[y];
        return static_cast<int64_t>(gj[x].k_blocks) * (tile_m(x) + gj[x].bn) >
               static_cast<int64_t>(gj[y].k_blocks) * (tile_m(y) + gj[y].bn);
    });
    std::vector<GramTile> tiles(static_cast<size_t>(ntiles));
    int64_t pos = 0;
    for (int64_t i : order) {
        const GramJob& g = gj[i];
        gram_tiles(static_cast<int>(i), g.n_a, g.n_b, g.bn, g.symmetric != 0, rt::g_opt.group_cols,
                   tiles.data() + pos, tile_m(i));
        pos += gram_tile_count(g.n_a, g.n_b, g.bn, g.symmetric != 0, tile_m(i));
    }

    // device tables through the slot's pinned staging buffer
    const size_t b_pack = pj.size() * sizeof(PackJob), b_jobs = gj.size() * sizeof(GramJob);
    const size_t b_tiles = tiles.size() * sizeof(GramTile);
    const size_t need = Arena::round(b_pack) + Arena::round(b_jobs) + Arena::round(b_tiles) + 256;
    if (sl.pin_cap < need) {
        if (sl.pin) cudaFreeHost(sl.pin);
        sl.pin = nullptr;
        GBMI_CUDA(cudaMallocHost(&sl.pin, need * 2), "serve staging");
        sl.pin_cap = need * 2;
    }
    sl.pin_err = reinterpret_cast<unsigned int*>(static_cast<uint8_t*>(sl.pin) + sl.pin_cap - 256);
    GBMI_TRY(rt::ensure(sl.dpack, std::max<size_t>(b_pack, 256), "serve pack table"));
    GBMI_TRY(rt::ensure(sl.djobs, std::max<size_t>(b_jobs, 256), "serve job table"));
    GBMI_TRY(rt::ensure(sl.dtiles, std::max<size_t>(b_tiles, 256), "serve tile list"));
    size_t po = 0;
    if (b_pack) GBMI_CUDA(stage_upload(sl, sl.dpack, pj.data(), b_pack, po), "serve upload");
    po += Arena::round(b_pack);
    GBMI_CUDA(stage_upload(sl, sl.djobs, gj.data(), b_jobs, po), "serve upload");
    po += Arena::round(b_jobs);
    GBMI_CUDA(stage_upload(sl, sl.dtiles, tiles.data(), b_tiles, po), "serve upload");

    if (!pj.empty()) {
        GBMI_CUDA(launch_pack_grouped(static_cast<const PackJob*>(sl.dpack.p),
                                      static_cast<int>(pj.size()), ctas, nullptr, sl.s),
                  "serve pack");
        for (int64_t id : sl.packs) {
            const Dataset& d = S->datasets[id];
            GBMI_CUDA(launch_mi_vars(v_of(S, d), d.n, rt::mi_params_plain(d.m, 0, nullptr),
                                     vars_of(S, d), sl.s),
                      "serve mi_vars");
        }
    }
    GBMI_CUDA(cudaEventRecord(sl.packed, sl.s), "serve event");
    unsigned int* ctrl = reinterpret_cast<unsigned int*>(at(S, sl.off_ctrl));
    GBMI_CUDA(cudaMemsetAsync(ctrl, 0, 3 * sizeof(unsigned int), sl.s), "serve counter");
    GramLaunch L;
    std::memset(&L, 0, sizeof(L));
    L.jobs = static_cast<const GramJob*>(sl.djobs.p);
    L.mode = kTcModeMI;
    L.fp4 = S->fp4 ? 1 : 0;
    L.err = ctrl + 1;
    L.timeout_ns = rt::g_opt.timeout_ns;
    uint64_t launches = sl.packs.size() + (sl.packs.empty() ? 0 : 1);
    if (npair > 0) {   // the large requests, on CTA pairs
        GramLaunch Pl = L;
        Pl.tiles = static_cast<const GramTile*>(sl.dtiles.p);
        Pl.num_tiles = static_cast<int>(npair);
        Pl.pair = 1;
        Pl.counter = ctrl + 2;   // its own tile counter (zeroed with the others)
        const int pgrid = 2 * static_cast<int>(std::min<int64_t>(S->pair_clusters, npair));
        GBMI_CUDA(launch_gram_tc(S->maps, Pl, pgrid, sl.s), "serve gram (pairs)");
        ++launches;
    }
    if (ntiles > npair) {
        L.tiles = static_cast<const GramTile*>(sl.dtiles.p) + npair;
        L.num_tiles = static_cast<int>(ntiles - npair);
        L.counter = ctrl;
        const int grid = static_cast<int>(
            std::max<int64_t>(1, std::min<int64_t>(S->sm_count, ntiles - npair)));
        GBMI_CUDA(launch_gram_tc(S->maps, L, grid, sl.s), "serve gram");
        ++launches;
    }
    rt::g_launches.fetch_add(launches, std::memory_order_relaxed);
    GBMI_CUDA(cudaMemcpyAsync(sl.pin_err, ctrl + 1, sizeof(unsigned int), cudaMemcpyDeviceToHost,
                              sl.s),
              "serve error word");
    GBMI_CUDA(cudaEventRecord(sl.done, sl.s), "serve event");
    sl.busy = true;
    S->batches += 1;
    S->batched += static_cast<int64_t>(tickets.size());
    return GBMI_OK;
}

// Requests finished by slot k (called with S->mu held).
void complete_slot(gbmi_server* S, int k, cudaError_t st) {
    Slot& sl = S->slots[k];
    const bool failed = st != cudaSuccess || *sl.pin_err != 0;
    const Clock::time_point now = Clock::now();
    for (int64_t t : sl.tickets) {
        Request& r = S->reqs[t];
        r.state = failed ? 3 : 2;
        r.err = failed ? (st != cudaSuccess ? GBMI_ERR_CUDA : GBMI_ERR_TIMEOUT) : GBMI_OK;
        r.t_done = now;
        if (!failed) {
            S->lat_ms.push_back(std::chrono::duration<double, std::milli>(now - r.t_submit).count());
            S->pairs_done += r.pairs;
            S->t_last = now;
        }
        for (int64_t id : {r.a, r.b}) {
            if (id < 0) continue;
            S->datasets[id].users -= 1;
        }
    }
    for (int64_t id : sl.packs) {
        Dataset& d = S->datasets[id];
        d.pack_slot = -1;
        d.X = nullptr;   // packed: the caller's buffer is no longer read
    }
    for (int64_t t : sl.tickets) {
        const Request& r = S->reqs[t];
        for (int64_t id : {r.a, r.b})
            if (id >= 0) drop_dataset_if_done(S, id);
    }
    sl.tickets.clear();
    sl.packs.clear();
    sl.busy = false;
}

// Admit queued requests for one batch (called with S->mu held).
std::vector<int64_t> admit(gbmi_server* S) {
    std::vector<int64_t> out;
    for (auto it = S->queue.begin(); it != S->queue.end() && static_cast<int>(out.size()) < S->max_batch;) {
        Request& r = S->reqs[*it];
        Dataset& da = S->datasets[r.a];
        Dataset* db = r.b >= 0 ? &S->datasets[r.b] : nullptr;
        const bool had_a = da.off_p >= 0, had_b = db == nullptr || db->off_p >= 0;
        bool ok = make_resident(S, da) && (db == nullptr || make_resident(S, *db));
        if (ok) {
            r.off_out = S->arena.alloc(r.bytes_out);
            ok = r.off_out >= 0;
        }
        if (!ok) {   // roll back what this request allocated; it waits for memory
            if (!had_a && da.off_p >= 0) {
                S->arena.release(da.off_p, da.bytes_p);
                S->arena.release(da.off_v, da.bytes_v);
                da.off_p = da.off_v = -1;
            }
            if (db != nullptr && !had_b && db->off_p >= 0) {
                S->arena.release(db->off_p, db->bytes_p);
                S->arena.release(db->off_v, db->bytes_v);
                db->off_p = db->off_v = -1;
            }
            ++it;
            continue;
        }
        r.state = 1;
        out.push_back(*it);
        it = S->queue.erase(it);
    }
    return out;
}

void worker_main(gbmi_server* S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        bool progressed = false;
        for (int k = 0; k < 2; ++k) {
            Slot& sl = S->slots[k];
            if (!sl.busy) continue;
            const cudaError_t q = cudaEventQuery(sl.done);
            if (q == cudaErrorNotReady) continue;
            complete_slot(S, k, q == cudaSuccess ? cudaSuccess : q);
            if (q != cudaSuccess) cudaGetLastError();
            progressed = true;
        }
        if (progressed) S->cv_done.notify_all();
        for (int k = 0; k < 2; ++k) {
            if (S->slots[k].busy || S->queue.empty()) continue;
            std::vector<int64_t> batch = admit(S);
            if (batch.empty()) break;
            if (launch_batch(S, k, batch) != GBMI_OK) {
                Slot& sl = S->slots[k];
                for (int64_t id : sl.packs) S->datasets[id].pack_slot = -1;   // packed again later
                sl.packs.clear();
                sl.tickets.clear();
                sl.busy = false;
                for (int64_t t : batch) {
                    Request& r = S->reqs[t];
                    r.state = 3;
                    r.err = GBMI_ERR_CUDA;
                    for (int64_t id : {r.a, r.b})
                        if (id >= 0) S->datasets[id].users -= 1;
                }
                S->cv_done.notify_all();
            }
        }
        const bool busy = S->slots[0].busy || S->slots[1].busy;
        if (S->stop) {   // shutting down: queued requests fail, running ones finish
            for (int64_t t : S->queue) {
                Request& r = S->reqs[t];
                r.state = 3;
                r.err = GBMI_ERR_ARG;
                for (int64_t id : {r.a, r.b})
                    if (id >= 0) S->datasets[id].users -= 1;
            }
            if (!S->queue.empty()) S->cv_done.notify_all();
            S->queue.clear();
            if (!busy) break;
        }
        if (busy)
            S->cv_work.wait_for(lk, std::chrono::microseconds(20));
        else
            S->cv_work.wait_for(lk, std::chrono::milliseconds(5));
    }
}

gbmi_status create(int64_t budget, int max_batch, gbmi_server** out) {
    if (out == nullptr || budget < (int64_t{1} << 20)) return rt::fail(GBMI_ERR_ARG, "budget too small");
    if (max_batch < 1) return rt::fail(GBMI_ERR_ARG, "max_batch must be >= 1");
    rt::DeviceCtx* cp = nullptr;
    {
        std::lock_guard<std::recursive_mutex> lk(rt::g_mu);
        GBMI_TRY(rt::get_ctx(&cp));
    }
    gbmi_server* S = new gbmi_server();
    S->max_batch = max_batch;
    S->sm_count = cp->sm_count;
    S->pair_clusters = cp->pair_clusters;
    S->fp4 = rt::g_opt.fp4 != 0;
    cudaGetDevice(&S->device);
    const size_t bytes = static_cast<size_t>(budget) & ~static_cast<size_t>(255);
    gbmi_status st = rt::ensure(S->mem, bytes, "server arena");
    if (st != GBMI_OK) {
        delete S;
        return st;
    }
    S->arena.init(bytes);
    if (!make_operand_maps(&S->maps, static_cast<const uint8_t*>(S->mem.p),
                           static_cast<int64_t>(bytes / kTcBK))) {
        rt::release(S->mem);
        delete S;
        return rt::fail(GBMI_ERR_ARG, "budget too large for the operand descriptors");
    }
    for (Slot& sl : S->slots) {
        cudaStreamCreateWithFlags(&sl.s, cudaStreamNonBlocking);
        cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
        cudaEventCreateWithFlags(&sl.packed, cudaEventDisableTiming);
        sl.off_ctrl = S->arena.alloc(256);
    }
    S->worker = std::thread(worker_main, S);
    *out = S;
    return GBMI_OK;
}

}  // namespace
}  // namespace gbmi

using namespace gbmi;

extern "C" {

gbmi_status gbmi_server_create(int64_t budget_bytes, int max_batch, gbmi_server** srv) {
    if (srv != nullptr) *srv = nullptr;
    return create(budget_bytes, max_batch, srv);
}

gbmi_status gbmi_server_add_dataset(gbmi_server* S, const uint8_t* X, int64_t m, int64_t n,
                                    int64_t* id) {
    if (S == nullptr || X == nullptr || id == nullptr) return rt::fail(GBMI_ERR_ARG, "null pointer");
    if (m < 1 || m > (int64_t{1} << 24)) return rt::fail(GBMI_ERR_ARG, "served datasets need 1 <= m <= 2^24");
    if (n < 1 || n > (int64_t{1} << 20)) return rt::fail(GBMI_ERR_ARG, "n out of range");
    std::lock_guard<std::mutex> lk(S->mu);
    Dataset d;
    d.X = X;
    d.m = m;
    d.n = n;
    d.kb = pack_ld_of(m, S->fp4) / kb_samples(S->fp4);
    d.rows_p = pack_rows(n);
    *id = S->next_ds++;
    S->datasets[*id] = d;
    return GBMI_OK;
}

gbmi_status gbmi_server_remove_dataset(gbmi_server* S, int64_t id) {
    if (S == nullptr) return rt::fail(GBMI_ERR_ARG, "null server");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->datasets.find(id);
    if (it == S->datasets.end() || it->second.removed) return rt::fail(GBMI_ERR_ARG, "unknown dataset");
    it->second.removed = true;
    drop_dataset_if_done(S, id);
    return GBMI_OK;
}

gbmi_status gbmi_server_submit(gbmi_server* S, int64_t a, int64_t b, int64_t* ticket) {
    if (S == nullptr || ticket == nullptr) return rt::fail(GBMI_ERR_ARG, "null pointer");
    std::unique_lock<std::mutex> lk(S->mu);
    auto ia = S->datasets.find(a);
    if (ia == S->datasets.end() || ia->second.removed) return rt::fail(GBMI_ERR_ARG, "unknown dataset a");
    Request r;
    r.a = a;
    r.b = b;
    r.m = ia->second.m;
    r.n_a = ia->second.n;
    r.n_b = r.n_a;
    if (b >= 0) {
        auto ib = S->datasets.find(b);
        if (ib == S->datasets.end() || ib->second.removed) return rt::fail(GBMI_ERR_ARG, "unknown dataset b");
        if (ib->second.m != r.m) return rt::fail(GBMI_ERR_ARG, "cross datasets need the same m");
        r.n_b = ib->second.n;
        ib->second.users += 1;
    }
    ia->second.users += 1;
    r.bytes_out = static_cast<size_t>(r.n_a) * r.n_b * 4;
    r.pairs = b >= 0 ? r.n_a * r.n_b : r.n_a * (r.n_a - 1) / 2;
    // a request that cannot fit even in an empty arena fails now
    const Dataset& da = ia->second;
    size_t need = Arena::round(r.bytes_out) + Arena::round(static_cast<size_t>(da.kb * da.rows_p) * kTcBK);
    if (b >= 0) {
        const Dataset& db = S->datasets[b];
        need += Arena::round(static_cast<size_t>(db.kb * db.rows_p) * kTcBK);
    }
    if (need + 1024 > S->arena.size()) {
        ia->second.users -= 1;
        if (b >= 0) S->datasets[b].users -= 1;
        return rt::fail(GBMI_ERR_OOM, "request needs more memory than the server's budget");
    }
    r.t_submit = Clock::now();
    if (!S->started) {
        S->started = true;
        S->t_first = r.t_submit;
    }
    *ticket = S->next_ticket++;
    S->reqs[*ticket] = r;
    S->queue.push_back(*ticket);
    lk.unlock();
    S->cv_work.notify_one();
    return GBMI_OK;
}

gbmi_status gbmi_server_wait(gbmi_server* S, int64_t ticket, int64_t timeout_ms, const float** out,
                             double* latency_ms) {
    if (S == nullptr) return rt::fail(GBMI_ERR_ARG, "null server");
    std::unique_lock<std::mutex> lk(S->mu);
    auto done = [&] {
        auto it = S->reqs.find(ticket);
        return it == S->reqs.end() || it->second.state >= 2;
    };
    if (timeout_ms > 0) {
        if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done))
            return rt::fail(GBMI_ERR_TIMEOUT, "request not finished within the timeout");
    } else {
        S->cv_done.wait(lk, done);
    }
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return rt::fail(GBMI_ERR_ARG, "unknown ticket");
    const Request& r = it->second;
    if (r.state == 3)
        return rt::fail(r.err, r.err == GBMI_ERR_ARG ? "request was cancelled (or the server closed)"
                                                     : "request failed on the device");
    if (out) *out = reinterpret_cast<const float*>(at(S, r.off_out));
    if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r.t_done - r.t_submit).count();
    return GBMI_OK;
}

gbmi_status gbmi_server_cancel(gbmi_server* S, int64_t ticket) {
    if (S == nullptr) return rt::fail(GBMI_ERR_ARG, "null server");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return rt::fail(GBMI_ERR_ARG, "unknown ticket");
    Request& r = it->second;
    if (r.state != 0) return rt::fail(GBMI_ERR_ARG, "request is not queued (running or done)");
    for (auto q = S->queue.begin(); q != S->queue.end(); ++q)
        if (*q == ticket) {
            S->queue.erase(q);
            break;
        }
    r.state = 3;
    r.err = GBMI_ERR_ARG;
    r.t_done = Clock::now();
    for (int64_t id : {r.a, r.b}) {
        if (id < 0) continue;
        S->datasets[id].users -= 1;
        drop_dataset_if_done(S, id);
    }
    lk.unlock();
    S->cv_done.notify_all();
    return GBMI_OK;
}

gbmi_status gbmi_server_state(gbmi_server* S, int64_t* queued, int64_t* running,
                              int64_t* datasets, int64_t* bytes_in_use) {
    if (S == nullptr) return rt::fail(GBMI_ERR_ARG, "null server");
    std::lock_guard<std::mutex> lk(S->mu);
    int64_t run = 0;
    for (const Slot& sl : S->slots)
        if (sl.busy) run += static_cast<int64_t>(sl.tickets.size());
    if (queued) *queued = static_cast<int64_t>(S->queue.size());
    if (running) *running = run;
    if (datasets) *datasets = static_cast<int64_t>(S->datasets.size());
    if (bytes_in_use) *bytes_in_use = static_cast<int64_t>(S->arena.used());
    return GBMI_OK;
}

gbmi_status gbmi_server_release(gbmi_server* S, int64_t ticket) {
    if (S == nullptr) return rt::fail(GBMI_ERR_ARG, "null server");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return rt::fail(GBMI_ERR_ARG, "unknown ticket");
    if (it->second.state < 2) return rt::fail(GBMI_ERR_ARG, "request still running");
    S->arena.release(it->second.off_out, it->second.bytes_out);
    S->reqs.erase(it);
    S->cv_work.notify_one();
    return GBMI_OK;
}

gbmi_status gbmi_server_stats(gbmi_server* S, double* st) {
    if (S == nullptr || st == nullptr) return rt::fail(GBMI_ERR_ARG, "null pointer");
    std::lock_guard<std::mutex> lk(S->mu);
    std::vector<double> l = S->lat_ms;
    std::sort(l.begin(), l.end());
    auto pct = [&](double p) {
        if (l.empty()) return 0.0;
        const size_t i = std::min(l.size() - 1, static_cast<size_t>(p * (l.size() - 1) + 0.5));
        return l[i];
    };
    const double span = S->started ? std::chrono::duration<double>(S->t_last - S->t_first).count() : 0.0;
    st[0] = static_cast<double>(l.size());
    st[1] = pct(0.50);
    st[2] = pct(0.99);
    st[3] = l.empty() ? 0.0 : std::accumulate(l.begin(), l.end(), 0.0) / l.size();
    st[4] = l.empty() ? 0.0 : l.back();
    st[5] = span > 0 ? static_cast<double>(S->pairs_done) / span : 0.0;
    st[6] = static_cast<double>(S->batches);
    st[7] = S->batches ? static_cast<double>(S->batched) / S->batches : 0.0;
    return GBMI_OK;
}

gbmi_status gbmi_server_destroy(gbmi_server* S) {
    if (S == nullptr) return GBMI_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->worker.joinable()) S->worker.join();
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(S->device);
    for (Slot& sl : S->slots) {
        if (sl.s) cudaStreamSynchronize(sl.s);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.packed) cudaEventDestroy(sl.packed);
        if (sl.s) cudaStreamDestroy(sl.s);
        if (sl.pin) cudaFreeHost(sl.pin);
        rt::release(sl.dpack);
        rt::release(sl.djobs);
        rt::release(sl.dtiles);
    }
    rt::release(S->mem);
    delete S;
    cudaSetDevice(prev);
    return GBMI_OK;
}

}  // extern "C"
