// Co-occurrence Gram N11 = X^T X (G11, Sec. 2 step 2) on the tcgen05 tensor
// cores, with the count derivation of Eq. 6-7 and the MI of Eq. 1/Eq. 2
// fused into the epilogue (the paper's "only one matrix multiplication",
// Sec. 3.1, with everything after it done per tile while it is on chip).
//
// Operands: K-block-major packed matrices (for each block of 128 samples, one
// 128-byte row per variable, FP8 E4M3 0x00/0x38), or their FP4 form (for each
// block of 256 samples, one 128-byte row of E2M1 nibbles 0x0/0x2, multiplied
// by the block-scaled MMA kind::mxf4 with every scale factor 1.0), or, on the
// direct path, the caller's row-major uint8 0/1 matrix itself read as MN-major
// E4M3 (a byte 1 is the subnormal 2^-9; counts come out scaled by 2^-18, still
// exact; the epilogue scales them back).  0 and 1 are exact in E4M3 and E2M1,
// every product is 0 or 1 and the FP32 accumulator holds integers exactly
// below 2^24, so a tile's counts are exact as long as one launch accumulates
// at most 2^24 samples (k_blocks x 128 or 256).  One launch can serve many
// datasets: every tile names its job (dataset), whose descriptor gives the
// operands' first rows in the shared buffer, its sample range, its tile width
// bn (64, 128 or 256; at most 240 in an FP4 launch), its epilogue terms and its
// output.
//
// Persistent, warp-specialised CTA, one per SM (448 threads), or CTA pairs
// (clusters of 2, kPair):
//   warp 0      TMA producer: per stage one 128 x 128-byte box of A (the
//               variables of row block I) and one bn x 128-byte box of B
//               (column block J) into a 4-stage shared-memory ring
//               (128-byte swizzle).  In a pair, CTA 0's producer loads both
//               CTAs' halves (128 rows of A and of B each) into a 6-stage
//               ring, the partner's through the cluster window.
//   warp 1      allocates 512 TMEM columns; one thread issues
//               tcgen05.mma.kind::f8f6f4 M=128 N=bn K=32 (4 per stage; in a
//               pair, CTA 0 issues cta_group::2 M=256 N=256) into one of two
//               256-column FP32 accumulators, commits each stage back to the
//               ring and each finished tile to the epilogue.  The ragged last
//               column block runs at its valid width rounded up to 32.  FP4
//               launches issue kind::mxf4.block_scale K=64 instead (N <= 240;
//               the scale factors, all 1.0, sit in columns 240-255 and 496-511,
//               filled by the epilogue warps before the first MMA).
//   warps 2-13  epilogue, three warps per TMEM lane quadrant (tcgen05.ld
//               only reaches lanes 32*(warp%4)..+31), each taking a third of
//               the tile's columns: load accumulator columns (one TMEM lane = one
//               variable i per thread), derive n10, n01, n00, evaluate MI (with
//               the FP64 combine for small pairs when it is on) and store
//               (i, j) as 16-, 8- or 4-byte pieces as the row's alignment
//               allows and, for a symmetric problem, (j, i) as coalesced rows
//               (or, for a panel of an out-of-core run, (j, i) into a separate
//               mirror buffer).  The second accumulator lets tile t+1's MMAs
//               run meanwhile.
// Tiles come from a host-built list: for all-pairs only blocks that touch
// the upper triangle (j >= i), in groups of column blocks, jobs one after
// another, so that CTAs running at the same time share operand panels in L2.
// The producer takes the CTA's next tile from a shared atomic counter
// (dynamic order: the tiles in flight are always a contiguous window of the
// list, whatever their lengths) or from the static round-robin sequence, and
// hands its id to the MMA thread and the epilogue warps (in a CTA pair, also
// to the partner's epilogue warps, by a cluster store and a remote arrive;
// their slot releases come back to CTA 0) through an 8-entry
// shared-memory queue (queue full / queue empty mbarriers; -1 ends the run).
//
// Every mbarrier wait is bounded (timeout_ns from its start, %globaltimer).
// A role whose wait runs out sets a bit in the device error word and a
// CTA-wide abort flag; the other roles see the flag and unwind; the producer
// waits (bounded) for its copies still in flight, the MMA thread for its
// MMAs, and warp 1 frees the tensor memory before the CTA exits.
#include <algorithm>
#include <cstring>

#include "internal.cuh"
#include "ptx.cuh"

namespace gbmi {

namespace {

// Kernel-only mode: MI with the FP64 combine compiled out (launched for MI
// whenever the combine is off, so the epilogue's code stays small).
constexpr int kTcModeMI32 = 3;
template <int kMode>
__host__ __device__ constexpr bool is_mi() { return kMode == kTcModeMI || kMode == kTcModeMI32; }
// Epilogue warps: 12 (three per TMEM lane quadrant) hide the latency of the
// per-pair arithmetic and of the FP64 combine's table reads; more of them
// delay the producer and MMA threads, which share sub-partitions 0 and 1 with
// them (measured at 10^5 x 10^4: 16 warps 1.791 / 3.089 ms per call without /
// with the FP64 combine, 12 warps 1.785 / 2.769 ms).  Epilogue warp
// w (w = 2, 3, ...) serves TMEM lane
// quadrant w % 4 (the only lanes its tcgen05.ld reaches), which is also the
// SM sub-partition it is scheduled on; warp 0 (producer) and warp 1 (MMA
// issuer) share sub-partitions 0 and 1 with the epilogue warps of quadrants 0
// and 1.  Any count >= 4 works: a quadrant's warps split the tile's columns.
constexpr int kEpiWarpsMain = 12;
__host__ __device__ constexpr int epi_warps(int mode) { return kEpiWarpsMain; }
// Epilogue warps serving the TMEM lane quadrant of warp w.
__host__ __device__ constexpr int quadrant_warps(int nepi, int w) {
    return (nepi - ((w - 2) & 3) + 3) / 4;
}
constexpr size_t kColVarTotal = 32768;   // staged column terms of all epilogue warps
// Shared-memory bytes of one epilogue warp's column terms: an equal share,
// rounded down to 32 bytes so that every warp's MiVar / MiVarF entries are
// aligned for their vector stores and loads.
__host__ __device__ constexpr size_t colvar_bytes(int nepi) {
    return (kColVarTotal / nepi) & ~static_cast<size_t>(31);
}
// Most columns one epilogue warp takes of a 256-wide tile (its quadrant has at
// least nepi / 4 warps; a warp's share is a multiple of 16).
__host__ __device__ constexpr int max_part_cols(int nepi) {
    return ((kTcBNMax + nepi / 4 - 1) / (nepi / 4) + 15) & ~15;
}
// int32 entries of one unit of a split tile (FP32 epilogue kernels): both CTAs
// of a pair, every epilogue warp, its columns, 32 lanes.
__host__ __device__ constexpr int64_t part_slot_ints() {
    return int64_t{2} * kEpiWarpsMain * max_part_cols(kEpiWarpsMain) * 32;
}
__host__ __device__ constexpr int threads_of(int mode) { return 64 + 32 * epi_warps(mode); }
constexpr int kUmmaK = 32;                       // bytes of K per MMA (32 FP8 or 64 FP4 samples)
constexpr int kABytes = kTcBM * kTcBK;           // 16 KB: 128 rows of A
constexpr int kAccCols = kTcBNMax;               // TMEM columns per accumulator buffer
constexpr int kTmemCols = 2 * kAccCols;          // 512: the whole tensor memory
// FP4 launches: scale factors (all 1.0, UE8M0 0x7F) in the 16 columns after
// each accumulator's first 240; A's in buffer 0's, B's in buffer 1's
constexpr int kSfaCol = kTcBNFp4;
constexpr int kSfbCol = kAccCols + kTcBNFp4;
constexpr uint32_t kScaleOnes = 0x7F7F7F7Fu;
constexpr int kGroup = 16;                       // accumulator columns per tcgen05.ld
constexpr int kQ = 8;                            // tile-id queue between the roles

// full, empty, tmem full x2, tmem empty x2, drain, queue full x kQ, queue empty x kQ
constexpr int kNumBarsFor(int stages) { return 2 * stages + 4 + 1 + 2 * kQ; }

// Pipeline stages of a kernel: single CTA 4, CTA pairs 6, one fewer for the
// kernels with the FP64 combine: their epilogue waits on reads scattered over
// the n log2 n table, and the stage they give up drops shared memory to the
// next carveout, leaving L1 about 60 KB instead of 28 (measured at 10^5 x
// 10^4: the pair Gram 2.41 -> 1.92 ms, the single-CTA one 2.87 -> 2.27 ms,
// while the FP32 epilogue kernels are slower with fewer stages).
__host__ __device__ constexpr int stages_for(int mode, bool pair) {
    return mode == kTcModeMI ? (pair ? 5 : 3) : (pair ? 6 : 4);
}

// Shared-memory plan.  Single CTA: kSt stages of A (128 rows) + B (up to 256
// rows).  CTA pair: kSt stages of this CTA's halves, 128 rows of A and 128 rows
// of B (the pair's tile is 256 x 256).
template <bool kPair, int kSt = stages_for(kTcModeMI32, kPair)>
struct Plan {
    static constexpr int stages = kSt;
    static constexpr int b_bytes = kPair ? kTcBM * kTcBK : kTcBNMax * kTcBK;
    static constexpr int stage_bytes = kABytes + b_bytes;
    static constexpr int tile_m = kPair ? 2 * kTcBM : kTcBM;   // rows of A per tile
    static constexpr size_t off_colvars = static_cast<size_t>(stages) * stage_bytes;
    static constexpr size_t off_bars = off_colvars + kColVarTotal;
    static constexpr int num_bars = kNumBarsFor(stages);
    static constexpr size_t off_misc = off_bars + num_bars * 8;
    static constexpr size_t off_queue = off_misc + 64;
    static constexpr size_t smem_bytes = 1024 + off_queue + kQ * 4;
    static_assert(stage_bytes % 1024 == 0, "stages must keep 1024-byte alignment");
    static_assert(smem_bytes <= 232448, "shared memory budget");
};

template <bool kPair, int kSt = stages_for(kTcModeMI32, kPair)>
struct Smem {
    using P = Plan<kPair, kSt>;
    uint8_t* base;
    uint32_t rank;   // CTA rank in the pair (0 when single)
    __device__ uint8_t* a(int s) const { return base + s * P::stage_bytes; }
    __device__ uint8_t* b(int s) const { return base + s * P::stage_bytes + kABytes; }
    // column terms of epilogue warp e of nepi (colvar_bytes(nepi) bytes each)
    __device__ void* colvars(int e, int nepi) const {
        return base + P::off_colvars + e * colvar_bytes(nepi);
    }
    __device__ uint64_t* bar(int k) const {
        return reinterpret_cast<uint64_t*>(base + P::off_bars) + k;
    }
    __device__ uint32_t full(int s) const { return ptx::smem_u32(bar(s)); }
    __device__ uint32_t empty(int s) const { return ptx::smem_u32(bar(P::stages + s)); }
    __device__ uint32_t tfull(int b) const { return ptx::smem_u32(bar(2 * P::stages + b)); }
    __device__ uint32_t tempty(int b) const { return ptx::smem_u32(bar(2 * P::stages + 2 + b)); }
    __device__ uint32_t drain() const { return ptx::smem_u32(bar(2 * P::stages + 4)); }
    __device__ uint32_t qfull(int q) const { return ptx::smem_u32(bar(2 * P::stages + 5 + q)); }
    __device__ uint32_t qempty(int q) const {
        return ptx::smem_u32(bar(2 * P::stages + 5 + kQ + q));
    }
    __device__ volatile int* queue() const {
        return reinterpret_cast<volatile int*>(base + P::off_queue);
    }
    __device__ uint32_t* tmem_holder() const {
        return reinterpret_cast<uint32_t*>(base + P::off_misc);
    }
    __device__ volatile int* abort_flag() const {
        return reinterpret_cast<volatile int*>(base + P::off_misc + 4);
    }
};

template <bool kPair, int kSt>
__device__ __forceinline__ void raise_abort(const Smem<kPair, kSt>& sm, unsigned int* err,
                                            uint32_t code) {
    atomicOr(err, code);
    *sm.abort_flag() = 1;
    if constexpr (kPair)   // the partner CTA unwinds too
        ptx::st_cluster_u32(
            ptx::mapa_shared(ptx::smem_u32(const_cast<int*>(sm.abort_flag())), sm.rank ^ 1u), 1u);
}

__device__ __forceinline__ const GramJob& job_of(const GramLaunch& L, int j) {
    return L.jobs != nullptr ? L.jobs[j] : L.job0;
}

// Column window [lo, hi) of a tile that its MMAs compute (gram_tile_window).
__device__ __forceinline__ ColWindow tile_window(const GramJob& job, const GramTile& tile,
                                                 int tile_m, bool direct) {
    return gram_tile_window(job.n_b, job.symmetric != 0, job.bn, tile, tile_m, direct);
}

// K blocks [kb0, kb1) of the job that a tile accumulates: all of them, or its
// part's share for a split tile.
__device__ __forceinline__ void tile_krange(const GramJob& job, const GramTile& tile, int& kb0,
                                            int& kb1) {
    if (!split_is_k(tile.split)) {
        kb0 = 0;
        kb1 = job.k_blocks;
        return;
    }
    const int parts = tile.split & 15, part = (tile.split >> 4) & 15;
    kb0 = static_cast<int>(static_cast<int64_t>(job.k_blocks) * part / parts);
    kb1 = static_cast<int>(static_cast<int64_t>(job.k_blocks) * (part + 1) / parts);
}

// ------------------------------------------------------------------ producer
// Next tile of this CTA: from the shared counter (dynamic order) or the static
// round-robin sequence.
// Next tile of this CTA (of CTA 0 of a pair): from the shared counter (dynamic
// order) or the static sequence of the CTA (of the cluster).
template <bool kPair>
__device__ __forceinline__ int next_tile(const GramLaunch& L, int s) {
    if (L.counter != nullptr) return static_cast<int>(atomicAdd(L.counter, 1u));
    if constexpr (kPair)
        return static_cast<int>(ptx::cluster_id_x() + s * ptx::nclusters_x());
    else
        return blockIdx.x + s * gridDim.x;
}

template <bool kPair, int kSt>
__device__ void run_producer(const Smem<kPair, kSt>& sm, const OperandMaps& maps,
                             const GramLaunch& L) {
    constexpr int kStages = kSt;
    // stages with a copy issued (bit s), and the barrier phase parity it
    // completes (bit s): registers, where an array indexed by the run-time
    // stage would live in local memory
    uint32_t issued = 0, issued_par = 0;
    const uint32_t full0 = sm.full(0), empty0 = sm.empty(0);
    const uint32_t a_smem0 = ptx::smem_u32(sm.a(0)), b_smem0 = ptx::smem_u32(sm.b(0));
    constexpr uint32_t kStageBytes = static_cast<uint32_t>(Plan<kPair>::stage_bytes);
    int stage = 0;
    uint32_t phase = 0;
    int qslot = 0;
    uint32_t qphase = 0;
    bool ok = true;
    int s = 0;
    int t = next_tile<kPair>(L, 0);
    while (ok) {
        // publish the tile id (-1 at the end) to the MMA thread and the epilogue
        if (!ptx::mbar_wait_bounded(sm.qempty(qslot), qphase ^ 1u, L.timeout_ns,
                                    sm.abort_flag())) {
            raise_abort(sm, L.err, kErrTimeoutLoad);
            ok = false;
            break;
        }
        const int tid = t < L.num_tiles ? t : -1;
        sm.queue()[qslot] = tid;
        ptx::mbar_arrive(sm.qfull(qslot));
        if constexpr (kPair) {   // the partner CTA's epilogue takes the same tile
            ptx::st_cluster_u32(
                ptx::mapa_shared(ptx::smem_u32(const_cast<int*>(sm.queue() + qslot)), 1u),
                static_cast<uint32_t>(tid));
            ptx::mbar_arrive_cluster(ptx::mapa_shared(sm.qfull(qslot), 1u));
        }
        if (++qslot == kQ) {
            qslot = 0;
            qphase ^= 1u;
        }
        if (tid < 0) break;
        if (L.debug_flags & 1) break;   // test hook: issue no copies, consumers must time out
        const int t_next = next_tile<kPair>(L, ++s);   // its latency overlaps this tile's copies
        const GramTile tile = L.tiles[tid];
        const GramJob& job = job_of(L, tile.job);
        const int bn = job.bn;
        // rows of B per stage on one CTA: the tile width, 256 for a 240-wide FP4
        // tile (its MMAs read the first 240); a pair loads two 128-row boxes of A
        // and two boxes of B (below)
        const int brows = bn > kTcBM ? kTcBNMax : bn;
        const CUtensorMap* mapB = brows == 256 ? &maps.box256 : (brows == 128 ? &maps.box128
                                                                               : &maps.box64);
        // pair: the partner CTA holds B rows [N/2, N) of the tile's MMA width N;
        // each CTA's half is one box of 120 rows when N = 240, else of 128
        const ColWindow win = tile_window(job, tile, Plan<kPair>::tile_m, L.direct != 0);
        const int nhalf = kPair ? (win.hi - win.lo) / 2 : 0;
        // (64 rows when N <= 128: column shares and tiles cut by the diagonal)
        const int hrows = nhalf == 120 ? 120 : (nhalf <= 64 ? 64 : kTcBM);
        const CUtensorMap* mapH =
            hrows == 120 ? &maps.box120 : (hrows == 64 ? &maps.box64 : &maps.box128);
        const uint32_t bytes = static_cast<uint32_t>(
            (Plan<kPair>::tile_m + (kPair ? 2 * hrows : brows)) * kTcBK);
        const int64_t a0 = job.rowA + static_cast<int64_t>(tile.I) * Plan<kPair>::tile_m;
        const int64_t b0 = job.rowB + static_cast<int64_t>(tile.J) * bn + win.lo;
        if (L.direct && ((a0 | b0) & 15) != 0) {
            // a direct copy's x coordinate (a variable index) must be a multiple
            // of 16 bytes: record it and issue nothing
            raise_abort(sm, L.err, kErrBadOperand);
            ok = false;
            break;
        }
        int kb_lo = 0, kb_hi = 0;
        tile_krange(job, tile, kb_lo, kb_hi);
        if (kPair || !L.direct) {
            // One K block of packed operands: wait for a free stage, then load
            // A and B (a pair's CTA 0 loads both CTAs' halves, rows +0 and +128
            // of A and +0 and +N/2 of B, every copy completing on CTA 0's full
            // barrier).  Stage s's addresses are stage 0's plus s stages, the
            // row coordinates advance by the operand strides, and the loop runs
            // two K blocks per iteration, so that a freed stage is refilled with
            // little delay.
            const int64_t k0 = static_cast<int64_t>(job.k_begin) + kb_lo;
            int32_t ya = static_cast<int32_t>(a0 + k0 * job.strideA);
            int32_t yb = static_cast<int32_t>(b0 + k0 * job.strideB);
            const int32_t dya = static_cast<int32_t>(job.strideA);
            const int32_t dyb = static_cast<int32_t>(job.strideB);
            auto load = [&]() -> bool {
                const uint32_t st = static_cast<uint32_t>(stage);
                const uint32_t eb = empty0 + 8u * st, fb = full0 + 8u * st;
                if (!ptx::mbar_try_wait(eb, phase ^ 1u) &&
                    !ptx::mbar_wait_bounded(eb, phase ^ 1u, L.timeout_ns, sm.abort_flag()))
                    return false;
                ptx::mbar_arrive_expect_tx(fb, bytes);
                const uint32_t a_s = a_smem0 + kStageBytes * st;
                const uint32_t b_s = b_smem0 + kStageBytes * st;
                ptx::tma_load_2d(a_s, &maps.box128, fb, 0, ya);
                if constexpr (kPair) {
                    ptx::tma_load_2d(b_s, mapH, fb, 0, yb);
                    ptx::tma_load_2d_peer(ptx::mapa_shared(a_s, 1u), &maps.box128, fb, 0,
                                          ya + kTcBM);
                    ptx::tma_load_2d_peer(ptx::mapa_shared(b_s, 1u), mapH, fb, 0, yb + nhalf);
                } else {
                    ptx::tma_load_2d(b_s, mapB, fb, 0, yb);
                }
                issued |= 1u << st;
                issued_par = (issued_par & ~(1u << st)) | (phase << st);
                ya += dya;
                yb += dyb;
                if (++stage == kStages) {
                    stage = 0;
                    phase ^= 1u;
                }
                return true;
            };
            int kb = kb_lo;
            for (; kb + 1 < kb_hi; kb += 2) {
                if (!load() || !load()) {
                    ok = false;
                    break;
                }
            }
            if (ok && kb < kb_hi && !load()) ok = false;
            if (!ok) {
                raise_abort(sm, L.err, kErrTimeoutLoad);
                break;
            }
            t = t_next;
            continue;
        }
        // direct operands (single CTA): 128 variables x 128 samples of X per
        // box, B in bn / 128 boxes
        for (int kb = kb_lo; kb < kb_hi; ++kb) {
            if (!ptx::mbar_wait_bounded(sm.empty(stage), phase ^ 1u, L.timeout_ns,
                                        sm.abort_flag())) {
                raise_abort(sm, L.err, kErrTimeoutLoad);
                ok = false;
                break;
            }
            const int64_t k = job.k_begin + kb;
            ptx::mbar_arrive_expect_tx(sm.full(stage), bytes);
            const int32_t y = static_cast<int32_t>(k * kTcBK);
            ptx::tma_load_2d(ptx::smem_u32(sm.a(stage)), &maps.xa, sm.full(stage),
                             static_cast<int32_t>(a0), y);
            for (int h = 0; h < bn; h += kTcBM)
                ptx::tma_load_2d(ptx::smem_u32(sm.b(stage) + h * kTcBK), &maps.xb,
                                 sm.full(stage), static_cast<int32_t>(b0 + h), y);
            issued |= 1u << stage;
            issued_par = (issued_par & ~(1u << stage)) | (phase << stage);
            if (++stage == kStages) {
                stage = 0;
                phase ^= 1u;
            }
        }
        t = t_next;
    }
    if (!ok || *sm.abort_flag()) {
        // Unwinding: wait (bounded) until every copy this thread issued has landed.
        const uint64_t d2 = ptx::globaltimer_ns() + 100000000ull;
        for (int s2 = 0; s2 < kStages; ++s2) {
            if (((issued >> s2) & 1u) == 0) continue;
            const uint32_t bar = sm.full(s2);
            const uint32_t par = (issued_par >> s2) & 1u;
            while (!ptx::mbar_try_wait(bar, par)) {
                if (ptx::globaltimer_ns() > d2) {
                    atomicOr(L.err, kErrTimeoutDrain);
                    break;
                }
            }
        }
    }
}

// ------------------------------------------------------------------ MMA issuer
// The MMAs of one K block of K-major operands (128 bytes of K: four MMAs of 32
// bytes, stepping the descriptors' start address inside the swizzled rows);
// acc0 = 0 starts the accumulator over with the first.
template <bool kPair, bool kFp4>
__device__ __forceinline__ void mma_kblock(uint32_t d, uint64_t adesc, uint64_t bdesc,
                                           uint32_t idesc, uint32_t sfa, uint32_t sfb,
                                           uint32_t acc0) {
#pragma unroll
    for (int kk = 0; kk < kTcBK / kUmmaK; ++kk) {
        const uint64_t off = static_cast<uint64_t>((kk * kUmmaK) >> 4);
        const uint32_t accumulate = kk == 0 ? acc0 : 1u;
        if constexpr (kPair && kFp4)
            ptx::mma_mxf4_pair(d, adesc + off, bdesc + off, idesc, sfa, sfb, accumulate);
        else if constexpr (kPair)
            ptx::mma_f8f6f4_pair(d, adesc + off, bdesc + off, idesc, accumulate);
        else if constexpr (kFp4)
            ptx::mma_mxf4(d, adesc + off, bdesc + off, idesc, sfa, sfb, accumulate);
        else
            ptx::mma_f8f6f4(d, adesc + off, bdesc + off, idesc, accumulate);
    }
}

// kFp4: the launch's operands are the FP4 form (block-scaled MMA); one copy of
// the issue loop per form, so the per-K-block loop carries no branch on it.
template <bool kPair, bool kFp4, int kSt>
__device__ void run_mma(const Smem<kPair, kSt>& sm, const GramLaunch& L, uint32_t tmem_base) {
    constexpr int kStages = kSt;
    int stage = 0;
    uint32_t phase = 0;
    int acc = 0;
    uint32_t acc_phase = 0;
    int qslot = 0;
    uint32_t qphase = 0;
    bool ok = true;
    // Stage s's barriers and operand descriptors are stage 0's plus s times a
    // constant (barriers 8 bytes apart; descriptors count 16-byte units in
    // their 14-bit start-address field, which no stage of the 227 KB shared
    // memory overflows).
    const uint32_t full0 = sm.full(0), empty0 = sm.empty(0);
    constexpr uint32_t kStageDesc = static_cast<uint32_t>(Plan<kPair>::stage_bytes >> 4);
    const bool mn_major = !kFp4 && !kPair && L.direct;
    const uint64_t adesc0 =
        mn_major ? ptx::smem_desc_mnmajor_sw128(ptx::smem_u32(sm.a(0)), kTcBM * kTcBK)
                 : ptx::smem_desc_kmajor_sw128(ptx::smem_u32(sm.a(0)));
    const uint64_t bdesc0 =
        mn_major ? ptx::smem_desc_mnmajor_sw128(ptx::smem_u32(sm.b(0)), kTcBM * kTcBK)
                 : ptx::smem_desc_kmajor_sw128(ptx::smem_u32(sm.b(0)));
    while (ok) {
        if (!ptx::mbar_wait_bounded(sm.qfull(qslot), qphase, L.timeout_ns, sm.abort_flag())) {
            raise_abort(sm, L.err, kErrTimeoutMma);
            break;
        }
        const int t = sm.queue()[qslot];
        ptx::mbar_arrive(sm.qempty(qslot));
        if (++qslot == kQ) {
            qslot = 0;
            qphase ^= 1u;
        }
        if (t < 0) break;
        const GramTile tile = L.tiles[t];
        const GramJob& job = job_of(L, tile.job);
        const ColWindow win = tile_window(job, tile, Plan<kPair>::tile_m, L.direct != 0);
        const uint32_t mma_n = static_cast<uint32_t>(win.hi - win.lo);
        const uint32_t idesc =
            kFp4 ? ptx::idesc_mxf4_f32(kPair ? 2 * kTcBM : kTcBM, mma_n)
            : kPair ? ptx::idesc_e4m3_f32(2 * kTcBM, mma_n)
            : L.direct ? ptx::idesc_e4m3_f32_mnmajor(kTcBM, static_cast<uint32_t>(job.bn))
                       : ptx::idesc_e4m3_f32(kTcBM, mma_n);
        const uint32_t sfa = tmem_base + kSfaCol, sfb = tmem_base + kSfbCol;
        int kb_lo = 0, kb_hi = 0;
        tile_krange(job, tile, kb_lo, kb_hi);
        const int k_blocks = kb_hi - kb_lo;
        if (!ptx::mbar_wait_bounded(sm.tempty(acc), acc_phase ^ 1u, L.timeout_ns,
                                    sm.abort_flag())) {
            raise_abort(sm, L.err, kErrTimeoutMma);
            break;
        }
        ptx::tc_fence_after();
        const uint32_t d_tmem = tmem_base + static_cast<uint32_t>(acc * kAccCols);
        // One K block: wait for its stage, issue its MMAs, release the stage
        // when they complete.  The tensor pipe queues few MMAs, so the cycles
        // this thread spends between K blocks show up as idle tensor time: the
        // loop below runs two K blocks per iteration with the addresses above
        // (measured with the copies and the epilogue switched off: 560 -> 483
        // SM cycles per K block of a 256 x 240 FP4 tile, the MMAs' own rate).
        auto kblock = [&](int kb) -> bool {
            const uint32_t st = static_cast<uint32_t>(stage);
            const uint32_t fb = full0 + 8u * st;
            if (!ptx::mbar_try_wait(fb, phase) &&
                !ptx::mbar_wait_bounded(fb, phase, L.timeout_ns, sm.abort_flag()))
                return false;
            ptx::tc_fence_after();
            const uint64_t adesc = adesc0 + kStageDesc * st;
            const uint64_t bdesc = bdesc0 + kStageDesc * st;
            const uint32_t acc0 = kb != 0 ? 1u : 0u;
            if (mn_major) {
                // MN-major: 128-sample K-rows of 128 bytes, 128-variable atoms of
                // B 16 KB apart; K step kk starts kk * 32 rows (4 atoms) further
#pragma unroll
                for (int kk = 0; kk < kTcBK / kUmmaK; ++kk) {
                    const uint64_t off = static_cast<uint64_t>((kk * kUmmaK * kTcBK) >> 4);
                    ptx::mma_f8f6f4(d_tmem, adesc + off, bdesc + off, idesc,
                                    kk == 0 ? acc0 : 1u);
                }
            } else {
                mma_kblock<kPair, kFp4>(d_tmem, adesc, bdesc, idesc, sfa, sfb, acc0);
            }
            if constexpr (kPair)
                ptx::mma_commit_pair(empty0 + 8u * st);
            else
                ptx::mma_commit(empty0 + 8u * st);   // frees the slot when these MMAs finish
            if (++stage == kStages) {
                stage = 0;
                phase ^= 1u;
            }
            return true;
        };
        int kb = 0;
        for (; kb + 1 < k_blocks; kb += 2) {
            if (!kblock(kb) || !kblock(kb + 1)) {
                ok = false;
                break;
            }
        }
        if (ok && kb < k_blocks && !kblock(kb)) ok = false;
        if (!ok) raise_abort(sm, L.err, kErrTimeoutMma);
        if (!ok) break;
        if constexpr (kPair)                    // both CTAs' halves are ready
            ptx::mma_commit_pair_multicast(sm.tfull(acc), static_cast<uint16_t>(3u));
        else
            ptx::mma_commit(sm.tfull(acc));     // accumulator ready for the epilogue
        if (++acc == 2) {
            acc = 0;
            acc_phase ^= 1u;
        }
    }
    // Wait (bounded) for every MMA issued by this thread before TMEM is freed.
    if constexpr (kPair)
        ptx::mma_commit_pair(sm.drain());
    else
        ptx::mma_commit(sm.drain());
    const uint64_t d2 = ptx::globaltimer_ns() + 100000000ull;
    while (!ptx::mbar_try_wait(sm.drain(), 0)) {
        if (ptx::globaltimer_ns() > d2) {
            atomicOr(L.err, kErrTimeoutDrain);
            break;
        }
    }
}

// ------------------------------------------------------------------ epilogue
template <int kMode>
__device__ __forceinline__ void store_one(const GramJob& g, int64_t row, int64_t col,
                                          uint32_t x) {
    if (is_mi<kMode>()) {
        g.out_f[row * g.ld_out + col] = __uint_as_float(x);
    } else if (kMode == kTcModeCounts) {
        g.out_c[row * g.ld_out + col] = static_cast<int32_t>(x);
    } else {
        g.out_c[row * g.ld_out + col] += static_cast<int32_t>(x);
    }
}

template <int kMode, bool kPair>
__device__ void run_epilogue(const Smem<kPair, stages_for(kMode, kPair)>& sm, const GramLaunch& L,
                             uint32_t tmem_base) {
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int lane_base = (warp & 3) * 32;             // TMEM lanes this warp may access
    constexpr int kNepi = epi_warps(kMode);
    const int nparts = quadrant_warps(kNepi, warp);    // warps of this TMEM lane quadrant
    const int part = (warp - 2) >> 2;                  // which part of the tile's columns
    // this warp's column terms: the 16-byte FP32 part of each MiVar and, with
    // the FP64 combine, its FP64 entropy term in a second array
    MiVarF* cvf = static_cast<MiVarF*>(sm.colvars(warp - 2, kNepi));
    double* cvh = reinterpret_cast<double*>(cvf + max_part_cols(kNepi));
    static_assert(!is_mi<kMode>() ||
                      colvar_bytes(kNepi) >=
                          max_part_cols(kNepi) *
                              (sizeof(MiVarF) + (kMode == kTcModeMI ? sizeof(double) : 0)),
                  "column-term staging does not fit");
    const float cscale = L.direct ? 262144.f : 1.f;    // 2^18: direct operands hold 2^-9
    constexpr bool kFix = kMode == kTcModeMI;          // FP64 combine compiled in
    int acc = 0;
    uint32_t acc_phase = 0;
    int qslot = 0;
    uint32_t qphase = 0;
    for (;;) {
        // pair: CTA 0's producer fills both CTAs' queues (cluster-scope acquire)
        if (!ptx::mbar_wait_bounded<kPair>(sm.qfull(qslot), qphase, L.timeout_ns,
                                           sm.abort_flag())) {
            raise_abort(sm, L.err, kErrTimeoutEpilogue);
            break;
        }
        const int t = sm.queue()[qslot];
        __syncwarp();
        if (lane == 0) {   // the slot goes back to CTA 0's producer
            if (kPair && sm.rank != 0)
                ptx::mbar_arrive_cluster(ptx::mapa_shared(sm.qempty(qslot), 0u));
            else
                ptx::mbar_arrive(sm.qempty(qslot));
        }
        if (++qslot == kQ) {
            qslot = 0;
            qphase ^= 1u;
        }
        if (t < 0) break;
        const GramTile tile = L.tiles[t];
        const GramJob& job = job_of(L, tile.job);
        // copies in registers: the epilogue's stores could otherwise alias the
        // job table and force these fields to be reloaded after every store
        const MiParams P = job.mp;
        // columns of this warp: an equal share of the unit's column window, a
        // multiple of 16 (a whole 240-wide tile on three warps: 80 each)
        const ColWindow win = tile_window(job, tile, Plan<kPair>::tile_m, L.direct != 0);
        const int per = ((win.hi - win.lo + nparts - 1) / nparts + 15) & ~15;
        const int col_base = win.lo + part * per;
        const int cols = max(0, min(per, win.hi - col_base));
        const int64_t n_a = job.n_a, n_b = job.n_b;
        const bool sym = job.symmetric != 0;
        const int64_t ibase = static_cast<int64_t>(tile.I) * Plan<kPair>::tile_m +
                              static_cast<int64_t>(sm.rank) * kTcBM + lane_base;
        const int64_t i = ibase + lane;
        const int64_t jstart = static_cast<int64_t>(tile.J) * job.bn + col_base;
        const bool row_ok = i < n_a;
        MiVar A;
        A.v = 0;
        A.r1 = A.r0 = A.rchi = 0.f;
        A.h = 0.0;
        A.unused = 0.0;
        if (is_mi<kMode>()) {
            // stage the per-variable terms of this warp's columns while the
            // accumulator is still being produced
            __syncwarp();
            for (int k = lane; k < cols; k += 32) {
                const int64_t j = jstart + k;
                cvf[k] = j < n_b ? load_var_f(job.vb + j) : MiVarF{0, 0.f, 0.f, 0.f};
                if (kFix) cvh[k] = j < n_b ? __ldg(&job.vb[j].h) : 0.0;
            }
            if (row_ok) A = load_var(job.va + i);
            __syncwarp();
        }
        if (!ptx::mbar_wait_bounded(sm.tfull(acc), acc_phase, L.timeout_ns, sm.abort_flag())) {
            raise_abort(sm, L.err, kErrTimeoutEpilogue);
            break;
        }
        ptx::tc_fence_after();
        // accumulator column of tile column col_base + c: col_base + c - win.lo
        const uint32_t taddr = tmem_base + (static_cast<uint32_t>(lane_base) << 16) +
                               static_cast<uint32_t>(acc * kAccCols + col_base - win.lo);
        if constexpr (is_mi<kMode>()) {
            // MI: chunks of 4 columns in one small loop body; the next chunk's
            // accumulator columns load from TMEM during this chunk's math.
            // With the FP64 combine compiled in (kFix), pairs whose FP32 value
            // is below the threshold (or surely below it by the chi-square
            // bound) are recomputed in FP64 from the n log2 n table, the four
            // pairs' table reads of a chunk issued together.
            const int64_t c_end64 = n_b - jstart < cols ? n_b - jstart : cols;
            int c_end = c_end64 <= 0 ? 0 : static_cast<int>((c_end64 + 3) & ~int64_t{3});
            int c = 0;
            if (sym && ibase > jstart)   // chunks entirely below the diagonal for all 32 rows
                c = static_cast<int>(((ibase - jstart) / 4) * 4);
            float* const out_f = job.out_f;
            float* const out_t = job.out_t;
            const int64_t ld_out = job.ld_out, ld_t = job.ld_t;
            // counts of earlier sample chunks (or null): n11 = prefix + this launch's
            const int32_t* const prefix = job.out_c;
            // split tile: units 0 .. parts-2 store their exact counts in their
            // slots and count themselves in; the last unit (listed, so taken,
            // after the others) waits for them, adds their counts to its
            // accumulator in tensor memory (exact: a launch counts at most
            // 2^24 samples) and evaluates MI as for a whole tile.  The wait
            // ends: the units it waits for are earlier in the tile list, so
            // none of them waits on it.
            if (split_is_k(tile.split)) {
                const int parts = tile.split & 15, part = (tile.split >> 4) & 15;
                const int64_t slot = (tile.split >> 8) - 1;
                const int64_t wbase = (static_cast<int64_t>(sm.rank) * kNepi + (warp - 2)) *
                                      max_part_cols(kNepi) * 32;
                int32_t* const slot_base = L.part_counts + slot * (parts - 1) * part_slot_ints();
                unsigned int* const arrive =
                    L.part_arrive + (slot * 2 + sm.rank) * kNepi + (warp - 2);
                if (part < parts - 1) {
                    int32_t* mine = slot_base + part * part_slot_ints() + wbase;
#pragma unroll 1
                    for (int cc = c; cc < c_end; cc += 4) {
                        uint32_t r4[4];
                        ptx::tmem_ld_32x32b_x4(taddr + static_cast<uint32_t>(cc), r4);
                        ptx::tmem_wait_ld();
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            mine[(cc + q) * 32 + lane] =
                                __float2int_rn(__uint_as_float(r4[q]) * cscale);
                    }
                    __threadfence();
                    __syncwarp();
                    if (lane == 0) atomicAdd(arrive, 1u);
                    c_end = c;   // the last unit evaluates this tile
                } else {
                    bool ready = true;
                    if (lane == 0) {
                        const uint64_t t0 = ptx::globaltimer_ns();
                        while (*reinterpret_cast<volatile unsigned int*>(arrive) + 1u <
                               static_cast<unsigned int>(parts)) {
                            if (*sm.abort_flag() || ptx::globaltimer_ns() - t0 > L.timeout_ns) {
                                ready = false;
                                break;
                            }
                        }
                    }
                    ready = __shfl_sync(0xffffffffu, ready ? 1 : 0, 0) != 0;
                    if (!ready) {
                        if (lane == 0) raise_abort(sm, L.err, kErrTimeoutEpilogue);
                        c_end = c;
                    } else {
                        __threadfence();   // the other units' counts are visible past this point
                        const int32_t* others = slot_base + wbase;
#pragma unroll 1
                        for (int cc = c; cc < c_end; cc += 4) {
                            uint32_t r4[4];
                            ptx::tmem_ld_32x32b_x4(taddr + static_cast<uint32_t>(cc), r4);
                            ptx::tmem_wait_ld();
#pragma unroll
                            for (int q = 0; q < 4; ++q) {
                                float f = __uint_as_float(r4[q]);
                                for (int pp = 0; pp < parts - 1; ++pp)
                                    f += static_cast<float>(__ldcg(
                                        others + pp * part_slot_ints() + (cc + q) * 32 + lane));
                                r4[q] = __float_as_uint(f);
                            }
                            ptx::tmem_st_32x32b_x4(taddr + static_cast<uint32_t>(cc), r4);
                        }
                        ptx::tmem_wait_st();
                    }
                }
            }
            uint32_t cur[4];
            if (c < c_end) {
                ptx::tmem_ld_32x32b_x4(taddr + static_cast<uint32_t>(c), cur);
                ptx::tmem_wait_ld();
            }
            // Interior chunks take a lean body with no per-pair predicate: the
            // FP32 epilogue without earlier-chunk counts or a transposed output,
            // packed operands, all 32 rows valid and 16-byte aligned output
            // rows, and (per chunk, warp-uniform) all 4 columns valid and
            // strictly above the diagonal of all 32 rows.  det = 0 needs no
            // test there: every x_c is then 0 and the series gives exactly 0.
            const bool lean_rows = !kFix && prefix == nullptr && out_t == nullptr && !L.direct &&
                                   ibase + 32 <= n_a && (ld_out & 3) == 0 &&
                                   (reinterpret_cast<uintptr_t>(out_f) & 15u) == 0;
            const bool lean_rows8 = lean_rows && (ld_out & 7) == 0 &&
                                    (reinterpret_cast<uintptr_t>(out_f) & 31u) == 0;
#pragma unroll 1
            for (; c < c_end; c += 4) {
                uint32_t nxt[4];
                const bool more = c + 4 < c_end;
                if (more) ptx::tmem_ld_32x32b_x4(taddr + static_cast<uint32_t>(c + 4), nxt);
                const int64_t j0 = jstart + c;
                if (lean_rows8 && (j0 & 7) == 0 && c + 8 <= c_end && j0 + 8 <= n_b &&
                    (!sym || j0 > ibase + 31)) {
                    // two chunks at once (the second is in flight in nxt): each
                    // row's 8 values leave as one 32-byte store
                    uint32_t nx2[4];
                    const bool more2 = c + 8 < c_end;
                    ptx::tmem_wait_ld();
                    if (more2) ptx::tmem_ld_32x32b_x4(taddr + static_cast<uint32_t>(c + 8), nx2);
                    float v[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const MiVarF B = cvf[c + q];
                        const uint32_t w = q < 4 ? cur[q] : nxt[q - 4];
                        const MiCounts cc = mi_counts(__float2int_rn(__uint_as_float(w)), A.v, B.v, P);
                        v[q] = fmaxf(mi_fp32(cc, det_to_float(cc.det), A, B, P), 0.f);
                    }
                    if (sym) {
#pragma unroll
                        for (int q = 0; q < 8; ++q) out_f[(j0 + q) * ld_out + i] = v[q];
                    }
                    ptx::st_global_v8(out_f + i * ld_out + j0, v);
                    if (more2) {
                        ptx::tmem_wait_ld();
#pragma unroll
                        for (int q = 0; q < 4; ++q) cur[q] = nx2[q];
                    }
                    c += 4;   // + 4 by the loop
                    continue;
                }
                if (lean_rows && j0 + 4 <= n_b && (!sym || j0 > ibase + 31)) {
                    float v[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const MiVarF B = cvf[c + q];
                        const MiCounts cc =
                            mi_counts(__float2int_rn(__uint_as_float(cur[q])), A.v, B.v, P);
                        v[q] = fmaxf(mi_fp32(cc, det_to_float(cc.det), A, B, P), 0.f);
                    }
                    if (sym) {
#pragma unroll
                        for (int q = 0; q < 4; ++q) out_f[(j0 + q) * ld_out + i] = v[q];
                    }
                    *reinterpret_cast<float4*>(out_f + i * ld_out + j0) =
                        make_float4(v[0], v[1], v[2], v[3]);
                    if (more) {
                        ptx::tmem_wait_ld();
#pragma unroll
                        for (int q = 0; q < 4; ++q) cur[q] = nxt[q];
                    }
                    continue;
                }
                float v[4];
                int32_t n11s[4];
                uint32_t need = 0;   // kFix: pairs that go to the FP64 combine
                // kFix: the table reads of the chunk's pairs are issued before
                // their FP32 arithmetic, which hides their latency (the reads
                // are scattered over the table and mostly miss L1); almost every
                // pair of sparse data needs them
                double t[4][4];
                if constexpr (kFix) {
                    const bool early = P.fixup && P.T != nullptr;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int64_t j = j0 + q;
                        int32_t n11 = __float2int_rn(__uint_as_float(cur[q]) * cscale);
                        const bool ld = early && row_ok && j < n_b && (!sym || j >= i);
                        if (ld && prefix != nullptr) n11 += prefix[i * ld_out + j];
                        n11s[q] = n11;
                        const MiCounts cc =
                            mi_counts(ld ? n11 : 0, ld ? A.v : 0, ld ? cvf[c + q].v : 0, P);
                        t[q][0] = ld ? __ldg(P.T + cc.n11) : 0.0;
                        t[q][1] = ld ? __ldg(P.T + cc.n00) : 0.0;
                        t[q][2] = ld ? __ldg(P.T + cc.n10) : 0.0;
                        t[q][3] = ld ? __ldg(P.T + cc.n01) : 0.0;
                    }
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int64_t j = j0 + q;
                    int32_t n11 = __float2int_rn(__uint_as_float(cur[q]) * cscale);
                    float mi = 0.f;
                    if (row_ok && j < n_b && (!sym || j >= i)) {
                        if (prefix != nullptr) n11 += prefix[i * ld_out + j];
                        if constexpr (kFix) {
                            const MiVarF B = cvf[c + q];
                            const MiCounts cc = mi_counts(n11, A.v, B.v, P);
                            if (cc.det != 0) {
                                const float fdet = det_to_float(cc.det);
                                bool small = P.fixup && mi_surely_small(fdet, A, B, P);
                                if (!small) {
                                    mi = fmaxf(mi_fp32(cc, fdet, A, B, P), 0.f);
                                    small = P.fixup && mi < P.fixup_below;
                                }
                                if (small) need |= 1u << q;
                            }
                        } else {
                            const MiVarF B = cvf[c + q];
                            const MiCounts cc = mi_counts(n11, A.v, B.v, P);
                            if (cc.det != 0)
                                mi = fmaxf(mi_fp32(cc, det_to_float(cc.det), A, B, P), 0.f);
                        }
                    }
                    v[q] = mi;
                    n11s[q] = n11;
                }
                if constexpr (kFix) {
                    if (!(P.fixup && P.T != nullptr) && __any_sync(0xffffffffu, need != 0)) {
                        // (no table: the terms evaluated here, for the pairs that need them)
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const bool on = (need >> q) & 1u;
                            const MiCounts cc = mi_counts(on ? n11s[q] : 0, on ? A.v : 0,
                                                          on ? cvf[c + q].v : 0, P);
                            t[q][0] = on ? nlog2n(cc.n11, P) : 0.0;
                            t[q][1] = on ? nlog2n(cc.n00, P) : 0.0;
                            t[q][2] = on ? nlog2n(cc.n10, P) : 0.0;
                            t[q][3] = on ? nlog2n(cc.n01, P) : 0.0;
                        }
                    }
                    if (need != 0) {
                        // m MI = T[n11] + T[n10] + T[n01] + T[n00] + K_i + K_j
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            if ((need >> q) & 1u) {
                                const double sum = (t[q][0] + t[q][1]) + (t[q][2] + t[q][3]);
                                const double r = sum + (A.h + cvh[c + q]);
                                v[q] = fmaxf(static_cast<float>(r) * P.inv_m, 0.f);
                            }
                        }
                    }
                }
                if (row_ok) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int64_t j = j0 + q;
                        if (sym && j < n_b && j > i) out_f[j * ld_out + i] = v[q];
                        if (out_t != nullptr && j < n_b) out_t[j * ld_t + i] = v[q];
                    }
                    // (i, j): one 16-byte vector, or two 8-byte ones, as the row's
                    // alignment allows (rows of an odd-width output differ)
                    float* const rowp = out_f + i * ld_out + j0;
                    const uint32_t al =
                        static_cast<uint32_t>(reinterpret_cast<uintptr_t>(rowp)) & 15u;
                    if (j0 + 4 <= n_b && (!sym || j0 >= i) && (al & 7u) == 0) {
                        if (al == 0) {
                            *reinterpret_cast<float4*>(rowp) = make_float4(v[0], v[1], v[2], v[3]);
                        } else {
                            reinterpret_cast<float2*>(rowp)[0] = make_float2(v[0], v[1]);
                            reinterpret_cast<float2*>(rowp)[1] = make_float2(v[2], v[3]);
                        }
                    } else {
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const int64_t j = j0 + q;
                            if (j < n_b && (!sym || j >= i)) out_f[i * ld_out + j] = v[q];
                        }
                    }
                }
                if (more) {
                    ptx::tmem_wait_ld();
#pragma unroll
                    for (int q = 0; q < 4; ++q) cur[q] = nxt[q];
                }
            }
        } else
#pragma unroll 1
        for (int g = 0; g < cols; g += kGroup) {
            const int64_t j0 = jstart + g;
            // warp-uniform skips: group beyond the last variable, or (symmetric)
            // entirely below the diagonal for this warp's 32 rows
            if (j0 >= n_b) break;
            if (sym && j0 + kGroup - 1 < ibase) continue;
            uint32_t r[kGroup];
            ptx::tmem_ld_32x32b_x16(taddr + static_cast<uint32_t>(g), r);
            ptx::tmem_wait_ld();
            // counts: the accumulator's exact integers
#pragma unroll
            for (int q = 0; q < kGroup; ++q)
                r[q] = static_cast<uint32_t>(__float2int_rn(__uint_as_float(r[q]) * cscale));
            // (j, i): lanes hold consecutive i -> each store is one coalesced row segment
            if (sym && row_ok) {
#pragma unroll
                for (int q = 0; q < kGroup; ++q) {
                    const int64_t j = j0 + q;
                    if (j < n_b && j > i) store_one<kMode>(job, j, i, r[q]);
                }
            }
            // (i, j): 16 consecutive columns of this thread's row
            if (!row_ok) continue;
            const bool full = (j0 + kGroup <= n_b) && (!sym || j0 >= i);
            const uintptr_t rowp = reinterpret_cast<uintptr_t>(job.out_c + i * job.ld_out + j0);
            if (full && (rowp & 15u) == 0) {
                {
                    int4* dst = reinterpret_cast<int4*>(job.out_c + i * job.ld_out + j0);
#pragma unroll
                    for (int q = 0; q < kGroup / 4; ++q) {
                        int4 v = make_int4(static_cast<int>(r[4 * q]),
                                           static_cast<int>(r[4 * q + 1]),
                                           static_cast<int>(r[4 * q + 2]),
                                           static_cast<int>(r[4 * q + 3]));
                        if (kMode == kTcModeCountsAdd) {
                            const int4 o = dst[q];
                            v.x += o.x;
                            v.y += o.y;
                            v.z += o.z;
                            v.w += o.w;
                        }
                        dst[q] = v;
                    }
                }
            } else {
#pragma unroll
                for (int q = 0; q < kGroup; ++q) {
                    const int64_t j = j0 + q;
                    if (j < n_b && (!sym || j >= i)) store_one<kMode>(job, i, j, r[q]);
                }
            }
        }
        if (L.panel_done != nullptr) {   // this warp's stores of the tile are done
            __syncwarp();
            __threadfence();
            if (lane == 0) {
                const int p = tile.I / L.panel_blocks;
                const unsigned int old = atomicAdd(L.panel_done + p, 1u);
                if (old + 1u == L.panel_target[p]) {
                    __threadfence_system();
                    *reinterpret_cast<volatile unsigned int*>(L.host_flags + p) = 1u;
                }
            }
        }
        ptx::tc_fence_before();
        if constexpr (kPair) {   // one arrival per warp, on CTA 0's barrier
            __syncwarp();
            if (lane == 0) {
                if (sm.rank == 0)
                    ptx::mbar_arrive(sm.tempty(acc));
                else
                    ptx::mbar_arrive_cluster(ptx::mapa_shared(sm.tempty(acc), 0u));
            }
        } else {
            ptx::mbar_arrive(sm.tempty(acc));
        }
        if (++acc == 2) {
            acc = 0;
            acc_phase ^= 1u;
        }
    }
}

template <int kMode, bool kPair>
__global__ void __launch_bounds__(threads_of(kMode), 1)
gram_tc_kernel(const __grid_constant__ OperandMaps maps, const __grid_constant__ GramLaunch L) {
    extern __shared__ uint8_t smem_raw[];
    constexpr int kStages = stages_for(kMode, kPair);
    Smem<kPair, kStages> sm;
    sm.base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                         ~static_cast<uintptr_t>(1023));
    sm.rank = kPair ? ptx::cluster_ctarank() : 0u;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const bool lead = sm.rank == 0;   // the CTA that loads and issues the MMAs

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            ptx::mbar_init(sm.full(s), 1);
            ptx::mbar_init(sm.empty(s), 1);
        }
        for (int b = 0; b < 2; ++b) {
            ptx::mbar_init(sm.tfull(b), 1);
            // pair: one arrival per epilogue warp of both CTAs, on CTA 0
            ptx::mbar_init(sm.tempty(b), kPair ? 2 * epi_warps(kMode) : epi_warps(kMode) * 32);
        }
        ptx::mbar_init(sm.drain(), 1);
        for (int q = 0; q < kQ; ++q) {
            ptx::mbar_init(sm.qfull(q), 1);
            // MMA thread + one lane per epilogue warp (pair: of both CTAs, on CTA 0)
            ptx::mbar_init(sm.qempty(q), 1 + (kPair ? 2 : 1) * epi_warps(kMode));
        }
        *sm.abort_flag() = 0;
        ptx::fence_barrier_init();
    }
    if (warp == 0 && lane == 0 && lead) {
        if (L.direct) {
            ptx::tma_prefetch_desc(&maps.xa);
            ptx::tma_prefetch_desc(&maps.xb);
        } else {
            ptx::tma_prefetch_desc(&maps.box64);
            ptx::tma_prefetch_desc(&maps.box120);
            ptx::tma_prefetch_desc(&maps.box128);
            ptx::tma_prefetch_desc(&maps.box256);
        }
    }
    if (warp == 1) {
        if constexpr (kPair) {
            ptx::tmem_alloc_pair(ptx::smem_u32(sm.tmem_holder()), kTmemCols);
            ptx::tmem_relinquish_pair();
        } else {
            ptx::tmem_alloc(ptx::smem_u32(sm.tmem_holder()), kTmemCols);
            ptx::tmem_relinquish();
        }
    }
    ptx::tc_fence_before();
    __syncthreads();
    // pair: the partner's barriers are initialised before anything reaches them
    if constexpr (kPair) ptx::cluster_sync();
    ptx::tc_fence_after();
    const uint32_t tmem_base = *sm.tmem_holder();
    if (L.fp4) {
        // every scale factor of the block-scaled MMA is 1.0: four epilogue warps
        // (one per TMEM lane quadrant) fill the two 16-column scale regions
        if (warp >= 2 && warp < 6) {
            const uint32_t lanes = static_cast<uint32_t>((warp & 3) * 32) << 16;
            ptx::tmem_st_32x32b_x16_fill(tmem_base + lanes + kSfaCol, kScaleOnes);
            ptx::tmem_st_32x32b_x16_fill(tmem_base + lanes + kSfbCol, kScaleOnes);
            ptx::tmem_wait_st();
        }
        ptx::tc_fence_before();
        __syncthreads();
        if constexpr (kPair) ptx::cluster_sync();
        ptx::tc_fence_after();
    }

    if (warp == 0) {
        if (lane == 0 && lead) run_producer<kPair>(sm, maps, L);
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0 && lead) {
            if (L.fp4)
                run_mma<kPair, true>(sm, L, tmem_base);
            else
                run_mma<kPair, false>(sm, L, tmem_base);
        }
        __syncwarp();
    } else {
        run_epilogue<kMode, kPair>(sm, L, tmem_base);
    }

    ptx::tc_fence_before();
    __syncthreads();
    // pair: neither CTA leaves (or frees tensor memory) while the other may
    // still signal its barriers or be written by its copies
    if constexpr (kPair) ptx::cluster_sync();
    if (warp == 1) {
        ptx::tc_fence_after();
        if constexpr (kPair)
            ptx::tmem_dealloc_pair(tmem_base, kTmemCols);
        else
            ptx::tmem_dealloc(tmem_base, kTmemCols);
    }
}

template <bool kPair>
cudaError_t set_smem_attrs() {
    // each mode's kernel: its own plan's shared memory (stages_for)
    cudaError_t e;
    e = cudaFuncSetAttribute(gram_tc_kernel<kTcModeMI, kPair>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(Plan<kPair, stages_for(kTcModeMI, kPair)>::smem_bytes));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(gram_tc_kernel<kTcModeMI32, kPair>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(Plan<kPair, stages_for(kTcModeMI32, kPair)>::smem_bytes));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(gram_tc_kernel<kTcModeCounts, kPair>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(Plan<kPair, stages_for(kTcModeCounts, kPair)>::smem_bytes));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(
        gram_tc_kernel<kTcModeCountsAdd, kPair>, cudaFuncAttributeMaxDynamicSharedMemorySize,
        static_cast<int>(Plan<kPair, stages_for(kTcModeCountsAdd, kPair)>::smem_bytes));
}

template <int kMode>
cudaError_t launch_pair(const OperandMaps& maps, const GramLaunch& L, int grid,
                        cudaStream_t s) {
    cudaLaunchConfig_t cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3(static_cast<unsigned>(grid), 1, 1);
    cfg.blockDim = dim3(threads_of(kMode), 1, 1);
    cfg.dynamicSmemBytes = Plan<true, stages_for(kMode, true)>::smem_bytes;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, gram_tc_kernel<kMode, true>, maps, L);
}

}  // namespace

size_t gram_tc_smem_bytes() { return Plan<false>::smem_bytes; }

cudaError_t gram_tc_prepare() {
    cudaError_t e = set_smem_attrs<false>();
    if (e != cudaSuccess) return e;
    return set_smem_attrs<true>();
}

int gram_tc_epilogue_warps(int mode, int fixup) {
    const int m = (mode == kTcModeMI && !fixup) ? kTcModeMI32 : mode;
    return epi_warps(m);
}

int64_t gram_part_slot_ints() { return part_slot_ints(); }
int gram_part_slot_counters() { return 2 * kEpiWarpsMain; }

int gram_tc_pair_clusters() {
    cudaLaunchConfig_t cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3(2, 1, 1);
    cfg.blockDim = dim3(threads_of(kTcModeMI32), 1, 1);
    cfg.dynamicSmemBytes = Plan<true>::smem_bytes;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, gram_tc_kernel<kTcModeMI32, true>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

int64_t gram_tile_count(int64_t n_a, int64_t n_b, int bn, bool symmetric, int bm) {
    const int64_t TI = (n_a + bm - 1) / bm, TJ = (n_b + bn - 1) / bn;
    if (!symmetric) return TI * TJ;
    int64_t c = 0;
    for (int64_t J = 0; J < TJ; ++J)   // row blocks I with bm I <= bn J + bn - 1
        c += std::min<int64_t>(TI, (J * bn + bn - 1) / bm + 1);
    return c;
}

void gram_tiles(int job, int64_t n_a, int64_t n_b, int bn, bool symmetric, int group_cols,
                GramTile* out, int bm) {
    const int64_t TI = (n_a + bm - 1) / bm, TJ = (n_b + bn - 1) / bn;
    const int64_t group = std::max(1, group_cols);
    int64_t k = 0;
    for (int64_t g0 = 0; g0 < TJ; g0 += group) {
        const int64_t g1 = std::min<int64_t>(TJ, g0 + group);
        for (int64_t I = 0; I < TI; ++I)
            for (int64_t J = g0; J < g1; ++J) {
                if (symmetric && I * bm > J * bn + bn - 1) continue;   // below the diagonal
                out[k++] = GramTile{job, static_cast<int32_t>(I), static_cast<int32_t>(J), 0};
            }
    }
}

cudaError_t launch_gram_tc(const OperandMaps& maps, const GramLaunch& L, int grid,
                           cudaStream_t s) {
    if (L.num_tiles <= 0 || grid <= 0) return cudaSuccess;
    // MI with the FP64 combine off runs the kernel without its code
    const int mode = (L.mode == kTcModeMI && !L.fixup) ? kTcModeMI32 : L.mode;
    if (L.fp4 && (L.direct || (L.jobs == nullptr && L.job0.bn > kTcBNFp4)))
        return cudaErrorInvalidValue;
    if (L.pair) {
        if (grid % 2 != 0 || L.direct) return cudaErrorInvalidValue;
        switch (mode) {
            case kTcModeMI32: return launch_pair<kTcModeMI32>(maps, L, grid, s);
            case kTcModeMI: return launch_pair<kTcModeMI>(maps, L, grid, s);
            case kTcModeCounts: return launch_pair<kTcModeCounts>(maps, L, grid, s);
            case kTcModeCountsAdd: return launch_pair<kTcModeCountsAdd>(maps, L, grid, s);
            default: return cudaErrorInvalidValue;
        }
    }
    // each mode's kernel takes its own plan's shared memory (stages_for)
    switch (mode) {
        case kTcModeMI32:
            gram_tc_kernel<kTcModeMI32, false><<<grid, threads_of(kTcModeMI32),
                Plan<false, stages_for(kTcModeMI32, false)>::smem_bytes, s>>>(maps, L);
            break;
        case kTcModeMI:
            gram_tc_kernel<kTcModeMI, false><<<grid, threads_of(kTcModeMI),
                Plan<false, stages_for(kTcModeMI, false)>::smem_bytes, s>>>(maps, L);
            break;
        case kTcModeCounts:
            gram_tc_kernel<kTcModeCounts, false><<<grid, threads_of(kTcModeCounts),
                Plan<false, stages_for(kTcModeCounts, false)>::smem_bytes, s>>>(maps, L);
            break;
        case kTcModeCountsAdd:
            gram_tc_kernel<kTcModeCountsAdd, false><<<grid, threads_of(kTcModeCountsAdd),
                Plan<false, stages_for(kTcModeCountsAdd, false)>::smem_bytes, s>>>(maps, L);
            break;
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace gbmi
