// Pack pass: one read of X (m samples x n variables, row-major uint8) writes
//   P  - the transposed FP8 operand of the tensor-core Gram in K-block-major
//        order (for each block of 128 samples, one 128-byte row per variable;
//        0x00 / 0x38 = E4M3 1.0 per sample), or its FP4 form (for each block of
//        256 samples, one 128-byte row of E2M1 nibbles 0x0 / 0x2), samples
//        beyond m zeroed (they would add to every count); rows beyond n are
//        not written (a garbage operand row only reaches accumulator rows or
//        columns that every epilogue masks),
//   Bp - the transposed bit-packed operand of the popcount Gram,
//   v  - the column counts v_j = sum_r X_rj (Sec. 3.1, Term 2: v = D^T 1;
//        also the diagonal of G11, Sec. 2 step 3).
// The complement matrix of Sec. 2 step 1 is never formed: Eq. 6-7 replace it.
//
// A CTA owns 128 variables and a run of 128-sample tiles.  Each tile is read
// with coalesced 16-byte loads (the next tile's loads are in flight while the
// current one is transposed; rows that are not 16-byte aligned are copied by
// cp.async as aligned granules and realigned from shared memory), transposed
// through shared memory in 4x4 byte blocks with byte permutes, and written
// out so that every warp store covers whole 128-byte rows of P (a tile's
// output is one contiguous 16 KB block).
// A grouped launch covers many datasets: CTA c works for the job whose CTA
// range holds c.
#include "internal.cuh"

namespace gbmi {

namespace {

constexpr int kPackThreads = 256;
constexpr int kTileR = 128;        // samples per tile
constexpr int kTileJ = 128;        // variables per CTA
constexpr int kTilesPerCta = 16;   // sample tiles walked by one CTA (at most, usually)
constexpr int64_t kPackCtasTarget = 152 * 8;   // CTAs one job should launch: 2 waves

// 1 in every byte that is non-zero, 0 elsewhere.
__device__ __forceinline__ uint32_t nz_bytes(uint32_t w) {
    uint32_t t = w | (w >> 4);
    t |= t >> 2;
    t |= t >> 1;
    return t & 0x01010101u;
}

// Transpose a 4x4 byte block: w[k] holds row k (4 bytes = 4 columns); c[q]
// receives column q (4 bytes = rows 0..3).
__device__ __forceinline__ void transpose4x4(const uint32_t w0, const uint32_t w1,
                                             const uint32_t w2, const uint32_t w3,
                                             uint32_t& c0, uint32_t& c1, uint32_t& c2,
                                             uint32_t& c3) {
    const uint32_t t0 = __byte_perm(w0, w1, 0x5140);
    const uint32_t t1 = __byte_perm(w2, w3, 0x5140);
    const uint32_t t2 = __byte_perm(w0, w1, 0x7362);
    const uint32_t t3 = __byte_perm(w2, w3, 0x7362);
    c0 = __byte_perm(t0, t1, 0x5410);
    c1 = __byte_perm(t0, t1, 0x7632);
    c2 = __byte_perm(t2, t3, 0x5410);
    c3 = __byte_perm(t2, t3, 0x7632);
}

// Asynchronous 16-byte copy global -> shared of the first `bytes` (0..16) bytes
// of a 16-byte aligned granule; the rest of the destination is zero-filled and
// no byte past `bytes` is read.
__device__ __forceinline__ void cp_async16(uint32_t dst_smem, const void* src, uint32_t bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst_smem), "l"(src),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// Unaligned rows: every warp stages its 16 rows of a tile (4 per quarter) as
// the 9 aligned 16-byte granules that cover each row's 128-byte slice (row
// stride 144 bytes).
constexpr int kRawRowBytes = 144;
constexpr int kRawWarpBytes = 16 * kRawRowBytes;

// Low bits of the four 0/1 bytes of x, packed into a nibble (byte k -> bit k).
__device__ __forceinline__ uint32_t bytes_to_nibble(uint32_t x) {
    return ((x * 0x01020408u) >> 24) & 0xFu;
}

// Thread layout of the transpose: warp w owns variables 16 w .. 16 w + 15 of
// the CTA's 128 and all 128 samples of the tile; lane = 4 sg + vg takes the
// 4 variables 16 w + 4 vg .. + 3 and the 16 samples 16 sg .. + 15.  A store
// instruction of the warp then writes 4 whole 128-byte rows of P (4 half rows
// of 64 bytes in the FP4 form).  The tile sits in shared memory with its
// 16-byte chunks XOR-swizzled by the row's 16-row group (chunk ^ (r / 16) % 8),
// which keeps both the row-wise fill and the column-wise reads of the
// transpose free of bank conflicts.
__device__ __forceinline__ int swz_chunk(int r, int chunk) { return chunk ^ ((r >> 4) & 7); }

// Transpose the tile in S (128 samples from r0, 128 variables from j0), add
// its column sums to colsum and store this thread's pieces of P and Bp.
// The pack is bound by instruction issue more than by HBM, so the FP4 form
// skips the byte transpose: the E2M1 byte of samples (2k, 2k + 1) of the four
// variables of a word column is (w_2k << 1) | (w_2k+1 << 5) of the 0/1 sample
// words, and two byte permutes per four samples regroup them by variable.
__device__ __forceinline__ void transpose_store(const PackJob& a, const uint8_t* S, int64_t tile,
                                                int64_t j0, int (&colsum)[4]) {
    const int t = threadIdx.x;
    const int w = t >> 5;
    const int lane = t & 31;
    const int vg = lane & 3;
    const int sg = lane >> 2;
    const int colw = 4 * w + vg;   // word column (4 variables) of this thread
    const uint32_t* S32 = reinterpret_cast<const uint32_t*>(S);
    const int swz = colw ^ (4 * sg);   // rows 16 sg .. +15 share one swizzle
    const int64_t jw = j0 + colw * 4;  // first of the thread's 4 variables
    uint32_t acc4 = 0;   // byte c: this tile's count of variable jw + c (<= 16)
    if (a.fp4 && a.Bp == nullptr) {
        uint32_t v01[4], v23[4];   // per 4 samples: variables 0, 1 and 2, 3 (16 bits each)
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            const int rr = sg * 16 + g * 4;
            const uint32_t w0 = nz_bytes(S32[(rr + 0) * (kTileJ / 4) + swz]);
            const uint32_t w1 = nz_bytes(S32[(rr + 1) * (kTileJ / 4) + swz]);
            const uint32_t w2 = nz_bytes(S32[(rr + 2) * (kTileJ / 4) + swz]);
            const uint32_t w3 = nz_bytes(S32[(rr + 3) * (kTileJ / 4) + swz]);
            acc4 += (w0 + w1) + (w2 + w3);
            const uint32_t A = (w0 << 1) | (w1 << 5);   // byte c: samples 0, 1 of variable c
            const uint32_t B = (w2 << 1) | (w3 << 5);   // samples 2, 3
            v01[g] = __byte_perm(A, B, 0x5140);
            v23[g] = __byte_perm(A, B, 0x7362);
        }
        // variable c: samples 16 sg .. + 15 as 8 bytes (64 h + 8 sg of its K-block row)
        const uint2 o[4] = {
            make_uint2(__byte_perm(v01[0], v01[1], 0x5410), __byte_perm(v01[2], v01[3], 0x5410)),
            make_uint2(__byte_perm(v01[0], v01[1], 0x7632), __byte_perm(v01[2], v01[3], 0x7632)),
            make_uint2(__byte_perm(v23[0], v23[1], 0x5410), __byte_perm(v23[2], v23[3], 0x5410)),
            make_uint2(__byte_perm(v23[0], v23[1], 0x7632), __byte_perm(v23[2], v23[3], 0x7632))};
        uint8_t* const dst = a.P + ((tile >> 1) * a.rows_p + jw) * kTileR +
                             (tile & 1) * (kTileR / 2) + sg * 8;
#pragma unroll
        for (int c = 0; c < 4; ++c)   // padding rows are left as they are: masked downstream
            if (jw + c < a.n) *reinterpret_cast<uint2*>(dst + c * kTileR) = o[c];
    } else {
        uint32_t col[4][4];   // col[c][g]: variable jw + c, samples 16 sg + 4 g .. +3
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            const int rr = sg * 16 + g * 4;
            const uint32_t w0 = nz_bytes(S32[(rr + 0) * (kTileJ / 4) + swz]);
            const uint32_t w1 = nz_bytes(S32[(rr + 1) * (kTileJ / 4) + swz]);
            const uint32_t w2 = nz_bytes(S32[(rr + 2) * (kTileJ / 4) + swz]);
            const uint32_t w3 = nz_bytes(S32[(rr + 3) * (kTileJ / 4) + swz]);
            acc4 += (w0 + w1) + (w2 + w3);
            transpose4x4(w0, w1, w2, w3, col[0][g], col[1][g], col[2][g], col[3][g]);
        }
        const int64_t rbase = tile * kTileR + sg * 16;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int64_t j = jw + c;
            if (j >= a.n) continue;   // padding rows are left as they are: masked downstream
            if (a.P != nullptr) {
                uint4 o;
                o.x = col[c][0] * 0x38u;
                o.y = col[c][1] * 0x38u;
                o.z = col[c][2] * 0x38u;
                o.w = col[c][3] * 0x38u;
                *reinterpret_cast<uint4*>(a.P + (tile * a.rows_p + j) * kTileR + sg * 16) = o;
            }
            if (a.Bp != nullptr) {
                const uint32_t bits = bytes_to_nibble(col[c][0]) |
                                      (bytes_to_nibble(col[c][1]) << 4) |
                                      (bytes_to_nibble(col[c][2]) << 8) |
                                      (bytes_to_nibble(col[c][3]) << 12);
                uint16_t* B16 = reinterpret_cast<uint16_t*>(a.Bp);
                B16[j * (a.ldp / 16) + rbase / 16] = static_cast<uint16_t>(bits);
            }
        }
    }
    colsum[0] += acc4 & 0xFF;
    colsum[1] += (acc4 >> 8) & 0xFF;
    colsum[2] += (acc4 >> 16) & 0xFF;
    colsum[3] += acc4 >> 24;
}

// Column sums of the CTA's variables: sum over the 8 sample groups of the warp
// (lane bits 2-4), one atomic add per variable.
__device__ __forceinline__ void flush_colsum(const PackJob& a, int64_t j0, const int (&colsum)[4]) {
    if (a.v == nullptr) return;
    const int t = threadIdx.x;
    const int lane = t & 31;
    const int colw = 4 * (t >> 5) + (lane & 3);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        int x = colsum[c];
        x += __shfl_xor_sync(0xffffffffu, x, 4);
        x += __shfl_xor_sync(0xffffffffu, x, 8);
        x += __shfl_xor_sync(0xffffffffu, x, 16);
        const int64_t j = j0 + colw * 4 + c;
        if ((lane >> 2) == 0 && j < a.n && x != 0) atomicAdd(a.v + j, x);
    }
}

// Rows that are 16-byte aligned: each tile is copied straight into its
// swizzled shared-memory slot by cp.async (lane l of a row's 8 lanes copies
// its 16-byte chunk; bytes outside [0, m) x [0, n) are zero-filled), in a ring
// of kStagesA tiles, so kStagesA - 1 tiles' loads are in flight while one is
// transposed and no registers hold them.
constexpr int kStagesA = 3;
constexpr int kTileBytes = kTileR * kTileJ;

__device__ __forceinline__ void pack_cta_aligned(const PackJob& a, const int64_t bx,
                                                 const int64_t by, uint8_t* S) {
    const int t = threadIdx.x;
    const int64_t j0 = bx * kTileJ;
    const int64_t tiles_total = a.ldp / kTileR;
    const int64_t tile_begin = by * a.tpc;
    const int64_t tile_end = min(tile_begin + a.tpc, tiles_total);
    const int64_t jl = j0 + (t & 7) * 16;
    auto issue = [&](int64_t tile, uint8_t* Sb) {
        if (tile < tile_end) {
            const int64_t r0 = tile * kTileR;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int r = q * 32 + (t >> 3);
                const int64_t rg = r0 + r;
                const bool in = rg < a.m && jl < a.n;
                const uint32_t dst = static_cast<uint32_t>(
                    __cvta_generic_to_shared(Sb + r * kTileJ + swz_chunk(r, t & 7) * 16));
                cp_async16(dst, in ? a.X + rg * a.ldx + jl : a.X, in ? 16u : 0u);
            }
        }
        cp_async_commit();   // one group per tile slot, empty past the end
    };
#pragma unroll
    for (int s = 0; s < kStagesA - 1; ++s) issue(tile_begin + s, S + s * kTileBytes);
    int colsum[4] = {0, 0, 0, 0};
    int slot = 0;
    for (int64_t tile = tile_begin; tile < tile_end; ++tile) {
        // this thread's copies of `tile` have landed, then everyone's; every
        // thread is also done with the slot the next issue refills
        asm volatile("cp.async.wait_group %0;" ::"n"(kStagesA - 2) : "memory");
        __syncthreads();
        const int refill = slot == 0 ? kStagesA - 1 : slot - 1;
        issue(tile + kStagesA - 1, S + refill * kTileBytes);
        transpose_store(a, S + slot * kTileBytes, tile, j0, colsum);
        slot = slot + 1 == kStagesA ? 0 : slot + 1;
    }
    cp_async_wait_all();
    flush_colsum(a, j0, colsum);
}

// Rows that are not 16-byte aligned: every warp stages its 16 rows of a tile
// (4 per quarter) in its raw rows by cp.async, as the aligned granules that
// cover each row's 128-byte slice (lane l of the row's 8 lanes copies granule
// l, lane 7 also granule 8), copying only bytes of [j0, min(j0 + 128, n)) of
// the row and zero-filling the rest; the next tile's copies are in flight
// while the current one is transposed.  The realignment (5 word reads and 4
// funnel shifts per lane and row) happens when the tile is written to S.
__device__ __forceinline__ void pack_cta_unaligned(const PackJob& a, const int64_t bx,
                                                   const int64_t by, uint8_t* S, uint8_t* raw) {
    const int t = threadIdx.x;
    const int64_t j0 = bx * kTileJ;
    const int64_t tiles_total = a.ldp / kTileR;
    const int64_t tile_begin = by * a.tpc;
    const int64_t tile_end = min(tile_begin + a.tpc, tiles_total);
    uint8_t* const wraw = raw + (t >> 5) * kRawWarpBytes;   // this warp's raw rows
    const int rr_w = (t >> 3) & 3;   // the lane's row among the warp's 4 per quarter
    const int gl = t & 7;            // and its granule
    // The lane's rows are r = 32 k + t / 8; 32 ldx is a multiple of 16, so all
    // of them start their slice at the same offset sft within a 16-byte
    // granule, and the valid bytes of each granule are the same for all of them.
    const int sft = static_cast<int>(
        (reinterpret_cast<uintptr_t>(a.X + j0) + static_cast<uint64_t>(t >> 3) * a.ldx) & 15);
    const int64_t keep_row = a.n - j0 < kTileJ ? a.n - j0 : kTileJ;   // >= 1
    const int64_t end = sft + keep_row;   // valid bytes: [sft, end) of the row's granules
    const uint32_t nb0 = static_cast<uint32_t>(
        end - 16 * gl <= 0 ? 0 : (end - 16 * gl > 16 ? 16 : end - 16 * gl));
    const uint32_t nb8 = static_cast<uint32_t>(end - 128 <= 0 ? 0 : end - 128);   // <= 16
    // + r * ldx: the lane's granule of row r (the aligned granule holding the
    // row's first byte, + 16 gl)
    const uintptr_t G0 = reinterpret_cast<uintptr_t>(a.X + j0) - sft + 16 * gl;
    auto issue_tile = [&](int64_t tile) {
        const int64_t r0 = tile * kTileR;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int64_t r = r0 + q * 32 + (t >> 3);
            const uint32_t dst = static_cast<uint32_t>(__cvta_generic_to_shared(
                wraw + (4 * q + rr_w) * kRawRowBytes + 16 * gl));
            const bool in = r < a.m;   // samples beyond m: zeros
            const uint8_t* G = reinterpret_cast<const uint8_t*>(G0 + r * a.ldx);
            cp_async16(dst, in ? G : a.X, in ? nb0 : 0u);
            if (gl == 7) cp_async16(dst + 16, in ? G + 16 : a.X, in ? nb8 : 0u);
        }
        cp_async_commit();
    };
    if (tile_begin < tile_end) issue_tile(tile_begin);

    int colsum[4] = {0, 0, 0, 0};
    const uint32_t sh = static_cast<uint32_t>(sft & 3) * 8u;
    for (int64_t tile = tile_begin; tile < tile_end; ++tile) {
        // this tile's raw rows have landed (the warp's own copies) -> realign
        cp_async_wait_all();
        __syncwarp();
        const uint32_t* wr =
            reinterpret_cast<const uint32_t*>(wraw) + (sft >> 2) + 4 * gl + rr_w * (kRawRowBytes / 4);
        uint4 pre[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t* row = wr + 4 * q * (kRawRowBytes / 4);
            const uint32_t w0 = row[0], w1 = row[1], w2 = row[2], w3 = row[3], w4 = row[4];
            pre[q] = make_uint4(__funnelshift_r(w0, w1, sh), __funnelshift_r(w1, w2, sh),
                                __funnelshift_r(w2, w3, sh), __funnelshift_r(w3, w4, sh));
        }
        __syncwarp();   // the raw rows are refilled by the next issue
        // ---- 128 samples x 128 variables into S (row r, swizzled 16-byte chunks)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int r = q * 32 + (t >> 3);
            *reinterpret_cast<uint4*>(S + r * kTileJ + swz_chunk(r, t & 7) * 16) = pre[q];
        }
        __syncthreads();
        if (tile + 1 < tile_end) issue_tile(tile + 1);
        transpose_store(a, S, tile, j0, colsum);
        __syncthreads();   // S is rewritten by the next tile
    }
    flush_colsum(a, j0, colsum);
}

// Shared memory of a pack CTA: the aligned ring (kStagesA tiles) or one tile
// plus the warps' raw rows, whichever is larger.
constexpr int kPackSmem = kStagesA * kTileBytes > kTileBytes + (kPackThreads / 32) * kRawWarpBytes
                              ? kStagesA * kTileBytes
                              : kTileBytes + (kPackThreads / 32) * kRawWarpBytes;
static_assert(kPackSmem <= 48 * 1024, "static shared memory of a pack CTA");

// One instantiation for 16-byte aligned rows, one for the rest.
template <bool kAligned>
__global__ void __launch_bounds__(kPackThreads, 4)   // 4 CTAs per SM: loads in flight
pack_kernel(const PackJob job) {
    __shared__ __align__(128) uint8_t smem[kAligned ? kStagesA * kTileBytes : kPackSmem];
    const int64_t c = blockIdx.x;
    if constexpr (kAligned)
        pack_cta_aligned(job, c % job.gx, c / job.gx, smem);
    else
        pack_cta_unaligned(job, c % job.gx, c / job.gx, smem, smem + kTileBytes);
}

__global__ void __launch_bounds__(kPackThreads, 4)
pack_grouped_kernel(const PackJob* __restrict__ jobs, int njobs,
                    const int32_t* __restrict__ cta_job) {
    __shared__ __align__(128) uint8_t smem[kPackSmem];
    const int64_t c = blockIdx.x;
    int lo = 0, hi = njobs - 1;   // last job whose cta_begin <= c
    if (cta_job != nullptr) {
        lo = __ldg(cta_job + c);
    } else {
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (jobs[mid].cta_begin <= c) lo = mid; else hi = mid - 1;
        }
    }
    const PackJob job = jobs[lo];
    const int64_t cl = c - job.cta_begin;
    if (job.vec)
        pack_cta_aligned(job, cl % job.gx, cl / job.gx, smem);
    else
        pack_cta_unaligned(job, cl % job.gx, cl / job.gx, smem, smem + kTileBytes);
}

__global__ void validate_kernel(const uint8_t* X, int64_t m, int64_t n, int64_t ldx,
                                unsigned int* flag) {
    const int64_t total = m * n;
    for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t r = e / n, j = e % n;
        if (X[r * ldx + j] > 1) {
            atomicOr(flag, 1u);
            return;
        }
    }
}

// Column counts for the direct operand path, which feeds the caller's X to the
// tensor cores without packing (n a multiple of 16, X 16-byte aligned): a
// block owns 512 columns (a warp reads 512 contiguous bytes of one row, one
// 16-byte load per lane) and a slice of rows split over its 8 warps.  Bytes
// are summed in 16-bit lanes (two per register, flushed every 255 rows, so
// any byte value is summed exactly), the warps' sums meet in shared memory
// and each column gets one atomic add per block.  A byte other than 0 / 1
// sets kErrNotBinary: the direct Gram reads bytes as E4M3 values, so
// non-binary data would not count as 1.
constexpr int kCsCols = 512;
constexpr int kCsWarps = 8;

__global__ void __launch_bounds__(kCsWarps * 32)
colsum_kernel(const uint8_t* __restrict__ X, int64_t m, int64_t n, int64_t rows_per_block,
              int32_t* __restrict__ v, unsigned int* err) {
    __shared__ int32_t red[kCsWarps][kCsCols + 16];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t c0 = static_cast<int64_t>(blockIdx.x) * kCsCols + lane * 16;
    const int64_t r0 = static_cast<int64_t>(blockIdx.y) * rows_per_block;
    const int64_t r1 = r0 + rows_per_block < m ? r0 + rows_per_block : m;
    int32_t tot[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) tot[k] = 0;
    uint32_t acc[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] = 0;
    uint32_t bad = 0;
    auto flush = [&]() {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            tot[4 * q + 0] += static_cast<int32_t>(acc[2 * q] & 0xFFFFu);
            tot[4 * q + 2] += static_cast<int32_t>(acc[2 * q] >> 16);
            tot[4 * q + 1] += static_cast<int32_t>(acc[2 * q + 1] & 0xFFFFu);
            tot[4 * q + 3] += static_cast<int32_t>(acc[2 * q + 1] >> 16);
            acc[2 * q] = acc[2 * q + 1] = 0;
        }
    };
    if (c0 < n) {   // n % 16 == 0: the lane's 16 bytes are inside the row
        int it = 0;
        for (int64_t r = r0 + w; r < r1; r += kCsWarps) {
            const uint4 q4 = __ldg(reinterpret_cast<const uint4*>(X + r * n + c0));
            const uint32_t ws[4] = {q4.x, q4.y, q4.z, q4.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                bad |= ws[q] & 0xFEFEFEFEu;
                acc[2 * q] += ws[q] & 0x00FF00FFu;
                acc[2 * q + 1] += (ws[q] >> 8) & 0x00FF00FFu;
            }
            if (++it == 255) {
                flush();
                it = 0;
            }
        }
        flush();
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) red[w][lane * 16 + k] = tot[k];
    if (__any_sync(0xffffffffu, bad != 0) && lane == 0) atomicOr(err, kErrNotBinary);
    __syncthreads();
    for (int c = threadIdx.x; c < kCsCols; c += kCsWarps * 32) {
        int32_t sum = 0;
#pragma unroll
        for (int k = 0; k < kCsWarps; ++k) sum += red[k][c];
        const int64_t col = static_cast<int64_t>(blockIdx.x) * kCsCols + c;
        if (col < n && sum != 0) atomicAdd(v + col, sum);
    }
}

}  // namespace

int64_t pack_job_ctas(PackJob& a, bool grouped) {
    const int64_t tiles_total = a.ldp / kTileR;
    // column blocks holding variables; the operand's padding rows (n .. rows_p)
    // are never written: every consumer masks rows and columns beyond n
    a.gx = static_cast<int32_t>((a.n + kTileJ - 1) / kTileJ);
    // Tiles per CTA: at most kTilesPerCta, fewer when the job has few column
    // blocks, so that a job alone still launches about kPackCtasTarget CTAs
    // (enough loads in flight to stream HBM); more for very long sample ranges,
    // to keep the CTA count moderate.  In a grouped launch the other jobs
    // supply the CTAs, and every CTA takes the most tiles (a CTA of one small
    // item would spend about as long starting as packing).
    int64_t tpc = grouped ? kTilesPerCta
                          : (tiles_total * a.gx + kPackCtasTarget - 1) / kPackCtasTarget;
    tpc = tpc < 1 ? 1 : (tpc > kTilesPerCta ? kTilesPerCta : tpc);
    while ((tiles_total + tpc - 1) / tpc > (int64_t{1} << 16)) tpc *= 2;
    a.tpc = static_cast<int32_t>(tpc);
    a.vec = (a.ldx % 16 == 0) && (a.n % 16 == 0) &&
            (reinterpret_cast<uintptr_t>(a.X) % 16 == 0);
    return static_cast<int64_t>(a.gx) * ((tiles_total + tpc - 1) / tpc);
}

cudaError_t launch_pack(const PackJob& job, cudaStream_t s) {
    if (job.rows_p % kTileJ != 0 || job.ldp % kTileR != 0) return cudaErrorInvalidValue;
    if (job.fp4 && job.ldp % (2 * kTileR) != 0) return cudaErrorInvalidValue;
    PackJob j = job;
    const int64_t ctas = pack_job_ctas(j);
    if (ctas <= 0 || ctas > 0x7FFFFFFF) return cudaErrorInvalidValue;
    if (j.vec)
        pack_kernel<true><<<static_cast<unsigned>(ctas), kPackThreads, 0, s>>>(j);
    else
        pack_kernel<false><<<static_cast<unsigned>(ctas), kPackThreads, 0, s>>>(j);
    return cudaGetLastError();
}

cudaError_t launch_pack_grouped(const PackJob* jobs, int njobs, int64_t total_ctas,
                                const int32_t* cta_job, cudaStream_t s) {
    if (njobs <= 0 || total_ctas <= 0) return cudaSuccess;
    if (total_ctas > 0x7FFFFFFF) return cudaErrorInvalidValue;
    pack_grouped_kernel<<<static_cast<unsigned>(total_ctas), kPackThreads, 0, s>>>(jobs, njobs,
                                                                                   cta_job);
    return cudaGetLastError();
}

cudaError_t launch_validate(const uint8_t* X, int64_t m, int64_t n, int64_t ldx,
                            unsigned int* flag, cudaStream_t s) {
    validate_kernel<<<1024, 256, 0, s>>>(X, m, n, ldx, flag);
    return cudaGetLastError();
}

cudaError_t launch_colsum_direct(const uint8_t* X, int64_t m, int64_t n, int32_t* v,
                                 unsigned int* err, int sm_count, cudaStream_t s) {
    if (m <= 0 || n <= 0) return cudaSuccess;
    if (n % 16 != 0 || (reinterpret_cast<uintptr_t>(X) & 15u) != 0) return cudaErrorInvalidValue;
    const int64_t gx = (n + kCsCols - 1) / kCsCols;
    const int64_t want = static_cast<int64_t>(sm_count > 0 ? sm_count : 152) * 8;
    int64_t gy = (want + gx - 1) / gx;
    gy = gy < 1 ? 1 : gy;
    int64_t rows = (m + gy - 1) / gy;
    rows = (rows + kCsWarps - 1) / kCsWarps * kCsWarps;
    gy = (m + rows - 1) / rows;
    if (gx > 0x7FFFFFFF || gy > 65535) return cudaErrorInvalidValue;
    colsum_kernel<<<dim3(static_cast<unsigned>(gx), static_cast<unsigned>(gy)), kCsWarps * 32, 0,
                    s>>>(X, m, n, rows, v, err);
    return cudaGetLastError();
}

}  // namespace gbmi
