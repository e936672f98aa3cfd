// Internal declarations shared by the kernels and the C ABI of libgbmi.so.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "mi_device.cuh"

namespace gbmi {

// ------------------------------------------------------------ packed layouts
//
// P  (tensor-core operand), K-block-major: for every block of 128 samples,
//    one 128-byte row per variable (FP8 E4M3 0x00 / 0x38 = 1.0 per sample):
//    byte (variable j, sample r) is at P[((r / 128) * rows_p + j) * 128 + r % 128].
//    rows_p = n rounded up to 256, k_blocks = m rounded up to 128, / 128.
//    Padding samples (beyond m) are zero; padding rows (beyond n) are not
//    written and hold whatever the buffer held: every consumer masks them.  Any number of operands can share one
//    buffer (each at its own first row), so one 2-D TMA descriptor of width
//    128 bytes reaches every tile of every dataset.
// P4 (the FP4 form of P, same buffer shape): for every block of 256 samples,
//    one 128-byte row per variable holding two samples per byte as E2M1
//    nibbles (0x0 / 0x2 = 1.0): samples 128 h + 16 g .. + 15 of the block
//    (h = 0, 1; g = 0..7) are the 8 bytes at 64 h + 8 g, sample 2 k and 2 k + 1
//    of those 16 in the low and high nibble of byte k.  k_blocks = m rounded up
//    to 256, / 256.  A and B always share this order, so the Gram's dot
//    products are the same sums as over samples in order.
// Bp (popcount operand): one row per variable, bit (r % 32) of 32-bit word
//    r / 32 holds sample r; wpr = ldp / 32 words per row, same row padding.
// v  column counts, int32, one per variable.
// MiVar per-variable epilogue terms (reciprocals, FP64 entropy term), one per
//    variable, computed from v once per call.
constexpr int64_t kRowPad = 256;
constexpr int64_t kColPad = 128;

inline int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }
inline int64_t pack_rows(int64_t n) { return round_up(n, kRowPad); }
inline int64_t pack_ld(int64_t m) { return round_up(m, kColPad); }
// Samples per K block (one 128-byte operand row): 128 FP8, 256 FP4.
constexpr int64_t kKbSamplesFp8 = 128;
constexpr int64_t kKbSamplesFp4 = 256;
inline int64_t kb_samples(bool fp4) { return fp4 ? kKbSamplesFp4 : kKbSamplesFp8; }
// Padded sample count of an operand of either form.
inline int64_t pack_ld_of(int64_t m, bool fp4) { return round_up(m, kb_samples(fp4)); }

// Device error word bits (set by kernels whose bounded waits gave up).
enum : uint32_t {
    kErrTimeoutLoad = 1u,
    kErrTimeoutMma = 2u,
    kErrTimeoutEpilogue = 4u,
    kErrTimeoutDrain = 8u,
    kErrNotBinary = 16u,     // the direct operand path met a byte other than 0 / 1
    kErrBadOperand = 32u,    // a direct operand tile did not start on a 16-byte boundary
    kErrBadCsr = 64u,        // a CSR row was out of bounds, out of range or not increasing
};

// -------------------------------------------------------------- pack kernel
struct PackJob {
    const uint8_t* X;    // m x n, leading dimension ldx
    int64_t m, n, ldx;
    uint8_t* P;          // K-block-major FP8 (or FP4) operand (this job's first row), or null
    uint32_t* Bp;        // bit-packed operand, rows_p x (ldp / 32) words, or null
    int32_t* v;          // column counts (zeroed before the launch), or null
    int64_t rows_p, ldp;
    int64_t cta_begin;   // first CTA of this job in a grouped launch
    int32_t gx;          // column blocks of 128 variables (rows_p / 128)
    int32_t tpc;         // 128-sample tiles walked by one CTA
    int32_t vec;         // 16-byte loads of X allowed
    int32_t fp4;         // P is the FP4 form (ldp a multiple of 256)
};
// Fill the launch fields (gx, tpc, vec) of a job; returns its CTA count.
// grouped: the job is one of many in a grouped launch (the most tiles per CTA).
int64_t pack_job_ctas(PackJob& j, bool grouped = false);
cudaError_t launch_pack(const PackJob& job, cudaStream_t s);
// Grouped pack: CTA c works for job cta_job[c] (device table), or, with a null
// table, for the last job whose cta_begin <= c (binary search).
cudaError_t launch_pack_grouped(const PackJob* jobs, int njobs, int64_t total_ctas,
                                const int32_t* cta_job, cudaStream_t s);
cudaError_t launch_validate(const uint8_t* X, int64_t m, int64_t n, int64_t ldx,
                            unsigned int* flag, cudaStream_t s);
// Column counts of X for the direct operand path (n % 16 == 0, X 16-byte
// aligned): v[j] += sum_r X[r][j] (v zeroed before); a byte other than 0 / 1
// sets kErrNotBinary in *err.
cudaError_t launch_colsum_direct(const uint8_t* X, int64_t m, int64_t n, int32_t* v,
                                 unsigned int* err, int sm_count, cudaStream_t s);

// ----------------------------------------------------- elementwise kernels
cudaError_t launch_zero_u32(void* p, int64_t words, cudaStream_t s);
cudaError_t launch_nlogn_table(double* T, int64_t len, cudaStream_t s);
cudaError_t launch_mi_vars(const int32_t* v, int64_t n, const MiParams& P, MiVar* out,
                           cudaStream_t s);
// Grouped: variables [var_begin[k], var_begin[k+1]) belong to dataset k, whose
// parameters are params[k]; v and out are indexed by the flat variable index.
cudaError_t launch_mi_vars_grouped(const int32_t* v, const int64_t* var_begin, int njobs,
                                   int64_t total, const MiParams* params, MiVar* out,
                                   cudaStream_t s);
// MI from counts.  slices > 1: the counts are the sums of `slices` partial
// count matrices slice_stride elements apart (the sample ranges of a split
// Gram), added exactly in int32.
cudaError_t launch_mi_from_counts(const int32_t* N11, int64_t ld_n11, const MiVar* va,
                                  const MiVar* vb, int64_t n1, int64_t n2, const MiParams& P,
                                  float* out, int64_t ld_out, cudaStream_t s, int slices = 1,
                                  int64_t slice_stride = 0);
// All pairs of one matrix (N11 symmetric): each unordered pair evaluated once,
// written to (i, j) and (j, i).  upper_only: only N11[a][b], a <= b, is read.
cudaError_t launch_mi_from_counts_sym(const int32_t* N11, int64_t ld_n11, const MiVar* vars,
                                      int64_t n, const MiParams& P, float* out, int64_t ld_out,
                                      cudaStream_t s, int upper_only = 0, int slices = 1,
                                      int64_t slice_stride = 0);
// out (rows x cols) = the sum of `slices` partial count matrices.
cudaError_t launch_slice_sum(const int32_t* N11, int64_t ld_n11, int slices, int64_t slice_stride,
                             int64_t rows, int64_t cols, int32_t* out, int64_t ld_out,
                             cudaStream_t s);

// ------------------------------------------------------------ sparse input
// Upper triangle (with the diagonal) of N11 from X in CSR by samples (N11
// zeroed before); a malformed row sets kErrBadCsr and is skipped.
cudaError_t launch_csr_pair_counts(const int64_t* row_ptr, const int32_t* col, int64_t m,
                                   int64_t n, int64_t nnz, int32_t* N11, unsigned int* err,
                                   int sm_count, cudaStream_t s);
// Dense uint8 0/1 form of a CSR matrix into X (m x n, zeroed before); a
// malformed row sets kErrBadCsr and writes nothing.
cudaError_t launch_csr_densify(const int64_t* row_ptr, const int32_t* col, int64_t m, int64_t n,
                               int64_t nnz, uint8_t* X, unsigned int* err, int sm_count,
                               cudaStream_t s);
cudaError_t launch_diag(const int32_t* N11, int64_t n, int32_t* v, cudaStream_t s);
cudaError_t launch_mirror_upper(int32_t* N11, int64_t n, cudaStream_t s);

// ---------------------------------------------------------- popcount Gram
struct PopcArgs {
    const uint32_t* Ba;  // rows x wpr
    const uint32_t* Bb;
    int64_t wpr;         // words per row (multiple of 4)
    int64_t n_a, n_b;
    int symmetric;       // Ba == Bb: compute j >= i tiles, write both halves
    const MiVar* va;     // per-variable terms (MI output only)
    const MiVar* vb;
    MiParams mp;
    float* out_f;        // MI output (or null)
    int32_t* out_c;      // counts output (or null)
    int64_t ld_out;
};
cudaError_t launch_popcount(const PopcArgs& a, cudaStream_t s);

// ------------------------------------------------------- tcgen05 FP8 Gram
constexpr int kTcBM = 128;     // A rows per tile = TMEM lanes
constexpr int kTcBNMax = 256;  // largest B rows per tile = accumulator columns
constexpr int kTcBK = 128;     // bytes per pipeline stage = one operand row
// Widest tile of an FP4 launch: the block-scaled MMA reads its scale factors
// from tensor memory, in the 16 columns each accumulator buffer leaves free.
constexpr int kTcBNFp4 = 240;

enum TcMode : int { kTcModeMI = 0, kTcModeCounts = 1, kTcModeCountsAdd = 2 };

// One dataset (or one cross pair) of a Gram launch.
struct GramJob {
    int64_t rowA, rowB;        // tensor-map row of (K block 0, variable 0) of A and B
    int64_t strideA, strideB;  // rows between consecutive K blocks (rows_p of A / B)
    int32_t k_begin;           // first K block accumulated by this launch
    int32_t k_blocks;          // K blocks (k_blocks * kb_samples <= 2^24: exact FP32 counts)
    int32_t n_a, n_b;          // valid variables of A and B
    int32_t symmetric;         // A == B: write (i, j) and (j, i) for j >= i only
    int32_t bn;                // B rows per tile: 64, 128 or 256 (240 for FP4)
    int32_t pad;
    const MiVar* va;           // per-variable terms (MI mode)
    const MiVar* vb;
    float* out_f;
    int32_t* out_c;            // counts modes: output; MI modes: counts of earlier sample
                               // chunks added to this launch's (or null)
    int64_t ld_out;
    float* out_t;              // MI mode, or null: also write (j, i) to out_t[j * ld_t + i]
    int64_t ld_t;
    MiParams mp;
};

// One 128 x bn output tile: job index, row block I, column block J.
// split = 0: the whole tile.  Otherwise either
// - a K share (bit 30 clear): the tile is one of `parts` units that each
//   accumulate a contiguous share of the job's K blocks:
//     split = ((slot + 1) << 8) | (part << 4) | parts   (2 <= parts <= 15)
//   Units 0 .. parts-2 store their exact int32 counts in the slot's part of
//   GramLaunch.part_counts and count themselves in on the slot's counters; unit
//   parts-1, listed after them, waits for them, adds their counts to its own
//   and runs the MI epilogue;
// - a column share (bit 30 set): split = kSplitCols | (part << 4) | parts; the
//   unit computes part `part` of `parts` of the tile's column window (below)
//   over all K blocks, with an MMA as wide as its share and no combining step.
// Either way the tail of a launch finishes in pieces of a tile, so fewer SMs
// idle.
struct GramTile {
    int32_t job, I, J, split;
};
constexpr int32_t kSplitCols = 1 << 30;
__host__ __device__ inline int32_t gram_split_code(int slot, int part, int parts) {
    return ((slot + 1) << 8) | (part << 4) | parts;
}
__host__ __device__ inline int32_t gram_cols_code(int part, int parts) {
    return kSplitCols | (part << 4) | parts;
}
__host__ __device__ inline bool split_is_k(int32_t split) {
    return split != 0 && (split & kSplitCols) == 0;
}

// MMA width of a tile: the job's tile width bn, or, for the ragged last column
// block, its valid columns rounded up to 32 (a valid N for M = 128 on one CTA
// and M = 256 on a pair), at most bn (240 = 15 x 16 is valid for both); the
// columns beyond are masked by every epilogue.
__host__ __device__ inline int gram_tile_n(int64_t n_b, int bn, int J) {
    const int64_t w = n_b - static_cast<int64_t>(J) * bn;
    if (w >= bn) return bn;
    const int n = static_cast<int>((w + 31) / 32 * 32);
    return n < 32 ? 32 : (n > bn ? bn : n);
}
// Columns [0, c0) of a tile of a symmetric job lie below the diagonal for all
// of its rows (tile rows start at tile_m I, its columns at bn J): its MMAs and
// B copies start at column c0, a multiple of 32.  0 for cross jobs and direct
// operands.
__host__ __device__ inline int gram_tile_c0(bool symmetric, int bn, int I, int J, int tile_m,
                                            bool direct) {
    if (!symmetric || direct) return 0;
    const int64_t skip = static_cast<int64_t>(I) * tile_m - static_cast<int64_t>(J) * bn;
    return skip > 0 ? static_cast<int>(skip & ~int64_t{31}) : 0;
}
// Column window [lo, hi) of the tile that a unit's MMAs compute: [c0, n) with
// n = gram_tile_n for a whole tile (or a K share); for a column share, piece
// `part` of `parts` of it, cut at multiples of 32 after c0.  Every piece is a
// non-empty multiple of 16 wide when hi - lo of the whole window is at least
// 32 * parts (the host splits no narrower tile).  Accumulator column a holds
// tile column lo + a.
struct ColWindow {
    int lo, hi;
};
__host__ __device__ inline ColWindow gram_tile_window(int64_t n_b, bool symmetric, int bn,
                                                      const GramTile& t, int tile_m,
                                                      bool direct) {
    const int c0 = gram_tile_c0(symmetric, bn, t.I, t.J, tile_m, direct);
    const int n = gram_tile_n(n_b, bn, t.J);
    ColWindow w{c0, n};
    if ((t.split & kSplitCols) != 0) {
        const int parts = t.split & 15, part = (t.split >> 4) & 15;
        const int width = n - c0;
        const int lo = part == 0 ? 0 : ((width * part / parts + 16) & ~31);
        const int hi = part + 1 == parts ? width : ((width * (part + 1) / parts + 16) & ~31);
        w.lo = c0 + lo;
        w.hi = c0 + hi;
    }
    return w;
}

struct GramLaunch {
    const GramJob* jobs;       // device table, or null: every tile uses job0
    GramJob job0;
    const GramTile* tiles;
    int num_tiles;
    int mode;                  // TcMode
    unsigned int* err;
    uint64_t timeout_ns;
    int debug_flags;
    // Operands: 0 = packed K-block-major FP8 buffer (box64/128/256, rowA/rowB
    // are buffer rows); 1 = direct: the caller's uint8 0/1 matrices read as
    // MN-major E4M3 through xa / xb (rowA/rowB are first variables, bn is 128
    // or 256, k_blocks count 128-sample steps).  A byte 1 is the E4M3
    // subnormal 2^-9, so the accumulator holds count * 2^-18 (exact below 2^24
    // samples) and the epilogue scales it back by 2^18.
    int direct;
    // 1: CTA-pair launch (clusters of 2, tcgen05 cta_group::2): tiles of 256 x
    // 256 (GramTile.I counts 256-row blocks; every job has bn = 256), packed
    // operands only, static tile order; the grid is an even number of CTAs.
    int pair;
    // Dynamic tile order: CTAs take the next tile from this counter (zero at
    // launch), so the tiles in flight are always a contiguous window of the
    // list.  Null: static round-robin (tile blockIdx.x + k * gridDim.x).
    unsigned int* counter;
    // Panel completion (or null): tile row block I belongs to panel
    // I / panel_blocks; every epilogue warp that finishes a tile adds 1 to
    // panel_done[panel], and the warp that brings it to panel_target[panel]
    // sets host_flags[panel] = 1 (mapped host memory, after a system fence),
    // so the host can copy the panel's rows while later panels compute.
    unsigned int* panel_done;
    const unsigned int* panel_target;
    unsigned int* host_flags;
    int panel_blocks;
    // MI mode: 1 if any job has the FP64 combine on (then the kernel that
    // contains it is launched; else the one without it)
    int fixup;
    // 1: the operands are the FP4 form (E2M1 nibbles, 256 samples per K
    // block) and the Gram runs the block-scaled FP4 MMA (kind::mxf4, every
    // scale factor 1.0): 0 and 1 are exact in E2M1, so the counts are the
    // same integers.  Packed operands only; every job has bn <= 240.
    int fp4;
    // Split tiles (GramTile.split != 0; FP32 MI epilogue only): per slot the
    // int32 counts of its first parts-1 units (gram_part_slot_ints() ints per
    // unit, laid out per CTA rank, epilogue warp, column and lane), and one
    // arrival counter per slot, CTA rank and epilogue warp (zero at launch).
    int32_t* part_counts;
    unsigned int* part_arrive;
};
// int32 entries of one part of a split tile in GramLaunch.part_counts (both
// CTAs of a pair, every epilogue warp, its columns, 32 lanes).
int64_t gram_part_slot_ints();
// Arrival counters of one split slot.
int gram_part_slot_counters();

// TMA descriptors of a K-block-major operand buffer of total_rows rows of 128
// bytes, for boxes of 64, 120, 128 and 256 rows (128-byte swizzle).
struct OperandMaps {
    CUtensorMap box64, box128, box256;
    CUtensorMap box120;   // a CTA's half of the B rows of a 240-wide FP4 pair tile
    // direct operands: X (A) and Y or X (B) themselves, row-major samples x
    // variables, boxes of 128 variables x 128 samples (128-byte swizzle)
    CUtensorMap xa, xb;
};
bool make_operand_maps(OperandMaps* maps, const uint8_t* P, int64_t total_rows);
// Direct-operand maps over X (m x n1) and Y (m x n2; Y = X for all pairs).
// Needs n1, n2 multiples of 16 and 16-byte aligned X, Y.
bool make_direct_maps(OperandMaps* maps, const uint8_t* X, int64_t m, int64_t n1,
                      const uint8_t* Y, int64_t n2);
// Tiles of one job in the kernel's order (groups of group_cols column blocks),
// bm rows (128; 256 for a CTA-pair launch) by bn columns.
int64_t gram_tile_count(int64_t n_a, int64_t n_b, int bn, bool symmetric, int bm = kTcBM);
void gram_tiles(int job, int64_t n_a, int64_t n_b, int bn, bool symmetric, int group_cols,
                GramTile* out, int bm = kTcBM);
cudaError_t launch_gram_tc(const OperandMaps& maps, const GramLaunch& L, int grid,
                           cudaStream_t s);
size_t gram_tc_smem_bytes();
cudaError_t gram_tc_prepare();   // set the kernels' shared-memory attribute (current device)
// CTA pairs (clusters of 2) of the pair kernel that fit on the device at once.
int gram_tc_pair_clusters();
// Epilogue warps per CTA of the kernel a launch of this mode runs (each
// signals a finished tile once in panel-completion counting).
int gram_tc_epilogue_warps(int mode, int fixup);

// Set the text gbmi_last_error_string() returns on this host thread.
void set_last_error(const char* msg);

}  // namespace gbmi
