// Internal declarations shared by the kernels and the C ABI of libgbmi.so.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "mi_device.cuh"

namespace gbmi {

// ------------------------------------------------------------ packed layouts
//
// P  (tensor-core operand): one row per variable, one byte per sample, FP8
//    E4M3 bit patterns 0x00 (0) and 0x38 (1.0).  rows_p = n rounded up to 256,
//    ldp = m rounded up to 128 bytes; padding rows and columns are zero.
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

// Device error word bits (set by kernels whose bounded waits gave up).
enum : uint32_t {
    kErrTimeoutLoad = 1u,
    kErrTimeoutMma = 2u,
    kErrTimeoutEpilogue = 4u,
    kErrTimeoutDrain = 8u,
};

// -------------------------------------------------------------- pack kernel
struct PackArgs {
    const uint8_t* X;
    int64_t m, n, ldx;
    uint8_t* P;        // may be null
    int64_t rows_p, ldp;
    uint32_t* Bp;      // may be null; rows_p x (ldp / 32) words
    int32_t* v;        // must be zeroed before the launch; may be null
};
cudaError_t launch_pack(const PackArgs& a, cudaStream_t s);
cudaError_t launch_validate(const uint8_t* X, int64_t m, int64_t n, int64_t ldx,
                            unsigned int* flag, cudaStream_t s);

// ----------------------------------------------------- elementwise kernels
cudaError_t launch_zero_u32(void* p, int64_t words, cudaStream_t s);
cudaError_t launch_nlogn_table(double* T, int64_t len, cudaStream_t s);
cudaError_t launch_mi_vars(const int32_t* v, int64_t n, const MiParams& P, MiVar* out,
                           cudaStream_t s);
cudaError_t launch_mi_from_counts(const int32_t* N11, int64_t ld_n11, const MiVar* va,
                                  const MiVar* vb, int64_t n1, int64_t n2, const MiParams& P,
                                  float* out, int64_t ld_out, cudaStream_t s);

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
constexpr int kTcBN = 256;     // B rows per tile = accumulator columns
constexpr int kTcBK = 128;     // K bytes per pipeline stage (one 128-byte swizzle row)

enum TcMode : int { kTcModeMI = 0, kTcModeCounts = 1, kTcModeCountsAdd = 2 };

struct TcArgs {
    const int2* tiles;   // (I, J) per tile: A rows [128 I, 128 I + 128), B rows [256 J, ...)
    int num_tiles;
    int k_begin;         // first K block (units of 128 samples)
    int k_blocks;        // K blocks to accumulate (k_blocks * 128 <= 2^24: exact FP32 counts)
    int64_t n_a, n_b;    // valid variables of A and B
    int symmetric;       // A == B: write (i, j) and (j, i) for j >= i only
    int mode;            // TcMode
    int vec_store;       // output rows are 16-byte aligned (ld % 4 == 0, aligned base)
    const MiVar* va;     // per-variable terms (MI mode)
    const MiVar* vb;
    MiParams mp;
    float* out_f;
    int32_t* out_c;
    int64_t ld_out;
    unsigned int* err;
    uint64_t timeout_ns;
    int debug_flags;
};
// Encode the TMA descriptor of a packed operand P viewed as box_rows x 128-byte
// tiles (128-byte swizzle).
bool make_operand_tmap(CUtensorMap* tm, const uint8_t* P, int64_t rows_p, int64_t ldp,
                       int box_rows);
cudaError_t launch_gram_tc(const CUtensorMap& tmA, const CUtensorMap& tmB, const TcArgs& a,
                           int grid, cudaStream_t s);
size_t gram_tc_smem_bytes();
cudaError_t gram_tc_prepare();   // set the kernel's shared-memory attribute (current device)

// Set the text gbmi_last_error_string() returns on this host thread.
void set_last_error(const char* msg);

}  // namespace gbmi
