/*
 * gbmi — all-pairs mutual information of binary variables on GB300 (sm_103a).
 *
 * C ABI of libgbmi.so.  The method is the matrix formulation of arXiv
 * 2411.19702 ("Fast Mutual Information Computation for Large Binary
 * Datasets"):
 *   - one co-occurrence Gram N11 = X^T X (Sec. 2 step 2, G11),
 *   - the other three contingency counts derived from the column counts v and
 *     the number of samples m (Sec. 3.1, Eq. 6 and Eq. 7: N01 = v_j - N11,
 *     N10 = v_i - N11, N00 = m - v_i - v_j + N11),
 *   - marginals from the diagonal / column counts (Sec. 2 step 3),
 *   - MI per pair in bits from the four cells (Eq. 1 written out as Eq. 2),
 *     with the limit 0*log 0 = 0 in place of the paper's unspecified epsilon.
 *
 * Conventions shared by every call:
 *   - X (and Y) are caller-owned DEVICE pointers on the current CUDA device:
 *     uint8, row-major, m rows (samples) by n columns (variables), leading
 *     dimension = number of columns, no alignment requirement.  An entry is
 *     read as 1 when its byte is non-zero (binary data, Sec. 2 step 1).
 *   - Outputs are caller-owned device pointers, row-major, fully overwritten.
 *   - m = samples, n = variables (the paper calls the data matrix n x m with the
 *     letters swapped; this header always uses m for samples).
 *   - Limits: 1 <= m <= 2^31 - 1, 1 <= n; outputs must not overlap inputs.
 *   - Work is enqueued on the library's current stream (gbmi_set_stream) and
 *     the calls return without waiting for it.  The returned status covers
 *     argument checks, workspace allocation and launch errors.  A device-side
 *     wait that times out (every wait inside the kernels is bounded) sets a
 *     device error word that gbmi_sync() reports as GBMI_ERR_TIMEOUT.
 *   - The library owns a grow-only device workspace (packed operands, column
 *     counts, the n*log2(n) table); gbmi_shutdown() frees it.  Calls from
 *     several host threads must be serialised by the caller.
 */
#ifndef GBMI_H_
#define GBMI_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GBMI_OK = 0,
    GBMI_ERR_ARG = 1,          /* bad argument (null pointer, size out of range, overlap) */
    GBMI_ERR_OOM = 2,          /* workspace allocation failed */
    GBMI_ERR_CUDA = 3,         /* a CUDA runtime/driver call or kernel launch failed */
    GBMI_ERR_TIMEOUT = 4,      /* a bounded device-side wait gave up (reported by gbmi_sync) */
    GBMI_ERR_NOT_BINARY = 5,   /* validation found an entry other than 0 or 1 */
    GBMI_ERR_UNSUPPORTED = 6   /* no GPU of compute capability 10.3 (sm_103a) */
} gbmi_status;

/* Computation paths.  AUTO picks the fused tensor-core path, or the popcount
 * path for tiny shapes.  The tensor-core Gram multiplies 0/1 operands packed
 * as FP4 E2M1 (GBMI_OPT_FP4, the default) or FP8 E4M3 and counts exactly in FP32 up to
 * 2^24 samples per launch; beyond that it runs in sample chunks of 2^24,
 * accumulating int32 counts in its workspace (n1 * n2 * 4 bytes), and the
 * fused path evaluates MI in the last chunk's epilogue. */
typedef enum {
    GBMI_PATH_AUTO = 0,
    GBMI_PATH_FUSED = 1,     /* tcgen05 FP4/FP8 Gram with the MI epilogue fused (one pass)  */
    GBMI_PATH_PLAIN = 2,     /* tcgen05 FP4/FP8 Gram -> int32 N11 in HBM, then elementwise MI */
    GBMI_PATH_POPCOUNT = 3   /* bit-packed AND + popcount Gram (exactness cross-check)      */
} gbmi_path;

/* Options for gbmi_set_option.  Their defaults can also be set in the
 * environment when the library loads: GBMI_FIXUP, GBMI_TILE_N, GBMI_PAIR,
 * GBMI_DIRECT, GBMI_FP4, GBMI_TIMEOUT_NS, GBMI_GROUP_COLS, GBMI_MAX_CTAS,
 * GBMI_TAIL_SPLIT, GBMI_TAIL_COLS (out-of-range
 * values are ignored).  GBMI_LOG=1 also writes every error text to stderr. */
typedef enum {
    GBMI_OPT_FIXUP = 1,          /* 1: FP64 n*log2(n) combine for pairs whose FP32 MI < 1e-4 (default 0) */
    GBMI_OPT_TIMEOUT_NS = 2,     /* bound of every device-side wait, ns (default 2e9)            */
    GBMI_OPT_DEBUG_FLAGS = 3,    /* test hooks; 1 = the fused kernel's loader issues no copies,
                                    so its consumer's bounded wait must run out; 2 = every new
                                    workspace allocation fails with GBMI_ERR_OOM (default 0)     */
    GBMI_OPT_GROUP_COLS = 4,     /* tile-order group width in 256-column blocks (default 8)      */
    GBMI_OPT_MAX_CTAS = 5,       /* cap on persistent CTAs, 0 = one per SM (default 0)           */
    GBMI_OPT_PROFILE = 6,        /* 1: time every kernel launch with CUDA events (default 0)     */
    GBMI_OPT_TILE_N = 7,         /* tensor-core tile width 64/128/256 (256 runs 240 wide with FP4
                                    operands); 0 = tuner / model (default)                        */
    GBMI_OPT_DIRECT = 8,         /* 1: tensor-core paths read X / Y directly, without the pack pass
                                    or its packed copy, when n (and n2) are multiples of 16 and X, Y
                                    are 16-byte aligned; bytes must then be 0 / 1 (others are
                                    reported as GBMI_ERR_NOT_BINARY by gbmi_sync).  Saves m*n bytes
                                    of device memory but measured slower (default 0)          */
    GBMI_OPT_PAIR = 9,           /* 1: the single-call and out-of-core tensor-core paths run the
                                    Gram on CTA pairs (clusters of two SMs sharing one tcgen05
                                    cta_group::2 MMA tile of 256 x 240 with FP4 operands, 256 x 256
                                    with FP8; each SM stages half of A and half of B) whenever
                                    that keeps at least as many SMs busy as
                                    single-CTA tiles would; 2: always; 0: single-CTA tiles only
                                    (default 1)                                                  */
    GBMI_OPT_CSR_PATH = 10,      /* CSR input (gbmi_*_csr): 0 = by a cost model (default), 1 = pair
                                    enumeration, 2 = dense 0/1 matrix + tensor-core path          */
    GBMI_OPT_SPLIT_K = 11,       /* a single-CTA tensor-core Gram with fewer tiles than SMs (few
                                    variables, many samples) is split over sample ranges, each
                                    part's exact int32 counts in its own workspace slice, summed by
                                    the MI (or counts) kernel: 0 = automatic (default), 1 = never,
                                    2 = whenever there are samples enough                        */
    GBMI_OPT_FP4 = 12,           /* 1: the tensor-core paths (single calls, cross, host buffers,
                                    out-of-core, CSR densified, batches and servers created while
                                    it is set; mi_all_pairs_noalloc always uses FP4, and
                                    GBMI_OPT_DIRECT reads X itself as FP8)
                                    pack X as FP4 (E2M1 0 / 1, two samples per byte) and run the
                                    block-scaled FP4 MMA (tcgen05 kind::mxf4, every scale factor
                                    1.0; tiles at most 240 wide): the same exact counts from half
                                    the operand bytes, about 1.7x the FP8 Gram's rate; 0: FP8
                                    operands (default 1)                                          */
    GBMI_OPT_TAIL_SPLIT = 13,    /* fused MI launch: its last (tiles mod slots) + slots tiles run
                                    as units of half the samples each; the second unit of a tile
                                    adds the first's exact int32 counts before the MI, so the
                                    launch ends in half-length pieces instead of a partial wave of
                                    whole tiles: 0 = off (default; at 10^5 x 10^4 the shorter tail
                                    was offset by the longer last epilogue), 1 = on, k in 2..15 =
                                    every tile in k parts (tests).  Results are bit-identical     */
    GBMI_OPT_TAIL_COLS = 14      /* tensor-core launches of one dataset or cross pair: the tiles of
                                    the last partial wave (tiles mod concurrent tile slots) run as
                                    2 to 4 column shares each, every share an MMA as wide as its
                                    columns over all samples (no combining step), the count chosen
                                    so the shares fill the fewest share-length waves: 1 = automatic
                                    (default), 0 = off, k in 2..4 = every tile in k shares (tests).
                                    Ignored while GBMI_OPT_TAIL_SPLIT is on.  Results are
                                    bit-identical                                                */
} gbmi_option;

/* ---------------------------------------------------------------- core calls */

/* MI of every pair of columns of X: out[i*n + j] = MI(X_i; X_j) in bits, FP32,
 * n x n.  The matrix is symmetric (out[i*n+j] and out[j*n+i] are the same
 * bits) and its diagonal is the entropy of each column.
 * Defined by Eq. 1 over all column pairs (Sec. 1, Sec. 2 steps 1-5); computed
 * with one Gram (Sec. 3.1, Eq. 4-7).  Accuracy: counts are exact; MI is within
 * 1e-6 absolute of the exact value. */
gbmi_status mi_all_pairs(const uint8_t* X, int64_t m, int64_t n, float* out);

/* MI between the columns of two datasets over the same m samples:
 * out[i*n2 + j] = MI(X_i; Y_j), n1 x n2, FP32 bits.  X is m x n1, Y is m x n2.
 * Same method with N11 = X^T Y and the column counts of each input. */
gbmi_status mi_cross(const uint8_t* X, const uint8_t* Y, int64_t m, int64_t n1, int64_t n2,
                     float* out);

/* One shard of mi_all_pairs on the fused path, for splitting one problem over
 * several GPUs (one call per GPU, each with its own X copy and out buffer):
 * the upper-triangle tile list of the Gram (the single call's list and order)
 * is cut into num_shards contiguous shares of equal tile count, and this call
 * computes share `shard` (0 <= shard < num_shards), writing out[i*n + j] and
 * out[j*n + i] for the pairs of its tiles only; other entries are untouched.
 * The shards' writes together are exactly mi_all_pairs's output.  Pack and
 * per-variable terms are computed in full by every shard (the Gram dominates).
 * Same limits and errors as mi_all_pairs, plus GBMI_ERR_ARG for a shard out
 * of range.  The paper has no counterpart: its method runs on one device. */
gbmi_status gbmi_mi_all_pairs_shard(const uint8_t* X, int64_t m, int64_t n, float* out,
                                    int shard, int num_shards);

/* The same two calls with an explicit path (gbmi_path). */
gbmi_status gbmi_mi_all_pairs_path(const uint8_t* X, int64_t m, int64_t n, float* out, int path);
gbmi_status gbmi_mi_cross_path(const uint8_t* X, const uint8_t* Y, int64_t m, int64_t n1,
                               int64_t n2, float* out, int path);

/* Host-buffer variants: X, Y and out are HOST pointers (pinned or pageable).
 * The call copies the inputs to the device, computes on the current stream,
 * copies the result back and returns only when out is filled. */
gbmi_status mi_all_pairs_host(const uint8_t* X, int64_t m, int64_t n, float* out);
gbmi_status mi_cross_host(const uint8_t* X, const uint8_t* Y, int64_t m, int64_t n1, int64_t n2,
                          float* out);

/* No-allocation variant of mi_all_pairs (the paper has no counterpart: this
 * is a service to callers of the library, not part of the method).
 *
 * For callers that must not allocate device memory: a host framework that
 * owns the device memory through its own pool, a latency-critical loop that
 * cannot afford cudaFree's device-wide synchronisation, a process under a
 * hard memory cap.  The call performs no cudaMalloc/cudaFree and calls no
 * allocating library routine.  Its scratch (packed operand, column counts,
 * per-variable terms, tile list, error word) is one 64 MiB array inside the
 * library, held by every GPU that loads the library until the process exits.
 *
 * X (m x n uint8 0/1) and out (n x n FP32) are caller-owned device pointers,
 * as for mi_all_pairs; the result is the fused tensor-core path's with the
 * FP32 epilogue and FP4 operands (GBMI_OPT_FIXUP and GBMI_OPT_FP4 are
 * ignored).  Limits: 1 <= m <= 2^24, and n_pad(n) * m_pad(m) / 2 bytes of
 * packed operand (n rounded up to 256, m to 256) plus about 36 n bytes must
 * fit in 64 MiB; larger problems return
 * GBMI_ERR_ARG with the required size in gbmi_last_error_string().
 *
 * The first call on each device looks up the array's device address (with
 * that device current); make that first call before any stream capture.  The
 * call runs on the library's current stream and returns after its work has
 * finished (GBMI_ERR_TIMEOUT if a bounded device-side wait gave up).  Every
 * call uses the same array: calls whose work overlaps on the GPU (from other
 * host threads or streams) race and must not be issued. */
gbmi_status mi_all_pairs_noalloc(const uint8_t* X, int64_t m, int64_t n, float* out);

/* ------------------------------------------------------ out-of-core output */

/* Out-of-core output (the blockwise computation the paper names as future
 * work, Sec. 5): for n where the n x n FP32 matrix does not fit in device
 * memory (n^2 * 4 bytes; n ~ 260,000 fills a GB300), or a cross problem with
 * a very large n2.  X (and Y) are device pointers as for mi_all_pairs /
 * mi_cross and must fit on the device together with their packed copy; the
 * result goes to host_out, HOST memory, row-major n x n (or n1 x n2), which
 * should be page-locked (cudaHostAlloc / cudaHostRegister) for the copies to
 * overlap the computation.  The matrix is computed in row panels of
 * panel_rows variables (0: automatic, within 4 GiB of device staging and at
 * least about eight panels) by the fused tensor-core path into two device
 * staging slots; each panel is copied to the host on a second stream while
 * the next one computes.  For all pairs, panel [i0, i1) computes rows
 * [i0, i1) x columns [i0, n) and writes the mirror of that block as well, so
 * every off-diagonal pair is evaluated once.  Values are bit-identical to
 * mi_all_pairs / mi_cross.  Synchronous: returns when host_out is complete.
 * Needs m <= 2^24 (each panel is one exact Gram launch). */
gbmi_status gbmi_mi_all_pairs_to_host(const uint8_t* X, int64_t m, int64_t n, float* host_out,
                                      int64_t panel_rows);
gbmi_status gbmi_mi_cross_to_host(const uint8_t* X, const uint8_t* Y, int64_t m, int64_t n1,
                                  int64_t n2, float* host_out, int64_t panel_rows);

/* ------------------------------------------------------------ sparse input */

/* Sparse input (the paper's sparse-matrix variant, Opt-SS, Sec. 4.2.3): X
 * given by samples in CSR form, device pointers: row_ptr[m + 1] (int64, row r
 * holds col_idx[row_ptr[r] .. row_ptr[r + 1])), col_idx[nnz] (int32) = the
 * variables that are 1 in that sample, strictly increasing.  A sample with k
 * ones adds 1 to N11[a][b] for each of its k (k + 1) / 2 pairs a <= b (atomic
 * adds; the diagonal gives the column counts), so the work follows
 * sum_r k_r^2 / 2 instead of m * n^2 / 2: it beats the dense tensor-core path
 * only for very sparse data.  Elsewhere (by a cost model of the two, from m, n
 * and nnz; GBMI_OPT_CSR_PATH forces either) the call writes the dense 0/1
 * matrix into its workspace (m * n bytes) and runs the tensor-core path on it.
 * gbmi_mi_all_pairs_csr writes the n x n FP32 MI matrix (out, as
 * mi_all_pairs; values identical to the dense paths, either way);
 * gbmi_counts_all_pairs_csr writes the symmetric n x n int32 counts.  A
 * malformed row (bounds outside [0, nnz], an index outside [0, n), indices not
 * strictly increasing) is skipped and reported as GBMI_ERR_ARG by gbmi_sync.
 * The library keeps an n x n int32 count matrix in its workspace for the MI
 * call.  Asynchronous on the library's stream. */
gbmi_status gbmi_mi_all_pairs_csr(const int64_t* row_ptr, const int32_t* col_idx, int64_t m,
                                  int64_t n, int64_t nnz, float* out);
gbmi_status gbmi_counts_all_pairs_csr(const int64_t* row_ptr, const int32_t* col_idx, int64_t m,
                                      int64_t n, int64_t nnz, int32_t* n11);

/* ------------------------------------------------------ counts and pieces */

/* Co-occurrence counts N11 = X^T X (G11 of Sec. 2 step 2) as int32, n x n,
 * both triangles written.  path = GBMI_PATH_PLAIN (tensor cores, FP4 or FP8 operands,
 * FP32 accumulation in exact chunks) or GBMI_PATH_POPCOUNT (bit-packed AND +
 * popcount).  Both must agree bit for bit. */
gbmi_status gbmi_counts_all_pairs(const uint8_t* X, int64_t m, int64_t n, int32_t* n11, int path);

/* N11 = X^T Y, n1 x n2 int32, with the same path choice. */
gbmi_status gbmi_counts_cross(const uint8_t* X, const uint8_t* Y, int64_t m, int64_t n1,
                              int64_t n2, int32_t* n11, int path);

/* Column counts v_j = number of ones in column j (Sec. 3.1, Term 2: v = D^T 1),
 * int32, length n. */
gbmi_status gbmi_column_counts(const uint8_t* X, int64_t m, int64_t n, int32_t* v);

/* Elementwise MI from counts (the second half of the plain path): for every
 * (i, j), n11 = N11[i*n2 + j], derive N10, N01, N00 by Eq. 6-7 from va[i],
 * vb[j] and m, and write MI in bits to out[i*n2 + j].  All pointers device. */
gbmi_status gbmi_mi_from_counts(const int32_t* N11, const int32_t* va, const int32_t* vb,
                                int64_t m, int64_t n1, int64_t n2, float* out);

/* Check that every entry of X is 0 or 1.  Synchronous; returns GBMI_OK or
 * GBMI_ERR_NOT_BINARY. */
gbmi_status gbmi_validate_binary(const uint8_t* X, int64_t m, int64_t n);

/* ------------------------------------------------------------ management */

/* Set the CUDA stream (a cudaStream_t, NULL = legacy default stream) used by
 * all subsequent calls from any host thread. */
gbmi_status gbmi_set_stream(void* stream);
void* gbmi_get_stream(void);

/* Set an option (gbmi_option) for subsequent calls. */
gbmi_status gbmi_set_option(int option, int64_t value);

/* Wait for the current stream, then report and clear the device error word:
 * GBMI_ERR_TIMEOUT if a bounded wait in a kernel gave up, GBMI_ERR_CUDA on an
 * asynchronous CUDA error, else GBMI_OK. */
gbmi_status gbmi_sync(void);

/* Human-readable text of the last error on this host thread ("" if none). */
const char* gbmi_last_error_string(void);

/* Number of kernels this library has launched since load (a monotone count). */
uint64_t gbmi_launch_count(void);

/* Free the workspace (waits for the device first). */
gbmi_status gbmi_shutdown(void);

/* ----------------------------------------------------------------- batches
 *
 * Many independent problems (datasets of uneven m and n) in one grouped run
 * (no counterpart in the paper, which treats one dataset at a time).  Each
 * job is the paper's all-pairs problem on its own X (Y == NULL) or the cross
 * problem between X and Y over the same samples.  A plan packs every job's
 * operands into one workspace and runs, on the library's current stream, a
 * CUDA graph of four kernels: column counts zeroing, one grouped pack, one
 * grouped per-variable-terms pass and ONE persistent tensor-core Gram launch
 * whose tile list holds the tiles of all jobs (largest tiles first; each
 * job's tile width from the tuner table).  Results are bit-identical to the
 * single calls (the counts are exact and the per-pair arithmetic is the same).
 * Limits per job: 1 <= m <= 2^24 (fused path), 1 <= n, n2.  Device pointers
 * X, Y, out as in mi_all_pairs / mi_cross.
 *
 * gbmi_batch_create allocates the plan's workspace, uploads its tables and
 * captures the graph (call it outside stream capture).  gbmi_batch_run
 * launches the graph (asynchronous).  gbmi_batch_set_io points the same plan
 * at new X / Y / out buffers of the same shapes (tables only; the graph is
 * reused).  gbmi_batch_destroy waits for the device and frees the plan.
 * gbmi_mi_batch is create + run + wait + destroy.  Device-side timeouts are
 * reported by gbmi_sync(). */
typedef struct {
    const uint8_t* X;   /* m x n samples x variables, uint8 0/1 */
    const uint8_t* Y;   /* m x n2 for cross MI, or NULL for all pairs of X */
    int64_t m;
    int64_t n;
    int64_t n2;         /* columns of Y; ignored when Y is NULL */
    float* out;         /* n x n (all pairs) or n x n2 (cross), FP32 bits */
} gbmi_job;

typedef struct gbmi_batch gbmi_batch;

gbmi_status gbmi_batch_create(const gbmi_job* jobs, int k, gbmi_batch** plan);
gbmi_status gbmi_batch_run(gbmi_batch* plan);
gbmi_status gbmi_batch_set_io(gbmi_batch* plan, const gbmi_job* jobs, int k);
gbmi_status gbmi_batch_destroy(gbmi_batch* plan);
gbmi_status gbmi_mi_batch(const gbmi_job* jobs, int k);
/* Number of tensor-core tiles in the plan's grouped launch. */
int64_t gbmi_batch_tiles(const gbmi_batch* plan);

/* ----------------------------------------------------------------- serving
 *
 * A request loop with continuous batching (no counterpart in the paper).
 * The server owns one device arena of budget_bytes from which it takes, per
 * dataset, the packed operand (FP4 or FP8 as GBMI_OPT_FP4 was when the server
 * was created), the column counts and the per-variable terms (resident until
 * the dataset is removed), and per request its output.
 * A worker thread admits queued requests in arrival order whenever their
 * memory fits and fewer than max_batch requests are waiting for the GPU,
 * merges them into one grouped launch (pack of the datasets not yet resident,
 * per-variable terms, one persistent tensor-core Gram over the tiles of all
 * admitted requests) and keeps up to two such batches in flight on two
 * streams, so requests that arrive while others run start without waiting for
 * them to finish.  Results are the same as the single calls (mi_all_pairs /
 * mi_cross with the FP32 epilogue).
 *
 * gbmi_server_add_dataset registers X (device pointer, m x n uint8 0/1, must
 * stay valid until the dataset has been packed, i.e. until the first request
 * on it completes) and returns its id.  gbmi_server_submit queues the
 * all-pairs problem of dataset a (b = -1) or the cross problem between a and
 * b (same m) and returns a ticket.  gbmi_server_wait blocks until the ticket
 * is done (or timeout_ms, 0 = forever), then gives the device pointer of the
 * FP32 result (n_a x n_a or n_a x n_b, valid until gbmi_server_release) and
 * the latency from submit to completion in ms.  gbmi_server_stats fills
 * stats[0..7] = completed requests, p50 ms, p99 ms, mean ms, max ms, pairs
 * per second over the server's busy span, batches launched, mean requests
 * per batch.  The server reads X on its own streams: its contents must be
 * complete on the device when the dataset is added.  Memory is returned by
 * gbmi_server_release (outputs) and gbmi_server_remove_dataset (datasets,
 * once no queued or running request reads them); a request that does not fit
 * waits in the queue until enough is returned.  Limits: m <= 2^24 per
 * dataset; a request whose memory could not fit even an empty arena fails
 * with GBMI_ERR_OOM at submit.  gbmi_server_destroy lets the running batches
 * finish, fails the queued requests, and frees the arena (result pointers
 * become invalid). */
typedef struct gbmi_server gbmi_server;

gbmi_status gbmi_server_create(int64_t budget_bytes, int max_batch, gbmi_server** srv);
gbmi_status gbmi_server_add_dataset(gbmi_server* srv, const uint8_t* X, int64_t m, int64_t n,
                                    int64_t* id);
gbmi_status gbmi_server_remove_dataset(gbmi_server* srv, int64_t id);
gbmi_status gbmi_server_submit(gbmi_server* srv, int64_t a, int64_t b, int64_t* ticket);
gbmi_status gbmi_server_wait(gbmi_server* srv, int64_t ticket, int64_t timeout_ms,
                             const float** out, double* latency_ms);
gbmi_status gbmi_server_release(gbmi_server* srv, int64_t ticket);
/* Cancel a request that is still queued (GBMI_ERR_ARG if it is running or
 * done): gbmi_server_wait then returns GBMI_ERR_ARG for it, and it must still
 * be released. */
gbmi_status gbmi_server_cancel(gbmi_server* srv, int64_t ticket);
/* Requests queued and running, datasets registered, and arena bytes in use
 * (packed datasets, per-variable terms, unreleased outputs); any pointer may
 * be NULL. */
gbmi_status gbmi_server_state(gbmi_server* srv, int64_t* queued, int64_t* running,
                              int64_t* datasets, int64_t* bytes_in_use);
gbmi_status gbmi_server_stats(gbmi_server* srv, double* stats);
gbmi_status gbmi_server_destroy(gbmi_server* srv);

/* Tile-width table of the autotuner (no counterpart in the paper).  The
 * tensor-core Gram works on tiles of 128 x tile_n variable pairs; narrow tiles
 * waste less padding on small n, wide tiles stream fewer operand bytes per
 * pair.  gbmi_tuner_set records the best width measured for problems in the
 * bucket of (m, n) (floor(log2 m), floor(2 log2 n)); gbmi_tile_n returns the
 * width an all-pairs call of that shape would use (GBMI_OPT_TILE_N, else the
 * table, else an operand-traffic cost model). */
gbmi_status gbmi_tuner_set(int64_t m, int64_t n, int tile_n);
gbmi_status gbmi_tuner_clear(void);
int gbmi_tile_n(int64_t m, int64_t n);
/* Kernel choice of the bucket of (m, n), measured by the autotuner: 1 = CTA
 * pairs (256-row tiles on clusters of two SMs), 0 = single-CTA tiles of the
 * bucket's tile width, -1 = the built-in rule (pairs when a single call fills
 * the GPU with them; in a batch, when both sides span >= 768 variables).
 * Applies to single calls, batches and servers created afterwards, unless
 * GBMI_OPT_PAIR forces a kernel.  gbmi_tuner_pair returns the current choice
 * (-1 for an untuned bucket).  Errors: GBMI_ERR_ARG. */
gbmi_status gbmi_tuner_set_pair(int64_t m, int64_t n, int pair);
int gbmi_tuner_pair(int64_t m, int64_t n);

/* Sample split of the (m, n) bucket's tensor-core Gram when it has fewer
 * tiles than the GPU runs at once (few variables, many samples): 0 = the
 * built-in cost model (default), 1 = never split, S in 2..128 = cut the
 * samples into S ranges whose exact int32 counts are summed by the MI (or
 * counts) kernel, where S keeps every range at least 2048 samples, at most
 * 2^24, and the ranges' counts within 2 GB (otherwise the model decides).
 * GBMI_OPT_SPLIT_K set to 1 or 2 overrides it.  Applies to single calls.
 * gbmi_tuner_split returns the current value (0 for an untuned bucket).
 * Errors: GBMI_ERR_ARG. */
gbmi_status gbmi_tuner_set_split(int64_t m, int64_t n, int parts);
int gbmi_tuner_split(int64_t m, int64_t n);

/* The tail plan a tensor-core launch of `tiles` tiles on `units` concurrent
 * tile slots would use under the current GBMI_OPT_TAIL_COLS: returns how many
 * tiles at the end of its list run as column shares (0: none) and stores the
 * shares per tile in *parts (if not null).  Automatic mode splits the last
 * partial wave (tiles mod units) into the 2-4 shares that fill the fewest
 * share-length waves, and nothing when that would not end before a whole-tile
 * wave.  A planning query: it launches nothing and needs no GPU. */
int gbmi_tail_cols_plan(int tiles, int units, int* parts);

/* Per-kernel launch profile (enable with GBMI_OPT_PROFILE).  Each kernel
 * launch is bracketed by CUDA events on the library's stream;
 * gbmi_profile_entries() waits for the recorded launches, folds them into
 * per-kernel totals and returns the number of kernel names k; entry k has a
 * name, a total device time in ms and a launch count.  gbmi_profile_reset()
 * clears the totals.  The returned name stays valid until the next reset. */
int gbmi_profile_entries(void);
const char* gbmi_profile_name(int k);
double gbmi_profile_ms(int k);
int64_t gbmi_profile_launches(int k);
gbmi_status gbmi_profile_reset(void);

/* Tensor-core throughput of the Gram kernel's MMA forms, for its roofline
 * (the paper has no counterpart; Sec. 3.2 puts the method's cost in the one
 * Gram, so this is the rate that bounds it).  Every SM (every CTA pair when
 * pair != 0) holds A and B tiles of random 0/1 values in shared memory and one
 * thread issues `mmas` back-to-back tcgen05.mma of M x n x K into tensor
 * memory: M = 128 (256 for a pair), K = 64 samples for fp4 != 0 (block-scaled
 * E2M1, kind::mxf4, every scale factor 1.0) or 32 for FP8 E4M3
 * (kind::f8f6f4), the instruction and shared-memory descriptors of the Gram
 * kernel.  No global memory is read in the loop.  n: multiple of 16 in
 * [16, 256]; mmas in [1, 2^32] (rounded up to a multiple of 16).  Synchronous
 * on the library stream: *flops_per_s = 2 M n K x MMAs issued / elapsed time
 * of the launch (CUDA events), *ms (may be null) = that time.  Errors:
 * GBMI_ERR_ARG, GBMI_ERR_CUDA, GBMI_ERR_TIMEOUT (a bounded wait gave up). */
gbmi_status gbmi_mma_peak(int fp4, int pair, int n, int64_t mmas, double* flops_per_s,
                          double* ms);

/* Library version, major*10000 + minor*100 + patch. */
int gbmi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GBMI_H_ */
