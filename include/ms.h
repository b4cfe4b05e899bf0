/*
 * libms — maximal all-ones square detection on one GB300 (sm_103a).
 *
 * Problem (S. Bhandari, "An Efficient Frequency-Based Approach for Maximal
 * Square Detection in Binary Matrices", arXiv 2503.18974, Sec. 1): given an
 * m x n 0/1 matrix, find the largest k such that some k x k submatrix is all
 * ones.  The paper's Algorithm 1 (Sec. 3.2) returns the area k*k; this
 * library returns the side k and a deterministic witness: the bottom-right
 * corner (row, col) of the first k-square in row-major order of that corner,
 * which is where Algorithm 1 makes its last validation.  Optionally it writes
 * the map dp[i][j] = side of the largest all-ones square whose bottom-right
 * corner is (i, j) (the table of Eq. 1, Sec. 2.1).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - All matrix, result and dp pointers are DEVICE pointers owned by the
 *   caller (for example torch tensors).  The library never frees them.
 * - Every call is asynchronous on the given stream; results are valid once
 *   that stream has been synchronised.  The library performs no host
 *   synchronisation on the hot path.
 * - Host-detectable problems (null pointers, negative sizes, ld < row width,
 *   unsupported format or size) return an error immediately and launch
 *   nothing.  Problems found on the device (a bounded wait that gave up) are
 *   reported in ms_result.status of the affected matrix; the context stays
 *   usable.
 * - An empty matrix (m == 0 or n == 0) yields side 0 and row = col = -1, as
 *   Algorithm 1 returns 0 for an empty input (Sec. 3.2).
 * - No C++ exception crosses this interface.  A context is not thread-safe:
 *   use one per host thread (contexts may share a device).  Calls on one
 *   context share its device workspace: issue them on one stream, or order
 *   them, rather than on streams that run at the same time.
 * - Size limits: m <= 65000 rows and min(m, n) <= 32768; larger inputs
 *   return MS_ERR_UNSUPPORTED.  n itself is limited by m*n < 2^40 and
 *   n < 2^31 - 4096.
 */
#ifndef MS_H
#define MS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* ms_stream_t; /* a cudaStream_t; NULL = legacy default stream */
typedef struct ms_ctx ms_ctx;

typedef enum {
  MS_OK = 0,
  MS_ERR_INVALID = 1,     /* bad argument */
  MS_ERR_OOM = 2,         /* device allocation failed or workspace budget too small */
  MS_ERR_CUDA = 3,        /* a CUDA runtime call failed */
  MS_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up (reported per matrix) */
  MS_ERR_BUDGET = 5,      /* request does not fit the serving memory budget */
  MS_ERR_UNSUPPORTED = 6, /* valid but outside the supported sizes or layouts */
  MS_ERR_CANCELLED = 7    /* a served request withdrawn by ms_server_cancel */
} ms_status;

typedef enum {
  MS_U8 = 0,    /* one byte per cell, row-major, ld = row stride in bytes (ld >= n);
                   any nonzero byte is a one */
  MS_BITS32 = 1 /* 32 cells per uint32 word, row-major, ld = row stride in words
                   (ld >= ceil(n/32)); bit b (LSB = 0) of word w is column 32*w+b;
                   bits for columns >= n are ignored */
} ms_format;

typedef struct {
  const void* data; /* device pointer to cell (0,0) */
  int64_t m, n;     /* rows, columns (>= 0) */
  int64_t ld;       /* row stride in elements of the format (bytes or words) */
  int32_t fmt;      /* ms_format */
  int32_t reserved; /* must be 0 */
} ms_matrix;

typedef struct {
  int32_t side;   /* largest all-ones square side, 0 if none */
  int32_t row;    /* bottom-right corner of the first side-k square, row-major; -1 if side == 0 */
  int32_t col;
  int32_t status; /* MS_OK, or MS_ERR_TIMEOUT if a device-side wait gave up */
} ms_result;

/* Create a context on `device`.  workspace_budget_bytes caps the device
 * workspace the context may hold (0 = no cap).  The workspace (job table,
 * per-matrix witness keys, fix-up carries) grows on demand up to the cap and
 * is owned by the context.  Returns MS_ERR_OOM if the initial workspace
 * cannot be allocated. */
ms_status ms_create(ms_ctx** out, int device, size_t workspace_budget_bytes);

/* Largest square side and witness of one matrix (Sec. 3.2, Algorithm 1's
 * result as a side, with the witness described above).  `out_dev` is one
 * ms_result in device memory. */
ms_status ms_max_square(ms_ctx* ctx, const ms_matrix* in, ms_result* out_dev, ms_stream_t s);

/* As ms_max_square, and also writes dp[i*ld_dp + j] (int32, device memory,
 * ld_dp >= n) for every cell: the side of the largest all-ones square with
 * bottom-right corner (i, j) (Eq. 1, Sec. 2.1).  Works for MS_U8 and
 * MS_BITS32 input. */
ms_status ms_dp_map(ms_ctx* ctx, const ms_matrix* in, int32_t* dp_dev, int64_t ld_dp,
                    ms_result* out_dev, ms_stream_t s);

/* All largest squares (the paper's "all maximal squares", Sec. 3.4 and
 * Sec. 6): the bottom-right corner of every all-ones square of the largest
 * side K, i.e. every cell with dp == K.  `out_dev` receives the same ms_result
 * as ms_max_square; `count_dev` (one int64, device memory) the number of
 * such corners, which may exceed `capacity`; `corners_dev` (device memory,
 * room for `capacity` pairs; may be null when capacity is 0) the first
 * min(count, capacity) of them as int32 (row, col) pairs, in unspecified
 * order (the set itself is unique).  Nothing is listed when K == 0.
 * MS_U8 and MS_BITS32 input (always through the tile kernels).  Returns
 * MS_ERR_OOM if the fix-up bitplane scratch cannot be allocated. */
ms_status ms_all_max_squares(ms_ctx* ctx, const ms_matrix* in, int32_t* corners_dev,
                             int64_t capacity, int64_t* count_dev, ms_result* out_dev,
                             ms_stream_t s);

/* Side and witness for `count` matrices of possibly different shapes and
 * formats in one pass: the descriptors are read from HOST memory (ins_host),
 * the results go to outs_dev[0..count-1] in device memory.  Work from all
 * matrices is scheduled together: by default matrices up to about 900 000
 * cells are solved whole, one per block, in a persistent launch per size
 * class (five classes; their bitplanes in shared memory), and larger ones as
 * bitplane tiles of one persistent launch followed by the exact fix-up of
 * their flagged boxes (see ms_tuning.tile_kind).  The size classes run on
 * streams of the context's own, forked from `s` and joined back into it
 * before the call returns, so all of the call's work stays ordered on `s`
 * for the caller.  After a first call with a given set of
 * shapes, the same call (same pointers, shapes and count) may be captured in
 * a CUDA graph: it then allocates nothing and performs no host-device copy
 * other than stream-ordered ones issued inside the call. */
ms_status ms_batch(ms_ctx* ctx, const ms_matrix* ins_host, int32_t count, ms_result* outs_dev,
                   ms_stream_t s);

/* Free the context and its workspace (after synchronising its device work). */
ms_status ms_destroy(ms_ctx* ctx);

/* ms_max_square for callers that may not allocate device memory.  The paper
 * has no counterpart: this is a library convenience.  Some callers cannot
 * call cudaMalloc, for example plug-ins inside an application whose own pool
 * allocator owns all device memory, or latency-critical services that must
 * not allocate after start-up because an allocation can synchronise the
 * device.  Such callers cannot create an ms_ctx, so this call needs none and
 * allocates nothing: it computes the same result as ms_max_square into
 * out_dev (one ms_result in device memory), using a fixed scratch array of
 * about 0.53 MiB that lives in the library's device image on every GPU that
 * loads the library, until the process exits.
 * - Limits: m <= 8192 and n <= 8192 (MS_U8 or MS_BITS32); a larger matrix
 *   returns MS_ERR_UNSUPPORTED and launches nothing.
 * - The first call on each device looks up the scratch array's device
 *   address (cudaGetSymbolAddress, with that device current) and raises the
 *   kernels' shared-memory limits; make that first call before any stream
 *   capture on that device.  A call in a new context of the device (after
 *   cudaDeviceReset) repeats that set-up, so it too should come before any
 *   capture.
 * - Every call on a device shares the one scratch array and clears the parts
 *   that must start at zero.  Calls whose work overlaps on the GPU (other
 *   streams, other host threads) race on it and give wrong results: order
 *   them on one stream or synchronise between them. */
ms_status ms_max_square_noalloc(const ms_matrix* in, ms_result* out_dev, ms_stream_t s);

/* ---- 3-D volumes (the paper's future-work extension, Sec. 6) ---------------
 * A uint8 volume in device memory: cell (z, i, j) at
 * data[z*ld_slice + i*ld + j] for z < d, i < m, j < n; nonzero = 1. */
typedef struct {
  const void* data;
  int64_t d, m, n;
  int64_t ld;        /* bytes between rows, >= n */
  int64_t ld_slice;  /* bytes between slices, >= (m-1)*ld + n */
  int32_t fmt;       /* MS_U8 */
  int32_t reserved;  /* 0 */
} ms_volume;

typedef struct {
  int32_t side;               /* largest all-ones cube */
  int32_t slice, row, col;    /* its first corner in (z, i, j) order, -1s if side == 0 */
  int32_t status;
  int32_t reserved;
} ms_cube_result;

/* Largest all-ones cube of a volume and the first corner (in (z, i, j)
 * order) of such a cube: the 3-D analogue of Eq. 1, computed by bitplane
 * growth (cube corners of side a + s from those of side a, 0 < s <= a).
 * `out_dev` is one ms_cube_result in device memory.  The call decides each
 * growth step from the previous one and so waits for the stream between
 * steps (it returns after the result is written).  Scratch (two bit volumes,
 * d*m*ceil(n/32) words each) is allocated stream-ordered for the call.
 * Limits: d, m, n < 2^31 and d*m*n < 2^62. */
ms_status ms_max_cube(ms_ctx* ctx, const ms_volume* in, ms_cube_result* out_dev, ms_stream_t s);

/* Static, human-readable name of a status code. */
const char* ms_status_string(ms_status st);

/* ---- serving ----------------------------------------------------------------
 * A request loop for a stream of independent detection requests (a library
 * feature; the paper has no counterpart).  ms_server_submit hands the server
 * a matrix in HOST memory (keep it valid until the request completes; pinned
 * memory copies fastest) and returns at once.  A scheduler thread owned by
 * the server then:
 *   - admits requests in arrival order while their device input buffer fits
 *     the memory budget (a request that could never fit is refused with
 *     MS_ERR_BUDGET at submit); admitted buffers stay resident in a device
 *     arena until the request completes;
 *   - copies admitted inputs host->device on a copy stream;
 *   - whenever one of `streams` compute streams is free, launches every
 *     copied, not yet launched request (up to max_batch) as one ms_batch, so
 *     requests arriving while others run join the next batch and batches on
 *     different streams overlap (continuous batching);
 *   - on completion reads the results back, frees the buffers and stamps the
 *     request's times.
 * Results are identical to ms_max_square on the same matrix.  Host clock
 * times are seconds on a monotonic clock (ms_server_now). */
typedef struct ms_server ms_server;

typedef struct {
  size_t memory_budget_bytes; /* device memory for resident request inputs */
  int32_t streams;            /* concurrent batches (default 2) */
  int32_t max_batch;          /* requests per batch (default 512) */
  /* Test hook for failure handling, 0 in normal use: when k > 0, the k-th
   * batch the server launches (counting from 1) is treated as a launch that
   * failed on the host: its requests complete with MS_ERR_CUDA and side 0,
   * while every other request is served normally. */
  int32_t test_fail_batch;
  int32_t reserved[3];
} ms_server_config;

typedef struct {
  uint64_t id;
  ms_result result;
  double t_submit, t_admit, t_launch, t_done;
} ms_server_completion;

typedef struct {
  int64_t submitted, completed, batches;
  int64_t peak_bytes;      /* largest arena use seen (never above the budget) */
  int32_t peak_inflight;   /* largest number of batches on the device at once */
  int32_t reserved;
  double host_batch_s;     /* scheduler time spent planning and launching batches */
  double host_copy_s;      /* scheduler time spent issuing input copies */
} ms_server_stats;

ms_status ms_server_create(ms_server** out, int device, const ms_server_config* cfg);
ms_status ms_server_submit(ms_server* srv, const ms_matrix* host_matrix, double t_arrival,
                           uint64_t* id);  /* t_arrival < 0: now */
ms_status ms_server_poll(ms_server* srv, ms_server_completion* out, int32_t max, int32_t* n_out);
/* Withdraw a request that is still waiting for admission: it completes at
 * once (its completion is returned by ms_server_poll) with status
 * MS_ERR_CANCELLED and side 0, and its host matrix is no longer read.
 * Returns MS_OK, or MS_ERR_INVALID when the id is unknown or the request has
 * already been admitted (its input is being copied, computed or done: it
 * then completes normally). */
ms_status ms_server_cancel(ms_server* srv, uint64_t id);
ms_status ms_server_wait_all(ms_server* srv);
ms_status ms_server_stats_get(ms_server* srv, ms_server_stats* out);
ms_status ms_server_destroy(ms_server* srv);
double ms_server_now(void);

/* ---- tuning -------------------------------------------------------------
 * Launch parameters: `band_rows` = rows of a matrix that one tile counts
 * (at most 16384)
 * (each tile also re-reads a halo of 32 rows above and 32 columns to its
 * left), `packed_path` selects, for MS_BITS32 size-only work, the bitplane
 * erosion search (1) or the byte-style tile kernel on unpacked bits (0).
 * `lane_cols` = columns each lane of a warp owns in a tile (1, 2, 4, 8, 16
 * or 32; a tile is 32 * lane_cols columns wide).  `tile_kind` selects the
 * size-only tile pass of ms_max_square: 1 = the dp recurrence on two tiles
 * per warp (16-bit lanes), 2 = bitplane tiles (one tile of 1024 columns per
 * warp, 32 cells per word, doubling and threshold tests); automatically
 * bitplane tiles when the matrix fills the GPU's resident tile warps with
 * bands of 64 rows or more.  For ms_batch, tile_kind 0 solves every matrix
 * whose two bitplanes fit one block's shared memory (about 28 000 words of
 * 32 cells each) whole in one block and sends the larger ones through
 * bitplane tiles and the box fix-up, 1 runs every matrix as dp-recurrence
 * tile pairs and 2 every matrix as bitplane tiles; ms_autotune chooses among
 * the three for a batch.
 * 0 for band_rows, lane_cols or tile_kind = choose automatically from the
 * matrix size. */
typedef struct {
  int32_t band_rows;
  int32_t packed_path;
  /* Test hook for failure detection, 0 in normal use: when 1, the first strip
   * of the exact fix-up never publishes its carries, so the next strip's
   * bounded wait (about 1 s) runs out and the matrix's ms_result.status is
   * MS_ERR_TIMEOUT; later calls with the hook off are unaffected. */
  int32_t test_hold_carries;
  int32_t lane_cols;
  int32_t tile_kind;
  int32_t reserved[3];
} ms_tuning;

ms_status ms_set_tuning(ms_ctx* ctx, const ms_tuning* t);
ms_status ms_get_tuning(ms_ctx* ctx, ms_tuning* t);

/* Autotuner (a library feature; the paper has no counterpart).  Times the
 * work of ms_max_square (count == 1) or ms_batch (count > 1) on the given
 * matrices for each candidate tuning -- band heights 32..1024 and the
 * automatic choice, lane widths 2..32 and the automatic choice (single
 * matrices only), and for
 * MS_BITS32 size-only work both packed paths, for batches the three tile
 * kinds and for single matrices bitplane tiles forced (tile_kind 2) with
 * each band height -- in three interleaved rounds, each candidate keeping its
 * fastest; batches are timed as replays of a CUDA graph of the call on a
 * private stream (ordered after the caller's work), so that the host's
 * planning of a call does not weigh in.  A candidate must beat the best
 * earlier one by 2% to replace it (near-ties keep the automatic choice, which
 * comes first).  Keeps the chosen one and caches it in the context under the workload's class
 * (entry point, format mix, log2 of the cell count, log2 of the matrix
 * count).  Later calls of that class with ms_tuning.band_rows == 0 and
 * lane_cols == 0 use the cached choice.  `outs_dev` receives results (count entries) and is
 * scratch.  Blocks the calling thread until the timing runs finish; must
 * not be called during stream capture, nor between ms_profile_start and
 * ms_profile_stop (the profile would time the candidates' launches too).  The chosen tuning is written to
 * `chosen` if non-null. */
ms_status ms_autotune(ms_ctx* ctx, const ms_matrix* ins_host, int32_t count, ms_result* outs_dev,
                      ms_stream_t s, ms_tuning* chosen);

/* ---- kernel timing --------------------------------------------------------
 * Between ms_profile_start and ms_profile_stop the context records a CUDA
 * event pair around every kernel it launches (on the caller's stream, so the
 * events time exactly those launches).  ms_profile_stop synchronises the
 * recorded events and returns per-kind launch counts and summed durations.
 * At most max_launches launches are timed; later ones run untimed and are
 * only counted.  The events add no device work. */
typedef struct {
  int64_t tile_launches;   /* tile-pass kernels (the bandwidth-bound hot kernel) */
  double tile_ms;
  int64_t fixup_launches;  /* exact fix-up / result kernels */
  double fixup_ms;
  int64_t other_launches;  /* packed-search kernels and helpers */
  double other_ms;
  int64_t untimed_launches;
  int64_t bit_tile_launches;  /* of the tile-pass kernels: bitplane tiles */
} ms_profile;

ms_status ms_profile_start(ms_ctx* ctx, int32_t max_launches);
ms_status ms_profile_stop(ms_ctx* ctx, ms_profile* out);

#ifdef __cplusplus
}
#endif
#endif /* MS_H */
