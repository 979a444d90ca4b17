/*
 * gbscan.h — C ABI of the GB300 (sm_103a) prefix-sum library.
 *
 * The operation (Zhang, Wang, Ross, "Parallel Prefix Sum with SIMD", ADMS'20,
 * Section 1): given [a_0, ..., a_{n-1}] and the operator +, the inclusive scan
 * is y_k = a_0 + ... + a_k; the exclusive scan is y_0 = 0, y_k = a_0 + ... +
 * a_{k-1}.  The paper's algorithms are multithreaded two-pass CPU schemes
 * (Section 2.1, Figure 1) and in-register SIMD scans (Section 3, Listing 1);
 * this library computes the same result on the GPU with four algorithms a
 * caller can pick (gbscan_algo): a single-pass chained scan with decoupled
 * look-back; the two-pass reduce-then-scan (the paper's "Accumulate + Prefix
 * Sum", Figure 1b); the partitioned scan (Section 2.2, Figure 2) with the
 * GPU's L2 as the cache, whose second pass over each chunk reads it from L2;
 * and, for inputs whose tiles all fit the SMs at once, the resident scan: the
 * same two passes with the whole array held in shared memory, one launch.
 * GBSCAN_ALGO_AUTO takes the resident scan where it fits and the single-pass
 * scan above that (see the plain scans).
 *
 * Conventions for every entry point:
 *  - Pointers named in/out/offsets/grad_* and the workspace are DEVICE
 *    pointers owned by the caller (scan_inclusive_i32_host takes host
 *    arrays).  The library allocates no device memory.
 *  - All work is enqueued on `stream` and is asynchronous; nothing blocks
 *    except scan_get_device_status().
 *  - `out == in` (in place, the paper's default, Section 2) is allowed; any
 *    other overlap of in and out returns GBSCAN_ERR_INVALID_ARG.
 *  - Integer arithmetic wraps (two's complement); float results are rounded
 *    sums whose rounding order depends on timing (float addition is not
 *    associative, Section 1.1), so they may differ in the last bits between runs.
 *  - n == 0 (or rows*cols == 0, or an empty segment list) is a no-op.
 *  - Argument errors return a status synchronously and launch nothing.
 *    Launch failures return GBSCAN_ERR_CUDA.  Errors found on the device (a
 *    bounded wait that ran out, malformed segment offsets) are recorded in the
 *    workspace and returned by scan_get_device_status().
 *  - Full speed needs `in` and `out` 16-byte aligned; other alignments are
 *    handled by a slower path (lanes instead of bulk copies).
 *  - The library never aborts, traps or prints.
 *
 * Workspace: query its size with gbscan_workspace_size(), allocate it on the
 * device, and zero it ONCE (gbscan_workspace_init or any memset to 0) before
 * first use.  It may then be reused by any number of calls issued on one
 * stream, including inside a captured CUDA graph: the kernels leave it ready
 * for the next call.  Calls that overlap in time must use separate workspaces.
 */
#ifndef GBSCAN_H
#define GBSCAN_H

#include <stddef.h>
#include <stdint.h>

#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GBSCAN_ABI_VERSION 2

typedef enum {
    GBSCAN_OK = 0,
    GBSCAN_ERR_INVALID_ARG = 1, /* null pointer, negative size, bad overlap, bad offsets */
    GBSCAN_ERR_ALIGNMENT = 2,   /* pointer not aligned to its element size */
    GBSCAN_ERR_WORKSPACE = 3,   /* workspace missing, misaligned or too small */
    GBSCAN_ERR_CUDA = 4,        /* a CUDA runtime call or kernel launch failed */
    GBSCAN_ERR_TIMEOUT = 5,     /* device: a bounded wait on another tile ran out */
    GBSCAN_ERR_UNSUPPORTED = 6  /* size or option outside what is built */
} gbscan_status;

typedef enum {
    GBSCAN_ALGO_AUTO = 0,         /* by size and type; see the plain scans below */
    GBSCAN_ALGO_SINGLE_PASS = 1,  /* chained scan with decoupled look-back */
    GBSCAN_ALGO_TWO_PASS = 2,     /* reduce tiles, scan the tile sums, scan with offsets */
    GBSCAN_ALGO_PARTITIONED = 3,  /* cache-friendly partitioned two-pass (Section 2.2):
                                     per L2-sized chunk, reduce then scan from L2, one launch */
    GBSCAN_ALGO_RESIDENT = 4      /* small inputs, one launch: every tile held in shared
                                     memory from its reduce until the sums of the tiles
                                     before it are written and its scan can finish
                                     (Figure 1b with Section 2.2's partitioning) */
} gbscan_algo;

typedef enum {
    GBSCAN_F32_PLAIN = 0,       /* all sums in fp32 */
    GBSCAN_F32_COMPENSATED = 1  /* per-thread and carried prefixes as (hi, lo) TwoSum pairs */
} gbscan_f32_mode;

typedef enum {
    GBSCAN_I32 = 0,
    GBSCAN_I64 = 1,
    GBSCAN_F32 = 2,
    GBSCAN_F64 = 3,
    GBSCAN_U32 = 4  /* sums share the int32 kernels (the same bits); max / min compare unsigned */
} gbscan_dtype;

typedef enum {
    GBSCAN_KIND_SCAN = 0,           /* one array: single-pass, two-pass or partitioned */
    GBSCAN_KIND_SEGMENTED = 1,      /* CSR segments, one persistent launch */
    GBSCAN_KIND_ROWS = 2,           /* rows x cols, along the last dim, forward or reverse */
    GBSCAN_KIND_SCAN_MAX = 3,       /* one array, running maximum (int32, int64, uint32, fp32) */
    GBSCAN_KIND_SCAN_MIN = 4,       /* one array, running minimum (int32, int64, uint32, fp32) */
    GBSCAN_KIND_COMPACT = 5,        /* stream compaction (int32, fp32) */
    GBSCAN_KIND_SEGMENTED_MAX = 6,  /* CSR segments, running maximum (int32, fp32) */
    GBSCAN_KIND_SEGMENTED_MIN = 7   /* CSR segments, running minimum (int32, fp32) */
} gbscan_kind;

/* Bytes of workspace needed by any call of `kind` on `dtype` with n elements
 * (and num_segments segments for GBSCAN_KIND_SEGMENTED), for every algorithm
 * and every variant.  Writes *bytes; returns GBSCAN_ERR_INVALID_ARG for a null
 * `bytes` or negative sizes and GBSCAN_ERR_UNSUPPORTED beyond the largest
 * supported size (2^31 tiles, 2^31 - 1 segments). */
gbscan_status gbscan_workspace_size(gbscan_dtype dtype, gbscan_kind kind, int64_t n,
                                    int64_t num_segments, size_t* bytes);

/* Zero a workspace on `stream` (cudaMemsetAsync).  Needed once per allocation. */
gbscan_status gbscan_workspace_init(void* ws, size_t ws_bytes, cudaStream_t stream);

/*
 * Plain scans of one contiguous array (Section 1 definition).
 *   in, out   : device arrays of n elements (out == in allowed).
 *   n         : element count, >= 0.
 *   ws        : zeroed workspace of ws_bytes >= gbscan_workspace_size(dtype, SCAN, n, 0).
 *   algo      : GBSCAN_ALGO_SINGLE_PASS (one launch), TWO_PASS (three launches:
 *               tile reduce, one-block scan of the tile sums, scan with offsets),
 *               PARTITIONED (one launch: the array is cut into chunks of about 8 MiB,
 *               environment variable GBSCAN_CHUNK_BYTES; each chunk is reduced tile by
 *               tile, its tile sums are scanned, and it is scanned a second time while
 *               still in L2, overlapped with the reduction of the chunk four ahead,
 *               GBSCAN_CHUNK_LAG), RESIDENT (one cooperative launch, one block per tile
 *               of 5120 4-byte or 2560 8-byte elements, every block resident at once:
 *               each block keeps its tile in shared memory, writes the tile's sum, and
 *               adds the sums of the tiles before it once they are written; for
 *               inputs of at most SMs x blocks-per-SM tiles, gbscan_resident_max_n;
 *               larger inputs return GBSCAN_ERR_UNSUPPORTED), or AUTO (RESIDENT where it fits;
 *               above that SINGLE_PASS, except fp64: TWO_PASS; the fastest choices
 *               measured on GB300).  SINGLE_PASS and PARTITIONED (and
 *               stream compaction) prefetch the input into L2 about 12 MiB ahead of their
 *               tile copies (environment variable GBSCAN_PREFETCH_BYTES; 1 turns it off).
 *   variant   : launch shape (threads, items per thread, pipeline stages), 0 = default;
 *               see gbscan_num_variants / gbscan_variant_info.  RESIDENT has one shape:
 *               the variant is checked but does not change the launch.
 *   mode      : (f32 only) plain fp32 or compensated two-sum carries.
 */
gbscan_status scan_inclusive_i32(const int32_t* in, int32_t* out, int64_t n, void* ws,
                                 size_t ws_bytes, gbscan_algo algo, int variant,
                                 cudaStream_t stream);
gbscan_status scan_exclusive_i32(const int32_t* in, int32_t* out, int64_t n, void* ws,
                                 size_t ws_bytes, gbscan_algo algo, int variant,
                                 cudaStream_t stream);
gbscan_status scan_inclusive_i64(const int64_t* in, int64_t* out, int64_t n, void* ws,
                                 size_t ws_bytes, gbscan_algo algo, int variant,
                                 cudaStream_t stream);
gbscan_status scan_exclusive_i64(const int64_t* in, int64_t* out, int64_t n, void* ws,
                                 size_t ws_bytes, gbscan_algo algo, int variant,
                                 cudaStream_t stream);
gbscan_status scan_inclusive_f32(const float* in, float* out, int64_t n, gbscan_f32_mode mode,
                                 void* ws, size_t ws_bytes, gbscan_algo algo, int variant,
                                 cudaStream_t stream);
gbscan_status scan_exclusive_f32(const float* in, float* out, int64_t n, gbscan_f32_mode mode,
                                 void* ws, size_t ws_bytes, gbscan_algo algo, int variant,
                                 cudaStream_t stream);
/* uint32 sums: modulo 2^32, the bits of the int32 sums of the same bits (they
 * run the int32 kernels); workspace and variants as for GBSCAN_I32. */
gbscan_status scan_inclusive_u32(const uint32_t* in, uint32_t* out, int64_t n, void* ws,
                                 size_t ws_bytes, gbscan_algo algo, int variant,
                                 cudaStream_t stream);
gbscan_status scan_exclusive_u32(const uint32_t* in, uint32_t* out, int64_t n, void* ws,
                                 size_t ws_bytes, gbscan_algo algo, int variant,
                                 cudaStream_t stream);
/* fp64 scans: used by the autograd layer for double-precision gradient checks. */
gbscan_status scan_inclusive_f64(const double* in, double* out, int64_t n, void* ws,
                                 size_t ws_bytes, gbscan_algo algo, int variant,
                                 cudaStream_t stream);
gbscan_status scan_exclusive_f64(const double* in, double* out, int64_t n, void* ws,
                                 size_t ws_bytes, gbscan_algo algo, int variant,
                                 cudaStream_t stream);

/*
 * Batched segmented scan (the Section 1 definition restarted at every segment
 * start; segments are not in the paper).  One persistent launch over the flat
 * array plus one small launch that locates each tile's first segment.
 *   offsets      : device int64 CSR array of num_segments + 1 entries, monotone,
 *                  offsets[0] = 0, offsets[num_segments] = n (the total length).
 *                  Empty segments are allowed.  Malformed offsets are reported by
 *                  scan_get_device_status() as GBSCAN_ERR_INVALID_ARG.
 *   n            : total length (offsets[num_segments], which the caller knows).
 *   exclusive    : 0 inclusive, 1 exclusive per segment (each segment starts at 0).
 * No host synchronisation: the call can be captured in a CUDA graph.
 */
gbscan_status scan_segmented_batched_i32(const int32_t* in, int32_t* out, int64_t n,
                                         const int64_t* offsets, int64_t num_segments,
                                         int exclusive, void* ws, size_t ws_bytes, int variant,
                                         cudaStream_t stream);
gbscan_status scan_segmented_batched_f32(const float* in, float* out, int64_t n,
                                         const int64_t* offsets, int64_t num_segments,
                                         int exclusive, void* ws, size_t ws_bytes, int variant,
                                         cudaStream_t stream);

/*
 * Row-wise scan along the last dimension of a row-major rows x cols array
 * (torch.cumsum(x, -1)): y[r, i] = sum_{k <= i} x[r, k] (exclusive: k < i).
 */
gbscan_status scan_rows_f32(const float* in, float* out, int64_t rows, int64_t cols,
                            int exclusive, void* ws, size_t ws_bytes, int variant,
                            cudaStream_t stream);
gbscan_status scan_rows_f64(const double* in, double* out, int64_t rows, int64_t cols,
                            int exclusive, void* ws, size_t ws_bytes, int variant,
                            cudaStream_t stream);

/*
 * Gradient of the row-wise scan: the reverse (suffix) scan of the incoming
 * gradient along the last dim.  The forward y_k = sum_{i<=k} x_i has Jacobian
 * dy_k/dx_i = [i <= k], so dx_i = sum_{k >= i} g_k; for the exclusive forward,
 * dx_i = sum_{k > i} g_k.  grad_out and grad_in are rows x cols, row-major;
 * grad_in == grad_out is allowed.
 */
gbscan_status scan_backward_f32(const float* grad_out, float* grad_in, int64_t rows, int64_t cols,
                                int exclusive, void* ws, size_t ws_bytes, int variant,
                                cudaStream_t stream);
gbscan_status scan_backward_f64(const double* grad_out, double* grad_in, int64_t rows,
                                int64_t cols, int exclusive, void* ws, size_t ws_bytes,
                                int variant, cudaStream_t stream);

/* Synchronises `stream`, returns the first device-side error recorded in the
 * workspace since the last call (GBSCAN_OK if none) and clears it. */
gbscan_status scan_get_device_status(void* ws, cudaStream_t stream);

/*
 * Scans under another associative operator (Section 1 defines the prefix sum;
 * the same scan exists for any associative operator, and + is the one the
 * paper measures):
 *   GBSCAN_OP_SUM  y_k = a_0 + ... + a_k    (the plain scans above)
 *   GBSCAN_OP_MAX  y_k = max(a_0, ..., a_k) (running maximum)
 *   GBSCAN_OP_MIN  y_k = min(a_0, ..., a_k) (running minimum)
 * Exclusive scans start from the operator's identity (0 for SUM; INT32_MIN,
 * INT64_MIN, 0 or -inf for MAX; INT32_MAX, INT64_MAX, UINT32_MAX or +inf for
 * MIN, for int32, int64, uint32, fp32).  uint32 MAX / MIN compare unsigned.
 * fp32 MAX / MIN follow IEEE maxNum / minNum (a NaN operand yields the other
 * operand).  Arguments, workspace (gbscan_workspace_size with
 * GBSCAN_KIND_SCAN or the operator's kind), algorithms and errors as for the
 * plain scans; variants per gbscan_num_variants(dtype, GBSCAN_KIND_SCAN_MAX /
 * _MIN).  An unknown op returns GBSCAN_ERR_INVALID_ARG.
 */
typedef enum { GBSCAN_OP_SUM = 0, GBSCAN_OP_MAX = 1, GBSCAN_OP_MIN = 2 } gbscan_op;

gbscan_status scan_op_i32(const int32_t* in, int32_t* out, int64_t n, gbscan_op op,
                          int exclusive, void* ws, size_t ws_bytes, gbscan_algo algo,
                          int variant, cudaStream_t stream);
gbscan_status scan_op_f32(const float* in, float* out, int64_t n, gbscan_op op, int exclusive,
                          void* ws, size_t ws_bytes, gbscan_algo algo, int variant,
                          cudaStream_t stream);
gbscan_status scan_op_i64(const int64_t* in, int64_t* out, int64_t n, gbscan_op op,
                          int exclusive, void* ws, size_t ws_bytes, gbscan_algo algo,
                          int variant, cudaStream_t stream);
gbscan_status scan_op_u32(const uint32_t* in, uint32_t* out, int64_t n, gbscan_op op,
                          int exclusive, void* ws, size_t ws_bytes, gbscan_algo algo,
                          int variant, cudaStream_t stream);

/*
 * Batched segmented scans under an operator: GBSCAN_OP_SUM is
 * scan_segmented_batched_*; MAX and MIN give each segment's running maximum
 * or minimum, an exclusive scan starting every segment from the operator's
 * identity.  Arguments and errors as for scan_segmented_batched_*; workspace
 * gbscan_workspace_size(dtype, GBSCAN_KIND_SEGMENTED_MAX / _MIN, n,
 * num_segments); variants per that kind.  An unknown op returns
 * GBSCAN_ERR_INVALID_ARG.
 */
gbscan_status scan_segmented_op_i32(const int32_t* in, int32_t* out, int64_t n,
                                    const int64_t* offsets, int64_t num_segments, gbscan_op op,
                                    int exclusive, void* ws, size_t ws_bytes, int variant,
                                    cudaStream_t stream);
gbscan_status scan_segmented_op_f32(const float* in, float* out, int64_t n,
                                    const int64_t* offsets, int64_t num_segments, gbscan_op op,
                                    int exclusive, void* ws, size_t ws_bytes, int variant,
                                    cudaStream_t stream);

/*
 * Stream compaction, an application of the exclusive scan (Section 1 names
 * stream compaction among the uses of prefix sums): the exclusive scan of the
 * keep flags (1 where flags[i] != 0) gives each kept element its output
 * position, so
 *   out[j] = in[i_j] for the kept indices i_0 < i_1 < ..., j < *count,
 *   *count = the number of kept elements (a DEVICE int64, written on `stream`).
 * One launch: the scan of the flags fused with the gather (no flag prefix
 * reaches memory); variants 0-2 run the partitioned scan, 3 the single-pass
 * chained scan with decoupled look-back (the faster below about 2^26
 * elements; the tuned choice by size takes it there).  in/out: device arrays of n 4-byte elements
 * (copied bit for bit), not overlapping; flags: n device bytes; out must hold
 * *count elements (n at most).  Workspace: gbscan_workspace_size(dtype,
 * GBSCAN_KIND_COMPACT, n, 0).  n = 0 writes *count = 0.  Null pointers,
 * overlap of in and out, or a count pointer not 8-byte aligned return
 * GBSCAN_ERR_INVALID_ARG / GBSCAN_ERR_ALIGNMENT; device errors as for scans.
 */
gbscan_status compact_i32(const int32_t* in, const uint8_t* flags, int32_t* out, int64_t n,
                          int64_t* count, void* ws, size_t ws_bytes, int variant,
                          cudaStream_t stream);
gbscan_status compact_f32(const float* in, const uint8_t* flags, float* out, int64_t n,
                          int64_t* count, void* ws, size_t ws_bytes, int variant,
                          cudaStream_t stream);

/*
 * End to end from host memory: the inclusive int32 scan (Section 1) of a HOST
 * array into a HOST array, through a device staging buffer.
 *   h_in, h_out : host arrays of n elements (pinned memory lets the copies run
 *                 asynchronously and overlap; pageable memory works, slower).
 *   d_buf       : device buffer of d_elems int32 elements, 16-byte aligned.  With
 *                 d_elems >= n the whole array stays resident; otherwise it is a
 *                 ring of at least two slots (d_elems >= 8192 required).
 *   ws          : workspace for a plain int32 scan of one piece (at most 16 Mi
 *                 elements: gbscan_workspace_size(I32, SCAN, min(n, 16Mi), 0)).
 * The array moves in pieces of up to 16 Mi elements: the upload of piece k
 * (on `stream`), its in-place partitioned scan continuing from the pieces
 * before it (the previous piece's last prefix, kept in the workspace header),
 * and its download run on three streams, so uploads, scans and downloads of
 * different pieces overlap.  Asynchronous: `stream` reaches the end of the
 * last download; h_out is valid after synchronising it.  Errors: null
 * pointers, negative sizes or a too small ring return GBSCAN_ERR_INVALID_ARG;
 * an unaligned d_buf GBSCAN_ERR_ALIGNMENT; a failed CUDA call GBSCAN_ERR_CUDA.
 */
gbscan_status scan_inclusive_i32_host(const int32_t* h_in, int32_t* h_out, int64_t n,
                                      int32_t* d_buf, int64_t d_elems, void* ws, size_t ws_bytes,
                                      cudaStream_t stream);

/* Test and tuning hooks, stored in the workspace header (not global state):
 *   spin_limit_us : bound of every wait on another tile, 0 = default (200 ms).
 *   drop_tile     : a tile index whose status is never published (-1 = none):
 *                   its successor's wait runs out and records GBSCAN_ERR_TIMEOUT.
 *   delay_ns_max  : before each status publication, sleep a pseudo-random
 *                   0..delay_ns_max ns to reorder tile completion (0 = off). */
gbscan_status gbscan_set_debug(void* ws, size_t ws_bytes, uint32_t spin_limit_us,
                               int64_t drop_tile, uint32_t delay_ns_max, cudaStream_t stream);

/* Launch shapes: number of variants for a (dtype, kind), and the shape of one:
 * threads per block, items per thread, pipeline stages, tile elements. */
int gbscan_num_variants(gbscan_dtype dtype, gbscan_kind kind);
gbscan_status gbscan_variant_info(gbscan_dtype dtype, gbscan_kind kind, int variant,
                                  int* threads, int* items, int* stages, int* tile);

/* The largest n that GBSCAN_ALGO_RESIDENT takes for a plain scan of `dtype` on
 * the current device: the blocks that fit the device at once (SMs x blocks per
 * SM, from the CUDA occupancy calculator) times the tile (5120 4-byte or 2560
 * 8-byte elements).  kind: GBSCAN_KIND_SCAN (for GBSCAN_F32, `mode` picks
 * plain or compensated sums; other types ignore it), GBSCAN_KIND_SCAN_MAX or
 * GBSCAN_KIND_SCAN_MIN.  Writes *n.  Returns GBSCAN_ERR_INVALID_ARG for a null
 * `n`, an unknown dtype or mode, GBSCAN_ERR_UNSUPPORTED for other kinds or
 * combinations without a resident scan, GBSCAN_ERR_CUDA if CUDA cannot report
 * the device or the occupancy. */
gbscan_status gbscan_resident_max_n(gbscan_dtype dtype, gbscan_kind kind, gbscan_f32_mode mode,
                                    int64_t* n);

/* Device-to-device copy of `bytes` bytes with a vectorised copy kernel: the
 * bandwidth reference the scan is measured against. */
gbscan_status gbscan_copy(const void* src, void* dst, size_t bytes, cudaStream_t stream);

const char* gbscan_status_string(gbscan_status status);
int gbscan_abi_version(void);

/*
 * Inclusive int32 scan that allocates nothing and takes no workspace (the
 * paper has no counterpart: this is a calling convention, not part of the
 * method).  It is for callers that cannot allocate device memory: code that
 * runs where cudaMalloc is forbidden or unavailable, such as inside a
 * fixed-budget memory pool that must not grow, an allocator callback or a
 * memory-accounting hook, or an embedding that hands out only the input and
 * output buffers.
 *
 * It runs the same single-pass kernel as scan_inclusive_i32 (default launch
 * shape), with its scratch (the tile status records) in a library-owned
 * static device array of GBSCAN_NOALLOC_SCRATCH_BYTES (8 MiB), which every GPU
 * that loads the library holds until the process exits.  That bounds n at
 * GBSCAN_NOALLOC_MAX_N elements; larger n returns GBSCAN_ERR_UNSUPPORTED and
 * launches nothing.
 *   in, out : device arrays of n int32 (out == in allowed), owned by the caller.
 *   n       : 0 <= n <= GBSCAN_NOALLOC_MAX_N; n == 0 scans nothing.
 * The first call on a device (n == 0 is enough: a warm-up call) looks up the
 * array's device address (cudaGetSymbolAddress) with that device current, and
 * may make CUDA load the library's device code and the array at that moment,
 * which allocates device memory.  So make one call per device at
 * initialisation, outside any no-allocation context and before any stream
 * capture.  Argument errors (null, misaligned or partly overlapping buffers)
 * return before the array is touched.  Every call clears the array's launch
 * counters and error
 * word (cudaMemsetAsync on `stream`), so device-side errors (bounded waits
 * that ran out) are not reported by this entry point.  All calls share the one
 * array: calls whose executions overlap on the GPU (other streams, or other
 * host threads) race and give wrong results; issue them on one stream, or
 * order them.  No cudaMalloc, cudaFree or allocating library call is made.
 */
#define GBSCAN_NOALLOC_SCRATCH_BYTES (8u << 20)
#define GBSCAN_NOALLOC_MAX_N ((int64_t)1340000000)
gbscan_status scan_inclusive_i32_noalloc(const int32_t* in, int32_t* out, int64_t n,
                                         cudaStream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* GBSCAN_H */
