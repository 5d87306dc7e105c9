/*
 * sell.h -- C ABI of the SELL-C-sigma library for NVIDIA GB300 (sm_103a).
 *
 * The library converts a sparse matrix from CRS (compressed row storage) into
 * the SELL-C-sigma format of Kreutzer, Hager, Wellein, Fehske and Bishop,
 * "A unified sparse matrix data format for efficient general sparse
 * matrix-vector multiply on modern processors with wide SIMD units"
 * (arXiv:1307.6209, SIAM J. Sci. Comput.), and multiplies it with vectors and
 * blocks of vectors on the GPU.  Every step runs in the library's own CUDA
 * kernels.
 *
 * Conventions that hold for every call:
 *   - Every call returns a sell_status; nothing is thrown across the ABI.
 *     sell_last_error() gives a message for the calling thread's last failure.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream).  sell_spmv, sell_spmmv and sell_batch_run are asynchronous on
 *     it.  sell_build synchronises the stream: it reads two sizes back and
 *     returns once the format is complete on the device;
 *     sell_export and sell_free synchronise the device.
 *   - Device pointers belong to the current CUDA device; a handle must be used
 *     on the device that was current when it was built.
 *   - Index types: row offsets int64, column indices int32 (Sec. 5: four-byte
 *     indices), chunk offsets int64.
 *   - The library allocates its device memory through sell_set_allocator's
 *     callbacks.  Default: stream-ordered allocation (cudaMallocFromPoolAsync
 *     / cudaFreeAsync) from one library-owned memory pool per device, which
 *     keeps freed memory for reuse; sell_free returns the pool's unused
 *     memory to the device.
 *   - Concurrency: a handle's products share its long-row scratch, so
 *     products of one handle must not overlap on the GPU (issue them on one
 *     stream, or order the streams), except that SELL_SPMV_HOST_IO products
 *     are ordered by the library, and sell_spmmv_noalloc / batch plans use
 *     scratch of their own.  Calls that change a handle (sell_set_launch,
 *     sell_free) must not race with other calls on it from other host
 *     threads.  A server (sell_server_*) may be used from any thread.
 */
#ifndef SELL_H
#define SELL_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define SELL_API __attribute__((visibility("default")))
#else
#define SELL_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- types */

/* Value types.  The paper stores binary64 only (Sec. 5); binary32 and
 * bfloat16 storage with binary32 accumulation are this library's extension. */
enum { SELL_F64 = 0, SELL_F32 = 1, SELL_BF16 = 2 };

typedef enum {
    SELL_OK = 0,
    SELL_EINVAL = 1,       /* bad argument or malformed CRS input */
    SELL_ENOMEM = 2,       /* an allocation failed; nothing leaked */
    SELL_ECUDA = 3,        /* a CUDA runtime call failed (message kept) */
    SELL_EBOUNDS = 4,      /* reserved for kernel-side bounds checks; no call
                              of this version returns it (sizes and indices
                              are validated on the host before a launch) */
    SELL_ETIMEOUT = 5,     /* a bounded device-side wait gave up */
    SELL_EUNSUPPORTED = 6  /* valid request this build does not support */
} sell_status;

/* CRS input (Sec. 3.1, Listing "crs"): row i holds entries rpt[i]..rpt[i+1]-1
 * of col[] and val[].  The matrix is borrowed for the duration of sell_build
 * only and never retained.  Requirements (checked, else SELL_EINVAL):
 * rpt[0] = 0, rpt non-decreasing, rpt[nrows] = nnz, every row length and
 * nrows below 2^31, 0 <= col[j] < ncols < 2^31.  Explicit zeros are stored
 * like any other entry.  val_type is SELL_F64 or SELL_F32. */
typedef struct {
    int64_t nrows;
    int64_t ncols;
    int64_t nnz;
    const int64_t *rpt;  /* nrows + 1 */
    const int32_t *col;  /* nnz */
    const void *val;     /* nnz elements of val_type */
    int32_t val_type;
    int32_t on_device;   /* 1: the three arrays are device pointers, 0: host */
} sell_csr;

/* Build flags. */
#define SELL_BUILD_PERMUTE_COLS 0x1u  /* renumber columns by the row permutation
                                         (square matrices only, Sec. 3.4): the
                                         handle then computes P A P^T and takes
                                         x, y in sorted-row order */

/* Build parameters (Sec. 3.3-3.4). */
typedef struct {
    int32_t C;          /* chunk height, >= 1 (GPU default 32: one warp/chunk) */
    int32_t store_type; /* SELL_F64, SELL_F32 or SELL_BF16: value storage */
    int64_t sigma;      /* sorting scope, >= 1; 1 = no sort, >= nrows = global */
    uint32_t flags;     /* SELL_BUILD_* */
    int32_t reserved;   /* must be 0 */
} sell_opts;

typedef struct sell_matrix *sell_handle;

/* What a handle holds (all counts of the built format). */
typedef struct {
    int64_t nrows, ncols, nnz;
    int64_t nchunks;      /* Nc = ceil(nrows / C), Eq. "nc" */
    int64_t stored;       /* cs[Nc] = sum_c C * cl[c], padding included */
    int64_t max_row_len;
    int64_t sigma;
    int32_t C;
    int32_t store_type;
    uint32_t flags;
    int32_t has_perm;     /* 0 when sigma <= 1 (the permutation is identity) */
    double beta;          /* Eq. "beta": nnz / stored (1 when stored = 0) */
    double zeta;          /* Eq. "cv": coefficient of variation of row lengths */
    size_t device_bytes;  /* device memory owned by the handle */
} sell_info_t;

/* Device-memory callbacks: alloc(bytes, ctx, stream) returns a device pointer
 * or NULL; release(ptr, ctx, stream) frees it (may be called with NULL). */
typedef void *(*sell_alloc_fn)(size_t bytes, void *ctx, void *stream);
typedef void (*sell_free_fn)(void *ptr, void *ctx, void *stream);

/* ---------------------------------------------------------------- calls */

/* Install process-wide allocation callbacks (both NULL restores the
 * default).  Handles keep the callbacks they were built with. */
SELL_API sell_status sell_set_allocator(sell_alloc_fn alloc, sell_free_fn release, void *ctx);

/* Convert CRS into SELL-C-sigma (Sec. 3.3 and 3.4, Eqs. "nc", "max"):
 *  1. rowLen[i] = rpt[i+1] - rpt[i];
 *  2. inside each window [w*sigma, min((w+1)*sigma, nrows)) rows are sorted by
 *     rowLen in descending order, equal lengths keeping their order;
 *     perm[r] = original row of sorted row r;
 *  3. chunks of C sorted rows; cl[c] = longest row of chunk c (rows past nrows
 *     count as empty);
 *  4. cs[0] = 0, cs[c+1] = cs[c] + C * cl[c];
 *  5. entry j of sorted row r = c*C + l is stored at cs[c] + j*C + l
 *     (column-major inside the chunk, Listing "sell"); padding has value 0 and
 *     column 0 (Sec. 4).  With SELL_BUILD_PERMUTE_COLS the stored column is
 *     invperm[col].
 * Values are converted to opts->store_type with one round-to-nearest-even.
 * On success *out owns all device arrays; release it with sell_free.
 * Errors: SELL_EINVAL (bad opts or CRS; *out untouched), SELL_ENOMEM,
 * SELL_ECUDA.  Synchronises `stream` (to read the maximum row length and the
 * stored size, and before returning), so the handle may be used on any stream
 * afterwards. */
SELL_API sell_status sell_build(const sell_csr *A, const sell_opts *opts, void *stream,
                       sell_handle *out);

/* SpMV flags. */
#define SELL_SPMV_ACCUMULATE 0x1u   /* y = y + A x instead of y = A x */
#define SELL_SPMV_COMPENSATED_LONG 0x8u /* F32/BF16 storage: compensated (Dot2)
                                          accumulation only for rows of more
                                          than 64 entries (the long-row path);
                                          shorter rows keep the binary32 chain.
                                          SELL_SPMV_COMPENSATED takes precedence */
#define SELL_SPMV_COMPENSATED 0x2u  /* F32/BF16 storage: compensated (Dot2)
                                       binary32 accumulation of each row */
#define SELL_SPMV_HOST_DIRECT 0x80u /* X and Y are page-locked host memory that
                                       the kernels read and write in place, over
                                       the host link, with no staging copies (on
                                       GB300 the x gather then mostly hits L2
                                       and y streams out).  The same arithmetic,
                                       so the same bits, as device buffers.
                                       Exclusive with SELL_SPMV_HOST_IO */
#define SELL_SPMV_RHS_BLOCK4 0x10u  /* SpMMV and batch items: multiply the right-hand
                                       sides in blocks of at most 4 (default 8);
                                       one of RHS_BLOCK4/2/1, the smallest wins.
                                       A tuning knob: every column keeps its own
                                       per-row operation order, so the results
                                       are the same bits for any block width */
#define SELL_SPMV_RHS_BLOCK2 0x20u  /* ... at most 2 */
#define SELL_SPMV_RHS_BLOCK1 0x40u  /* ... one at a time */
#define SELL_SPMV_HOST_IO 0x4u      /* x and y (X and Y) are host pointers
                                       (pinned for asynchronous copies); the
                                       copies to and from the handle's four
                                       staging slots, used in turn, are issued
                                       on `stream`.  Host-io products of one
                                       handle run one after another whatever
                                       their streams, so consecutive calls on
                                       two streams overlap one call's copies
                                       with the other's kernels.  The host
                                       buffers may be reused once the call's
                                       stream has passed it. */

/* y = A x over the SELL-C-sigma handle (Listing "sell", one GPU thread per
 * row of a chunk, each thread stopping at its own row length -- Sec. 3.4, the
 * "Sliced ELLR-T" variant with T = 1).  Each row is summed in CRS order with
 * fused multiply-adds.
 * Types: F64 storage -> x, y binary64; F32/BF16 storage -> x, y binary32 with
 * binary32 accumulation (SELL_SPMV_COMPENSATED: error-free product and sum
 * transformations, result rounded once; SELL_SPMV_COMPENSATED_LONG: the same
 * for rows of more than 64 entries only).  The segment sums of long rows are
 * added in binary64 for binary32 chains.
 * x has ncols elements and y nrows, both in the original row order unless the
 * handle was built with SELL_BUILD_PERMUTE_COLS (then both in sorted order).
 * x and y must not overlap.  Asynchronous on `stream`.
 * Errors: SELL_EINVAL (NULL handle/pointer), SELL_EUNSUPPORTED (COMPENSATED
 * or COMPENSATED_LONG on F64 storage), SELL_ENOMEM (HOST_IO staging),
 * SELL_ECUDA. */
SELL_API sell_status sell_spmv(sell_handle h, const void *x, void *y, uint32_t flags, void *stream);

/* y = A x (as sell_spmv, same flags but SELL_SPMV_HOST_IO) followed by
 * *dot = x . y in binary64 (a Krylov step's p . Ap; not in the paper, which
 * names other kernels over SELL-C-sigma as open work).  A must be square; x
 * and y are in the same order (original, or sorted with
 * SELL_BUILD_PERMUTE_COLS).  The dot is summed in a fixed order over the
 * vector (1024 contiguous ranges, fixed trees), so its bits depend only on x
 * and y, not on the format, the launch or the run.  dot is a device pointer.
 * Errors: those of sell_spmv, SELL_EINVAL (NULL dot, non-square A, HOST_IO). */
SELL_API sell_status sell_spmv_dot(sell_handle h, const void *x, void *y, uint32_t flags, double *dot,
                                   void *stream);

/* Y = A X for k right-hand sides (not in the paper; the matrix is streamed
 * once for up to 8 vectors).  X is ncols x k and Y nrows x k, row-major with
 * leading dimensions ldx >= k and ldy >= k (in elements); element types as in
 * sell_spmv.  k > 8 is processed in blocks of 8 columns, streaming the
 * matrix once per block.  Column c of Y equals sell_spmv of column c of X
 * bit for bit.  Errors as sell_spmv, plus SELL_EINVAL for k < 1, ldx < k,
 * ldy < k. */
SELL_API sell_status sell_spmmv(sell_handle h, const void *X, int64_t ldx, void *Y, int64_t ldy,
                       int32_t k, uint32_t flags, void *stream);

/* The product of sell_spmmv without allocating any memory.  The paper has no
 * counterpart; this entry point is for callers that cannot allocate device
 * memory at the time they multiply -- a serving loop held to a fixed memory
 * budget, code running inside another framework's memory pool, or a
 * latency-critical path that must not wait for an allocation.  (sell_spmmv
 * itself may allocate: staging buffers for SELL_SPMV_HOST_IO, and a larger
 * long-row scratch the first time a call uses more right-hand sides.)
 * Instead of memory owned by the handle, the partial sums of long rows
 * (rows longer than 64 entries) go to one fixed 4 MiB device array that the
 * library holds on every device where it is loaded, until the process exits.
 * Arguments and results are those of sell_spmmv, bit for bit; X and Y are
 * device buffers (SELL_SPMV_HOST_IO is rejected).  The right-hand sides are
 * processed in blocks of up to 8 columns, narrower if the array is too small
 * for 8.  Errors: SELL_EINVAL when even one column's long-row scratch exceeds
 * 4 MiB (the message states the need), plus those of sell_spmmv.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture.  Every call shares the one array and leaves its
 * contents behind (the counters are cleared at the start of every call): two
 * calls whose work overlaps on the GPU -- on different streams, or from
 * different threads -- race and give wrong results.  Calls issued on one
 * stream are ordered and safe. */
SELL_API sell_status sell_spmmv_noalloc(sell_handle h, const void *X, int64_t ldx, void *Y, int64_t ldy,
                                        int32_t k, uint32_t flags, void *stream);

/* Launch tuning of a handle's SpMV/SpMMV kernels (autotuner knob).  The
 * results do not depend on any of these settings.
 *   block    threads per block (32..512, multiple of 32); 0 keeps it.
 *   unroll   entries of a row loaded per step (1, 2, 4 or 8); 0 keeps it.
 *   pipeline how the matrix stream (val/col) is read; -1 keeps it:
 *            0 every thread loads its own entries;
 *            1 as 0, with the next step's loads issued before the current
 *              step's gathers (software pipelining, at every number of
 *              right-hand sides);
 *            2 bulk-staged: each warp copies whole pieces of its chunks into
 *              shared memory with asynchronous bulk copies while it multiplies
 *              the previous piece (single right-hand sides; C = 32, 64 or 128;
 *              block = warps per block x 32, unroll 1/2/4/8 = 1/2/3/4 pieces
 *              per warp; with 1 the next copy starts when the piece is used).
 *              Selecting it computes the per-warp work split of the handle on
 *              the device (synchronous; a few small allocations through the
 *              handle's allocator).
 * Errors: SELL_EINVAL (values), SELL_EUNSUPPORTED (pipeline 2 with another
 * C, or a block that does not fit on an SM), SELL_ENOMEM, SELL_ECUDA. */
SELL_API sell_status sell_set_launch(sell_handle h, int32_t block, int32_t unroll, int32_t pipeline);

/* Synchronise `stream`, then report whether a bounded device-side wait in a
 * kernel of this handle gave up since the last check (SELL_ETIMEOUT; the
 * products of that launch are incomplete) and clear the record.  Only the
 * bulk-staged SpMV (pipeline 2) waits on the device.  Errors: SELL_EINVAL,
 * SELL_ECUDA, SELL_ETIMEOUT. */
SELL_API sell_status sell_check(sell_handle h, void *stream);

/* Test hook of the failure route above (not in the paper): the next
 * single-vector product of h that runs on the bulk-staged kernel (launch mode
 * 2) makes its first warp wait, before its first piece, on a barrier that
 * nothing ever completes, for limit_us microseconds (1..1000000).  That wait
 * gives up; the warp drains its own copies in flight with the normal limit,
 * records the failure and ends, so the product is incomplete and sell_check
 * returns SELL_ETIMEOUT.  One launch only; later products are unaffected.
 * No GPU fault is involved.  Errors: SELL_EINVAL, SELL_EUNSUPPORTED (the
 * handle is not in launch mode 2). */
SELL_API sell_status sell_test_expire_wait(sell_handle h, uint32_t limit_us);

/* Fill *info (host struct).  Errors: SELL_EINVAL. */
SELL_API sell_status sell_info(sell_handle h, sell_info_t *info);

/* Copy the format to host buffers (any may be NULL to skip it): val (stored
 * elements of the storage type), col (stored), cs (nchunks + 1), cl
 * (nchunks), rl (nchunks * C: length of every sorted row, 0 past nrows), perm
 * (nrows; identity when sigma <= 1).  Synchronous.  Errors: SELL_EINVAL,
 * SELL_ECUDA. */
SELL_API sell_status sell_export(sell_handle h, void *val, int32_t *col, int64_t *cs, int32_t *cl,
                        int32_t *rl, int32_t *perm);

/* Release a handle and its device memory.  NULL is accepted (no-op). */
SELL_API sell_status sell_free(sell_handle h);

/* Static text for a status, and the calling thread's last error message. */
SELL_API const char *sell_strerror(sell_status s);
SELL_API const char *sell_last_error(void);

/* ------------------------------------------------------------- batching */

/* One product of a batch: Y = A X (or Y += A X) for k right-hand sides, with
 * the layout rules of sell_spmmv (k = 1 and ldx = ldy = 1 is a plain SpMV).
 * X and Y are device pointers. */
typedef struct {
    sell_handle A;
    const void *X;
    void *Y;
    int64_t ldx, ldy;
    int32_t k;
    uint32_t flags;  /* SELL_SPMV_ACCUMULATE | SELL_SPMV_COMPENSATED | SELL_SPMV_COMPENSATED_LONG */
} sell_batch_item;

typedef struct sell_batch *sell_batch_plan;

/* Prepare a batch of n products to run in a few launches (one per kernel
 * variant present -- value type, block of 1/2/4/8 right-hand sides, plain or
 * compensated accumulation -- and per 160 products).  Work units are tiles of
 * 128 sorted rows of one product, or 128 threads of its long-row segment
 * work (sell_batch_set_launch changes the size); every launch has one block
 * per unit, long-row work first and the biggest products first.  The
 * products may use matrices of different sizes and storage types; a matrix
 * with more than 8 right-hand sides is split into blocks of 8 (or of the
 * item's SELL_SPMV_RHS_BLOCK* width).  Each result is bit-identical to the same product run
 * alone by sell_spmmv.  The plan owns the long-row scratch of its products
 * (one allocation, cleared on `stream`; plans never share scratch with each
 * other or with sell_spmmv); the work units travel in the launch parameters;
 * the items' buffers are referenced, not copied.  Several products in one
 * plan must not write overlapping Y.  Does not synchronise.  Errors:
 * SELL_EINVAL, SELL_ENOMEM, SELL_ECUDA. */
SELL_API sell_status sell_batch_create(const sell_batch_item *items, int32_t n, void *stream,
                              sell_batch_plan *out);

/* Launch a plan on `stream` (kernel launches only: capturable in a CUDA
 * graph).  grid must be 0 (reserved).  Errors: SELL_EINVAL, SELL_ECUDA. */
SELL_API sell_status sell_batch_run(sell_batch_plan plan, int32_t grid, void *stream);

/* Launch tuning of a plan (autotuner knob): `block` threads per block, 64,
 * 128 (the default) or 256, and as many sorted rows (or long-row segment
 * threads) per work unit.  The results do not depend on it.  Takes effect
 * at the next sell_batch_run (a graph captured before keeps the old launch).
 * Errors: SELL_EINVAL, SELL_EUNSUPPORTED (too many units). */
SELL_API sell_status sell_batch_set_launch(sell_batch_plan plan, int32_t block);

/* Release a plan (NULL accepted).  The memory is returned stream-ordered on
 * the stream of the plan's latest sell_batch_run (no host wait); a plan run
 * on several streams must have finished its runs on the other streams. */
SELL_API sell_status sell_batch_free(sell_batch_plan plan);

/* ------------------------------------------------------------- serving */

/* A continuous-batching server over device-resident handles (an extension;
 * the paper stops at single products).  Requests Y = A_mid X arrive from any
 * thread.  A scheduler thread admits them in arrival order while their device
 * footprint -- the x block, the y block and the long-row scratch -- fits in
 * an arena of budget - resident bytes (allocated once at creation, so the
 * budget is never exceeded), packs the admitted ones into one batch plan
 * (sell_batch_create) on a free stream with the device-to-host copies after
 * it, and keeps up to `streams` batches in flight: requests that arrive while
 * others run are admitted as soon as a stream and memory are free, and their
 * work overlaps on the device.  The inputs of all batches go through one
 * copy stream of the server's in 4 MB pieces, the batch with the fewest bytes
 * left first -- a waiting batch's count falling by 200 GB per second of its
 * age, so that a large input is not starved by a stream of small ones -- so a
 * small request's input waits for at most one aged large input rather than
 * for every large one; a batch's kernels start once its inputs are issued.  A batch whose requests
 * differ widely in size runs in two parts, the small requests (work at most
 * 1/8 of its largest) first with their own completion.  Every result is
 * bitwise the result of the same product alone. */
typedef struct sell_server *sell_server_t;

typedef struct {
    int64_t budget_bytes; /* device bytes for the resident handles plus all requests in flight */
    int32_t max_batch;    /* requests per batch, 1..4096 */
    int32_t streams;      /* batches in flight, 1..16 */
    int32_t size_ratio;   /* 0 or 1: a batch takes queued requests in arrival order; r > 1: a batch takes
                             the oldest request, then later ones whose work (stored elements x k) is
                             within a factor r of it, so small requests do not wait for a large one */
    int32_t reserved;     /* 0 */
    int64_t max_batch_work; /* 0: no cap; w > 0: with size_ratio <= 1, a batch stops taking requests
                               once its work (stored elements x k) would exceed w (it always takes
                               at least one) */
} sell_server_opts;

typedef struct {
    double t_arrive, t_launch, t_done; /* seconds, steady clock (differences are latencies) */
    int32_t batch;                     /* requests in the batch it ran in */
    int32_t status;                    /* SELL_OK or the error of its batch */
} sell_request_info;

typedef struct {
    int64_t requests, batches, batched_requests, queued;
    int64_t resident_bytes, budget_bytes, in_use_bytes, peak_bytes; /* peak: resident + arena high-water mark */
} sell_server_stats_t;

/* Start a server over n handles (all on the current device; they must
 * outlive the server).  Errors: SELL_EINVAL (arguments, handles that fill the
 * budget), SELL_ENOMEM, SELL_ECUDA. */
SELL_API sell_status sell_server_create(const sell_handle *mats, int32_t n, const sell_server_opts *opts,
                                        sell_server_t *out);

/* Queue Y = A_mid X for k right-hand sides (row-major ncols x k and
 * nrows x k, binary64 for F64 handles, binary32 otherwise).  X is page-locked
 * host memory that stays unchanged until the request completes; Y is
 * page-locked host memory that receives the result, or NULL to keep the
 * result on the device (sell_server_result) until sell_server_release.
 * flags: SELL_SPMV_ACCUMULATE (host Y only: Y = Y + A X),
 * SELL_SPMV_COMPENSATED.  Does not block.  *id names the request.  Errors:
 * SELL_EINVAL (bad id/k/flags, pageable memory, a request larger than the
 * budget), SELL_EUNSUPPORTED, SELL_ENOMEM. */
SELL_API sell_status sell_server_submit(sell_server_t srv, int32_t mid, const void *X, int32_t k, void *Y,
                                        uint32_t flags, uint64_t *id);

/* Block until request id has completed (or timeout_s passed: SELL_ETIMEOUT)
 * and fill *info (may be NULL).  A request with a host Y is forgotten after
 * its wait; a device-result request stays until sell_server_release.
 * Errors: SELL_EINVAL (unknown id, or a request that another thread delivered
 * with sell_server_next or released while this call waited), SELL_ETIMEOUT,
 * the batch's error. */
SELL_API sell_status sell_server_wait(sell_server_t srv, uint64_t id, double timeout_s, sell_request_info *info);

/* Deliver the next completed request not yet delivered by a wait, in
 * completion order: *id and *info (may be NULL), with the same forgetting
 * rule as sell_server_wait.  Blocks up to timeout_s (SELL_ETIMEOUT). */
SELL_API sell_status sell_server_next(sell_server_t srv, double timeout_s, uint64_t *id, sell_request_info *info);

/* Device address of a completed device-result request's Y (nrows x k). */
SELL_API sell_status sell_server_result(sell_server_t srv, uint64_t id, void **dev_y);

/* Return a completed device-result request's Y to the arena. */
SELL_API sell_status sell_server_release(sell_server_t srv, uint64_t id);

/* Counters and the device-memory high-water mark. */
SELL_API sell_status sell_server_stats(sell_server_t srv, sell_server_stats_t *stats);

/* Finish every queued and running request, stop the scheduler and free the
 * server (NULL accepted).  Device results not yet released are dropped first
 * (their memory goes with the server).  No other call on the server may run
 * at the same time or follow it. */
SELL_API sell_status sell_server_destroy(sell_server_t srv);

/* ------------------------------------------------------------ measuring */

/* Read-only bandwidth kernel (the GPU analogue of Listing "reduction",
 * Sec. 2.1): reads `bytes` of device memory at `buf` (16-byte aligned, size
 * a multiple of 16) and writes one double per block to `sink` (device, at
 * least `grid` doubles) so the reads cannot be elided.  grid = 0 picks
 * 4 blocks per SM.  Used to measure the bandwidth b of the roofline model
 * (Eq. "roof_general").  Errors: SELL_EINVAL, SELL_ECUDA. */
SELL_API sell_status sell_bench_read(const void *buf, size_t bytes, double *sink, int32_t grid,
                            void *stream);

/* Random-gather rate kernel: grid x 256 threads each load iters x 8
 * 8-byte words x[h % n] at pseudo-random positions h (a linear congruential
 * sequence) and write one value each to `sink` (device, grid*256 doubles).
 * With x (n <= 2^32 - 1 words, 8-byte aligned) small enough to stay in L2,
 * gathers per second measure how fast L2 serves scattered 32-byte sectors:
 * the co-bound of an SpMV with random column indices, where every nonzero
 * gathers one x element (the access that alpha models in Sec. 4, whose
 * model assumes infinitely fast caches).  Errors: SELL_EINVAL, SELL_ECUDA. */
SELL_API sell_status sell_bench_gather(const void *x, int64_t n, double *sink, int32_t grid, int32_t iters,
                                       void *stream);

/* The random-gather rate through the tensor memory accelerator instead of
 * the load/store path: x (n words of 8 bytes, n even, 16-byte aligned) is
 * viewed as n / 2 rows of 16 bytes, and every thread of grid x 128 issues
 * `iters` tile::gather4 copies of four random rows each into shared memory
 * (a linear congruential sequence, as sell_bench_gather).  Rows gathered per
 * second = grid x 128 x iters x 4 / time; every row is one 32-byte sector
 * fetch from L2.  sink holds grid x 128 + 1 doubles, the last one 0 on
 * entry: it is set to 1 if a bounded wait for the copies gave up.  Errors:
 * SELL_EINVAL, SELL_EUNSUPPORTED (no tensor-map encoder), SELL_ECUDA. */
SELL_API sell_status sell_bench_gather4(const void *x, int64_t n, double *sink, int32_t grid, int32_t iters,
                                        void *stream);

/* Binary64 fused multiply-add throughput kernel: every thread of
 * grid x 256 threads runs `iters` x 64 dependent-chain FMAs on 8 independent
 * chains; `sink` (device, grid*256 doubles) receives the results.  Used to
 * measure the FP64 pipe's peak, a possible co-bound of the binary64 SpMV
 * (one FMA per stored nonzero).  Errors: SELL_EINVAL, SELL_ECUDA. */
SELL_API sell_status sell_bench_fma64(double *sink, int32_t grid, int32_t iters, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* SELL_H */
