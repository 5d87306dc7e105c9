// sell_internal.cuh -- shared internals of the SELL-C-sigma CUDA library.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "sell.h"
#include "sell_device.cuh"

namespace sell {

// ------------------------------------------------------------------ errors
void set_error(const std::string &msg);
sell_status fail(sell_status s, const std::string &msg);
sell_status cuda_fail(cudaError_t e, const char *what);

#define SELL_CUDA_TRY(expr)                                   \
    do {                                                      \
        cudaError_t _e = (expr);                              \
        if (_e != cudaSuccess) return ::sell::cuda_fail(_e, #expr); \
    } while (0)

#define SELL_TRY(expr)                         \
    do {                                       \
        sell_status _s = (expr);               \
        if (_s != SELL_OK) return _s;          \
    } while (0)

// --------------------------------------------------------------- allocator
struct Allocator {
    sell_alloc_fn alloc = nullptr;
    sell_free_fn release = nullptr;
    void *ctx = nullptr;
    void *get(size_t bytes, cudaStream_t s) const;
    void put(void *p, cudaStream_t s) const;
};
Allocator current_allocator();

// Device buffer released through the allocator it came from (RAII).
struct DevBuf {
    Allocator al;
    cudaStream_t stream = nullptr;
    void *p = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { reset(); }
    sell_status alloc(const Allocator &a, size_t n, cudaStream_t s);
    void reset();
    void *release_ownership() { void *q = p; p = nullptr; bytes = 0; return q; }
    template <class T> T *as() const { return static_cast<T *>(p); }
};

inline size_t value_size(int t) { return t == SELL_F64 ? 8 : (t == SELL_F32 ? 4 : 2); }

// Accumulation of reduced-precision products: 0 binary32 chains, 1 Dot2 on
// every row, 2 Dot2 on rows longer than kSeg only.
inline int comp_mode(uint32_t flags) {
    if (flags & SELL_SPMV_COMPENSATED) return 1;
    return (flags & SELL_SPMV_COMPENSATED_LONG) ? 2 : 0;
}
constexpr uint32_t kCompFlags = SELL_SPMV_COMPENSATED | SELL_SPMV_COMPENSATED_LONG;
constexpr uint32_t kRhsFlags = SELL_SPMV_RHS_BLOCK4 | SELL_SPMV_RHS_BLOCK2 | SELL_SPMV_RHS_BLOCK1;

// The widest block of right-hand sides the flags allow (8 by default).
inline int max_rhs_block(uint32_t flags) {
    if (flags & SELL_SPMV_RHS_BLOCK1) return 1;
    if (flags & SELL_SPMV_RHS_BLOCK2) return 2;
    return (flags & SELL_SPMV_RHS_BLOCK4) ? 4 : 8;
}

// The next block of right-hand sides: the widest of 8, 4, 2, 1 that fits the
// remaining columns and the flags' limit.
inline int rhs_block(int rem, int maxw) {
    int kb = rem >= 8 ? 8 : rem >= 4 ? 4 : rem >= 2 ? 2 : 1;
    while (kb > maxw) kb >>= 1;
    return kb;
}

// How the kernels may load a row of X, or store a row of Y (base, row pitch
// ld elements of xs bytes): 2 with 32-byte vectors, 1 with 16-byte vectors,
// 0 value by value.  The kernels take X's in bits 0-1 and Y's in bits 2-3.
inline int x_vec(const void *X, int64_t ldx, size_t xs) {
    const uintptr_t a = (uintptr_t)X;
    const int64_t pitch = ldx * (int64_t)xs;
    if (a % 32 == 0 && pitch % 32 == 0) return 2;
    return (a % 16 == 0 && pitch % 16 == 0) ? 1 : 0;
}

}  // namespace sell

// ------------------------------------------------------------------ handle
struct sell_matrix {
    int64_t nrows = 0, ncols = 0, nnz = 0, nchunks = 0, stored = 0, sigma = 1, max_rl = 0;
    int32_t C = 32, store_type = SELL_F64;
    uint32_t flags = 0;
    double beta = 1.0, zeta = 0.0;
    int device = 0;
    int32_t block = 256, unroll = 4, pipeline = 0;
    sell::Allocator al;
    // device arrays (owned)
    void *val = nullptr;       // stored elements of store_type
    int32_t *col = nullptr;    // stored
    int64_t *cs = nullptr;     // nchunks + 1
    int32_t *cl = nullptr;     // nchunks
    int32_t *srl = nullptr;    // nchunks * C, length of each sorted row
    int32_t *perm = nullptr;   // nrows, sorted -> original (null: identity)
    int32_t *lchunk = nullptr; // nlong chunks holding rows longer than kSeg
    int64_t nlong = 0;
    int2 *lunit = nullptr;     // nunits long-row work units {long chunk, segment}
    int32_t *lrow = nullptr;   // nlong * C lanes of each long chunk's long rows
    int4 *lmeta = nullptr;     // nlong {long rows, mode, units, 0} (sell_build.cu k_long_rows)
    int64_t nunits = 0;
    int32_t *cnt = nullptr;    // nlong * C per-row segment counters (zero at rest)
    int32_t *cnt2 = nullptr;   // nunits * C group counters of very long rows (zero at rest)
    void *part = nullptr;      // segment partials: nunits * C * part_k * 8 bytes
    int32_t part_k = 0;
    // bulk-staged SpMV (launch mode 2), prepared by sell_set_launch
    int32_t *bsc = nullptr;    // nchunks staged columns per chunk
    int32_t *wsplit = nullptr; // wsplit_n + 1 per-warp chunk boundaries
    int64_t wsplit_n = 0;
    int32_t *dstat = nullptr;  // device status word: 1 after a bounded wait gave up
    int32_t bulk_grid = 0, bulk_warps = 0, bulk_ring = 0;
    mutable uint32_t expire_us = 0;  // one-shot test hook of sell_test_expire_wait (0: off),
                                     // consumed by the next bulk-staged launch
    double *dot_part = nullptr;  // range sums of sell_spmv_dot (lazily allocated)
    // host-io staging (lazily allocated): kIoSlots slots used in turn, so that
    // the copies of one call overlap the kernels of the previous ones when
    // calls alternate streams.  A slot is reused only after its result has
    // been copied out; with two slots that wait (the result copy of call i
    // before the input copy of call i + 2) bounds a call at half of the two
    // copies plus the kernel, with four the kernels set the pace.  done =
    // recorded after the slot's last device-to-host copy; kdone = recorded
    // after the latest host-io product's kernels.
    static constexpr int kIoSlots = 4;
    struct IoSlot {
        void *x = nullptr, *y = nullptr;
        size_t xb = 0, yb = 0;
        cudaEvent_t done = nullptr;
        bool used = false;
    } io[kIoSlots];
    int io_next = 0;
    cudaEvent_t kdone = nullptr;
    bool kdone_used = false;
    size_t device_bytes = 0;
};

struct sell_batch {
    struct Group {              // one launch: kernel variant, its products and units
        void *fn = nullptr;     // kernel entry
        void *params = nullptr; // host copy of the launch parameters (products and their unit ranges)
        int64_t nwork = 0;
        int32_t grid = 0;
    };
    int device = 0;
    sell::Allocator al;
    std::vector<void *> scratch;  // per-product segment scratch and counters
    std::vector<Group> groups;
    int64_t nwork = 0;
    int32_t nprod = 0;
    int32_t tile = 128;  // threads per block = rows (or segment threads) per work unit
    cudaStream_t last_stream = nullptr;  // stream of the latest sell_batch_run
    bool ran = false;
};

namespace sell {

// --------------------------------------------------------- launch entry points
// (defined in sell_spmv.cu / sell_build.cu / sell_batch.cu / sell_bench.cu)
sell_status launch_spmmv(sell_matrix *h, const void *X, int64_t ldx, void *Y, int64_t ldy,
                         int32_t k, uint32_t flags, cudaStream_t s);
sell_status launch_block_with_scratch(const sell_matrix *h, const void *X, int64_t ldx, void *Y,
                                      int64_t ldy, int kb, uint32_t flags, void *part, int32_t *cnt,
                                      int32_t *cnt2, cudaStream_t s);
sell_status build_format(const sell_csr *A, const sell_opts *o, cudaStream_t s, sell_matrix *h);
sell_status bulk_plan(sell_matrix *h, int64_t nwarps, cudaStream_t s);
sell_status bulk_prepare(sell_matrix *h);
sell_status launch_dot(sell_matrix *h, const void *x, const void *y, double *out, cudaStream_t s);
// scratch: per item, batch_item_scratch() bytes of device memory (or NULL for
// items without long rows); NULL: the plan allocates its own.
sell_status batch_create(const sell_batch_item *items, int32_t n, cudaStream_t s, sell_batch *b,
                         void *const *scratch = nullptr);
size_t batch_item_scratch(const sell_matrix *h, int32_t k, uint32_t flags, size_t *counter_offset);
sell_status batch_run(sell_batch *b, int32_t grid, cudaStream_t s);
sell_status batch_set_tile(sell_batch *b, int32_t tile);
void batch_release(sell_batch *b, cudaStream_t s);
sell_status bench_read(const void *buf, size_t bytes, double *sink, int32_t grid, cudaStream_t s);
sell_status bench_fma64(double *sink, int32_t grid, int32_t iters, cudaStream_t s);
sell_status bench_gather(const void *x, int64_t n, double *sink, int32_t grid, int32_t iters, cudaStream_t s);
sell_status bench_gather4(const void *x, int64_t n, double *sink, int32_t grid, int32_t iters, cudaStream_t s);

}  // namespace sell
