// sell_internal.cuh -- shared internals of the SELL-C-sigma CUDA library.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "sell.h"

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

// Entries per segment of a long row.  Part of the numerics: a row longer than
// kSeg is summed segment by segment (sell_rowdot.cuh), so changing it changes
// the rounding of long rows.
constexpr int kSeg = 64;
// Segments per group of the two-level fold of very long rows (more than
// kSeg * kSuper = 16384 entries); also part of the numerics.
constexpr int kSuper = 256;

inline size_t value_size(int t) { return t == SELL_F64 ? 8 : (t == SELL_F32 ? 4 : 2); }

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
    // host-io staging (lazily allocated)
    void *xstage = nullptr, *ystage = nullptr;
    size_t xstage_bytes = 0, ystage_bytes = 0;
    size_t device_bytes = 0;
};

struct sell_batch {
    struct Group {              // one launch: kernel variant, its products and units
        void *fn = nullptr;     // kernel entry
        void *params = nullptr; // host copy of the launch parameters (products + unit table pointer)
        void *units = nullptr;  // device work-unit table
        int64_t nwork = 0;
        int32_t grid = 0;
    };
    int device = 0;
    sell::Allocator al;
    std::vector<void *> scratch;  // per-product segment scratch and counters
    std::vector<Group> groups;
    int64_t nwork = 0;
    int32_t nprod = 0;
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
sell_status batch_create(const sell_batch_item *items, int32_t n, cudaStream_t s, sell_batch *b);
sell_status batch_run(sell_batch *b, int32_t grid, cudaStream_t s);
void batch_release(sell_batch *b, cudaStream_t s);
sell_status bench_read(const void *buf, size_t bytes, double *sink, int32_t grid, cudaStream_t s);
sell_status bench_fma64(double *sink, int32_t grid, int32_t iters, cudaStream_t s);
sell_status bench_gather(const void *x, int64_t n, double *sink, int32_t grid, int32_t iters, cudaStream_t s);

// --------------------------------------------------------- device helpers
// Streaming loads for data touched once per product (val/col): do not allocate
// in L1 and mark the L2 lines evict-first, so that the gathered vector x keeps
// its place in L2.
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ double ld_stream(const double *ptr, uint64_t pol) {
    double v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.f64 %0, [%1], %2;"
                 : "=d"(v) : "l"(ptr), "l"(pol));
    return v;
}
__device__ __forceinline__ float ld_stream(const float *ptr, uint64_t pol) {
    float v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.f32 %0, [%1], %2;"
                 : "=f"(v) : "l"(ptr), "l"(pol));
    return v;
}
__device__ __forceinline__ int32_t ld_stream(const int32_t *ptr, uint64_t pol) {
    int32_t v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.s32 %0, [%1], %2;"
                 : "=r"(v) : "l"(ptr), "l"(pol));
    return v;
}
__device__ __forceinline__ __nv_bfloat16 ld_stream(const __nv_bfloat16 *ptr, uint64_t pol) {
    unsigned short v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.b16 %0, [%1], %2;"
                 : "=h"(v) : "l"(ptr), "l"(pol));
    return __ushort_as_bfloat16(v);
}

}  // namespace sell
