// sell_api.cu -- the extern "C" entry points declared in include/sell.h:
// argument checks, error reporting, the allocator hook and handle lifetime.
// The kernels live in sell_build.cu, sell_spmv.cu, sell_batch.cu and
// sell_bench.cu.
#include <cstring>
#include <mutex>
#include <new>
#include <string>

#include "sell_internal.cuh"

namespace sell {

namespace {
thread_local std::string g_last_error;
std::mutex g_alloc_mu;
Allocator g_alloc;  // null callbacks = stream-ordered allocation from the library pool
}  // namespace

void set_error(const std::string &msg) { g_last_error = msg; }

sell_status fail(sell_status s, const std::string &msg) {
    g_last_error = msg;
    return s;
}

sell_status cuda_fail(cudaError_t e, const char *what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    if (e == cudaErrorMemoryAllocation) return SELL_ENOMEM;
    return SELL_ECUDA;
}

namespace {
// The default allocator draws from one library-owned memory pool per device.
// The pool keeps freed memory for reuse (release threshold: unlimited), so
// plans and staging buffers created in a serving loop do not map new memory
// each time; sell_free hands the unused part back to the device.
constexpr int kMaxDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pool[kMaxDevices] = {};

cudaMemPool_t library_pool(int dev) {
    if (dev < 0 || dev >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> g(g_pool_mu);
    if (!g_pool[dev]) {
        cudaMemPoolProps pr;
        std::memset(&pr, 0, sizeof(pr));
        pr.allocType = cudaMemAllocationTypePinned;
        pr.handleTypes = cudaMemHandleTypeNone;
        pr.location.type = cudaMemLocationTypeDevice;
        pr.location.id = dev;
        cudaMemPool_t p = nullptr;
        if (cudaMemPoolCreate(&p, &pr) != cudaSuccess) {
            (void)cudaGetLastError();
            return nullptr;
        }
        uint64_t keep = UINT64_MAX;
        (void)cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
        g_pool[dev] = p;
    }
    return g_pool[dev];
}
}  // namespace

void trim_library_pool(int dev) {
    cudaMemPool_t p = nullptr;
    {
        std::lock_guard<std::mutex> g(g_pool_mu);
        if (dev >= 0 && dev < kMaxDevices) p = g_pool[dev];
    }
    if (p) (void)cudaMemPoolTrimTo(p, 0);
}

void *Allocator::get(size_t bytes, cudaStream_t s) const {
    if (alloc) return alloc(bytes, ctx, s);
    void *p = nullptr;
    int dev = 0;
    cudaMemPool_t pool = cudaGetDevice(&dev) == cudaSuccess ? library_pool(dev) : nullptr;
    const cudaError_t e = pool ? cudaMallocFromPoolAsync(&p, bytes, pool, s) : cudaMallocAsync(&p, bytes, s);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();  // clear the sticky-free allocation error
        return nullptr;
    }
    return p;
}

void Allocator::put(void *p, cudaStream_t s) const {
    if (!p) return;
    if (release) release(p, ctx, s);
    else (void)cudaFreeAsync(p, s);
}

Allocator current_allocator() {
    std::lock_guard<std::mutex> g(g_alloc_mu);
    return g_alloc;
}

sell_status DevBuf::alloc(const Allocator &a, size_t n, cudaStream_t s) {
    reset();
    al = a;
    stream = s;
    if (n == 0) return SELL_OK;
    p = al.get(n, s);
    if (!p) return fail(SELL_ENOMEM, "device allocation of " + std::to_string(n) + " bytes failed");
    bytes = n;
    return SELL_OK;
}

void DevBuf::reset() {
    if (p) al.put(p, stream);
    p = nullptr;
    bytes = 0;
}

namespace {

void free_matrix(sell_matrix *h) {
    // every kernel that may still read the arrays must finish first
    (void)cudaDeviceSynchronize();
    void *ptrs[] = {h->val,    h->col,   h->cs,   h->cl,     h->srl,    h->perm,
                    h->lchunk, h->lunit, h->cnt, h->cnt2, h->part, h->bsc, h->wsplit, h->dstat, h->dot_part,
                    h->lrow,   h->lmeta};
    for (void *p : ptrs) h->al.put(p, nullptr);
    for (auto &sl : h->io) {
        h->al.put(sl.x, nullptr);
        h->al.put(sl.y, nullptr);
    }
    for (auto &sl : h->io)
        if (sl.done) (void)cudaEventDestroy(sl.done);
    if (h->kdone) (void)cudaEventDestroy(h->kdone);
    const bool own_pool = !h->al.alloc;
    const int dev = h->device;
    (void)cudaDeviceSynchronize();
    delete h;
    if (own_pool) trim_library_pool(dev);
}

// The device address of a page-locked host buffer (SELL_SPMV_HOST_DIRECT);
// anything else is refused.
sell_status host_device_pointer(const void *p, void **out, const char *name) {
    if (!p) {
        *out = nullptr;
        return SELL_OK;
    }
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(SELL_EINVAL, std::string("HOST_DIRECT: ") + name + " is not page-locked host memory");
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer)
        return fail(SELL_EINVAL, std::string("HOST_DIRECT: ") + name + " is not page-locked host memory");
    *out = a.devicePointer;
    return SELL_OK;
}

// Grow a staging buffer of a slot whose previous use has been waited for.
sell_status ensure_stage(sell_matrix *h, void **buf, size_t *have, size_t need, cudaStream_t s) {
    if (*have >= need) return SELL_OK;
    if (*buf) {
        h->al.put(*buf, s);
        *buf = nullptr;
        *have = 0;
    }
    *buf = h->al.get(need, s);
    if (!*buf) return fail(SELL_ENOMEM, "host-io staging buffer allocation failed");
    *have = need;
    return SELL_OK;
}

}  // namespace
}  // namespace sell

using namespace sell;

extern "C" {

sell_status sell_set_allocator(sell_alloc_fn alloc, sell_free_fn release, void *ctx) {
    if ((alloc == nullptr) != (release == nullptr))
        return fail(SELL_EINVAL, "sell_set_allocator: give both callbacks or neither");
    std::lock_guard<std::mutex> g(g_alloc_mu);
    g_alloc.alloc = alloc;
    g_alloc.release = release;
    g_alloc.ctx = alloc ? ctx : nullptr;
    return SELL_OK;
}

sell_status sell_build(const sell_csr *A, const sell_opts *opts, void *stream, sell_handle *out) {
    if (!out) return fail(SELL_EINVAL, "sell_build: NULL output handle");
    sell_matrix *h = new (std::nothrow) sell_matrix();
    if (!h) return fail(SELL_ENOMEM, "sell_build: host allocation failed");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        delete h;
        return cuda_fail(e, "cudaGetDevice");
    }
    h->device = dev;
    sell_status st = build_format(A, opts, static_cast<cudaStream_t>(stream), h);
    if (st != SELL_OK) {
        std::string msg = g_last_error;
        free_matrix(h);
        g_last_error = msg;
        return st;
    }
    *out = h;
    return SELL_OK;
}

sell_status sell_spmmv(sell_handle h, const void *X, int64_t ldx, void *Y, int64_t ldy, int32_t k,
                       uint32_t flags, void *stream) {
    if (!h) return fail(SELL_EINVAL, "sell_spmmv: NULL handle");
    if (k < 1 || ldx < k || ldy < k) return fail(SELL_EINVAL, "sell_spmmv: need k >= 1, ldx >= k, ldy >= k");
    if (flags & ~(SELL_SPMV_ACCUMULATE | kCompFlags | kRhsFlags | SELL_SPMV_HOST_IO | SELL_SPMV_HOST_DIRECT))
        return fail(SELL_EINVAL, "sell_spmmv: unknown flags");
    if ((flags & SELL_SPMV_HOST_IO) && (flags & SELL_SPMV_HOST_DIRECT))
        return fail(SELL_EINVAL, "sell_spmmv: HOST_IO and HOST_DIRECT are exclusive");
    if ((flags & kCompFlags) && h->store_type == SELL_F64)
        return fail(SELL_EUNSUPPORTED, "compensated accumulation needs F32/BF16 storage");
    if (h->nrows == 0) return SELL_OK;
    if (!Y || (!X && h->ncols > 0)) return fail(SELL_EINVAL, "sell_spmmv: NULL vector");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (flags & SELL_SPMV_HOST_DIRECT) {
        // page-locked host buffers, read and written in place by the kernels
        void *xd = nullptr, *yd = nullptr;
        SELL_TRY(host_device_pointer(X, &xd, "X"));
        SELL_TRY(host_device_pointer(Y, &yd, "Y"));
        return launch_spmmv(h, xd, ldx, yd, ldy, k, flags & ~SELL_SPMV_HOST_DIRECT, s);
    }
    if (!(flags & SELL_SPMV_HOST_IO)) return launch_spmmv(h, X, ldx, Y, ldy, k, flags, s);

    // host buffers: stage through device memory owned by the handle, in
    // kIoSlots slots used in turn.  A slot is reused only after its previous
    // device-to-host copy (event wait on this stream), and the products of
    // host-io calls run one after another whatever their streams (they share
    // the long-row scratch), so calls may alternate streams to overlap their
    // copies with the previous call's kernels.  The slots hold X and Y
    // densely (leading dimension k); only the k used columns of each host row
    // are copied, so host columns k..ld-1 are neither read nor written.
    const size_t xs = h->store_type == SELL_F64 ? 8 : 4;
    const size_t xb = (size_t)h->ncols * k * xs, yb = (size_t)h->nrows * k * xs;
    sell_matrix::IoSlot &sl = h->io[h->io_next];
    if (!sl.done) SELL_CUDA_TRY(cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming));
    if (!h->kdone) SELL_CUDA_TRY(cudaEventCreateWithFlags(&h->kdone, cudaEventDisableTiming));
    if (sl.used) SELL_CUDA_TRY(cudaStreamWaitEvent(s, sl.done, 0));
    SELL_TRY(ensure_stage(h, &sl.x, &sl.xb, xb > 0 ? xb : 16, s));
    SELL_TRY(ensure_stage(h, &sl.y, &sl.yb, yb, s));
    h->io_next = (h->io_next + 1) % sell_matrix::kIoSlots;
    const size_t row = (size_t)k * xs;
    if (xb) {
        if (ldx == k) SELL_CUDA_TRY(cudaMemcpyAsync(sl.x, X, xb, cudaMemcpyHostToDevice, s));
        else SELL_CUDA_TRY(cudaMemcpy2DAsync(sl.x, row, X, (size_t)ldx * xs, row, (size_t)h->ncols,
                                             cudaMemcpyHostToDevice, s));
    }
    if (flags & SELL_SPMV_ACCUMULATE) {
        if (ldy == k) SELL_CUDA_TRY(cudaMemcpyAsync(sl.y, Y, yb, cudaMemcpyHostToDevice, s));
        else SELL_CUDA_TRY(cudaMemcpy2DAsync(sl.y, row, Y, (size_t)ldy * xs, row, (size_t)h->nrows,
                                             cudaMemcpyHostToDevice, s));
    }
    if (h->kdone_used) SELL_CUDA_TRY(cudaStreamWaitEvent(s, h->kdone, 0));
    SELL_TRY(launch_spmmv(h, sl.x, k, sl.y, k, k, flags & ~SELL_SPMV_HOST_IO, s));
    SELL_CUDA_TRY(cudaEventRecord(h->kdone, s));
    h->kdone_used = true;
    if (ldy == k) SELL_CUDA_TRY(cudaMemcpyAsync(Y, sl.y, yb, cudaMemcpyDeviceToHost, s));
    else SELL_CUDA_TRY(cudaMemcpy2DAsync(Y, (size_t)ldy * xs, sl.y, row, row, (size_t)h->nrows,
                                         cudaMemcpyDeviceToHost, s));
    SELL_CUDA_TRY(cudaEventRecord(sl.done, s));
    sl.used = true;
    return SELL_OK;
}

sell_status sell_spmv(sell_handle h, const void *x, void *y, uint32_t flags, void *stream) {
    return sell_spmmv(h, x, 1, y, 1, 1, flags, stream);
}

sell_status sell_spmv_dot(sell_handle h, const void *x, void *y, uint32_t flags, double *dot, void *stream) {
    if (!h || !dot) return fail(SELL_EINVAL, "sell_spmv_dot: NULL argument");
    if (h->nrows != h->ncols) return fail(SELL_EINVAL, "sell_spmv_dot: the matrix must be square");
    if (flags & (SELL_SPMV_HOST_IO | SELL_SPMV_HOST_DIRECT))
        return fail(SELL_EINVAL, "sell_spmv_dot: device vectors only");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    SELL_TRY(sell_spmmv(h, x, 1, y, 1, 1, flags, stream));
    if (h->nrows == 0) {
        SELL_CUDA_TRY(cudaMemsetAsync(dot, 0, sizeof(double), s));
        return SELL_OK;
    }
    return launch_dot(h, x, y, dot, s);
}

sell_status sell_set_launch(sell_handle h, int32_t block, int32_t unroll, int32_t pipeline) {
    if (!h) return fail(SELL_EINVAL, "sell_set_launch: NULL handle");
    if (block != 0 && (block < 32 || block > 512 || block % 32 != 0))
        return fail(SELL_EINVAL, "sell_set_launch: block must be a multiple of 32 in [32, 512]");
    if (unroll != 0 && unroll != 1 && unroll != 2 && unroll != 4 && unroll != 8)
        return fail(SELL_EINVAL, "sell_set_launch: unroll must be 1, 2, 4 or 8");
    if (pipeline < -1 || pipeline > 2)
        return fail(SELL_EINVAL, "sell_set_launch: pipeline must be -1, 0, 1 or 2");
    const int32_t nb = block ? block : h->block, nu = unroll ? unroll : h->unroll;
    const int32_t np = pipeline >= 0 ? pipeline : h->pipeline;
    if (np == 2) {
        const int32_t ob = h->block, ou = h->unroll;
        h->block = nb;
        h->unroll = nu;
        sell_status st = bulk_prepare(h);
        if (st != SELL_OK) {
            h->block = ob;
            h->unroll = ou;
            return st;
        }
    }
    h->block = nb;
    h->unroll = nu;
    h->pipeline = np;
    return SELL_OK;
}

sell_status sell_check(sell_handle h, void *stream) {
    if (!h) return fail(SELL_EINVAL, "sell_check: NULL handle");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    SELL_CUDA_TRY(cudaStreamSynchronize(s));
    if (!h->dstat) return SELL_OK;
    int32_t v = 0;
    SELL_CUDA_TRY(cudaMemcpy(&v, h->dstat, sizeof(v), cudaMemcpyDeviceToHost));
    if (v == 0) return SELL_OK;
    SELL_CUDA_TRY(cudaMemset(h->dstat, 0, sizeof(v)));
    return fail(SELL_ETIMEOUT, "sell_check: a bounded wait of the bulk-staged SpMV gave up");
}

sell_status sell_test_expire_wait(sell_handle h, uint32_t limit_us) {
    if (!h) return fail(SELL_EINVAL, "sell_test_expire_wait: NULL handle");
    if (limit_us == 0 || limit_us > 1000000u)
        return fail(SELL_EINVAL, "sell_test_expire_wait: the limit must be 1..1000000 microseconds");
    if (h->pipeline != 2 || h->bulk_grid <= 0)
        return fail(SELL_EUNSUPPORTED, "sell_test_expire_wait: only the bulk-staged SpMV (launch mode 2) "
                                       "waits on the device");
    h->expire_us = limit_us;
    return SELL_OK;
}

sell_status sell_info(sell_handle h, sell_info_t *info) {
    if (!h || !info) return fail(SELL_EINVAL, "sell_info: NULL argument");
    std::memset(info, 0, sizeof(*info));
    info->nrows = h->nrows;
    info->ncols = h->ncols;
    info->nnz = h->nnz;
    info->nchunks = h->nchunks;
    info->stored = h->stored;
    info->max_row_len = h->max_rl;
    info->sigma = h->sigma;
    info->C = h->C;
    info->store_type = h->store_type;
    info->flags = h->flags;
    info->has_perm = h->perm != nullptr;
    info->beta = h->beta;
    info->zeta = h->zeta;
    info->device_bytes = h->device_bytes;
    return SELL_OK;
}

sell_status sell_export(sell_handle h, void *val, int32_t *col, int64_t *cs, int32_t *cl, int32_t *rl,
                        int32_t *perm) {
    if (!h) return fail(SELL_EINVAL, "sell_export: NULL handle");
    SELL_CUDA_TRY(cudaDeviceSynchronize());
    const size_t vs = value_size(h->store_type);
    if (val && h->stored) SELL_CUDA_TRY(cudaMemcpy(val, h->val, h->stored * vs, cudaMemcpyDeviceToHost));
    if (col && h->stored)
        SELL_CUDA_TRY(cudaMemcpy(col, h->col, h->stored * sizeof(int32_t), cudaMemcpyDeviceToHost));
    if (cs) SELL_CUDA_TRY(cudaMemcpy(cs, h->cs, (h->nchunks + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost));
    if (cl && h->nchunks)
        SELL_CUDA_TRY(cudaMemcpy(cl, h->cl, h->nchunks * sizeof(int32_t), cudaMemcpyDeviceToHost));
    if (rl && h->nchunks)
        SELL_CUDA_TRY(cudaMemcpy(rl, h->srl, h->nchunks * h->C * sizeof(int32_t), cudaMemcpyDeviceToHost));
    if (perm) {
        if (h->perm) {
            SELL_CUDA_TRY(cudaMemcpy(perm, h->perm, h->nrows * sizeof(int32_t), cudaMemcpyDeviceToHost));
        } else {
            for (int64_t i = 0; i < h->nrows; ++i) perm[i] = (int32_t)i;
        }
    }
    return SELL_OK;
}

sell_status sell_free(sell_handle h) {
    if (h) free_matrix(h);
    return SELL_OK;
}

const char *sell_strerror(sell_status s) {
    switch (s) {
        case SELL_OK: return "success";
        case SELL_EINVAL: return "invalid argument";
        case SELL_ENOMEM: return "out of memory";
        case SELL_ECUDA: return "CUDA error";
        case SELL_EBOUNDS: return "bounds check failed";
        case SELL_ETIMEOUT: return "device wait timed out";
        case SELL_EUNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

const char *sell_last_error(void) { return g_last_error.c_str(); }

sell_status sell_batch_create(const sell_batch_item *items, int32_t n, void *stream, sell_batch_plan *out) {
    if (!out || n < 0 || (n > 0 && !items)) return fail(SELL_EINVAL, "sell_batch_create: bad arguments");
    sell_batch *b = new (std::nothrow) sell_batch();
    if (!b) return fail(SELL_ENOMEM, "sell_batch_create: host allocation failed");
    sell_status st = batch_create(items, n, static_cast<cudaStream_t>(stream), b);
    if (st != SELL_OK) {
        std::string msg = g_last_error;
        (void)cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
        batch_release(b, nullptr);
        (void)cudaDeviceSynchronize();
        delete b;
        g_last_error = msg;
        return st;
    }
    *out = b;
    return SELL_OK;
}

sell_status sell_batch_run(sell_batch_plan plan, int32_t grid, void *stream) {
    if (!plan || grid < 0) return fail(SELL_EINVAL, "sell_batch_run: bad arguments");
    return batch_run(plan, grid, static_cast<cudaStream_t>(stream));
}

sell_status sell_batch_set_launch(sell_batch_plan plan, int32_t block) {
    if (!plan) return fail(SELL_EINVAL, "sell_batch_set_launch: NULL plan");
    return batch_set_tile(plan, block);
}

sell_status sell_batch_free(sell_batch_plan plan) {
    if (!plan) return SELL_OK;
    // stream-ordered release after the latest run (no host wait), so a
    // scheduler can retire finished plans while other batches still run
    cudaStream_t s = plan->ran ? plan->last_stream : nullptr;
    batch_release(plan, s);
    delete plan;
    return SELL_OK;
}

sell_status sell_bench_read(const void *buf, size_t bytes, double *sink, int32_t grid, void *stream) {
    return bench_read(buf, bytes, sink, grid, static_cast<cudaStream_t>(stream));
}

sell_status sell_bench_gather(const void *x, int64_t n, double *sink, int32_t grid, int32_t iters,
                              void *stream) {
    return bench_gather(x, n, sink, grid, iters, static_cast<cudaStream_t>(stream));
}

sell_status sell_bench_gather4(const void *x, int64_t n, double *sink, int32_t grid, int32_t iters,
                               void *stream) {
    return bench_gather4(x, n, sink, grid, iters, static_cast<cudaStream_t>(stream));
}

sell_status sell_bench_fma64(double *sink, int32_t grid, int32_t iters, void *stream) {
    return bench_fma64(sink, grid, iters, static_cast<cudaStream_t>(stream));
}

}  // extern "C"
