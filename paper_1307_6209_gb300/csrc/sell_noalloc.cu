// sell_noalloc.cu -- sell_spmmv_noalloc: a product that allocates no memory.
//
// Some callers cannot allocate device memory when they multiply: a serving
// loop that runs under a fixed memory budget, code that runs inside another
// framework's memory pool, or a latency-critical path where an allocation
// (and the synchronisation it may imply) is not acceptable.  sell_spmmv can
// allocate in two cases -- host-buffer staging, and a larger long-row scratch
// the first time more right-hand sides are used -- so this entry point
// computes the same product with its long-row scratch in one fixed device
// array that the library holds for the whole process.
//
// The array has kScratchBytes bytes on every device that loads the library.
// In host code `g_noalloc_scratch` names a host-side stand-in, not the device
// memory: the device address is taken once per device with
// cudaGetSymbolAddress (with that device current) and passed to the kernel.
#include <mutex>

#include "sell_internal.cuh"

namespace sell {
namespace {

constexpr size_t kScratchBytes = 4u << 20;  // 4 MiB: segment partials + counters
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
void *g_addr[kMaxDevices] = {};

// The device address of the array on the current device (set up on first use).
sell_status scratch_address(void **out) {
    int dev = 0;
    SELL_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(SELL_EUNSUPPORTED, "sell_spmmv_noalloc: device index too large");
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return SELL_OK;
}

}  // namespace
}  // namespace sell

using namespace sell;

extern "C" sell_status sell_spmmv_noalloc(sell_handle h, const void *X, int64_t ldx, void *Y, int64_t ldy,
                                          int32_t k, uint32_t flags, void *stream) {
    if (!h) return fail(SELL_EINVAL, "sell_spmmv_noalloc: NULL handle");
    if (k < 1 || ldx < k || ldy < k)
        return fail(SELL_EINVAL, "sell_spmmv_noalloc: need k >= 1, ldx >= k, ldy >= k");
    if (flags & ~(SELL_SPMV_ACCUMULATE | kCompFlags))
        return fail(SELL_EINVAL, "sell_spmmv_noalloc: only ACCUMULATE and COMPENSATED are accepted "
                                 "(HOST_IO needs staging memory)");
    if ((flags & kCompFlags) && h->store_type == SELL_F64)
        return fail(SELL_EUNSUPPORTED, "compensated accumulation needs F32/BF16 storage");
    if (h->nrows == 0) return SELL_OK;
    if (!Y || (!X && h->ncols > 0)) return fail(SELL_EINVAL, "sell_spmmv_noalloc: NULL vector");
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    // scratch layout: [row counters: nlong * C int32][group counters: nunits * C
    // int32][partials], each region padded to 256 bytes
    const size_t cnt1_bytes = ((size_t)h->nlong * h->C * sizeof(int32_t) + 255) / 256 * 256;
    const size_t cnt2_bytes = ((size_t)h->nunits * h->C * sizeof(int32_t) + 255) / 256 * 256;
    const size_t cnt_bytes = cnt1_bytes + cnt2_bytes;
    const size_t per_col = (size_t)h->nunits * h->C * 8;
    int kmax = 8;
    while (kmax > 1 && cnt_bytes + per_col * kmax > kScratchBytes) kmax >>= 1;
    if (cnt_bytes + per_col * kmax > kScratchBytes)
        return fail(SELL_EINVAL, "sell_spmmv_noalloc: the matrix's long rows need " +
                                     std::to_string(cnt_bytes + per_col) + " bytes of scratch, more than the " +
                                     std::to_string(kScratchBytes) + "-byte limit");
    void *base = nullptr;
    SELL_TRY(scratch_address(&base));
    int32_t *cnt = static_cast<int32_t *>(base);
    int32_t *cnt2 = reinterpret_cast<int32_t *>(static_cast<unsigned char *>(base) + cnt1_bytes);
    void *part = static_cast<unsigned char *>(base) + cnt_bytes;
    const size_t xs = h->store_type == SELL_F64 ? 8 : 4;
    for (int32_t done = 0; done < k;) {
        int rem = k - done;
        int kb = rem >= 8 ? 8 : rem >= 4 ? 4 : rem >= 2 ? 2 : 1;
        while (kb > kmax) kb >>= 1;
        // the array keeps the previous call's contents: counters start at zero
        if (h->nlong > 0) SELL_CUDA_TRY(cudaMemsetAsync(cnt, 0, cnt_bytes, s));
        SELL_TRY(launch_block_with_scratch(h, static_cast<const char *>(X) + done * xs, ldx,
                                           static_cast<char *>(Y) + done * xs, ldy, kb, flags, part, cnt, cnt2,
                                           s));
        done += kb;
    }
    return SELL_OK;
}
