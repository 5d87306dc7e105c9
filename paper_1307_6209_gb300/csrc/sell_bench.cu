// sell_bench.cu -- measuring kernels for the roofline model (Sec. 2.1, Sec. 4).
//
// k_read_bw is the GPU analogue of the read-only reduction benchmark of
// Listing "reduction": every thread sums 16-byte vectors of a large buffer in
// a grid-stride loop; one partial sum per block is written so that the loads
// cannot be removed.  Its bandwidth is the b of Eq. "roof_general".
//
// k_gather measures the rate of random 8-byte gathers (L2-resident x).
// k_gather4 measures the same access through the tensor memory accelerator:
// x viewed as rows of 16 bytes, four random rows per tile::gather4 copy.
// k_fma64 measures the binary64 FMA issue rate, which bounds the binary64
// SpMV as well (one FMA per stored nonzero).
#include <cuda.h>

#include "sell_spmv_bulk.cuh"

namespace sell {
namespace {

// The loaded words are combined with integer operations: on GB300 the
// binary64 pipe is too slow to keep up with HBM, so a floating-point sum
// would measure the FP64 adder instead of the memory.  A plain grid-stride
// loop over 16-byte words with many resident blocks reads fastest.
__global__ void __launch_bounds__(256) k_read_bw(const uint4 *__restrict__ a, int64_t n16,
                                                 double *__restrict__ sink) {
    __shared__ unsigned int red[8];
    unsigned int s = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n16; i += stride) {
        uint4 v = a[i];
        s += v.x ^ v.y ^ v.z ^ v.w;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        sink[blockIdx.x] = (double)t;
    }
}

// Random gathers of 8-byte words from x[0..n): every thread draws `iters`
// x 8 indices from a linear congruential sequence and sums the words as
// integers.  With x resident in L2 this measures the rate at which L2 serves
// scattered sectors, the bound of an SpMV whose column indices are random
// (Sec. 4 assumes infinitely fast caches; the access to x is what alpha
// models).
__global__ void __launch_bounds__(256) k_gather(const unsigned long long *__restrict__ x, uint32_t n,
                                                int iters, double *__restrict__ sink) {
    uint32_t h = (blockIdx.x * blockDim.x + threadIdx.x) * 2654435761u + 12345u;
    unsigned long long s = 0;
    for (int it = 0; it < iters; ++it) {
        unsigned long long v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            h = h * 1664525u + 1013904223u;
            v[u] = __ldg(x + (h % n));
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) s += v[u];
    }
    sink[blockIdx.x * (int64_t)blockDim.x + threadIdx.x] = (double)(s & 0xFFFFu);
}

// Random rows through TMA gather4: every lane of every warp issues one copy
// of four random 16-byte rows of x (a 2 x nrows binary64 tensor, box 2 x 1)
// per step into its own 128-byte slot; two slots per lane, each warp's copies
// of a step counted on one mbarrier (32 x 64 bytes).  Lane l then reads one
// word of its slot, so the copies are used.  Waits are bounded (the bulk
// kernel's limit); a warp whose wait gives up sets sink[grid * blockDim]
// to 1, waits (bounded) for its copies still in flight and ends.
constexpr int kG4Warps = 4;
constexpr int kG4Slot = 128;  // bytes per lane and step (64 used)

__device__ __forceinline__ void gather4_rows(void *dst, const CUtensorMap *tm, const uint32_t (&r)[4], uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile::gather4.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(bulk::smem_addr(dst)),
        "l"(tm), "r"(0), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(bulk::smem_addr(bar))
        : "memory");
}

__global__ void __launch_bounds__(kG4Warps * 32) k_gather4(const __grid_constant__ CUtensorMap tm, uint32_t nrows,
                                                            int iters, double *__restrict__ sink) {
    __shared__ __align__(128) unsigned char buf[kG4Warps][2][32 * kG4Slot];
    __shared__ __align__(8) uint64_t bar[kG4Warps][2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t h = (blockIdx.x * blockDim.x + threadIdx.x) * 2654435761u + 12345u;
    if (lane == 0) {
        bulk::mbar_init(&bar[warp][0], 1);
        bulk::mbar_init(&bar[warp][1], 1);
        bulk::fence_mbar_init();
    }
    __syncwarp();
    auto issue = [&](int i) {
        const int slot = i & 1;
        bulk::fence_proxy_async();  // this lane's reads of its slot's previous use come first
        if (lane == 0) bulk::mbar_expect_tx(&bar[warp][slot], 32 * 64);
        __syncwarp();
        uint32_t r[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            h = h * 1664525u + 1013904223u;
            r[q] = h % nrows;
        }
        gather4_rows(&buf[warp][slot][lane * kG4Slot], &tm, r, &bar[warp][slot]);
    };
    double s = 0.0;
    issue(0);
    int issued = 1;
    for (int i = 0; i < iters; ++i) {
        if (i + 1 < iters) {
            issue(i + 1);
            issued = i + 2;
        }
        const int slot = i & 1;
        const bool ok = bulk::mbar_wait(&bar[warp][slot], (uint32_t)((i >> 1) & 1));
        if (__any_sync(0xffffffffu, !ok)) {
            if (lane == 0) sink[(int64_t)gridDim.x * blockDim.x] = 1.0;
            for (int k = i; k < issued; ++k) (void)bulk::mbar_wait(&bar[warp][k & 1], (uint32_t)((k >> 1) & 1));
            return;
        }
        s += reinterpret_cast<const double *>(&buf[warp][slot][lane * kG4Slot])[lane & 7];
        __syncwarp();
    }
    sink[blockIdx.x * (int64_t)blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_fma64(double *__restrict__ sink, int iters) {
    const double a = 1.0000001, b = 0.9999999;
    double c[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) c[q] = threadIdx.x * 1e-3 + q;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int rep = 0; rep < 8; ++rep)
#pragma unroll
            for (int q = 0; q < 8; ++q) c[q] = fma(c[q], a, b);
    }
    double t = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) t += c[q];
    sink[blockIdx.x * (int64_t)blockDim.x + threadIdx.x] = t;
}

}  // namespace

sell_status bench_read(const void *buf, size_t bytes, double *sink, int32_t grid, cudaStream_t s) {
    if (!buf || !sink || bytes == 0 || (bytes % 16) != 0 || ((uintptr_t)buf % 16) != 0 || grid < 0)
        return fail(SELL_EINVAL, "sell_bench_read: need a 16-byte aligned buffer, size % 16 == 0");
    int g = grid;
    if (g == 0) {
        int dev = 0, sms = 0;
        SELL_CUDA_TRY(cudaGetDevice(&dev));
        SELL_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        g = sms * 16;
    }
    k_read_bw<<<g, 256, 0, s>>>(static_cast<const uint4 *>(buf), (int64_t)(bytes / 16), sink);
    SELL_CUDA_TRY(cudaGetLastError());
    return SELL_OK;
}

sell_status bench_gather(const void *x, int64_t n, double *sink, int32_t grid, int32_t iters,
                         cudaStream_t s) {
    if (!x || !sink || n < 1 || n > 0xFFFFFFFFll || grid < 1 || iters < 1 || ((uintptr_t)x % 8) != 0)
        return fail(SELL_EINVAL, "sell_bench_gather: bad arguments");
    k_gather<<<grid, 256, 0, s>>>(static_cast<const unsigned long long *>(x), (uint32_t)n, iters, sink);
    SELL_CUDA_TRY(cudaGetLastError());
    return SELL_OK;
}

sell_status bench_gather4(const void *x, int64_t n, double *sink, int32_t grid, int32_t iters, cudaStream_t s) {
    if (!x || !sink || n < 2 || (n % 2) != 0 || n / 2 > 0xFFFFFFFFll || grid < 1 || iters < 1 ||
        ((uintptr_t)x % 16) != 0)
        return fail(SELL_EINVAL, "sell_bench_gather4: need a 16-byte aligned x of an even number of words");
    using EncodeFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    void *fp = nullptr;
    cudaDriverEntryPointQueryResult q;
    SELL_CUDA_TRY(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fp, 12000, cudaEnableDefault, &q));
    if (q != cudaDriverEntryPointSuccess || !fp)
        return fail(SELL_EUNSUPPORTED, "sell_bench_gather4: cuTensorMapEncodeTiled is not available");
    // x as a 2 x (n / 2) tensor of binary64: rows of 16 bytes, a box of one row
    CUtensorMap tm;
    const cuuint64_t dims[2] = {2, (cuuint64_t)(n / 2)};
    const cuuint64_t strides[1] = {16};
    const cuuint32_t box[2] = {2, 1};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = reinterpret_cast<EncodeFn>(fp)(&tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<void *>(x),
                                                      dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                                      CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                                                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(SELL_ECUDA, "sell_bench_gather4: cuTensorMapEncodeTiled failed");
    k_gather4<<<grid, kG4Warps * 32, 0, s>>>(tm, (uint32_t)(n / 2), iters, sink);
    SELL_CUDA_TRY(cudaGetLastError());
    return SELL_OK;
}

sell_status bench_fma64(double *sink, int32_t grid, int32_t iters, cudaStream_t s) {
    if (!sink || grid < 1 || iters < 1) return fail(SELL_EINVAL, "sell_bench_fma64: bad arguments");
    k_fma64<<<grid, 256, 0, s>>>(sink, iters);
    SELL_CUDA_TRY(cudaGetLastError());
    return SELL_OK;
}

}  // namespace sell
