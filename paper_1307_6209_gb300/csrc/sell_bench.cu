// sell_bench.cu -- measuring kernels for the roofline model (Sec. 2.1, Sec. 4).
//
// k_read_bw is the GPU analogue of the read-only reduction benchmark of
// Listing "reduction": every thread sums 16-byte vectors of a large buffer in
// a grid-stride loop; one partial sum per block is written so that the loads
// cannot be removed.  Its bandwidth is the b of Eq. "roof_general".
//
// k_gather measures the rate of random 8-byte gathers (L2-resident x).
// k_fma64 measures the binary64 FMA issue rate, which bounds the binary64
// SpMV as well (one FMA per stored nonzero).
#include "sell_internal.cuh"

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

sell_status bench_fma64(double *sink, int32_t grid, int32_t iters, cudaStream_t s) {
    if (!sink || grid < 1 || iters < 1) return fail(SELL_EINVAL, "sell_bench_fma64: bad arguments");
    k_fma64<<<grid, 256, 0, s>>>(sink, iters);
    SELL_CUDA_TRY(cudaGetLastError());
    return SELL_OK;
}

}  // namespace sell
