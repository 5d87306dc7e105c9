// sell_dot.cu -- the dot product x . y that follows an SpMV in a Krylov step
// (the p . Ap of conjugate gradients), in binary64 and in a fixed order.
//
// The sum does not depend on the format, the launch or the run: element i of
// the n-vector belongs to range b = i / ceil(n / kDotBlocks) of kDotBlocks
// contiguous ranges; inside a range, thread t of kDotThreads adds elements
// t, t + kDotThreads, ... in that order (fma of the binary64 products), the
// block's threads are then added in a fixed tree, and one thread adds the
// kDotBlocks range sums in a fixed tree too.  y is read right after the SpMV
// wrote it, mostly from L2.
#include "sell_internal.cuh"

namespace sell {
namespace {

constexpr int kDotBlocks = 1024;
constexpr int kDotThreads = 256;

__device__ __forceinline__ double as_f64(double v) { return v; }
__device__ __forceinline__ double as_f64(float v) { return (double)v; }

template <class T>
__global__ void __launch_bounds__(kDotThreads) k_dot_ranges(const T *__restrict__ x, const T *__restrict__ y,
                                                            int64_t n, double *__restrict__ part) {
    __shared__ double red[kDotThreads];
    const int64_t len = (n + kDotBlocks - 1) / kDotBlocks;
    const int64_t b0 = blockIdx.x * len, b1 = min(n, b0 + len);
    double s = 0.0;
    for (int64_t i = b0 + threadIdx.x; i < b1; i += kDotThreads) s = fma(as_f64(x[i]), as_f64(y[i]), s);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = kDotThreads / 2; w > 0; w >>= 1) {  // fixed pairwise tree
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void __launch_bounds__(kDotThreads) k_dot_final(const double *__restrict__ part, double *__restrict__ out) {
    __shared__ double red[kDotBlocks];
    for (int i = threadIdx.x; i < kDotBlocks; i += kDotThreads) red[i] = part[i];
    __syncthreads();
    for (int w = kDotBlocks / 2; w > 0; w >>= 1) {  // fixed pairwise tree
        for (int i = threadIdx.x; i < w; i += kDotThreads) red[i] += red[i + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

}  // namespace

sell_status launch_dot(sell_matrix *h, const void *x, const void *y, double *out, cudaStream_t s) {
    if (!h->dot_part) {
        h->dot_part = static_cast<double *>(h->al.get(kDotBlocks * sizeof(double), s));
        if (!h->dot_part) return fail(SELL_ENOMEM, "dot scratch allocation failed");
    }
    const int64_t n = h->nrows;
    if (h->store_type == SELL_F64)
        k_dot_ranges<double><<<kDotBlocks, kDotThreads, 0, s>>>(static_cast<const double *>(x),
                                                               static_cast<const double *>(y), n, h->dot_part);
    else
        k_dot_ranges<float><<<kDotBlocks, kDotThreads, 0, s>>>(static_cast<const float *>(x),
                                                              static_cast<const float *>(y), n, h->dot_part);
    k_dot_final<<<1, kDotThreads, 0, s>>>(h->dot_part, out);
    SELL_CUDA_TRY(cudaGetLastError());
    return SELL_OK;
}

}  // namespace sell
