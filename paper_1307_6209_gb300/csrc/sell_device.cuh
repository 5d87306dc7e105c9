// sell_device.cuh -- the constants and device helpers that the SpMV kernels'
// arithmetic and memory behaviour depend on (kept apart from the host-side
// internals so that a change here is a change of the kernels).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace sell {

// Entries per segment of a long row.  Part of the numerics: a row longer than
// kSeg is summed segment by segment (sell_rowdot.cuh), so changing it changes
// the rounding of long rows.
constexpr int kSeg = 64;
// Segments per group of the two-level fold of very long rows (more than
// kSeg * kSuper = 16384 entries); also part of the numerics.
constexpr int kSuper = 256;

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
