// sell_spmv_impl.cuh -- the SpMV / SpMMV kernel template and its launch
// helpers, included by one translation unit per value type
// (sell_spmv_f64.cu, sell_spmv_f32.cu, sell_spmv_bf16.cu).
//
// Mapping (Sec. 3.4, "Sliced ELLR-T"; Sec. 5: one thread per row): thread r
// handles sorted row r = c*C + l and walks its own row length over
// val[cs[c] + j*C + l] -- for a fixed j the C threads of a chunk read C
// consecutive elements, so the loads of val/col are coalesced when C is a
// multiple of 32, and no thread loads padding.  Rows longer than kSeg are
// cut into kSeg-entry segments; the (long chunk, segment) work units occupy
// the first blocks of the same launch, C threads per unit (sell_rowdot.cuh).
// The result goes to y[perm[r]] (original order) or y[r] (permuted space).
// Matrices without long rows use an instantiation with that path compiled
// out.
//
// Memory behaviour: val/col are read once per product (L1 no-allocate, L2
// evict-first); x is gathered through the read-only path and stays
// L2-resident; U entries of a row are loaded per step (the last, partial
// group predicated), so each thread keeps up to 2U streaming loads and U
// gathers in flight.
#pragma once

#include <type_traits>

#include "sell_rowdot.cuh"
#include "sell_spmv_bulk.cuh"

namespace sell {
namespace spmv_impl {


// AccL: the accumulation of the long rows' segments (Acc unless only long
// rows are compensated, SELL_SPMV_COMPENSATED_LONG).
template <class VT, int K, int U, bool PIPE, class Acc, bool LONG, class AccL = Acc>
__device__ __forceinline__ void spmmv_body(
        const VT *__restrict__ val, const int32_t *__restrict__ col, const int64_t *__restrict__ cs,
        const int32_t *__restrict__ srl, const int32_t *__restrict__ perm, const int32_t *__restrict__ lchunk,
        const int2 *__restrict__ lunit, const int4 *__restrict__ lmeta, const int32_t *__restrict__ lrow,
        int64_t long_threads, int64_t long_blocks, AccL *part, int32_t *cnt,
        int32_t *cnt2,
        const typename XType<VT>::T *__restrict__ X, int64_t ldx, typename XType<VT>::T *Y, int64_t ldy,
        int64_t N, int C, int accumulate, int vec) {
    using XT = typename XType<VT>::T;
    const uint64_t pol = l2_evict_first_policy();
    if constexpr (LONG) {
        if (blockIdx.x < long_blocks) {
            const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
            if (v < long_threads)
                long_unit<VT, XT, K, U, PIPE, AccL>(val, col, cs, srl, perm, lchunk, lunit, lmeta, lrow, part, cnt,
                                                    cnt2, X, ldx, Y, ldy, N, C, v, accumulate, vec, pol);
            return;
        }
    }
    const int64_t r = (blockIdx.x - long_blocks) * (int64_t)blockDim.x + threadIdx.x;
    if (r >= N) return;
    short_row<VT, XT, K, U, PIPE, Acc>(val, col, cs, srl, perm, X, ldx, Y, ldy, C, r, accumulate, vec, pol);
}

#define SELL_SPMMV_PARAMS                                                                                        \
    const VT *__restrict__ val, const int32_t *__restrict__ col, const int64_t *__restrict__ cs,               \
        const int32_t *__restrict__ srl, const int32_t *__restrict__ perm, const int32_t *__restrict__ lchunk, \
        const int2 *__restrict__ lunit, const int4 *__restrict__ lmeta, const int32_t *__restrict__ lrow,      \
        int64_t long_threads, int64_t long_blocks, AccL *part, int32_t *cnt, int32_t *cnt2,                    \
        const typename XType<VT>::T *__restrict__ X, int64_t ldx, typename XType<VT>::T *Y, int64_t ldy,      \
        int64_t N, int C, int accumulate, int vec
#define SELL_SPMMV_ARGS                                                                                 \
    val, col, cs, srl, perm, lchunk, lunit, lmeta, lrow, long_threads, long_blocks, part, cnt, cnt2, X, ldx, \
        Y, ldy, N, C, accumulate, vec

template <class VT, int K, int U, bool PIPE, class Acc, bool LONG, class AccL = Acc>
__global__ void __launch_bounds__(512) k_spmmv(SELL_SPMMV_PARAMS) {
    spmmv_body<VT, K, U, PIPE, Acc, LONG, AccL>(SELL_SPMMV_ARGS);
}

// Occupancy: the one-vector kernel of matrices without long rows asks for 4
// resident blocks of 512 threads, i.e. 32 registers -- every warp slot of
// the SM at any block size.  Its pipelined forms would otherwise take 39-40
// registers (48 of 64 warps); capped they spill 12-28 bytes and still run
// faster, measured on the 200^3 stencil: binary64 (unroll 2, pipelined)
// 467 -> 420 us, the best launch overall (425.5 us before); binary32
// (unroll 4, pipelined) 319 -> 295 us; bfloat16 unchanged.  The other
// kernels keep the allocation ptxas picks (capping the wider ones spills
// hundreds of bytes).
template <class VT, int U, bool PIPE, class Acc, class AccL = Acc>
__global__ void __launch_bounds__(512, 4) k_spmv_short(SELL_SPMMV_PARAMS) {
    spmmv_body<VT, 1, U, PIPE, Acc, false, AccL>(SELL_SPMMV_ARGS);
}

#undef SELL_SPMMV_PARAMS
#undef SELL_SPMMV_ARGS

// One launch of k_spmmv with the given long-row scratch (the handle's own,
// or the caller's for sell_spmmv_noalloc).
template <class VT, int K, int U, bool PIPE, class Acc, class AccL = Acc>
cudaError_t run_with(const sell_matrix *h, const void *X, int64_t ldx, void *Y, int64_t ldy, int acc,
                     int vec, void *part, int32_t *cnt, int32_t *cnt2, cudaStream_t s) {
    using XT = typename XType<VT>::T;
    const int64_t long_threads = h->nunits * h->C;
    const int64_t long_blocks = (long_threads + h->block - 1) / h->block;
    const int64_t grid = long_blocks + (h->nrows + h->block - 1) / h->block;
    // without long rows the long-row path is compiled out, so that it does
    // not cost the per-row path registers or scheduling freedom; one vector
    // without long rows runs at full occupancy (k_spmv_short)
    auto pick = [&]() {
        if constexpr (K == 1)
            return h->nunits ? k_spmmv<VT, 1, U, PIPE, Acc, true, AccL> : k_spmv_short<VT, U, PIPE, Acc, AccL>;
        else
            return h->nunits ? k_spmmv<VT, K, U, PIPE, Acc, true, AccL> : k_spmmv<VT, K, U, PIPE, Acc, false, AccL>;
    };
    auto kern = pick();
    kern<<<(unsigned)grid, h->block, 0, s>>>(
        static_cast<const VT *>(h->val), h->col, h->cs, h->srl,
        (h->flags & SELL_BUILD_PERMUTE_COLS) ? nullptr : h->perm, h->lchunk, h->lunit, h->lmeta, h->lrow,
        long_threads, long_blocks, static_cast<AccL *>(part), cnt, cnt2, static_cast<const XT *>(X), ldx,
        static_cast<XT *>(Y), ldy, h->nrows, h->C, acc, vec);
    return cudaGetLastError();
}

template <class VT, int K, int U, bool PIPE, class Acc, class AccL>
cudaError_t run(const sell_matrix *h, const void *X, int64_t ldx, void *Y, int64_t ldy, int acc,
                int vec, cudaStream_t s) {
    return run_with<VT, K, U, PIPE, Acc, AccL>(h, X, ldx, Y, ldy, acc, vec, h->part, h->cnt, h->cnt2, s);
}

template <class VT, class Acc, class AccL>
cudaError_t pick_with(const sell_matrix *h, const void *X, int64_t ldx, void *Y, int64_t ldy, int kb,
                      int acc, int vec, void *part, int32_t *cnt, int32_t *cnt2, cudaStream_t s) {
    switch (kb) {
        case 1: return run_with<VT, 1, 4, false, Acc, AccL>(h, X, ldx, Y, ldy, acc, vec, part, cnt, cnt2, s);
        case 2: return run_with<VT, 2, 4, false, Acc, AccL>(h, X, ldx, Y, ldy, acc, vec, part, cnt, cnt2, s);
        case 4: return run_with<VT, 4, 2, false, Acc, AccL>(h, X, ldx, Y, ldy, acc, vec, part, cnt, cnt2, s);
        default: return run_with<VT, 8, 2, false, Acc, AccL>(h, X, ldx, Y, ldy, acc, vec, part, cnt, cnt2, s);
    }
}

// Unroll choices keep U * K <= 16 gathered values per thread.
template <class VT, int K, bool PIPE, class Acc, class AccL>
cudaError_t pick_u(const sell_matrix *h, const void *X, int64_t ldx, void *Y, int64_t ldy, int acc, int vec,
                   cudaStream_t s) {
    int u = h->unroll;
    if constexpr (K >= 8) {
        return u >= 2 ? run<VT, K, 2, PIPE, Acc, AccL>(h, X, ldx, Y, ldy, acc, vec, s)
                      : run<VT, K, 1, PIPE, Acc, AccL>(h, X, ldx, Y, ldy, acc, vec, s);
    } else if constexpr (K >= 4) {
        if (u >= 4) return run<VT, K, 4, PIPE, Acc, AccL>(h, X, ldx, Y, ldy, acc, vec, s);
        if (u >= 2) return run<VT, K, 2, PIPE, Acc, AccL>(h, X, ldx, Y, ldy, acc, vec, s);
        return run<VT, K, 1, PIPE, Acc, AccL>(h, X, ldx, Y, ldy, acc, vec, s);
    } else {
        if (u >= 8) return run<VT, K, 8, PIPE, Acc, AccL>(h, X, ldx, Y, ldy, acc, vec, s);
        if (u >= 4) return run<VT, K, 4, PIPE, Acc, AccL>(h, X, ldx, Y, ldy, acc, vec, s);
        if (u >= 2) return run<VT, K, 2, PIPE, Acc, AccL>(h, X, ldx, Y, ldy, acc, vec, s);
        return run<VT, K, 1, PIPE, Acc, AccL>(h, X, ldx, Y, ldy, acc, vec, s);
    }
}

// Launch mode 1 runs the software-pipelined chain at every block width.
template <class VT, int K, class Acc, class AccL>
cudaError_t pick_unroll(const sell_matrix *h, const void *X, int64_t ldx, void *Y, int64_t ldy,
                        int acc, int vec, cudaStream_t s) {
    if (h->pipeline == 1) return pick_u<VT, K, true, Acc, AccL>(h, X, ldx, Y, ldy, acc, vec, s);
    return pick_u<VT, K, false, Acc, AccL>(h, X, ldx, Y, ldy, acc, vec, s);
}

template <class VT, class Acc, class AccL>
cudaError_t pick_k(const sell_matrix *h, const void *X, int64_t ldx, void *Y, int64_t ldy, int kb,
                   int acc, int vec, cudaStream_t s) {
    switch (kb) {
        case 1: return pick_unroll<VT, 1, Acc, AccL>(h, X, ldx, Y, ldy, acc, vec, s);
        case 2: return pick_unroll<VT, 2, Acc, AccL>(h, X, ldx, Y, ldy, acc, vec, s);
        case 4: return pick_unroll<VT, 4, Acc, AccL>(h, X, ldx, Y, ldy, acc, vec, s);
        default: return pick_unroll<VT, 8, Acc, AccL>(h, X, ldx, Y, ldy, acc, vec, s);
    }
}

}  // namespace spmv_impl

// Launch one column block (kb in {1, 2, 4, 8}) of the given storage type and
// accumulation; part/cnt/cnt2 = nullptr uses the handle's scratch.  A single
// column with launch mode 2 goes to the bulk-staged kernel.
template <class VT, class Acc, class AccL = Acc>
cudaError_t spmv_block(const sell_matrix *h, const void *X, int64_t ldx, void *Y, int64_t ldy, int kb,
                       int acc, int vec, void *part, int32_t *cnt, int32_t *cnt2, cudaStream_t s) {
    using namespace spmv_impl;
    if constexpr (std::is_same<Acc, AccL>::value) {  // the bulk kernel has one accumulation for all rows
        if (!part && kb == 1 && h->pipeline == 2 && h->bulk_grid > 0)
            return bulk::run<VT, Acc>(h, X, ldx, Y, ldy, acc, s);
    }
    if (!part) return pick_k<VT, Acc, AccL>(h, X, ldx, Y, ldy, kb, acc, vec, s);
    return pick_with<VT, Acc, AccL>(h, X, ldx, Y, ldy, kb, acc, vec, part, cnt, cnt2, s);
}

}  // namespace sell
