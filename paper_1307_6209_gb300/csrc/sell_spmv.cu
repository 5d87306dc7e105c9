// sell_spmv.cu -- SELL-C-sigma SpMV / SpMMV kernels for sm_103a.
//
// Mapping (Sec. 3.4, "Sliced ELLR-T"; Sec. 5: one thread per row): thread r
// handles sorted row r = c*C + l and walks its own row length over
// val[cs[c] + j*C + l] -- for a fixed j the C threads of a chunk read C
// consecutive elements, so the loads of val/col are coalesced when C is a
// multiple of 32, and no thread loads padding.  Rows longer than kSeg are
// taken by the first nlong blocks of the same launch, one block per chunk that
// holds such rows, many threads per row (sell_rowdot.cuh); those blocks come
// first in the grid so that they start early.  The result goes to y[perm[r]]
// (original order) or y[r] (permuted space).
//
// Memory behaviour: val/col are read once per product (L1 no-allocate, L2
// evict-first); x is gathered through the read-only path and stays
// L2-resident; U entries of a row are loaded per step (predicated), so each
// thread keeps up to 2U streaming loads and U gathers in flight.
#include "sell_rowdot.cuh"

namespace sell {
namespace {

template <class VT, int K, int U, class Acc>
__global__ void __launch_bounds__(512)
k_spmmv(const VT *__restrict__ val, const int32_t *__restrict__ col, const int64_t *__restrict__ cs,
        const int32_t *__restrict__ srl, const int32_t *__restrict__ perm, const int32_t *__restrict__ lchunk,
        const int2 *__restrict__ lunit, int64_t long_threads, int64_t long_blocks, Acc *part, int32_t *cnt,
        int32_t *cnt2,
        const typename XType<VT>::T *__restrict__ X, int64_t ldx, typename XType<VT>::T *Y, int64_t ldy,
        int64_t N, int C, int accumulate, int vec) {
    using XT = typename XType<VT>::T;
    const uint64_t pol = l2_evict_first_policy();
    if (blockIdx.x < long_blocks) {
        const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
        if (v < long_threads)
            long_unit<VT, XT, K, U, Acc>(val, col, cs, srl, perm, lchunk, lunit, part, cnt, cnt2, X, ldx, Y, ldy,
                                         N, C, v, accumulate, vec != 0, pol);
        return;
    }
    const int64_t r = (blockIdx.x - long_blocks) * (int64_t)blockDim.x + threadIdx.x;
    if (r >= N) return;
    short_row<VT, XT, K, U, Acc>(val, col, cs, srl, perm, X, ldx, Y, ldy, C, r, accumulate, vec != 0, pol);
}

template <class VT, int K, int U, class Acc>
cudaError_t run(const sell_matrix *h, const void *X, int64_t ldx, void *Y, int64_t ldy, int acc,
                int vec, cudaStream_t s) {
    using XT = typename XType<VT>::T;
    const int64_t long_threads = h->nunits * h->C;
    const int64_t long_blocks = (long_threads + h->block - 1) / h->block;
    const int64_t grid = long_blocks + (h->nrows + h->block - 1) / h->block;
    k_spmmv<VT, K, U, Acc><<<(unsigned)grid, h->block, 0, s>>>(
        static_cast<const VT *>(h->val), h->col, h->cs, h->srl,
        (h->flags & SELL_BUILD_PERMUTE_COLS) ? nullptr : h->perm, h->lchunk, h->lunit, long_threads,
        long_blocks, static_cast<Acc *>(h->part), h->cnt, h->cnt2, static_cast<const XT *>(X), ldx,
        static_cast<XT *>(Y), ldy, h->nrows, h->C, acc, vec);
    return cudaGetLastError();
}

// Same launch with caller-chosen segment scratch (used by sell_spmmv_noalloc).
template <class VT, int K, int U, class Acc>
cudaError_t run_with(const sell_matrix *h, const void *X, int64_t ldx, void *Y, int64_t ldy, int acc,
                     int vec, void *part, int32_t *cnt, int32_t *cnt2, cudaStream_t s) {
    using XT = typename XType<VT>::T;
    const int64_t long_threads = h->nunits * h->C;
    const int64_t long_blocks = (long_threads + h->block - 1) / h->block;
    const int64_t grid = long_blocks + (h->nrows + h->block - 1) / h->block;
    k_spmmv<VT, K, U, Acc><<<(unsigned)grid, h->block, 0, s>>>(
        static_cast<const VT *>(h->val), h->col, h->cs, h->srl,
        (h->flags & SELL_BUILD_PERMUTE_COLS) ? nullptr : h->perm, h->lchunk, h->lunit, long_threads,
        long_blocks, static_cast<Acc *>(part), cnt, cnt2, static_cast<const XT *>(X), ldx, static_cast<XT *>(Y),
        ldy, h->nrows, h->C, acc, vec);
    return cudaGetLastError();
}

template <class VT, class Acc>
cudaError_t pick_with(const sell_matrix *h, const void *X, int64_t ldx, void *Y, int64_t ldy, int kb,
                      int acc, int vec, void *part, int32_t *cnt, int32_t *cnt2, cudaStream_t s) {
    switch (kb) {
        case 1: return run_with<VT, 1, 4, Acc>(h, X, ldx, Y, ldy, acc, vec, part, cnt, cnt2, s);
        case 2: return run_with<VT, 2, 4, Acc>(h, X, ldx, Y, ldy, acc, vec, part, cnt, cnt2, s);
        case 4: return run_with<VT, 4, 2, Acc>(h, X, ldx, Y, ldy, acc, vec, part, cnt, cnt2, s);
        default: return run_with<VT, 8, 2, Acc>(h, X, ldx, Y, ldy, acc, vec, part, cnt, cnt2, s);
    }
}

// Unroll choices keep U * K <= 16 gathered values per thread.
template <class VT, int K, class Acc>
cudaError_t pick_unroll(const sell_matrix *h, const void *X, int64_t ldx, void *Y, int64_t ldy,
                        int acc, int vec, cudaStream_t s) {
    int u = h->unroll;
    if constexpr (K >= 8) {
        return u >= 2 ? run<VT, K, 2, Acc>(h, X, ldx, Y, ldy, acc, vec, s)
                      : run<VT, K, 1, Acc>(h, X, ldx, Y, ldy, acc, vec, s);
    } else if constexpr (K >= 4) {
        if (u >= 4) return run<VT, K, 4, Acc>(h, X, ldx, Y, ldy, acc, vec, s);
        if (u >= 2) return run<VT, K, 2, Acc>(h, X, ldx, Y, ldy, acc, vec, s);
        return run<VT, K, 1, Acc>(h, X, ldx, Y, ldy, acc, vec, s);
    } else {
        if (u >= 8) return run<VT, K, 8, Acc>(h, X, ldx, Y, ldy, acc, vec, s);
        if (u >= 4) return run<VT, K, 4, Acc>(h, X, ldx, Y, ldy, acc, vec, s);
        if (u >= 2) return run<VT, K, 2, Acc>(h, X, ldx, Y, ldy, acc, vec, s);
        return run<VT, K, 1, Acc>(h, X, ldx, Y, ldy, acc, vec, s);
    }
}

template <class VT, class Acc>
cudaError_t pick_k(const sell_matrix *h, const void *X, int64_t ldx, void *Y, int64_t ldy, int kb,
                   int acc, int vec, cudaStream_t s) {
    switch (kb) {
        case 1: return pick_unroll<VT, 1, Acc>(h, X, ldx, Y, ldy, acc, vec, s);
        case 2: return pick_unroll<VT, 2, Acc>(h, X, ldx, Y, ldy, acc, vec, s);
        case 4: return pick_unroll<VT, 4, Acc>(h, X, ldx, Y, ldy, acc, vec, s);
        default: return pick_unroll<VT, 8, Acc>(h, X, ldx, Y, ldy, acc, vec, s);
    }
}

}  // namespace

// Splits k into kernel blocks of 8, 4, 2, 1 columns (every column keeps the
// same per-row operation order, so the split does not change any result).
// The segment scratch grows on the first product with a wider block.
sell_status launch_spmmv(sell_matrix *h, const void *X, int64_t ldx, void *Y, int64_t ldy,
                         int32_t k, uint32_t flags, cudaStream_t s) {
    if (h->nrows == 0) return SELL_OK;
    if (h->nunits > 0) {
        const int need = k >= 8 ? 8 : k >= 4 ? 4 : k >= 2 ? 2 : 1;
        if (need > h->part_k) {
            void *p = h->al.get((size_t)h->nunits * h->C * need * 8, s);
            if (!p) return fail(SELL_ENOMEM, "segment scratch allocation failed");
            h->al.put(h->part, s);
            h->part = p;
            h->part_k = need;
        }
    }
    const int acc = (flags & SELL_SPMV_ACCUMULATE) ? 1 : 0;
    const bool comp = (flags & SELL_SPMV_COMPENSATED) != 0;
    const size_t xs = h->store_type == SELL_F64 ? 8 : 4;
    int32_t done = 0;
    while (done < k) {
        int rem = k - done;
        int kb = rem >= 8 ? 8 : rem >= 4 ? 4 : rem >= 2 ? 2 : 1;
        const char *Xb = static_cast<const char *>(X) + (size_t)done * xs;
        char *Yb = static_cast<char *>(Y) + (size_t)done * xs;
        int vec = (((uintptr_t)Xb % 16) == 0 && ((ldx * xs) % 16) == 0) ? 1 : 0;
        cudaError_t e;
        switch (h->store_type) {
            case SELL_F64:
                e = pick_k<double, Plain<double>>(h, Xb, ldx, Yb, ldy, kb, acc, vec, s);
                break;
            case SELL_F32:
                e = comp ? pick_k<float, Dot2>(h, Xb, ldx, Yb, ldy, kb, acc, vec, s)
                         : pick_k<float, Plain<float>>(h, Xb, ldx, Yb, ldy, kb, acc, vec, s);
                break;
            default:
                e = comp ? pick_k<__nv_bfloat16, Dot2>(h, Xb, ldx, Yb, ldy, kb, acc, vec, s)
                         : pick_k<__nv_bfloat16, Plain<float>>(h, Xb, ldx, Yb, ldy, kb, acc, vec, s);
                break;
        }
        if (e != cudaSuccess) return cuda_fail(e, "SpMV kernel launch");
        done += kb;
    }
    return SELL_OK;
}

// One column block of up to 8 right-hand sides with the given segment scratch
// `part` (nunits * C * kb * 8 bytes) and zeroed counters `cnt` (nlong * C).
sell_status launch_block_with_scratch(const sell_matrix *h, const void *X, int64_t ldx, void *Y,
                                      int64_t ldy, int kb, uint32_t flags, void *part, int32_t *cnt,
                                      int32_t *cnt2, cudaStream_t s) {
    const int acc = (flags & SELL_SPMV_ACCUMULATE) ? 1 : 0;
    const bool comp = (flags & SELL_SPMV_COMPENSATED) != 0;
    const size_t xs = h->store_type == SELL_F64 ? 8 : 4;
    const int vec = (((uintptr_t)X % 16) == 0 && ((ldx * xs) % 16) == 0) ? 1 : 0;
    cudaError_t e;
    switch (h->store_type) {
        case SELL_F64:
            e = pick_with<double, Plain<double>>(h, X, ldx, Y, ldy, kb, acc, vec, part, cnt, cnt2, s);
            break;
        case SELL_F32:
            e = comp ? pick_with<float, Dot2>(h, X, ldx, Y, ldy, kb, acc, vec, part, cnt, cnt2, s)
                     : pick_with<float, Plain<float>>(h, X, ldx, Y, ldy, kb, acc, vec, part, cnt, cnt2, s);
            break;
        default:
            e = comp ? pick_with<__nv_bfloat16, Dot2>(h, X, ldx, Y, ldy, kb, acc, vec, part, cnt, cnt2, s)
                     : pick_with<__nv_bfloat16, Plain<float>>(h, X, ldx, Y, ldy, kb, acc, vec, part, cnt, cnt2, s);
            break;
    }
    if (e != cudaSuccess) return cuda_fail(e, "SpMV kernel launch");
    return SELL_OK;
}

}  // namespace sell
