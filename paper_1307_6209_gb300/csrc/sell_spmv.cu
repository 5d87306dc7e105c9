// sell_spmv.cu -- host side of the SELL-C-sigma SpMV / SpMMV: splits the
// right-hand sides into column blocks of 8/4/2/1, grows the long-row scratch
// and dispatches to the per-type kernels (sell_spmv_impl.cuh, instantiated in
// sell_spmv_f64.cu, sell_spmv_f32.cu, sell_spmv_bf16.cu).

#include "sell_internal.cuh"

namespace sell {

// per-type entry points (sell_spmv_f64.cu / sell_spmv_f32.cu / sell_spmv_bf16.cu)
cudaError_t spmv_block_f64(const sell_matrix *h, const void *X, int64_t ldx, void *Y, int64_t ldy, int kb,
                           int acc, int vec, void *part, int32_t *cnt, int32_t *cnt2, cudaStream_t s);
cudaError_t spmv_block_f32(const sell_matrix *h, const void *X, int64_t ldx, void *Y, int64_t ldy, int kb,
                           int acc, int vec, int comp, void *part, int32_t *cnt, int32_t *cnt2, cudaStream_t s);
cudaError_t spmv_block_bf16(const sell_matrix *h, const void *X, int64_t ldx, void *Y, int64_t ldy, int kb,
                            int acc, int vec, int comp, void *part, int32_t *cnt, int32_t *cnt2, cudaStream_t s);

int bulk_blocks_per_sm_f64(const sell_matrix *h, int W, int R);
int bulk_blocks_per_sm_f32(const sell_matrix *h, int W, int R);
int bulk_blocks_per_sm_bf16(const sell_matrix *h, int W, int R);

namespace {

cudaError_t dispatch(const sell_matrix *h, const void *X, int64_t ldx, void *Y, int64_t ldy, int kb, int acc,
                     int vec, int comp, void *part, int32_t *cnt, int32_t *cnt2, cudaStream_t s) {
    switch (h->store_type) {
        case SELL_F64: return spmv_block_f64(h, X, ldx, Y, ldy, kb, acc, vec, part, cnt, cnt2, s);
        case SELL_F32: return spmv_block_f32(h, X, ldx, Y, ldy, kb, acc, vec, comp, part, cnt, cnt2, s);
        default: return spmv_block_bf16(h, X, ldx, Y, ldy, kb, acc, vec, comp, part, cnt, cnt2, s);
    }
}

}  // namespace

// Splits k into kernel blocks of 8, 4, 2, 1 columns, at most the flags' block
// width (every column keeps the same per-row operation order, so the split
// does not change any result).  The segment scratch grows on the first
// product with a wider block.
sell_status launch_spmmv(sell_matrix *h, const void *X, int64_t ldx, void *Y, int64_t ldy,
                         int32_t k, uint32_t flags, cudaStream_t s) {
    if (h->nrows == 0) return SELL_OK;
    const int maxw = max_rhs_block(flags);
    if (h->nunits > 0) {
        const int need = rhs_block(k, maxw);
        if (need > h->part_k) {
            void *p = h->al.get((size_t)h->nunits * h->C * need * 8, s);
            if (!p) return fail(SELL_ENOMEM, "segment scratch allocation failed");
            h->al.put(h->part, s);
            h->part = p;
            h->part_k = need;
        }
    }
    const int acc = (flags & SELL_SPMV_ACCUMULATE) ? 1 : 0;
    const int comp = comp_mode(flags);
    const size_t xs = h->store_type == SELL_F64 ? 8 : 4;
    int32_t done = 0;
    while (done < k) {
        const int kb = rhs_block(k - done, maxw);
        const char *Xb = static_cast<const char *>(X) + (size_t)done * xs;
        char *Yb = static_cast<char *>(Y) + (size_t)done * xs;
        int vec = x_vec(Xb, ldx, xs) | (x_vec(Yb, ldy, xs) << 2);
        cudaError_t e = dispatch(h, Xb, ldx, Yb, ldy, kb, acc, vec, comp, nullptr, nullptr, nullptr, s);
        if (e != cudaSuccess) return cuda_fail(e, "SpMV kernel launch");
        done += kb;
    }
    return SELL_OK;
}

// One column block of up to 8 right-hand sides with the given segment scratch
// `part` (nunits * C * kb * 8 bytes) and zeroed counters `cnt` (nlong * C) and
// `cnt2` (nunits * C).
sell_status launch_block_with_scratch(const sell_matrix *h, const void *X, int64_t ldx, void *Y,
                                      int64_t ldy, int kb, uint32_t flags, void *part, int32_t *cnt,
                                      int32_t *cnt2, cudaStream_t s) {
    const int acc = (flags & SELL_SPMV_ACCUMULATE) ? 1 : 0;
    const int comp = comp_mode(flags);
    const size_t xs = h->store_type == SELL_F64 ? 8 : 4;
    const int vec = x_vec(X, ldx, xs) | (x_vec(Y, ldy, xs) << 2);
    cudaError_t e = dispatch(h, X, ldx, Y, ldy, kb, acc, vec, comp, part, cnt, cnt2, s);
    if (e != cudaSuccess) return cuda_fail(e, "SpMV kernel launch");
    return SELL_OK;
}

// Launch shape and work split of the bulk-staged SpMV for the handle's
// block (warps per block) and unroll (slots per warp: 1, 2, 3, 4 for unroll
// 1, 2, 4, 8; fewer if shared memory does not hold them): one persistent
// wave, every SM filled with as many blocks as fit.
sell_status bulk_prepare(sell_matrix *h) {
    h->bulk_grid = 0;  // the bulk kernel stays off until the plan below exists
    if (h->C != 32 && h->C != 64 && h->C != 128)
        return fail(SELL_EUNSUPPORTED, "bulk-staged SpMV needs C = 32, 64 or 128");
    // bulk copies need 16-byte aligned sources (chunk offsets are multiples of C)
    if (((uintptr_t)h->val | (uintptr_t)h->col | (uintptr_t)h->srl) % 16 != 0)
        return fail(SELL_EUNSUPPORTED, "bulk-staged SpMV needs 16-byte aligned format arrays");
    const int W = h->block / 32;
    int R = h->unroll >= 8 ? 4 : (h->unroll >= 4 ? 3 : (h->unroll >= 2 ? 2 : 1));
    int bps = 0;
    for (; R >= 1; --R) {
        switch (h->store_type) {
            case SELL_F64: bps = bulk_blocks_per_sm_f64(h, W, R); break;
            case SELL_F32: bps = bulk_blocks_per_sm_f32(h, W, R); break;
            default: bps = bulk_blocks_per_sm_bf16(h, W, R); break;
        }
        if (bps > 0) break;
    }
    if (bps <= 0) return fail(SELL_EUNSUPPORTED, "bulk-staged SpMV: the block does not fit on an SM");
    int nsm = 0;
    SELL_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device));
    const int grid = nsm * bps;
    SELL_TRY(bulk_plan(h, (int64_t)grid * W, nullptr));
    h->bulk_grid = grid;
    h->bulk_warps = W;
    h->bulk_ring = R;
    return SELL_OK;
}

}  // namespace sell
