// sell_spmv_f32.cu -- SpMV / SpMMV kernels for float storage (instantiations
// of sell_spmv_impl.cuh, kept in their own translation unit to compile in
// parallel).
#include "sell_spmv_impl.cuh"

namespace sell {

cudaError_t spmv_block_f32(const sell_matrix *h, const void *X, int64_t ldx, void *Y, int64_t ldy, int kb,
                           int acc, int vec, int comp, void *part, int32_t *cnt, int32_t *cnt2, cudaStream_t s) {
    if (comp == 1) return spmv_block<float, Dot2>(h, X, ldx, Y, ldy, kb, acc, vec, part, cnt, cnt2, s);
    if (comp == 2)  // Dot2 on the long rows only
        return spmv_block<float, Plain<float>, Dot2>(h, X, ldx, Y, ldy, kb, acc, vec, part, cnt, cnt2, s);
    return spmv_block<float, Plain<float>>(h, X, ldx, Y, ldy, kb, acc, vec, part, cnt, cnt2, s);
}

// Resident blocks per SM of the bulk-staged kernels of this storage type.
int bulk_blocks_per_sm_f32(const sell_matrix *h, int W, int R) {
    int a = bulk::blocks_per_sm<float, Plain<float>>(h, W, R);
    int b = bulk::blocks_per_sm<float, Dot2>(h, W, R);
    return a < b ? a : b;
}

}  // namespace sell
