// sell_spmv_f64.cu -- SpMV / SpMMV kernels for double storage (instantiations
// of sell_spmv_impl.cuh, kept in their own translation unit to compile in
// parallel).
#include "sell_spmv_impl.cuh"

namespace sell {

cudaError_t spmv_block_f64(const sell_matrix *h, const void *X, int64_t ldx, void *Y, int64_t ldy, int kb,
                           int acc, int vec, void *part, int32_t *cnt, int32_t *cnt2, cudaStream_t s) {
    return spmv_block<double, Plain<double>>(h, X, ldx, Y, ldy, kb, acc, vec, part, cnt, cnt2, s);
}

// Resident blocks per SM of the bulk-staged kernels of this storage type.
int bulk_blocks_per_sm_f64(const sell_matrix *h, int W, int R) {
    int a = bulk::blocks_per_sm<double, Plain<double>>(h, W, R);
    return a;
}

}  // namespace sell
