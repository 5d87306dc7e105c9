// sell_spmv_f64.cu -- SpMV / SpMMV kernels for double storage (instantiations
// of sell_spmv_impl.cuh, kept in their own translation unit to compile in
// parallel).
#include "sell_spmv_impl.cuh"

namespace sell {

cudaError_t spmv_block_f64(const sell_matrix *h, const void *X, int64_t ldx, void *Y, int64_t ldy, int kb,
                           int acc, int vec, void *part, int32_t *cnt, int32_t *cnt2, cudaStream_t s) {
    return spmv_block<double, Plain<double>>(h, X, ldx, Y, ldy, kb, acc, vec, part, cnt, cnt2, s);
}

}  // namespace sell
