// sell_spmv.cu -- SELL-C-sigma SpMV / SpMMV kernels for sm_103a.
//
// Mapping (Sec. 3.4, "Sliced ELLR-T" with T = 1; Sec. 5: one thread per row):
// thread r handles sorted row r = c*C + l and walks j < rowLen(r) over
// val[cs[c] + j*C + l] -- for a fixed j the C threads of a chunk read C
// consecutive elements, so every load of val/col is coalesced when C is a
// multiple of 32, and no thread loads its row's padding.  The result goes to
// y[perm[r]] (original order) or y[r] (permuted space).
//
// Memory behaviour: val/col are read exactly once per product (L1
// no-allocate, L2 evict-first); x is gathered through the read-only path and
// stays L2-resident.  U independent (val, col) pairs are issued before their
// x gathers so that each thread keeps several loads in flight.
//
// Arithmetic: each row is summed in CRS order with fused multiply-adds
// (binary64 for F64 storage; binary32 for F32/BF16 storage, optionally with
// the compensated Dot2 scheme: TwoProduct by FMA and Knuth's TwoSum, the
// error terms summed separately and added once at the end).  The order of
// operations inside a row does not depend on C, sigma, the launch shape or on
// how many right-hand sides are processed together.
#include "sell_internal.cuh"

namespace sell {
namespace {

template <class VT> struct Types;
template <> struct Types<double> { using X = double; };
template <> struct Types<float> { using X = float; };
template <> struct Types<__nv_bfloat16> { using X = float; };

__device__ __forceinline__ double widen(double v) { return v; }
__device__ __forceinline__ float widen(float v) { return v; }
__device__ __forceinline__ float widen(__nv_bfloat16 v) { return __bfloat162float(v); }

// K consecutive right-hand-side values of row `ci` of X (row-major, ldx).
template <int K, class XT>
__device__ __forceinline__ void load_x(const XT *__restrict__ X, int64_t ldx, int32_t ci, bool vec,
                                       XT (&xv)[K]) {
    const XT *p = X + (int64_t)ci * ldx;
    if constexpr (K == 1) {
        xv[0] = __ldg(p);
    } else {
        constexpr int V = 16 / sizeof(XT);  // elements per 16-byte vector
        if (vec && (K % V) == 0) {
            if constexpr (sizeof(XT) == 8) {
#pragma unroll
                for (int q = 0; q < K; q += 2) {
                    double2 t = __ldg(reinterpret_cast<const double2 *>(p + q));
                    xv[q] = t.x;
                    xv[q + 1] = t.y;
                }
            } else {
#pragma unroll
                for (int q = 0; q < K; q += 4) {
                    float4 t = __ldg(reinterpret_cast<const float4 *>(p + q));
                    xv[q] = t.x;
                    xv[q + 1] = t.y;
                    xv[q + 2] = t.z;
                    xv[q + 3] = t.w;
                }
            }
        } else {
#pragma unroll
            for (int q = 0; q < K; ++q) xv[q] = __ldg(p + q);
        }
    }
}

template <class AT>
struct Plain {
    AT s;
    __device__ __forceinline__ void init(AT y0) { s = y0; }
    __device__ __forceinline__ void add(AT a, AT b) { s = fma(a, b, s); }
    __device__ __forceinline__ AT result() const { return s; }
};

// Dot2 (Ogita, Rump, Oishi 2005): p carries the running sum, s the
// accumulated rounding errors of every product and every addition.
struct Dot2 {
    float p, s;
    __device__ __forceinline__ void init(float y0) { p = y0; s = 0.0f; }
    __device__ __forceinline__ void add(float a, float b) {
        float h = __fmul_rn(a, b);
        float r = __fmaf_rn(a, b, -h);  // exact: a*b = h + r
        float t = __fadd_rn(p, h);
        float z = __fsub_rn(t, p);
        float q = __fadd_rn(__fsub_rn(p, __fsub_rn(t, z)), __fsub_rn(h, z));  // p + h = t + q
        p = t;
        s = __fadd_rn(s, __fadd_rn(q, r));
    }
    __device__ __forceinline__ float result() const { return __fadd_rn(p, s); }
};

template <class VT, int K, int U, class Acc>
__global__ void __launch_bounds__(1024)
k_spmmv(const VT *__restrict__ val, const int32_t *__restrict__ col, const int64_t *__restrict__ cs,
        const int32_t *__restrict__ srl, const int32_t *__restrict__ perm,
        const typename Types<VT>::X *__restrict__ X, int64_t ldx, typename Types<VT>::X *Y,
        int64_t ldy, int64_t N, int C, int accumulate, int vec) {
    using XT = typename Types<VT>::X;
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= N) return;
    const int64_t c = r / C;
    const int l = (int)(r - c * C);
    const int len = srl[r];
    const int64_t out = perm ? (int64_t)perm[r] : r;
    const uint64_t pol = l2_evict_first_policy();
    const VT *vp = val + cs[c] + l;
    const int32_t *cp = col + cs[c] + l;

    Acc acc[K];
#pragma unroll
    for (int q = 0; q < K; ++q) acc[q].init(accumulate ? Y[out * ldy + q] : XT(0));

    int j = 0;
    for (; j + U <= len; j += U) {
        VT v[U];
        int32_t ci[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            v[u] = ld_stream(vp + (int64_t)u * C, pol);
            ci[u] = ld_stream(cp + (int64_t)u * C, pol);
        }
        XT xv[U][K];
#pragma unroll
        for (int u = 0; u < U; ++u) load_x<K>(X, ldx, ci[u], vec, xv[u]);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            XT a = widen(v[u]);
#pragma unroll
            for (int q = 0; q < K; ++q) acc[q].add(a, xv[u][q]);
        }
        vp += (int64_t)U * C;
        cp += (int64_t)U * C;
    }
    for (; j < len; ++j) {
        VT v = ld_stream(vp, pol);
        int32_t ci = ld_stream(cp, pol);
        XT xv[K];
        load_x<K>(X, ldx, ci, vec, xv);
        XT a = widen(v);
#pragma unroll
        for (int q = 0; q < K; ++q) acc[q].add(a, xv[q]);
        vp += C;
        cp += C;
    }
#pragma unroll
    for (int q = 0; q < K; ++q) Y[out * ldy + q] = acc[q].result();
}

template <class VT, int K, int U, class Acc>
cudaError_t run(const sell_matrix *h, const void *X, int64_t ldx, void *Y, int64_t ldy, int acc,
                int vec, cudaStream_t s) {
    using XT = typename Types<VT>::X;
    const int64_t grid = (h->nrows + h->block - 1) / h->block;
    k_spmmv<VT, K, U, Acc><<<(unsigned)grid, h->block, 0, s>>>(
        static_cast<const VT *>(h->val), h->col, h->cs, h->srl,
        (h->flags & SELL_BUILD_PERMUTE_COLS) ? nullptr : h->perm,
        static_cast<const XT *>(X), ldx, static_cast<XT *>(Y), ldy, h->nrows, h->C, acc, vec);
    return cudaGetLastError();
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
sell_status launch_spmmv(const sell_matrix *h, const void *X, int64_t ldx, void *Y, int64_t ldy,
                         int32_t k, uint32_t flags, cudaStream_t s) {
    if (h->nrows == 0) return SELL_OK;
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

}  // namespace sell
