// sell_rowdot.cuh -- the per-row arithmetic shared by every SpMV kernel
// (single products in sell_spmv.cu, batches in sell_batch.cu), so that a row
// gives the same bits whichever kernel, launch shape, (C, sigma) or batch it
// runs in.
//
// Definition of a row's result (row length L, initial value y0 = 0, or the
// old y with SELL_SPMV_ACCUMULATE):
//   L <= kSeg : one chain over the entries in CRS order, starting at y0 --
//               s = fma(a_j, x_cj, s) (binary64 / binary32), or one Dot2 step;
//   L >  kSeg : the row is cut into segments of kSeg consecutive entries;
//               segment 0 is a chain starting at y0, every other segment a
//               chain starting at 0; the segment results are then added in
//               segment order (Dot2: merged with TwoSum, errors carried).
// The segments let one block work on a long chunk with many threads at once
// (Sec. 3.4 notes that one thread per row leaves a warp waiting for its
// longest row; Sec. 5.2 suggests several threads per row for such rows).
#pragma once

#include "sell_internal.cuh"

namespace sell {

template <class VT> struct XType;
template <> struct XType<double> { using T = double; };
template <> struct XType<float> { using T = float; };
template <> struct XType<__nv_bfloat16> { using T = float; };

__device__ __forceinline__ double widen(double v) { return v; }
__device__ __forceinline__ float widen(float v) { return v; }
__device__ __forceinline__ float widen(__nv_bfloat16 v) { return __bfloat162float(v); }

template <class AT>
struct Plain {
    AT s;
    __device__ __forceinline__ void init(AT y0) { s = y0; }
    __device__ __forceinline__ void add(AT a, AT b) { s = fma(a, b, s); }
    __device__ __forceinline__ void merge(const Plain &o) { s = s + o.s; }
    __device__ __forceinline__ AT result() const { return s; }
};

// Dot2 (Ogita, Rump, Oishi 2005): p is the running sum, e the sum of the
// exact rounding errors of every product (TwoProduct by FMA) and every
// addition (Knuth's TwoSum); the result p + e is rounded once.
struct Dot2 {
    float p, e;
    __device__ __forceinline__ void init(float y0) { p = y0; e = 0.0f; }
    __device__ __forceinline__ static void two_sum(float a, float b, float &t, float &q) {
        t = __fadd_rn(a, b);
        float z = __fsub_rn(t, a);
        q = __fadd_rn(__fsub_rn(a, __fsub_rn(t, z)), __fsub_rn(b, z));
    }
    __device__ __forceinline__ void add(float a, float b) {
        float h = __fmul_rn(a, b);
        float r = __fmaf_rn(a, b, -h);  // a*b = h + r exactly
        float t, q;
        two_sum(p, h, t, q);
        p = t;
        e = __fadd_rn(e, __fadd_rn(q, r));
    }
    __device__ __forceinline__ void merge(const Dot2 &o) {
        float t, q;
        two_sum(p, o.p, t, q);
        p = t;
        e = __fadd_rn(e, __fadd_rn(q, o.e));
    }
    __device__ __forceinline__ float result() const { return __fadd_rn(p, e); }
};

// K consecutive right-hand-side values of row `ci` of X (row-major, ldx).
template <int K, class XT>
__device__ __forceinline__ void load_x(const XT *__restrict__ X, int64_t ldx, int32_t ci, bool vec,
                                       XT (&xv)[K]) {
    const XT *p = X + (int64_t)ci * ldx;
    if constexpr (K == 1) {
        xv[0] = __ldg(p);
    } else {
        constexpr int V = 16 / sizeof(XT);  // elements per 16-byte vector
        if ((K % V) == 0 && vec) {
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

// One chain over entries j0..j1-1 of a row whose entry j sits at vp[j*C]
// (values) and cp[j*C] (columns).  U entries are loaded per step, predicated
// on j < j1, so that short rows still keep U loads in flight; the FMAs are
// applied in entry order.
template <class VT, class XT, int K, int U, class Acc>
__device__ __forceinline__ void chain(Acc (&acc)[K], const VT *__restrict__ vp,
                                      const int32_t *__restrict__ cp, int C, int j0, int j1,
                                      const XT *__restrict__ X, int64_t ldx, bool vec, uint64_t pol) {
    const int64_t stride = C;
    vp += (int64_t)j0 * stride;
    cp += (int64_t)j0 * stride;
    for (int j = j0; j < j1; j += U) {
        VT v[U];
        int32_t ci[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (j + u < j1) {
                v[u] = ld_stream(vp + u * stride, pol);
                ci[u] = ld_stream(cp + u * stride, pol);
            }
        }
        XT xv[U][K];
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (j + u < j1) load_x<K>(X, ldx, ci[u], vec, xv[u]);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (j + u < j1) {
                XT a = widen(v[u]);
#pragma unroll
                for (int q = 0; q < K; ++q) acc[q].add(a, xv[u][q]);
            }
        }
        vp += U * stride;
        cp += U * stride;
    }
}

// A block works on the long rows (L > kSeg) of chunk c.  Lp = min(C, block)
// lanes form a group; the G = block / Lp groups take segments g, g+G, ...;
// after every round the partial results go through shared memory and the
// first group folds them in segment order.  `part` holds block * K Accs.
template <class VT, class XT, int K, int U, class Acc>
__device__ __forceinline__ void long_chunk(const VT *__restrict__ val, const int32_t *__restrict__ col,
                                           const int64_t *__restrict__ cs, const int32_t *__restrict__ srl,
                                           const int32_t *__restrict__ cl, const int32_t *__restrict__ perm,
                                           const XT *__restrict__ X, int64_t ldx, XT *Y, int64_t ldy,
                                           int64_t N, int C, int64_t c, int accumulate, bool vec,
                                           uint64_t pol, Acc *part) {
    const int B = blockDim.x;
    const int Lp = C < B ? C : B;
    const int G = B / Lp;
    const int g = threadIdx.x / Lp;
    const int l0 = threadIdx.x - g * Lp;
    const int nseg_max = (cl[c] + kSeg - 1) / kSeg;
    const int rounds = (nseg_max + G - 1) / G;
    const int64_t base = cs[c];
    for (int lb = 0; lb < C; lb += Lp) {
        const int l = lb + l0;
        const int64_t r = c * C + l;
        const bool in = g < G && l < C && r < N;
        const int L = in ? srl[r] : 0;
        const bool active = in && L > kSeg;
        const int nseg = active ? (L + kSeg - 1) / kSeg : 0;
        const int64_t out = active ? (perm ? (int64_t)perm[r] : r) : 0;
        Acc tot[K];
        for (int k = 0; k < rounds; ++k) {
            const int s = k * G + g;
            if (active && s < nseg) {
                Acc acc[K];
#pragma unroll
                for (int q = 0; q < K; ++q)
                    acc[q].init((s == 0 && accumulate) ? Y[out * ldy + q] : XT(0));
                const int j0 = s * kSeg;
                const int j1 = min(L, j0 + kSeg);
                chain<VT, XT, K, U, Acc>(acc, val + base + l, col + base + l, C, j0, j1, X, ldx, vec, pol);
#pragma unroll
                for (int q = 0; q < K; ++q) part[threadIdx.x * K + q] = acc[q];
            }
            __syncthreads();
            if (g == 0 && active) {
                for (int gg = 0; gg < G; ++gg) {
                    const int s2 = k * G + gg;
                    if (s2 >= nseg) break;
#pragma unroll
                    for (int q = 0; q < K; ++q) {
                        const Acc &p = part[(gg * Lp + l0) * K + q];
                        if (s2 == 0) tot[q] = p;
                        else tot[q].merge(p);
                    }
                }
            }
            __syncthreads();
        }
        if (g == 0 && active) {
#pragma unroll
            for (int q = 0; q < K; ++q) Y[out * ldy + q] = tot[q].result();
        }
    }
}

// The thread's own row when it is short (L <= kSeg); long rows return.
template <class VT, class XT, int K, int U, class Acc>
__device__ __forceinline__ void short_row(const VT *__restrict__ val, const int32_t *__restrict__ col,
                                          const int64_t *__restrict__ cs, const int32_t *__restrict__ srl,
                                          const int32_t *__restrict__ perm, const XT *__restrict__ X,
                                          int64_t ldx, XT *Y, int64_t ldy, int C, int64_t r, int accumulate,
                                          bool vec, uint64_t pol) {
    const int L = srl[r];
    if (L > kSeg) return;
    const int64_t c = r / C;
    const int l = (int)(r - c * C);
    const int64_t out = perm ? (int64_t)perm[r] : r;
    const int64_t base = cs[c] + l;
    Acc acc[K];
#pragma unroll
    for (int q = 0; q < K; ++q) acc[q].init(accumulate ? Y[out * ldy + q] : XT(0));
    chain<VT, XT, K, U, Acc>(acc, val + base, col + base, C, 0, L, X, ldx, vec, pol);
#pragma unroll
    for (int q = 0; q < K; ++q) Y[out * ldy + q] = acc[q].result();
}

}  // namespace sell
