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
//               segment order (binary32 chains: in binary64, rounded to
//               binary32 once at the end; Dot2: merged with TwoSum, errors
//               carried) -- for more than kSuper (256) segments, first within
//               each group of kSuper consecutive segments, then the group
//               results in order.
// Every segment of a long row is an independent work unit, so long rows are
// spread over the whole grid instead of holding one warp for their full
// length (Sec. 3.4 notes that one thread per row leaves a warp waiting for
// its longest row; Sec. 5.2 suggests several threads per row for such rows).
// A segment's partial result goes to scratch memory; the thread that
// completes the last segment of a row (per-row counter) folds the partials
// in segment order, so the result does not depend on which segment finished
// last.
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
    __device__ __forceinline__ static Plain load_l2(const Plain *p) {
        Plain r;
        r.s = __ldcg(&p->s);
        return r;
    }
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
    __device__ __forceinline__ static Dot2 load_l2(const Dot2 *q) {
        float2 t = __ldcg(reinterpret_cast<const float2 *>(q));
        Dot2 r;
        r.p = t.x;
        r.e = t.y;
        return r;
    }
};

// The type a long row's segment partials are kept and folded in.  Binary32
// chains (Plain<float>) are folded in binary64 -- a segment result converts
// exactly, the fold rounds in binary64, and the row's result is rounded to
// binary32 once at the end; binary64 and Dot2 fold in their own type.  Every
// partial slot of the scratch is 8 bytes, so both fit.
template <class Acc>
struct PartOf {
    using T = Acc;
    __device__ __forceinline__ static T from(const Acc &a) { return a; }
};
template <>
struct PartOf<Plain<float>> {
    using T = Plain<double>;
    __device__ __forceinline__ static T from(const Plain<float> &a) {
        T t;
        t.s = (double)a.s;
        return t;
    }
};

// 32 bytes of x at p (32-byte aligned) in one 256-bit load (sm_100 and later).
__device__ __forceinline__ void ld_x32(const float *p, float *v) {
    asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
        : "l"(p));
}
__device__ __forceinline__ void ld_x32(const double *p, double *v) {
    asm("ld.global.nc.v4.f64 {%0,%1,%2,%3}, [%4];" : "=d"(v[0]), "=d"(v[1]), "=d"(v[2]), "=d"(v[3]) : "l"(p));
}

// K consecutive right-hand-side values of row `ci` of X (row-major, ldx).
// vec & 3: 2 when X and its row pitch are 32-byte aligned (rows of a
// multiple of 32 bytes then take one 256-bit load per 32 bytes: a random row
// costs one L1 request instead of two), 1 when they are 16-byte aligned
// (16-byte vector loads), 0 otherwise (one load per value); bits 2-3 hold the
// same for Y (store_y).  The values loaded are the same in every case.
template <int K, class XT>
__device__ __forceinline__ void load_x(const XT *__restrict__ X, int64_t ldx, int32_t ci, int vec,
                                       XT (&xv)[K]) {
    const XT *p = X + (int64_t)ci * ldx;
    vec &= 3;
    if constexpr (K == 1) {
        xv[0] = __ldg(p);
    } else {
        constexpr int V = 16 / sizeof(XT);  // elements per 16-byte vector
        constexpr int W = 32 / sizeof(XT);  // elements per 32-byte vector
        if ((K % W) == 0 && vec >= 2) {
#pragma unroll
            for (int q = 0; q < K; q += W) ld_x32(p + q, xv + q);
        } else if ((K % V) == 0 && vec) {
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

// 32 bytes of Y at p (32-byte aligned) in one 256-bit store or load.
__device__ __forceinline__ void st_y32(float *p, const float *v) {
    asm volatile("st.global.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "f"(v[0]), "f"(v[1]), "f"(v[2]),
                 "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7])
                 : "memory");
}
__device__ __forceinline__ void st_y32(double *p, const double *v) {
    asm volatile("st.global.v4.f64 [%0], {%1,%2,%3,%4};" ::"l"(p), "d"(v[0]), "d"(v[1]), "d"(v[2]), "d"(v[3])
                 : "memory");
}
__device__ __forceinline__ void ld_y32(const float *p, float *v) {
    asm volatile("ld.global.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
                 : "l"(p)
                 : "memory");
}
__device__ __forceinline__ void ld_y32(const double *p, double *v) {
    asm volatile("ld.global.v4.f64 {%0,%1,%2,%3}, [%4];"
                 : "=d"(v[0]), "=d"(v[1]), "=d"(v[2]), "=d"(v[3])
                 : "l"(p)
                 : "memory");
}

// Row i of Y (K values, row-major, ldy) written, or read for accumulation,
// with the widest vectors that bits 2-3 of vec allow (the layout of load_x).
// One vector store per 32 bytes instead of K scalar stores: each scalar
// store of a scattered row is an L2 request of its own.
template <int K, class XT>
__device__ __forceinline__ void store_y(XT *Y, int64_t ldy, int64_t i, int vec, const XT (&v)[K]) {
    XT *p = Y + i * ldy;
    const int yv = (vec >> 2) & 3;
    if constexpr (K == 1) {
        p[0] = v[0];
    } else {
        constexpr int V = 16 / sizeof(XT);
        constexpr int W = 32 / sizeof(XT);
        if ((K % W) == 0 && yv >= 2) {
#pragma unroll
            for (int q = 0; q < K; q += W) st_y32(p + q, v + q);
        } else if ((K % V) == 0 && yv) {
            if constexpr (sizeof(XT) == 8) {
#pragma unroll
                for (int q = 0; q < K; q += 2) *reinterpret_cast<double2 *>(p + q) = make_double2(v[q], v[q + 1]);
            } else {
#pragma unroll
                for (int q = 0; q < K; q += 4)
                    *reinterpret_cast<float4 *>(p + q) = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
            }
        } else {
#pragma unroll
            for (int q = 0; q < K; ++q) p[q] = v[q];
        }
    }
}
template <int K, class XT>
__device__ __forceinline__ void load_y(const XT *Y, int64_t ldy, int64_t i, int vec, XT (&v)[K]) {
    const XT *p = Y + i * ldy;
    const int yv = (vec >> 2) & 3;
    if constexpr (K == 1) {
        v[0] = p[0];
    } else {
        constexpr int V = 16 / sizeof(XT);
        constexpr int W = 32 / sizeof(XT);
        if ((K % W) == 0 && yv >= 2) {
#pragma unroll
            for (int q = 0; q < K; q += W) ld_y32(p + q, v + q);
        } else if ((K % V) == 0 && yv) {
            if constexpr (sizeof(XT) == 8) {
#pragma unroll
                for (int q = 0; q < K; q += 2) {
                    const double2 t = *reinterpret_cast<const double2 *>(p + q);
                    v[q] = t.x;
                    v[q + 1] = t.y;
                }
            } else {
#pragma unroll
                for (int q = 0; q < K; q += 4) {
                    const float4 t = *reinterpret_cast<const float4 *>(p + q);
                    v[q] = t.x;
                    v[q + 1] = t.y;
                    v[q + 2] = t.z;
                    v[q + 3] = t.w;
                }
            }
        } else {
#pragma unroll
            for (int q = 0; q < K; ++q) v[q] = p[q];
        }
    }
}

// One chain over entries j0..j1-1 of a row whose entry j sits at vp[j*C]
// (values) and cp[j*C] (columns), in entry order.  Full groups of U entries
// are loaded before their gathers and FMAs; the last, partial group is loaded
// with predicates so that short rows keep all their loads in flight.  With
// PIPE the stream loads of the next group are issued before the gathers and
// FMAs of the current one (software pipelining: more bytes in flight per
// thread; the order of the FMAs is unchanged).
template <class VT, class XT, int K, int U, bool PIPE, class Acc>
__device__ __forceinline__ void chain(Acc (&acc)[K], const VT *__restrict__ vp,
                                      const int32_t *__restrict__ cp, int C, int j0, int j1,
                                      const XT *__restrict__ X, int64_t ldx, int vec, uint64_t pol) {
    const int64_t stride = C;
    vp += (int64_t)j0 * stride;
    cp += (int64_t)j0 * stride;
    int j = j0;
    if constexpr (PIPE) {
        if (j + U <= j1) {
            VT v[U];
            int32_t ci[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                v[u] = ld_stream(vp + u * stride, pol);
                ci[u] = ld_stream(cp + u * stride, pol);
            }
            for (;;) {
                const bool more = j + 2 * U <= j1;
                VT vn[U];
                int32_t cn[U];
                if (more) {
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        vn[u] = ld_stream(vp + (U + u) * stride, pol);
                        cn[u] = ld_stream(cp + (U + u) * stride, pol);
                    }
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
                vp += U * stride;
                cp += U * stride;
                j += U;
                if (!more) break;
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    v[u] = vn[u];
                    ci[u] = cn[u];
                }
            }
        }
    } else {
        for (; j + U <= j1; j += U) {
            VT v[U];
            int32_t ci[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                v[u] = ld_stream(vp + u * stride, pol);
                ci[u] = ld_stream(cp + u * stride, pol);
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
            vp += U * stride;
            cp += U * stride;
        }
    }
    if constexpr (U > 1) {
        if (j < j1) {
            VT v[U];
            int32_t ci[U];
#pragma unroll
            for (int u = 0; u < U - 1; ++u) {
                if (j + u < j1) {
                    v[u] = ld_stream(vp + u * stride, pol);
                    ci[u] = ld_stream(cp + u * stride, pol);
                }
            }
            XT xv[U][K];
#pragma unroll
            for (int u = 0; u < U - 1; ++u)
                if (j + u < j1) load_x<K>(X, ldx, ci[u], vec, xv[u]);
#pragma unroll
            for (int u = 0; u < U - 1; ++u) {
                if (j + u < j1) {
                    XT a = widen(v[u]);
#pragma unroll
                    for (int q = 0; q < K; ++q) acc[q].add(a, xv[u][q]);
                }
            }
        }
    }
}

// Fold `count` partials of lane l, found at units base, base + stride, ...,
// in that order (loads issued FB at a time, folds strictly in order).
template <int K, class Acc>
__device__ __forceinline__ void fold_partials(const Acc *part, int64_t base, int64_t stride, int count, int C,
                                              int l, Acc (&tot)[K]) {
#pragma unroll
    for (int q = 0; q < K; ++q) tot[q] = Acc::load_l2(part + (base * C + l) * K + q);
    constexpr int FB = K >= 8 ? 2 : (K >= 4 ? 4 : 16 / K);
    int i = 1;
    for (; i + FB <= count; i += FB) {
        Acc buf[FB][K];
#pragma unroll
        for (int f = 0; f < FB; ++f)
#pragma unroll
            for (int q = 0; q < K; ++q) buf[f][q] = Acc::load_l2(part + ((base + (i + f) * stride) * C + l) * K + q);
#pragma unroll
        for (int f = 0; f < FB; ++f)
#pragma unroll
            for (int q = 0; q < K; ++q) tot[q].merge(buf[f][q]);
    }
    for (; i < count; ++i) {
#pragma unroll
        for (int q = 0; q < K; ++q) tot[q].merge(Acc::load_l2(part + ((base + i * stride) * C + l) * K + q));
    }
}

// One thread of a long-row work unit.  Units are (long chunk lc, segment s)
// pairs, numbered chunk by chunk (lunit[u] = {lc, s}); a unit has C threads,
// virtual thread v = u*C + l takes lane l.  part holds K Accs per (unit,
// lane); cnt one counter per (long chunk, lane) and cnt2 one per (unit,
// lane), all zero between products.
//
// Folding: a row of at most kSuper segments is folded in segment order by the
// thread that completes its last segment.  A longer row folds in two levels:
// each group of kSuper consecutive segments is folded in order by the thread
// that completes the group (its result replaces the group's first partial),
// then the thread that completes the last group folds the group results in
// order.  Either way the result depends only on the row's entries.
template <class VT, class XT, int K, int U, bool PIPE, class Acc>
__device__ __forceinline__ void long_unit(const VT *__restrict__ val, const int32_t *__restrict__ col,
                                          const int64_t *__restrict__ cs, const int32_t *__restrict__ srl,
                                          const int32_t *__restrict__ perm, const int32_t *__restrict__ lchunk,
                                          const int2 *__restrict__ lunit, const int4 *__restrict__ lmeta,
                                          const int32_t *__restrict__ lrow, Acc *part, int32_t *cnt,
                                          int32_t *cnt2, const XT *__restrict__ X, int64_t ldx, XT *Y,
                                          int64_t ldy, int64_t N, int C, int64_t v, int accumulate, int vec,
                                          uint64_t pol) {
    const int64_t u = v / C;
    const int t = (int)(v - u * C);
    const int2 us = lunit[u];
    const int4 meta = lmeta[us.x];
    int l, s;
    if (meta.y == 0) {  // thread t takes lane t
        l = t;
        s = us.y;
    } else {  // the chunk's threads take consecutive segments of each long row
        const int64_t i = (int64_t)us.y * C + t;  // beyond 32 bits for rows of more than 2^31 / C segments
        const int64_t k = i / meta.z;
        if (k >= meta.x) return;
        s = (int)(i - k * meta.z);
        l = lrow[(int64_t)us.x * C + k];
    }
    const int64_t c = lchunk[us.x];
    const int64_t r = c * C + l;
    if (r >= N) return;
    const int L = srl[r];
    if (L <= kSeg) return;  // short rows belong to the per-row path
    const int nseg = (L - 1) / kSeg + 1;  // L > kSeg here; no overflow near 2^31
    if (s >= nseg) return;
    const int64_t u0 = u - us.y;  // the chunk's first unit; segment s's partial sits in unit u0 + s
    const int64_t out = perm ? (int64_t)perm[r] : r;
    Acc acc[K];
#pragma unroll
    for (int q = 0; q < K; ++q) acc[q].init((s == 0 && accumulate) ? Y[out * ldy + q] : XT(0));
    const int64_t base = cs[c] + l;
    chain<VT, XT, K, U, PIPE, Acc>(acc, val + base, col + base, C, s * kSeg, min(L, (s + 1) * kSeg), X, ldx,
                                   vec & 3, pol);
    using PT = typename PartOf<Acc>::T;
    PT *pp = reinterpret_cast<PT *>(part);
#pragma unroll
    for (int q = 0; q < K; ++q) pp[((u0 + s) * C + l) * K + q] = PartOf<Acc>::from(acc[q]);
    int32_t *ct = cnt + (int64_t)us.x * C + l;
    PT tot[K];
    if (nseg <= kSuper) {
        __threadfence();
        if (atomicAdd(ct, 1) != nseg - 1) return;
        __threadfence();  // this thread completed the row
        fold_partials<K, PT>(pp, u0, 1, nseg, C, l, tot);
    } else {
        const int s0 = (s / kSuper) * kSuper;
        const int ng = min(kSuper, nseg - s0);
        int32_t *cg = cnt2 + (u0 + s0) * C + l;
        __threadfence();
        if (atomicAdd(cg, 1) != ng - 1) return;
        __threadfence();  // this thread completed the group
        fold_partials<K, PT>(pp, u0 + s0, 1, ng, C, l, tot);
        *cg = 0;
#pragma unroll
        for (int q = 0; q < K; ++q) pp[((u0 + s0) * C + l) * K + q] = tot[q];
        __threadfence();
        const int ngroups = (nseg + kSuper - 1) / kSuper;
        if (atomicAdd(ct, 1) != ngroups - 1) return;
        __threadfence();  // ... and the last group of the row
        fold_partials<K, PT>(pp, u0, kSuper, ngroups, C, l, tot);
    }
#pragma unroll
    for (int q = 0; q < K; ++q) Y[out * ldy + q] = static_cast<XT>(tot[q].result());
    *ct = 0;
}

// The thread's own row when it is short (L <= kSeg); long rows return.
template <class VT, class XT, int K, int U, bool PIPE, class Acc>
__device__ __forceinline__ void short_row(const VT *__restrict__ val, const int32_t *__restrict__ col,
                                          const int64_t *__restrict__ cs, const int32_t *__restrict__ srl,
                                          const int32_t *__restrict__ perm, const XT *__restrict__ X,
                                          int64_t ldx, XT *Y, int64_t ldy, int C, int64_t r, int accumulate,
                                          int vec, uint64_t pol) {
    const int L = srl[r];
    if (L > kSeg) return;
    const int64_t c = r / C;
    const int l = (int)(r - c * C);
    const int64_t out = perm ? (int64_t)perm[r] : r;
    const int64_t base = cs[c] + l;
    Acc acc[K];
    if (accumulate) {
        XT y0[K];
        load_y<K>(Y, ldy, out, vec, y0);
#pragma unroll
        for (int q = 0; q < K; ++q) acc[q].init(y0[q]);
    } else {
#pragma unroll
        for (int q = 0; q < K; ++q) acc[q].init(XT(0));
    }
    chain<VT, XT, K, U, PIPE, Acc>(acc, val + base, col + base, C, 0, L, X, ldx, vec & 3, pol);
    XT yo[K];
#pragma unroll
    for (int q = 0; q < K; ++q) yo[q] = acc[q].result();
    store_y<K>(Y, ldy, out, vec, yo);
}

}  // namespace sell
