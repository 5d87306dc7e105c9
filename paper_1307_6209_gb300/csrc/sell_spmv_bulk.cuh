// sell_spmv_bulk.cuh -- the bulk-staged SpMV (one right-hand side, C = 32,
// 64 or 128), included by the per-type translation units.
//
// The same product as k_spmmv (Listing "sell", one thread per row, Sec. 3.4 /
// Sec. 5), with a different route for the matrix stream: instead of every
// thread loading its own val/col entries, each warp copies whole pieces of
// its chunks into shared memory with asynchronous bulk copies
// (cp.async.bulk, completion counted on an mbarrier) and its lanes read them
// from there.  The warp's load/store unit then only carries the gathers of x,
// and the copies of the next pieces are in flight while the current piece is
// multiplied.
//
// Work split.  Rows of at most kSeg entries ("short rows") are taken from a
// per-warp stream: warp w owns the chunks [wsplit[w], wsplit[w+1]), balanced
// by bsc[c] + 1, where bsc[c] = the longest short row of chunk c, or -1 if
// the chunk has none.  A chunk of short rows is staged whole, a chunk that
// also holds long rows up to its longest short row, a chunk of long rows not
// at all; a chunk of empty rows is one piece with no columns (its rows still
// get their result).  Rows longer than kSeg are the long-row work units of
// sell_rowdot.cuh, spread over the warps before their streams start.  The arithmetic of every row is the
// one of sell_rowdot.cuh, so the result is bitwise that of k_spmmv.
//
// Pipeline per warp (R slots of kStageElems elements): lane 0 issues the copy
// of piece k + R - 1 into the slot that piece k - 1 used, then all lanes wait
// for piece k, gather x for all its entries at once, and run the FMA chains
// in entry order.  With R = 1 (one piece per warp, twice the resident warps
// of R = 2) the next piece is issued once the current one is consumed.  Every wait is bounded (kWaitNs); a wait that gives up sets
// *dstat, waits (bounded) for the warp's copies still in flight and ends the
// warp, and sell_check reports it.  For testing that route, a launch may ask
// (Args::expire_ns) that the first warp of the grid first waits, with that
// short limit, on a barrier that nothing ever completes; the warp's real
// copies are then drained with the normal limit before it ends.
#pragma once

#include "sell_rowdot.cuh"

namespace sell {
namespace bulk {

constexpr int kStageElems = 512;                // val/col elements per piece
constexpr int kMaxC = 128;                      // largest C of the bulk path
constexpr unsigned long long kWaitNs = 2000000000ull;  // bounded wait: 2 s

template <class VT>
struct Slot {  // byte offsets inside one slot (all 16-byte aligned)
    static constexpr int val = 0;
    static constexpr int col = kStageElems * (int)sizeof(VT);
    static constexpr int srl = col + kStageElems * 4;
    static constexpr int desc = srl + kMaxC * 4;
    static constexpr int bytes = desc + 16;
};

// Byte size of the barrier region: R barriers per warp plus one that no copy
// ever completes (the test barrier of Args::expire_ns).
constexpr int bars_bytes(int W, int R) { return ((W * R + 1) * 8 + 15) / 16 * 16; }

// Dynamic shared memory of a block of W warps with R slots each.
template <class VT>
constexpr size_t smem_bytes(int W, int R) {
    return (size_t)bars_bytes(W, R) + (size_t)W * R * Slot<VT>::bytes;
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for the phase of the given parity to complete; false after limit_ns
// (or 2^26 polls) without completion.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint64_t limit_ns = kWaitNs) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t i = 0; i < (1u << 26); ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 255u) == 255u && global_ns() - t0 > limit_ns) return false;
    }
    return false;
}

// Global -> shared bulk copy; bytes and both addresses are multiples of 16.
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar,
                                          uint64_t pol) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1], %2, [%3], %4;" ::"r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(pol)
        : "memory");
}

template <class VT, class Acc>
struct Args {
    const VT *val;
    const int32_t *col;
    const int64_t *cs;
    const int32_t *srl;
    const int32_t *perm;     // null: permuted-space output
    const int32_t *bsc;      // staged columns per chunk (-1: none, no short rows)
    const int32_t *wsplit;   // nwarps + 1 chunk boundaries
    const int32_t *lchunk;
    const int2 *lunit;
    const int4 *lmeta;
    const int32_t *lrow;
    Acc *part;
    int32_t *cnt, *cnt2;
    int32_t *dstat;
    const typename XType<VT>::T *X;
    typename XType<VT>::T *Y;
    int64_t ldx, ldy, N, long_threads;
    int ring, accumulate;
    uint64_t expire_ns;  // 0, or: warp 0 of block 0 first waits this long on the test barrier
};

// RPL = C / 32 rows per lane: lane l of a warp takes rows l, l + 32, ... of
// each of its chunks.
template <class VT, class Acc, int RPL, bool LONG>
__global__ void __launch_bounds__(512) k_spmv_bulk(const __grid_constant__ Args<VT, Acc> a) {
    using XT = typename XType<VT>::T;
    using S = Slot<VT>;
    constexpr int C = RPL * 32;
    constexpr int T = kStageElems / C;  // chunk columns per piece
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, W = blockDim.x >> 5;
    const int R = a.ring;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem) + warp * R;
    uint64_t *never = reinterpret_cast<uint64_t *>(smem) + W * R;  // no copy ever completes it
    unsigned char *slots = smem + bars_bytes(W, R) + (size_t)warp * R * S::bytes;
    const int64_t wg = (int64_t)blockIdx.x * W + warp;
    const int64_t NW = (int64_t)gridDim.x * W;
    const uint64_t pol = l2_evict_first_policy();

    if (lane == 0) {
        for (int i = 0; i < R; ++i) mbar_init(bars + i, 1);
        if (warp == 0) mbar_init(never, 1);
        fence_mbar_init();
    }
    __syncwarp();

    // ---- producer: the warp's pieces in order (state is warp-uniform)
    const int64_t ce = a.wsplit[wg + 1];
    int64_t pc = a.wsplit[wg];  // chunk of the next piece
    int pj = 0;                 // its first column
    int64_t wbase = -1;         // metadata window: lane i holds chunk wbase + i
    int64_t wcs = 0;
    int wsc = 0;
    int64_t issued = 0;
    auto issue_next = [&]() -> bool {
        for (;;) {
            if (pc >= ce) return false;
            if (wbase < 0 || pc - wbase >= 32) {
                wbase = pc;
                const int64_t cc = pc + lane;
                wcs = cc < ce ? a.cs[cc] : 0;
                wsc = cc < ce ? a.bsc[cc] : 0;
            }
            const int i = (int)(pc - wbase);
            const int sc = __shfl_sync(0xffffffffu, wsc, i);
            if (sc >= 0) {  // the chunk has short rows: piece (pc, pj), pj < sc or sc == 0
                const int64_t c0 = __shfl_sync(0xffffffffu, wcs, i);
                const int n = min(T, sc - pj);
                const bool last = pj + n >= sc;
                const int slot = (int)(issued % R);
                unsigned char *sp = slots + (size_t)slot * S::bytes;
                if (lane == 0) {
                    int4 d;
                    d.x = (int)(uint32_t)pc;
                    d.y = (int)(pc >> 32);
                    d.z = pj | (last ? (1 << 16) : 0);
                    d.w = n;
                    *reinterpret_cast<int4 *>(sp + S::desc) = d;
                    const uint32_t vb = (uint32_t)(n * C * sizeof(VT)), cb = (uint32_t)(n * C * 4);
                    const uint32_t sb = pj == 0 ? (uint32_t)(C * 4) : 0u;
                    fence_proxy_async();  // earlier reads of this slot precede the copy's writes
                    mbar_expect_tx(bars + slot, vb + cb + sb);
                    const int64_t e0 = c0 + (int64_t)pj * C;
                    if (n > 0) {
                        bulk_load(sp + S::val, a.val + e0, vb, bars + slot, pol);
                        bulk_load(sp + S::col, a.col + e0, cb, bars + slot, pol);
                    }
                    if (sb) bulk_load(sp + S::srl, a.srl + pc * C, sb, bars + slot, pol);
                }
                ++issued;
                if (last) {
                    ++pc;
                    pj = 0;
                } else {
                    pj += n;
                }
                return true;
            }
            ++pc;  // only long rows: the long-row units cover the chunk
            pj = 0;
        }
    };

    for (int i = 0; i < (R > 1 ? R - 1 : 1); ++i)
        if (!issue_next()) break;
    __syncwarp();

    // ---- long-row work units first (their copies above are already in flight)
    if constexpr (LONG) {
        for (int64_t v = wg * 32 + lane; v < a.long_threads; v += NW * 32)
            long_unit<VT, XT, 1, 4, false, Acc>(a.val, a.col, a.cs, a.srl, a.perm, a.lchunk, a.lunit, a.lmeta,
                                                a.lrow, a.part, a.cnt, a.cnt2, a.X, a.ldx, a.Y, a.ldy, a.N, C, v,
                                                a.accumulate, false, pol);
        __syncwarp();
    }

    // ---- consumer
    Acc acc[RPL];
    int rl[RPL];
    int64_t out[RPL];
#pragma unroll
    for (int q = 0; q < RPL; ++q) {
        rl[q] = 0;
        out[q] = -1;
    }
    for (int64_t k = 0; k < issued; ++k) {
        if (R > 1) issue_next();  // piece k + R - 1 into the slot of piece k - 1
        const int slot = (int)(k % R);
        bool ok = true;
        if (a.expire_ns && k == 0 && wg == 0) ok = mbar_wait(never, 0, a.expire_ns);  // runs out
        ok = ok && mbar_wait(bars + slot, (uint32_t)((k / R) & 1));
        if (__any_sync(0xffffffffu, !ok)) {
            if (lane == 0) atomicExch(a.dstat, 1);
            for (int64_t kk = k; kk < issued; ++kk) (void)mbar_wait(bars + kk % R, (uint32_t)((kk / R) & 1));
            return;
        }
        const unsigned char *sp = slots + (size_t)slot * S::bytes;
        const int4 d = *reinterpret_cast<const int4 *>(sp + S::desc);
        const int64_t c = (int64_t)(uint32_t)d.x | ((int64_t)d.y << 32);
        const int j0 = d.z & 0xffff;
        const bool last = (d.z >> 16) != 0;
        if (j0 == 0) {
            const int32_t *ssrl = reinterpret_cast<const int32_t *>(sp + S::srl);
#pragma unroll
            for (int q = 0; q < RPL; ++q) {
                const int64_t r = c * C + q * 32 + lane;
                const int len = ssrl[q * 32 + lane];
                const bool mine = r < a.N && len <= kSeg;
                rl[q] = mine ? len : 0;
                out[q] = mine ? (a.perm ? (int64_t)a.perm[r] : r) : -1;
                acc[q].init((mine && a.accumulate) ? a.Y[out[q] * a.ldy] : XT(0));
            }
        }
        const VT *sv = reinterpret_cast<const VT *>(sp + S::val);
        const int32_t *sc = reinterpret_cast<const int32_t *>(sp + S::col);
        XT xv[T][RPL];
#pragma unroll
        for (int t = 0; t < T; ++t)
#pragma unroll
            for (int q = 0; q < RPL; ++q)
                if (j0 + t < rl[q]) xv[t][q] = __ldg(a.X + (int64_t)sc[t * C + q * 32 + lane] * a.ldx);
#pragma unroll
        for (int t = 0; t < T; ++t)
#pragma unroll
            for (int q = 0; q < RPL; ++q)
                if (j0 + t < rl[q]) acc[q].add(widen(sv[t * C + q * 32 + lane]), xv[t][q]);
        if (last) {
#pragma unroll
            for (int q = 0; q < RPL; ++q)
                if (out[q] >= 0) a.Y[out[q] * a.ldy] = acc[q].result();
        }
        __syncwarp();
        if (R == 1) issue_next();  // the one slot is free again: piece k + 1
    }
}

template <class VT, class Acc, int RPL>
void *kernel_for(bool has_long) {
    return has_long ? (void *)k_spmv_bulk<VT, Acc, RPL, true> : (void *)k_spmv_bulk<VT, Acc, RPL, false>;
}

template <class VT, class Acc>
void *kernel_for_c(int C, bool has_long) {
    switch (C) {
        case 32: return kernel_for<VT, Acc, 1>(has_long);
        case 64: return kernel_for<VT, Acc, 2>(has_long);
        default: return kernel_for<VT, Acc, 4>(has_long);
    }
}

// Resident blocks per SM of the kernel the handle would launch with W warps
// and R slots (0 if it does not fit); sets the kernel's shared-memory limit.
// The kernels may use up to the device's opt-in shared memory per block (the
// same value for every caller, so concurrent handles do not undo each other).
inline cudaError_t allow_smem(const void *fn, int device) {
    int optin = 0;
    cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
}

template <class VT, class Acc>
int blocks_per_sm(const sell_matrix *h, int W, int R) {
    const size_t smem = smem_bytes<VT>(W, R);
    const void *fn = kernel_for_c<VT, Acc>(h->C, h->nunits > 0);
    if (allow_smem(fn, h->device) != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, W * 32, smem) != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    return nb;
}

template <class VT, class Acc>
cudaError_t run(const sell_matrix *h, const void *X, int64_t ldx, void *Y, int64_t ldy, int acc,
                cudaStream_t s) {
    using XT = typename XType<VT>::T;
    Args<VT, Acc> a;
    a.val = static_cast<const VT *>(h->val);
    a.col = h->col;
    a.cs = h->cs;
    a.srl = h->srl;
    a.perm = (h->flags & SELL_BUILD_PERMUTE_COLS) ? nullptr : h->perm;
    a.bsc = h->bsc;
    a.wsplit = h->wsplit;
    a.lchunk = h->lchunk;
    a.lunit = h->lunit;
    a.lmeta = h->lmeta;
    a.lrow = h->lrow;
    a.part = static_cast<Acc *>(h->part);
    a.cnt = h->cnt;
    a.cnt2 = h->cnt2;
    a.dstat = h->dstat;
    a.X = static_cast<const XT *>(X);
    a.Y = static_cast<XT *>(Y);
    a.ldx = ldx;
    a.ldy = ldy;
    a.N = h->nrows;
    a.long_threads = h->nunits * h->C;
    a.ring = h->bulk_ring;
    a.accumulate = acc;
    a.expire_ns = (uint64_t)h->expire_us * 1000u;
    h->expire_us = 0;  // the test hook applies to one launch
    const size_t smem = smem_bytes<VT>(h->bulk_warps, h->bulk_ring);
    const void *fn = kernel_for_c<VT, Acc>(h->C, h->nunits > 0);
    cudaError_t e = allow_smem(fn, h->device);
    if (e != cudaSuccess) return e;
    void *args[] = {&a};
    return cudaLaunchKernel(fn, dim3((unsigned)h->bulk_grid), dim3((unsigned)(h->bulk_warps * 32)), args, smem,
                            s);
}

}  // namespace bulk
}  // namespace sell
