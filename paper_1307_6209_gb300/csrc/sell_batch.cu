// sell_batch.cu -- many SELL-C-sigma products in persistent launches.
//
// A plan splits every product into column blocks of 8, 4, 2 or 1 right-hand
// sides (at most the item's SELL_SPMV_RHS_BLOCK* width) and groups the blocks
// by kernel variant (value type, block width,
// plain or compensated accumulation).  Each variant present gets one launch
// (per 160 products): its products and the block ranges of their work units
// travel in the kernel's parameter space -- a unit is one block's worth of
// sorted rows of one product (its short rows; 128 by default, 64 or 256
// after sell_batch_set_launch), or as many threads of the product's long-row
// segment units.  Creating a plan makes one device allocation (the
// products' long-row scratch) and no copies, and does not synchronise.  One
// block per unit, long-row units first and biggest products first; the
// hardware block scheduler balances the uneven products.  (A grid-stride "persistent" form of this kernel was measured:
// its loop-carried state raised the register count from 40 to 64, cut the
// resident blocks per SM from 6 to 4 and made the batch slower.)
//
// Every row is computed by the same per-row arithmetic as sell_spmmv
// (sell_rowdot.cuh), so a product's result is bit-identical whether it runs
// alone or inside any batch.
#include <algorithm>
#include <map>
#include <new>
#include <tuple>
#include <type_traits>
#include <vector>

#include "sell_rowdot.cuh"

namespace sell {
namespace {

constexpr int kTileRows = 256;

struct Prod {
    const void *val;
    const int32_t *col;
    const int64_t *cs;
    const int32_t *srl;
    const int32_t *perm;
    const int32_t *lchunk;
    const int2 *lunit;
    const int4 *lmeta;
    const int32_t *lrow;
    void *part;    // this product's own segment scratch (owned by the plan)
    int32_t *cnt;  // this product's own segment counters (owned by the plan)
    int32_t *cnt2; // this product's own group counters (owned by the plan)
    const void *X;
    void *Y;
    int64_t ldx, ldy, N, long_threads;
    int32_t C, kb, type, acc, comp, vec;
};

// The products of one launch travel in the kernel's parameter space (read
// through the constant cache when a unit needs a field), which keeps the
// register footprint at that of the single-product kernel.  The work units
// need no table: block w belongs to range i of `start` (start[i] <= w <
// start[i+1]); ranges 0..nprod-1 are the products' long-row units
// (blockDim.x segment threads per block), ranges nprod..2*nprod-1 their short
// rows (blockDim.x rows per block).
constexpr int kLaunchProds = 160;  // 160 * 168 B + the ranges fit the 32 KB parameter limit

struct LaunchParams {
    Prod prods[kLaunchProds];
    int32_t start[2 * kLaunchProds + 1];
    int32_t nprod;
};

// One block per work unit, long-row units first in the grid so that they
// start early (the same shape as the single-product kernel).  Every variant
// issues the next group's val/col loads before the current group's gathers
// (software pipelining, as launch mode 1 of the single product; the FMA
// order and so the bits are unchanged).  Measured on 256-matrix binary32
// batches: banded k = 1 3 % faster (the 512-matrix mixed one 2 %); at k = 8
// banded 2.16 -> 1.79 ms and lognormal 2.45 -> 2.15 ms, at k = 4 banded
// 1.84 -> 1.67 ms and lognormal unchanged -- without it the wide variants,
// at 64 registers and half the SM's warps, kept too few stream bytes in
// flight.
template <class VT, int K, class Acc, class AccL, bool LONG = true>
__device__ __forceinline__ void batch_unit(const LaunchParams &lp) {
    using XT = typename XType<VT>::T;
    constexpr int U = K >= 4 ? 2 : 4;
    constexpr bool PIPE = true;
    const uint64_t pol = l2_evict_first_policy();
    const int32_t w = (int32_t)blockIdx.x;
    if (w >= lp.start[2 * lp.nprod]) return;
    int lo = 0, hi = 2 * lp.nprod;  // last range with start <= w
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (lp.start[mid] <= w) lo = mid;
        else hi = mid;
    }
    const bool is_long = lo < lp.nprod;
    const Prod &P = lp.prods[is_long ? lo : lo - lp.nprod];
    const int64_t first = (int64_t)(w - lp.start[lo]) * blockDim.x;
    if (LONG && is_long) {
        const int64_t v = first + threadIdx.x;
        if (v < P.long_threads)
            long_unit<VT, XT, K, U, PIPE, AccL>(static_cast<const VT *>(P.val), P.col, P.cs, P.srl, P.perm,
                                         P.lchunk, P.lunit, P.lmeta, P.lrow, static_cast<AccL *>(P.part), P.cnt, P.cnt2,
                                         static_cast<const XT *>(P.X),
                                         P.ldx, static_cast<XT *>(P.Y), P.ldy, P.N, P.C, v, P.acc, P.vec, pol);
        return;
    }
    const int64_t r = first + threadIdx.x;
    if (r < P.N)
        short_row<VT, XT, K, U, PIPE, Acc>(static_cast<const VT *>(P.val), P.col, P.cs, P.srl, P.perm,
                                     static_cast<const XT *>(P.X), P.ldx, static_cast<XT *>(P.Y), P.ldy, P.C, r, P.acc,
                                     P.vec, pol);
}

// The kernel holds both the long-row path (segment folds) and the short-row
// path.  Left alone, ptxas gives the one- and two-vector variants 60-64
// registers (4 blocks of 256 threads per SM, half the SM's warps) for the
// sake of the long-row path, although the short rows carry most of the work.
// Their entry point therefore asks for 6 resident blocks (5 for bfloat16 and
// for two vectors), which fits them in 40-48 registers with no spills (ptxas
// -v).  The four-vector variants ask for 5 blocks (48 registers; binary32
// without spills): measured against ptxas's own 64 registers (4 blocks) on
// 256 lognormal binary32 matrices 2.17 -> 1.90 ms and on the 512-matrix
// mixed batch 7.00 -> 5.01 ms; binary64 unchanged.  The eight-vector
// variants would take 64-76 (3 blocks per SM for binary32).  4 resident
// blocks (64 registers) measured 5 % faster than that on the 512-matrix
// binary32 batch; binary32 and bfloat16 now ask for 5 (48 registers, 92
// bytes of spills): 256 lognormal binary32 matrices 2.17 -> 2.12 ms, a
// 512-matrix mixed batch 6.28 -> 5.55 ms.  Binary64 keeps 4 (5 measured 6 %
// slower).
template <class VT, int K>
constexpr int narrow_min_blocks() {
    return K == 1 && !std::is_same<VT, __nv_bfloat16>::value ? 6 : 5;
}

template <class VT, int K, class Acc, class AccL = Acc>
__global__ void __launch_bounds__(kTileRows, (narrow_min_blocks<VT, K>()))
k_batch_narrow(const __grid_constant__ LaunchParams lp) {
    batch_unit<VT, K, Acc, AccL>(lp);
}

template <class VT, int K, class Acc, class AccL = Acc>
__global__ void __launch_bounds__(kTileRows, 5) k_batch(const __grid_constant__ LaunchParams lp) {
    batch_unit<VT, K, Acc, AccL>(lp);
}

template <class VT>
constexpr int wide_min_blocks() {
    return sizeof(VT) == 8 ? 4 : 5;
}

template <class VT, int K, class Acc, class AccL = Acc>
__global__ void __launch_bounds__(kTileRows, (wide_min_blocks<VT>()))
k_batch_wide(const __grid_constant__ LaunchParams lp) {
    batch_unit<VT, K, Acc, AccL>(lp);
}

// Products without long rows (every row at most kSeg entries) at one right-
// hand side get an entry point of their own, capped at 32 registers: 8
// resident blocks of 256 threads, every warp slot of the SM.  ptxas places
// its spills (96-112 bytes) in the long-row path, which these products never
// enter.  Measured on the 256 banded matrices of the benchmark batch
// (binary32): 0.766 -> 0.837 of the HBM copy bandwidth.  (The same cap on
// the products with long rows made the mixed 512-matrix batch 1 % slower;
// an entry point with the long-row path compiled out reached only 0.807.)
template <class VT, class Acc>
__global__ void __launch_bounds__(kTileRows, 8) k_batch_short(const __grid_constant__ LaunchParams lp) {
    batch_unit<VT, 1, Acc, Acc, true>(lp);
}

// The same for four and eight right-hand sides of binary32 and bfloat16
// storage: 6 and 5 resident blocks (40 and 48 registers) instead of the 4
// of the general variants.  (Binary64 rows of four and eight values do not
// fit: ptxas spills 208 and 856 bytes there, so those keep the general
// variants.)
template <int K>
constexpr int short_min_blocks() {
    return K == 4 ? 6 : 5;
}

template <class VT, int K, class Acc>
__global__ void __launch_bounds__(kTileRows, (short_min_blocks<K>()))
k_batch_short_wide(const __grid_constant__ LaunchParams lp) {
    batch_unit<VT, K, Acc, Acc, true>(lp);
}

using KernelFn = void (*)(const LaunchParams);

template <class VT, class Acc, class AccL = Acc>
KernelFn kernel_for_k(int kb) {
    switch (kb) {
        case 1: return k_batch_narrow<VT, 1, Acc, AccL>;
        case 2: return k_batch_narrow<VT, 2, Acc, AccL>;
        case 4: return k_batch<VT, 4, Acc, AccL>;
        default: return k_batch_wide<VT, 8, Acc, AccL>;
    }
}

// comp: 0 binary32 chains, 1 Dot2 on every row, 2 Dot2 on the long rows only.
template <class VT>
KernelFn kernel_for_reduced(int comp, int kb) {
    if (comp == 1) return kernel_for_k<VT, Dot2>(kb);
    if (comp == 2) return kernel_for_k<VT, Plain<float>, Dot2>(kb);
    return kernel_for_k<VT, Plain<float>>(kb);
}

template <class VT, class Acc>
KernelFn short_for_k(int kb) {
    switch (kb) {
        case 1: return k_batch_short<VT, Acc>;
        case 4: return k_batch_short_wide<VT, 4, Acc>;
        default: return k_batch_short_wide<VT, 8, Acc>;
    }
}

// The entry point of products without long rows at 1, 4 or 8 right-hand
// sides (Dot2 on long rows only is then plain accumulation: there is no long
// row).
KernelFn kernel_for_short(int type, int comp, int kb) {
    if (type == SELL_F64) return k_batch_short<double, Plain<double>>;  // kb == 1 only
    if (type == SELL_F32) return comp == 1 ? short_for_k<float, Dot2>(kb) : short_for_k<float, Plain<float>>(kb);
    return comp == 1 ? short_for_k<__nv_bfloat16, Dot2>(kb) : short_for_k<__nv_bfloat16, Plain<float>>(kb);
}

KernelFn kernel_for(int type, int comp, int kb) {
    if (type == SELL_F64) return kernel_for_k<double, Plain<double>>(kb);
    if (type == SELL_F32) return kernel_for_reduced<float>(comp, kb);
    return kernel_for_reduced<__nv_bfloat16>(comp, kb);
}

}  // namespace

namespace {
size_t up256(size_t x) { return (x + 255) / 256 * 256; }
}  // namespace

// Long-row scratch of one batch item (all its column blocks): the segment
// partials of every block, then the counters of every block (cleared
// together).  0 for matrices without long rows.
size_t batch_item_scratch(const sell_matrix *h, int32_t k, uint32_t flags, size_t *counter_offset) {
    size_t pb = 0, cb = 0;
    if (h->nunits > 0 && h->nrows > 0) {
        for (int32_t done = 0; done < k;) {
            const int kb = rhs_block(k - done, max_rhs_block(flags));
            pb += up256((size_t)h->nunits * h->C * kb * 8);
            cb += up256((size_t)(h->nlong + h->nunits) * h->C * sizeof(int32_t));
            done += kb;
        }
    }
    if (counter_offset) *counter_offset = pb;
    return pb + cb;
}

namespace {
// The block ranges of a launch's products for blocks of `tile` threads:
// long-row units of every product first, then their short rows.  Returns the
// number of blocks.
int64_t assign_units(LaunchParams *lp, int tile) {
    const int np = lp->nprod;
    int64_t w = 0;
    for (int j = 0; j < np; ++j) {
        lp->start[j] = (int32_t)std::min<int64_t>(w, 0x7FFFFFFF);
        w += (lp->prods[j].long_threads + tile - 1) / tile;
    }
    for (int j = 0; j < np; ++j) {
        lp->start[np + j] = (int32_t)std::min<int64_t>(w, 0x7FFFFFFF);
        w += (lp->prods[j].N + tile - 1) / tile;
    }
    lp->start[2 * np] = (int32_t)std::min<int64_t>(w, 0x7FFFFFFF);
    return w;
}
}  // namespace

sell_status batch_create(const sell_batch_item *items, int32_t n, cudaStream_t s, sell_batch *b,
                         void *const *scratch) {
    std::vector<Prod> prods;
    std::vector<const sell_matrix *> owner;
    b->al = current_allocator();
    // each item with long rows gets its own scratch (given by the caller, or
    // one allocation for the whole plan), so products of one plan -- even on
    // the same matrix -- never share segment partials or counters
    char *own = nullptr;
    if (!scratch) {
        size_t total = 0;
        for (int32_t i = 0; i < n; ++i)
            if (items[i].A && items[i].k >= 1) total += batch_item_scratch(items[i].A, items[i].k, items[i].flags, nullptr);
        if (total > 0) {
            own = static_cast<char *>(b->al.get(total, s));
            if (!own) return fail(SELL_ENOMEM, "sell_batch_create: segment scratch allocation failed");
            b->scratch.push_back(own);
        }
    }
    size_t own_off = 0;
    for (int32_t i = 0; i < n; ++i) {
        const sell_batch_item &it = items[i];
        const sell_matrix *h = it.A;
        if (!h) return fail(SELL_EINVAL, "sell_batch_create: NULL matrix");
        if (it.k < 1 || it.ldx < it.k || it.ldy < it.k)
            return fail(SELL_EINVAL, "sell_batch_create: need k >= 1, ldx >= k, ldy >= k");
        if (h->nrows > 0 && (!it.X || !it.Y)) return fail(SELL_EINVAL, "sell_batch_create: NULL X/Y");
        if (it.flags & ~(SELL_SPMV_ACCUMULATE | kCompFlags | kRhsFlags))
            return fail(SELL_EINVAL, "sell_batch_create: unsupported flags");
        if ((it.flags & kCompFlags) && h->store_type == SELL_F64)
            return fail(SELL_EUNSUPPORTED, "compensated accumulation needs F32/BF16 storage");
        if (h->nrows == 0) continue;
        size_t coff = 0;
        const size_t sbytes = batch_item_scratch(h, it.k, it.flags, &coff);
        char *sc = nullptr;
        if (sbytes > 0) {
            sc = scratch ? static_cast<char *>(scratch[i]) : own + own_off;
            own_off += scratch ? 0 : sbytes;
            if (!sc) return fail(SELL_EINVAL, "sell_batch_create: missing scratch");
            SELL_CUDA_TRY(cudaMemsetAsync(sc + coff, 0, sbytes - coff, s));
        }
        size_t poff = 0, cpos = coff;
        const size_t xs = h->store_type == SELL_F64 ? 8 : 4;
        for (int32_t done = 0; done < it.k;) {
            const int kb = rhs_block(it.k - done, max_rhs_block(it.flags));
            Prod P;
            P.val = h->val;
            P.col = h->col;
            P.cs = h->cs;
            P.srl = h->srl;
            P.lchunk = h->lchunk;
            P.lunit = h->lunit;
            P.lmeta = h->lmeta;
            P.lrow = h->lrow;
            P.part = nullptr;
            P.cnt = nullptr;
            P.cnt2 = nullptr;
            if (sc) {
                P.part = sc + poff;
                P.cnt = reinterpret_cast<int32_t *>(sc + cpos);
                P.cnt2 = P.cnt + h->nlong * h->C;
                poff += up256((size_t)h->nunits * h->C * kb * 8);
                cpos += up256((size_t)(h->nlong + h->nunits) * h->C * sizeof(int32_t));
            }
            P.long_threads = h->nunits * h->C;
            P.perm = (h->flags & SELL_BUILD_PERMUTE_COLS) ? nullptr : h->perm;
            P.X = static_cast<const char *>(it.X) + done * xs;
            P.Y = static_cast<char *>(it.Y) + done * xs;
            P.ldx = it.ldx;
            P.ldy = it.ldy;
            P.N = h->nrows;
            P.C = h->C;
            P.kb = kb;
            P.type = h->store_type;
            P.acc = (it.flags & SELL_SPMV_ACCUMULATE) ? 1 : 0;
            P.comp = h->store_type != SELL_F64 ? comp_mode(it.flags) : 0;
            P.vec = x_vec(P.X, it.ldx, xs) | (x_vec(P.Y, it.ldy, xs) << 2);
            prods.push_back(P);
            owner.push_back(h);
            done += kb;
        }
    }
    // group by kernel variant (products without long rows at 1, 4 or 8
    // right-hand sides apart: their entry points hold fewer registers);
    // inside a group: long-row work first, biggest first
    std::map<std::tuple<int, int, int, int>, std::vector<int32_t>> groups;
    for (size_t i = 0; i < prods.size(); ++i) {
        const Prod &P = prods[i];
        const int short_only =
            (P.long_threads == 0 && (P.kb == 1 || (P.kb >= 4 && P.type != SELL_F64))) ? 1 : 0;
        groups[std::make_tuple(P.type, P.comp, P.kb, short_only)].push_back((int32_t)i);
    }
    int dev = 0;
    SELL_CUDA_TRY(cudaGetDevice(&dev));
    b->device = dev;
    b->nprod = (int32_t)prods.size();
    b->nwork = 0;
    std::vector<std::pair<int64_t, int>> order;  // (work, group index) biggest group first
    std::vector<std::vector<int32_t>> gids;
    std::vector<std::tuple<int, int, int, int>> gkey;
    for (auto &kv : groups) {
        std::vector<int32_t> ids = kv.second;
        std::stable_sort(ids.begin(), ids.end(), [&](int32_t a, int32_t c) {
            return owner[a]->stored > owner[c]->stored;
        });
        int64_t work = 0;
        for (int32_t id : ids) work += prods[id].N * prods[id].kb;
        order.push_back({work, (int)gids.size()});
        gids.push_back(std::move(ids));
        gkey.push_back(kv.first);
    }
    std::stable_sort(order.begin(), order.end(),
                     [](const std::pair<int64_t, int> &a, const std::pair<int64_t, int> &c) { return a.first > c.first; });
    for (auto &o : order) {
        const int g = o.second;
        // launches of at most kLaunchProds products each
        KernelFn fn = std::get<3>(gkey[g]) ? kernel_for_short(std::get<0>(gkey[g]), std::get<1>(gkey[g]),
                                                              std::get<2>(gkey[g]))
                                           : kernel_for(std::get<0>(gkey[g]), std::get<1>(gkey[g]), std::get<2>(gkey[g]));
        const std::vector<int32_t> &ids = gids[g];
        for (size_t p0 = 0; p0 < ids.size(); p0 += kLaunchProds) {
            const int np = (int)(std::min(ids.size(), p0 + (size_t)kLaunchProds) - p0);
            auto *lp = new (std::nothrow) LaunchParams();
            if (!lp) return fail(SELL_ENOMEM, "sell_batch_create: host allocation failed");
            lp->nprod = np;
            for (int j = 0; j < np; ++j) lp->prods[j] = prods[ids[p0 + j]];
            const int64_t w = assign_units(lp, b->tile);
            if (w > 0x7FFFFFFF) {
                delete lp;
                return fail(SELL_EUNSUPPORTED, "sell_batch_create: too many work units in one launch");
            }
            if (w == 0) {
                delete lp;
                continue;
            }
            sell_batch::Group G;
            G.fn = reinterpret_cast<void *>(fn);
            G.params = lp;
            G.nwork = w;
            G.grid = (int32_t)w;  // one block per unit
            b->groups.push_back(G);
            b->nwork += G.nwork;
        }
    }
    return SELL_OK;
}

void batch_release(sell_batch *b, cudaStream_t s) {
    for (auto &G : b->groups) delete static_cast<LaunchParams *>(G.params);
    b->groups.clear();
    for (void *p : b->scratch) b->al.put(p, s);
    b->scratch.clear();
}

sell_status batch_set_tile(sell_batch *b, int32_t tile) {
    if (tile != 64 && tile != 128 && tile != 256)
        return fail(SELL_EINVAL, "sell_batch_set_launch: block must be 64, 128 or 256");
    std::vector<int64_t> ws;
    for (const sell_batch::Group &G : b->groups) {
        LaunchParams tmp = *static_cast<const LaunchParams *>(G.params);
        const int64_t w = assign_units(&tmp, tile);
        if (w > 0x7FFFFFFF) return fail(SELL_EUNSUPPORTED, "sell_batch_set_launch: too many work units in one launch");
        ws.push_back(w);
    }
    b->tile = tile;
    b->nwork = 0;
    for (size_t g = 0; g < b->groups.size(); ++g) {
        sell_batch::Group &G = b->groups[g];
        assign_units(static_cast<LaunchParams *>(G.params), tile);
        G.nwork = ws[g];
        G.grid = (int32_t)ws[g];
        b->nwork += ws[g];
    }
    return SELL_OK;
}

sell_status batch_run(sell_batch *b, int32_t grid, cudaStream_t s) {
    if (grid != 0) return fail(SELL_EINVAL, "sell_batch_run: grid must be 0 (one block per work unit)");
    b->last_stream = s;
    b->ran = true;
    for (const sell_batch::Group &G : b->groups) {
        KernelFn fn = reinterpret_cast<KernelFn>(G.fn);
        fn<<<G.grid, b->tile, 0, s>>>(*static_cast<const LaunchParams *>(G.params));
        SELL_CUDA_TRY(cudaGetLastError());
    }
    return SELL_OK;
}

}  // namespace sell
