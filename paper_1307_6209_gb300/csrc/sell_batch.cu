// sell_batch.cu -- many SELL-C-sigma products in one persistent launch.
//
// A plan holds a device table of products and one of work units; a unit is
// (product, first sorted row, first right-hand-side column), i.e. a tile of
// kTileRows sorted rows of one product for up to 8 right-hand sides.  The
// persistent kernel runs one or a few blocks per SM; each block claims units
// with an atomic counter until the table is exhausted, so small and large
// matrices share the machine without per-matrix launches or tail gaps.
//
// Every row is computed by the same per-thread loop as sell_spmmv (CRS order,
// one FMA or one Dot2 step per stored nonzero), so a product's result is
// bit-identical whether it runs alone or inside any batch.
#include <algorithm>
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
    void *part;    // this product's own segment scratch (owned by the plan)
    int32_t *cnt;  // this product's own segment counters (owned by the plan)
    const void *X;
    void *Y;
    int64_t ldx, ldy, N, long_threads;
    int32_t C, kb, type, acc, comp, vec;
};

// kind 0: a tile of kTileRows sorted rows starting at row idx (short rows);
// kind 1: kTileRows long-row work-unit threads starting at virtual thread idx.
struct Unit {
    int32_t prod;
    int32_t kind;
    int64_t idx;
};

template <class VT, int K, class Acc>
__device__ __noinline__ void do_unit(const Prod &P, const Unit &u, uint64_t pol) {
    using XT = typename XType<VT>::T;
    constexpr int U = K >= 8 ? 2 : (K >= 4 ? 4 : 8);
    const VT *val = static_cast<const VT *>(P.val);
    const XT *X = static_cast<const XT *>(P.X);
    XT *Y = static_cast<XT *>(P.Y);
    if (u.kind == 1) {
        const int64_t v = u.idx + threadIdx.x;
        if (v < P.long_threads)
            long_unit<VT, XT, K, U, Acc>(val, P.col, P.cs, P.srl, P.perm, P.lchunk, P.lunit,
                                         static_cast<Acc *>(P.part), P.cnt, X, P.ldx, Y, P.ldy, P.N, P.C, v,
                                         P.acc, P.vec != 0, pol);
    } else {
        const int64_t r = u.idx + threadIdx.x;
        if (r < P.N)
            short_row<VT, XT, K, U, Acc>(val, P.col, P.cs, P.srl, P.perm, X, P.ldx, Y, P.ldy, P.C, r, P.acc,
                                         P.vec != 0, pol);
    }
}

template <class VT, class Acc>
__device__ __forceinline__ void dispatch_k(const Prod &P, const Unit &u, uint64_t pol) {
    switch (P.kb) {
        case 1: do_unit<VT, 1, Acc>(P, u, pol); break;
        case 2: do_unit<VT, 2, Acc>(P, u, pol); break;
        case 4: do_unit<VT, 4, Acc>(P, u, pol); break;
        default: do_unit<VT, 8, Acc>(P, u, pol); break;
    }
}

__global__ void __launch_bounds__(kTileRows)
k_batch(const Prod *__restrict__ prods, const Unit *__restrict__ units, int64_t nwork,
        unsigned int *counter) {
    __shared__ int64_t s_unit;
    const uint64_t pol = l2_evict_first_policy();
    for (;;) {
        if (threadIdx.x == 0) s_unit = (int64_t)atomicAdd(counter, 1u);
        __syncthreads();
        const int64_t w = s_unit;
        __syncthreads();
        if (w >= nwork) break;
        const Unit u = units[w];
        const Prod P = prods[u.prod];
        if (P.type == SELL_F64) {
            dispatch_k<double, Plain<double>>(P, u, pol);
        } else if (P.type == SELL_F32) {
            if (P.comp) dispatch_k<float, Dot2>(P, u, pol);
            else dispatch_k<float, Plain<float>>(P, u, pol);
        } else {
            if (P.comp) dispatch_k<__nv_bfloat16, Dot2>(P, u, pol);
            else dispatch_k<__nv_bfloat16, Plain<float>>(P, u, pol);
        }
        __syncthreads();
    }
}

}  // namespace

sell_status batch_create(const sell_batch_item *items, int32_t n, cudaStream_t s, sell_batch *b) {
    std::vector<Prod> prods;
    std::vector<const sell_matrix *> owner;
    std::vector<std::pair<int64_t, int32_t>> order;  // (stored elements, product) for ordering
    for (int32_t i = 0; i < n; ++i) {
        const sell_batch_item &it = items[i];
        const sell_matrix *h = it.A;
        if (!h) return fail(SELL_EINVAL, "sell_batch_create: NULL matrix");
        if (it.k < 1 || it.ldx < it.k || it.ldy < it.k)
            return fail(SELL_EINVAL, "sell_batch_create: need k >= 1, ldx >= k, ldy >= k");
        if (h->nrows > 0 && (!it.X || !it.Y)) return fail(SELL_EINVAL, "sell_batch_create: NULL X/Y");
        if (it.flags & ~(SELL_SPMV_ACCUMULATE | SELL_SPMV_COMPENSATED))
            return fail(SELL_EINVAL, "sell_batch_create: unsupported flags");
        if ((it.flags & SELL_SPMV_COMPENSATED) && h->store_type == SELL_F64)
            return fail(SELL_EUNSUPPORTED, "compensated accumulation needs F32/BF16 storage");
        const size_t xs = h->store_type == SELL_F64 ? 8 : 4;
        for (int32_t done = 0; done < it.k;) {
            int rem = it.k - done;
            int kb = rem >= 8 ? 8 : rem >= 4 ? 4 : rem >= 2 ? 2 : 1;
            Prod P;
            P.val = h->val;
            P.col = h->col;
            P.cs = h->cs;
            P.srl = h->srl;
            P.lchunk = h->lchunk;
            P.lunit = h->lunit;
            P.part = nullptr;
            P.cnt = nullptr;
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
            P.comp = (it.flags & SELL_SPMV_COMPENSATED) ? 1 : 0;
            P.vec = (((uintptr_t)P.X % 16) == 0 && ((it.ldx * xs) % 16) == 0) ? 1 : 0;
            if (h->nrows > 0) {
                order.push_back({h->stored * kb, (int32_t)prods.size()});
                prods.push_back(P);
                owner.push_back(h);
            }
            done += kb;
        }
    }
    // biggest products first: their tiles start early and small ones fill the tail
    std::stable_sort(order.begin(), order.end(),
                     [](const std::pair<int64_t, int32_t> &a, const std::pair<int64_t, int32_t> &b) {
                         return a.first > b.first;
                     });
    // each product with long rows gets its own segment scratch and counters,
    // so products of one plan (even on the same matrix) never share them
    b->al = current_allocator();
    for (size_t i = 0; i < prods.size(); ++i) {
        const sell_matrix *h = owner[i];
        if (h->nunits == 0) continue;
        void *p = b->al.get((size_t)h->nunits * h->C * prods[i].kb * 8, s);
        void *c = p ? b->al.get((size_t)h->nlong * h->C * sizeof(int32_t), s) : nullptr;
        if (p) b->scratch.push_back(p);
        if (c) b->scratch.push_back(c);
        if (!p || !c) return fail(SELL_ENOMEM, "sell_batch_create: segment scratch allocation failed");
        SELL_CUDA_TRY(cudaMemsetAsync(c, 0, (size_t)h->nlong * h->C * sizeof(int32_t), s));
        prods[i].part = p;
        prods[i].cnt = static_cast<int32_t *>(c);
    }
    // long-row work first (its units are the longest), then row tiles
    std::vector<Unit> units;
    for (auto &o : order) {
        const Prod &P = prods[o.second];
        for (int64_t v0 = 0; v0 < P.long_threads; v0 += kTileRows) units.push_back({o.second, 1, v0});
    }
    for (auto &o : order) {
        const Prod &P = prods[o.second];
        for (int64_t r0 = 0; r0 < P.N; r0 += kTileRows) units.push_back({o.second, 0, r0});
    }
    b->nprod = (int32_t)prods.size();
    b->nwork = (int64_t)units.size();
    DevBuf dp, du, dc;
    if (!prods.empty()) {
        SELL_TRY(dp.alloc(b->al, prods.size() * sizeof(Prod), s));
        SELL_TRY(du.alloc(b->al, units.size() * sizeof(Unit), s));
        SELL_CUDA_TRY(cudaMemcpyAsync(dp.p, prods.data(), prods.size() * sizeof(Prod),
                                      cudaMemcpyHostToDevice, s));
        SELL_CUDA_TRY(cudaMemcpyAsync(du.p, units.data(), units.size() * sizeof(Unit),
                                      cudaMemcpyHostToDevice, s));
    }
    SELL_TRY(dc.alloc(b->al, sizeof(unsigned int), s));
    SELL_CUDA_TRY(cudaStreamSynchronize(s));
    int dev = 0, sms = 0, occ = 0;
    SELL_CUDA_TRY(cudaGetDevice(&dev));
    SELL_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    SELL_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch, kTileRows, 0));
    b->device = dev;
    b->grid_default = std::max(1, sms * std::max(occ, 1));
    b->items = dp.release_ownership();
    b->units = du.release_ownership();
    b->counter = static_cast<unsigned int *>(dc.release_ownership());
    return SELL_OK;
}

sell_status batch_run(sell_batch *b, int32_t grid, cudaStream_t s) {
    b->last_stream = s;
    b->ran = true;
    if (b->nwork == 0) return SELL_OK;
    int g = grid > 0 ? grid : b->grid_default;
    SELL_CUDA_TRY(cudaMemsetAsync(b->counter, 0, sizeof(unsigned int), s));
    k_batch<<<g, kTileRows, 0, s>>>(static_cast<const Prod *>(b->items),
                                    static_cast<const Unit *>(b->units), b->nwork, b->counter);
    SELL_CUDA_TRY(cudaGetLastError());
    return SELL_OK;
}

}  // namespace sell
