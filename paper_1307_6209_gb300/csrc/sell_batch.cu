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

#include "sell_internal.cuh"

namespace sell {
namespace {

constexpr int kTileRows = 256;

struct Prod {
    const void *val;
    const int32_t *col;
    const int64_t *cs;
    const int32_t *srl;
    const int32_t *perm;
    const void *X;
    void *Y;
    int64_t ldx, ldy, N;
    int32_t C, kb, type, acc, comp, vec;
};

struct Unit {
    int32_t prod;
    int32_t row0;
};

__device__ __forceinline__ double widen_b(double v) { return v; }
__device__ __forceinline__ float widen_b(float v) { return v; }
__device__ __forceinline__ float widen_b(__nv_bfloat16 v) { return __bfloat162float(v); }

struct PlainD {
    double s;
    __device__ __forceinline__ void init(double y) { s = y; }
    __device__ __forceinline__ void add(double a, double b) { s = fma(a, b, s); }
    __device__ __forceinline__ double result() const { return s; }
};
struct PlainF {
    float s;
    __device__ __forceinline__ void init(float y) { s = y; }
    __device__ __forceinline__ void add(float a, float b) { s = fmaf(a, b, s); }
    __device__ __forceinline__ float result() const { return s; }
};
struct Dot2F {
    float p, s;
    __device__ __forceinline__ void init(float y) { p = y; s = 0.0f; }
    __device__ __forceinline__ void add(float a, float b) {
        float h = __fmul_rn(a, b);
        float r = __fmaf_rn(a, b, -h);
        float t = __fadd_rn(p, h);
        float z = __fsub_rn(t, p);
        float q = __fadd_rn(__fsub_rn(p, __fsub_rn(t, z)), __fsub_rn(h, z));
        p = t;
        s = __fadd_rn(s, __fadd_rn(q, r));
    }
    __device__ __forceinline__ float result() const { return __fadd_rn(p, s); }
};

template <class VT, class XT, int K, class Acc>
__device__ __forceinline__ void row_product(const Prod &P, int64_t r, uint64_t pol) {
    const int64_t c = r / P.C;
    const int l = (int)(r - c * P.C);
    const int len = P.srl[r];
    const int64_t out = P.perm ? (int64_t)P.perm[r] : r;
    const VT *vp = static_cast<const VT *>(P.val) + P.cs[c] + l;
    const int32_t *cp = P.col + P.cs[c] + l;
    const XT *X = static_cast<const XT *>(P.X);
    XT *Y = static_cast<XT *>(P.Y);
    Acc acc[K];
#pragma unroll
    for (int q = 0; q < K; ++q) acc[q].init(P.acc ? Y[out * P.ldy + q] : XT(0));
    constexpr int U = K >= 4 ? 2 : 4;
    int j = 0;
    for (; j + U <= len; j += U) {
        VT v[U];
        int32_t ci[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            v[u] = ld_stream(vp + (int64_t)u * P.C, pol);
            ci[u] = ld_stream(cp + (int64_t)u * P.C, pol);
        }
        XT xv[U][K];
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int q = 0; q < K; ++q) xv[u][q] = __ldg(X + (int64_t)ci[u] * P.ldx + q);
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int q = 0; q < K; ++q) acc[q].add(widen_b(v[u]), xv[u][q]);
        vp += (int64_t)U * P.C;
        cp += (int64_t)U * P.C;
    }
    for (; j < len; ++j) {
        VT v = ld_stream(vp, pol);
        int32_t ci = ld_stream(cp, pol);
#pragma unroll
        for (int q = 0; q < K; ++q) acc[q].add(widen_b(v), __ldg(X + (int64_t)ci * P.ldx + q));
        vp += P.C;
        cp += P.C;
    }
#pragma unroll
    for (int q = 0; q < K; ++q) Y[out * P.ldy + q] = acc[q].result();
}

template <class VT, class XT, class Acc>
__device__ __forceinline__ void row_dispatch_k(const Prod &P, int64_t r, uint64_t pol) {
    switch (P.kb) {
        case 1: row_product<VT, XT, 1, Acc>(P, r, pol); break;
        case 2: row_product<VT, XT, 2, Acc>(P, r, pol); break;
        case 4: row_product<VT, XT, 4, Acc>(P, r, pol); break;
        default: row_product<VT, XT, 8, Acc>(P, r, pol); break;
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
        const int64_t r = (int64_t)u.row0 + threadIdx.x;
        if (r < P.N) {
            if (P.type == SELL_F64) {
                row_dispatch_k<double, double, PlainD>(P, r, pol);
            } else if (P.type == SELL_F32) {
                if (P.comp) row_dispatch_k<float, float, Dot2F>(P, r, pol);
                else row_dispatch_k<float, float, PlainF>(P, r, pol);
            } else {
                if (P.comp) row_dispatch_k<__nv_bfloat16, float, Dot2F>(P, r, pol);
                else row_dispatch_k<__nv_bfloat16, float, PlainF>(P, r, pol);
            }
        }
    }
}

}  // namespace

sell_status batch_create(const sell_batch_item *items, int32_t n, cudaStream_t s, sell_batch *b) {
    std::vector<Prod> prods;
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
            P.vec = 0;
            if (h->nrows > 0) {
                order.push_back({h->stored * kb, (int32_t)prods.size()});
                prods.push_back(P);
            }
            done += kb;
        }
    }
    // biggest products first: their tiles start early and small ones fill the tail
    std::stable_sort(order.begin(), order.end(),
                     [](const std::pair<int64_t, int32_t> &a, const std::pair<int64_t, int32_t> &b) {
                         return a.first > b.first;
                     });
    std::vector<Unit> units;
    for (auto &o : order) {
        const Prod &P = prods[o.second];
        for (int64_t r0 = 0; r0 < P.N; r0 += kTileRows) units.push_back({o.second, (int32_t)r0});
    }
    b->al = current_allocator();
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

sell_status batch_run(const sell_batch *b, int32_t grid, cudaStream_t s) {
    if (b->nwork == 0) return SELL_OK;
    int g = grid > 0 ? grid : b->grid_default;
    SELL_CUDA_TRY(cudaMemsetAsync(b->counter, 0, sizeof(unsigned int), s));
    k_batch<<<g, kTileRows, 0, s>>>(static_cast<const Prod *>(b->items),
                                    static_cast<const Unit *>(b->units), b->nwork, b->counter);
    SELL_CUDA_TRY(cudaGetLastError());
    return SELL_OK;
}

}  // namespace sell
