// sell_build.cu -- CRS -> SELL-C-sigma conversion on the GPU (Sec. 3.3-3.4).
//
// Pipeline (one stream, two host synchronisations):
//   k_rowlen / k_colcheck   rowLen[i] = rpt[i+1] - rpt[i]; input validation;
//                           max row length and sum of squares (for Eq. "cv")
//   -- sync 1: validation word, max row length --
//   sorting scope sigma     sigma <= 1: identity (no permutation stored)
//                           sigma' = min(sigma, N) <= 4096: k_window_sort, a
//                             bitonic sort in shared memory of whole windows,
//                             several windows per block for small sigma
//                           larger: stable LSD radix sort over the key
//                             (window, maxlen - rowLen), 8-bit digits
//   k_chunk_len             sorted row lengths srl[r], cl[c] = max (Eq. "max")
//   scan                    cs = exclusive prefix sum of C * cl (cl[i] =
//                           (cs[i+1]-cs[i])/C)
//   -- sync 2: stored size cs[Nc] --
//   k_scatter               entry j of sorted row r = c*C + l -> cs[c] + j*C + l,
//                           zero padding (value 0, column 0), value rounding
//
// Every sort key is unique (it ends in the row's position), so any correct
// sort gives the stable order: ties in length keep the original row order.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "sell_internal.cuh"

namespace sell {
namespace {

constexpr int kWindowSortMax = 4096;  // rows per block of the shared-memory sort
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;          // items per thread in the scan
constexpr int kScanTile = kScanThreads * kScanItems;
constexpr int kRadixThreads = 256;
constexpr int kRadixRounds = 8;
constexpr int kRadixTile = kRadixThreads * kRadixRounds;

struct BuildStats {
    unsigned int err;
    int max_rl;
    unsigned long long sumsq;
};
enum : unsigned int {
    kErrRpt0 = 1u,
    kErrRptOrder = 2u,
    kErrRptEnd = 4u,
    kErrRowLong = 8u,
    kErrCol = 16u,
};

inline int grid_for(int64_t n, int threads, int64_t cap = 1 << 20) {
    int64_t g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    return (int)std::min<int64_t>(g, cap);
}

// ------------------------------------------------------------ row lengths
__global__ void k_rowlen(const int64_t *__restrict__ rpt, int64_t N, int64_t nnz,
                         int32_t *__restrict__ rl, BuildStats *st) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned int err = 0;
    int mx = 0;
    unsigned long long sq = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += stride) {
        int64_t a = rpt[i], b = rpt[i + 1];
        int64_t len = b - a;
        if (i == 0 && a != 0) err |= kErrRpt0;
        if (i == N - 1 && b != nnz) err |= kErrRptEnd;
        if (len < 0) { err |= kErrRptOrder; len = 0; }
        if (len > 0x7FFFFFFF) { err |= kErrRowLong; len = 0; }
        rl[i] = (int32_t)len;
        mx = max(mx, (int)len);
        sq += (unsigned long long)len * (unsigned long long)len;
    }
    for (int o = 16; o > 0; o >>= 1) {
        err |= __shfl_xor_sync(0xffffffffu, err, o);
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        sq += __shfl_xor_sync(0xffffffffu, sq, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (err) atomicOr(&st->err, err);
        atomicMax(&st->max_rl, mx);
        atomicAdd(&st->sumsq, sq);
    }
}

__global__ void k_colcheck(const int32_t *__restrict__ col, int64_t nnz, int64_t ncols,
                           BuildStats *st) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    bool bad = false;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nnz; j += stride) {
        int32_t c = col[j];
        bad |= (c < 0) | ((int64_t)c >= ncols);
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&st->err, kErrCol);
}

// ------------------------------------------------- window sort (small sigma)
// One block sorts `wpb` whole windows of W rows (wpb * W <= 4096) with a
// bitonic network over P = next power of two keys.  Key layout (ascending):
//   bits 43..63  window index inside the block
//   bits 12..42  0x7FFFFFFF - rowLen     (descending length)
//   bits  0..11  row position inside the block (tie-break: original order)
__global__ void k_window_sort(const int32_t *__restrict__ rl, int64_t N, int64_t W, int wpb,
                              int P, int32_t *__restrict__ perm) {
    extern __shared__ unsigned long long skey[];
    const int64_t tile = (int64_t)wpb * W;
    const int64_t base = blockIdx.x * tile;
    const int64_t nrow = min(tile, N - base);
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        unsigned long long k = ~0ull;
        if (i < nrow) {
            unsigned long long w = (unsigned long long)(i / W);
            unsigned long long inv = 0x7FFFFFFFull - (unsigned long long)rl[base + i];
            k = (w << 43) | (inv << 12) | (unsigned long long)i;
        }
        skey[i] = k;
    }
    __syncthreads();
    for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int t = threadIdx.x; t < (P >> 1); t += blockDim.x) {
                int lo = 2 * j * (t / j) + (t % j);
                int hi = lo + j;
                bool up = (lo & k) == 0;
                unsigned long long a = skey[lo], b = skey[hi];
                if ((a > b) == up) { skey[lo] = b; skey[hi] = a; }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < nrow; i += blockDim.x)
        perm[base + i] = (int32_t)(base + (int64_t)(skey[i] & 0xFFFull));
}

// --------------------------------------------------- radix sort (large sigma)
__global__ void k_radix_init(const int32_t *__restrict__ rl, int64_t N, int64_t sigma, int lbits,
                             int max_rl, unsigned long long *__restrict__ key,
                             int32_t *__restrict__ val) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += stride) {
        unsigned long long w = (unsigned long long)(i / sigma);
        key[i] = (w << lbits) | (unsigned long long)(max_rl - rl[i]);
        val[i] = (int32_t)i;
    }
}

__global__ void k_radix_hist(const unsigned long long *__restrict__ key, int64_t N, int shift,
                             int64_t ntiles, uint32_t *__restrict__ hist) {
    __shared__ uint32_t cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t t0 = blockIdx.x * (int64_t)kRadixTile;
    for (int r = 0; r < kRadixRounds; ++r) {
        int64_t i = t0 + r * kRadixThreads + threadIdx.x;
        if (i < N) atomicAdd(&cnt[(key[i] >> shift) & 0xFF], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];
}

// Stable scatter of one tile: items are taken in rounds of 256 (thread order
// inside a round, rounds in order); an item's rank is the number of earlier
// items of the tile with the same digit.
__global__ void __launch_bounds__(kRadixThreads)
k_radix_scatter(const unsigned long long *__restrict__ kin, const int32_t *__restrict__ vin,
                unsigned long long *__restrict__ kout, int32_t *__restrict__ vout, int64_t N,
                int shift, int64_t ntiles, const int64_t *__restrict__ off) {
    __shared__ int64_t base[256];
    __shared__ uint32_t running[256];
    __shared__ uint32_t wcount[kRadixThreads / 32][256];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    base[tid] = off[(int64_t)tid * ntiles + blockIdx.x];
    running[tid] = 0;
    const int64_t t0 = blockIdx.x * (int64_t)kRadixTile;
    const unsigned lt = (1u << lane) - 1u;
    for (int r = 0; r < kRadixRounds; ++r) {
        for (int w = 0; w < kRadixThreads / 32; ++w) wcount[w][tid] = 0;
        __syncthreads();
        int64_t i = t0 + r * kRadixThreads + tid;
        bool valid = i < N;
        unsigned long long k = valid ? kin[i] : 0ull;
        int32_t v = valid ? vin[i] : 0;
        unsigned d = valid ? (unsigned)((k >> shift) & 0xFF) : 256u;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        unsigned rank = __popc(peers & lt);
        if (valid && rank == 0) wcount[warp][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            uint32_t pre = 0;
            for (int w = 0; w < warp; ++w) pre += wcount[w][d];
            int64_t pos = base[d] + running[d] + pre + rank;
            kout[pos] = k;
            vout[pos] = v;
        }
        __syncthreads();
        uint32_t tot = 0;
        for (int w = 0; w < kRadixThreads / 32; ++w) tot += wcount[w][tid];
        running[tid] += tot;
        __syncthreads();
    }
}

// -------------------------------------------------------------- prefix scan
// Exclusive scan of mult * in[i] (int64 result, out has n + 1 entries with the
// total in out[n]).  Three kernels: tile sums, scan of tile sums (recursive),
// tile scan plus offset.
__device__ __forceinline__ int64_t block_exclusive(int64_t v, int64_t *warp_tot, int64_t *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t inc = v;
    for (int o = 1; o < 32; o <<= 1) {
        int64_t u = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += u;
    }
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int nw = blockDim.x >> 5;
        int64_t t = lane < nw ? warp_tot[lane] : 0;
        int64_t ti = t;
        for (int o = 1; o < 32; o <<= 1) {
            int64_t u = __shfl_up_sync(0xffffffffu, ti, o);
            if (lane >= o) ti += u;
        }
        if (lane < nw) warp_tot[lane] = ti - t;
        if (lane == nw - 1) *total = ti;
    }
    __syncthreads();
    return inc - v + warp_tot[warp];
}

template <class T>
__global__ void __launch_bounds__(kScanThreads)
k_scan_reduce(const T *__restrict__ in, int64_t mult, int64_t n, int64_t *__restrict__ bsum) {
    __shared__ int64_t wt[32];
    __shared__ int64_t tot;
    int64_t i0 = blockIdx.x * (int64_t)kScanTile + threadIdx.x * kScanItems;
    int64_t s = 0;
#pragma unroll
    for (int q = 0; q < kScanItems; ++q)
        if (i0 + q < n) s += (int64_t)in[i0 + q] * mult;
    block_exclusive(s, wt, &tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

template <class T>
__global__ void __launch_bounds__(kScanThreads)
k_scan_apply(const T *__restrict__ in, int64_t mult, int64_t n, const int64_t *__restrict__ boff,
             int64_t *__restrict__ out) {
    __shared__ int64_t wt[32];
    __shared__ int64_t tot;
    int64_t i0 = blockIdx.x * (int64_t)kScanTile + threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t s = 0;
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
        v[q] = (i0 + q < n) ? (int64_t)in[i0 + q] * mult : 0;
        s += v[q];
    }
    int64_t ex = block_exclusive(s, wt, &tot) + (boff ? boff[blockIdx.x] : 0);
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
        if (i0 + q < n) out[i0 + q] = ex;
        ex += v[q];
    }
    // the tile total (items past n are zero) completes the last tile
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = (boff ? boff[blockIdx.x] : 0) + tot;
}

template <class T>
sell_status scan_exclusive(const T *in, int64_t mult, int64_t n, int64_t *out, const Allocator &al,
                           cudaStream_t s) {
    if (n == 0) {
        SELL_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(int64_t), s));
        return SELL_OK;
    }
    int64_t nb = (n + kScanTile - 1) / kScanTile;
    DevBuf bsum, boff;
    if (nb > 1) {
        SELL_TRY(bsum.alloc(al, nb * sizeof(int64_t), s));
        SELL_TRY(boff.alloc(al, (nb + 1) * sizeof(int64_t), s));
        k_scan_reduce<T><<<(unsigned)nb, kScanThreads, 0, s>>>(in, mult, n, bsum.as<int64_t>());
        SELL_CUDA_TRY(cudaGetLastError());
        SELL_TRY(scan_exclusive<int64_t>(bsum.as<int64_t>(), 1, nb, boff.as<int64_t>(), al, s));
    }
    k_scan_apply<T><<<(unsigned)nb, kScanThreads, 0, s>>>(in, mult, n,
                                                          nb > 1 ? boff.as<int64_t>() : nullptr, out);
    SELL_CUDA_TRY(cudaGetLastError());
    return SELL_OK;
}

// ------------------------------------------------------------- chunk lengths
__global__ void k_chunk_len(const int32_t *__restrict__ rl, const int32_t *__restrict__ perm,
                            int64_t N, int64_t Np, int C, int32_t *__restrict__ srl,
                            int32_t *__restrict__ cl, int32_t *__restrict__ inv) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    bool warp_chunks = (C % 32) == 0;
    // the loop trip count is uniform across a warp because Np is a multiple of
    // C and the grid stride is a multiple of 32
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r - (threadIdx.x & 31) < Np;
         r += stride) {
        bool live = r < Np;
        int32_t len = 0;
        if (live && r < N) {
            int64_t old = perm ? perm[r] : r;
            len = rl[old];
            if (inv) inv[old] = (int32_t)r;
        }
        if (live) srl[r] = len;
        if (warp_chunks) {
            int32_t m = len;
            for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
            if (live && (threadIdx.x & 31) == 0 && m > 0) atomicMax(&cl[r / C], m);
        } else if (live && len > 0) {
            atomicMax(&cl[r / C], len);
        }
    }
}

// ---------------------------------------------------------- long-row chunks
__global__ void k_long_flags(const int32_t *__restrict__ cl, int64_t Nc, int32_t *__restrict__ flag) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < Nc; c += stride)
        flag[c] = cl[c] > kSeg ? 1 : 0;
}

__global__ void k_long_compact(const int32_t *__restrict__ cl, const int64_t *__restrict__ pos, int64_t Nc,
                               int32_t *__restrict__ lchunk) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < Nc; c += stride)
        if (cl[c] > kSeg) lchunk[pos[c]] = (int32_t)c;
}

// Long-row work units: chunk lc has ceil(cl / kSeg) segments; the units are
// numbered chunk by chunk (ubase = exclusive scan of the segment counts).
__global__ void k_long_nseg(const int32_t *__restrict__ cl, const int32_t *__restrict__ lchunk,
                            int64_t nlong, int32_t *__restrict__ nseg) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nlong; i += stride)
        nseg[i] = (cl[lchunk[i]] - 1) / kSeg + 1;  // cl > kSeg for a long chunk
}

__global__ void k_long_units(const int32_t *__restrict__ nseg, const int64_t *__restrict__ ubase,
                             int64_t nlong, int2 *__restrict__ lunit) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nlong; i += stride)
        for (int32_t sg = 0; sg < nseg[i]; ++sg) lunit[ubase[i] + sg] = make_int2((int)i, sg);
}

// Long rows of each long chunk: lrow[i*C + k] = the lane of its k-th row
// longer than kSeg (lane order), lmeta[i] = {m rows, mode, units of the
// chunk, 0}.  Mode 0: unit thread t takes lane t (its row's segment); mode 1,
// for chunks whose long rows are few (8 m <= C): the chunk's unit threads
// take consecutive segments of one long row after another, so a warp runs 32
// segments of a long row instead of one segment of each of 32 mostly short
// rows.  Either way each segment is the same chain and lands in the same
// partial slot (unit of the segment, lane of the row), so the results do not
// depend on the mode.
__global__ void k_long_rows(const int32_t *__restrict__ srl, int64_t N, int C, const int32_t *__restrict__ lchunk,
                            const int32_t *__restrict__ nseg, int64_t nlong, int32_t *__restrict__ lrow,
                            int4 *__restrict__ lmeta) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nlong; i += stride) {
        const int64_t c = lchunk[i];
        int m = 0;
        for (int l = 0; l < C; ++l) {
            const int64_t r = c * C + l;
            if (r < N && srl[r] > kSeg) lrow[i * C + m++] = l;
        }
        lmeta[i] = make_int4(m, 8 * m <= C ? 1 : 0, nseg[i], 0);
    }
}

// ------------------------------------------------- bulk-staged SpMV plan
// bsc[c] = the longest row of at most kSeg entries in chunk c, -1 if the
// chunk has no such row (the columns of chunk c that the bulk-staged SpMV
// copies), and its work weight bw[c] = bsc[c] + 1.  One warp per chunk.
__global__ void k_bulk_cols(const int32_t *__restrict__ srl, int64_t N, int64_t Nc, int C,
                            int32_t *__restrict__ bsc, int32_t *__restrict__ bw) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t c = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); c < Nc; c += nw) {
        int m = -1;
        for (int l = lane; l < C; l += 32) {
            const int len = srl[c * C + l];
            if (c * C + l < N && len <= kSeg) m = max(m, len);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) {
            bsc[c] = m;
            bw[c] = m + 1;
        }
    }
}

// wsplit[w] = first chunk c with bss[c] >= w * total / nw (bss = exclusive
// scan of the weights bw, bss[Nc] = total), wsplit[nw] = Nc: warp w stages
// chunks [wsplit[w], wsplit[w+1]), about total / nw weight.
__global__ void k_bulk_split(const int64_t *__restrict__ bss, int64_t Nc, int64_t nw, int32_t *__restrict__ wsplit) {
    const int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (w > nw) return;
    if (w == nw) {
        wsplit[w] = (int32_t)Nc;
        return;
    }
    const int64_t total = bss[Nc];
    const int64_t target = total * w / nw;  // total <= 64 * Nc < 2^37, w <= nw < 2^20
    int64_t lo = 0, hi = Nc;  // first index in [0, Nc] with bss >= target
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (bss[mid] < target) lo = mid + 1;
        else hi = mid;
    }
    wsplit[w] = (int32_t)lo;
}

// ------------------------------------------------------------------ scatter
template <class TI, class TO> __device__ __forceinline__ TO cvt(TI v);
template <> __device__ __forceinline__ double cvt<double, double>(double v) { return v; }
template <> __device__ __forceinline__ float cvt<double, float>(double v) { return __double2float_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 cvt<double, __nv_bfloat16>(double v) {
    return __double2bfloat16(v);
}
template <> __device__ __forceinline__ double cvt<float, double>(float v) { return (double)v; }
template <> __device__ __forceinline__ float cvt<float, float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 cvt<float, __nv_bfloat16>(float v) {
    return __float2bfloat16_rn(v);
}
template <class TO> __device__ __forceinline__ TO zero_of();
template <> __device__ __forceinline__ double zero_of<double>() { return 0.0; }
template <> __device__ __forceinline__ float zero_of<float>() { return 0.0f; }
template <> __device__ __forceinline__ __nv_bfloat16 zero_of<__nv_bfloat16>() {
    return __ushort_as_bfloat16((unsigned short)0);
}

// One thread per sorted row; the C threads of a chunk write one stored column
// (C consecutive elements) per step j, so stores are coalesced for C >= 32.
template <class TI, class TO>
__global__ void k_scatter(const int64_t *__restrict__ rpt, const int32_t *__restrict__ col_in,
                          const TI *__restrict__ val_in, const int32_t *__restrict__ perm,
                          const int32_t *__restrict__ inv, const int32_t *__restrict__ srl,
                          const int32_t *__restrict__ cl, const int64_t *__restrict__ cs, int64_t N,
                          int64_t Np, int C, TO *__restrict__ val, int32_t *__restrict__ col) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < Np; r += stride) {
        int64_t c = r / C;
        int l = (int)(r - c * C);
        int32_t width = cl[c];
        int32_t len = srl[r];
        int64_t src = 0;
        if (r < N && len > 0) src = rpt[perm ? perm[r] : r];
        int64_t pos = cs[c] + l;
        for (int32_t j = 0; j < width; ++j, pos += C) {
            if (j < len) {
                int32_t cidx = col_in[src + j];
                val[pos] = cvt<TI, TO>(val_in[src + j]);
                col[pos] = inv ? inv[cidx] : cidx;
            } else {
                val[pos] = zero_of<TO>();
                col[pos] = 0;
            }
        }
    }
}

template <class TI>
sell_status launch_scatter(const sell_csr &A, const int64_t *rpt, const int32_t *col_in,
                           const void *val_in, const int32_t *perm, const int32_t *inv,
                           const int32_t *srl, const int32_t *cl, const int64_t *cs, int64_t Np,
                           int C, int store, void *val, int32_t *col, cudaStream_t s) {
    int g = grid_for(Np, 256);
    const TI *vi = static_cast<const TI *>(val_in);
    switch (store) {
        case SELL_F64:
            k_scatter<TI, double><<<g, 256, 0, s>>>(rpt, col_in, vi, perm, inv, srl, cl, cs, A.nrows,
                                                    Np, C, (double *)val, col);
            break;
        case SELL_F32:
            k_scatter<TI, float><<<g, 256, 0, s>>>(rpt, col_in, vi, perm, inv, srl, cl, cs, A.nrows,
                                                   Np, C, (float *)val, col);
            break;
        default:
            k_scatter<TI, __nv_bfloat16><<<g, 256, 0, s>>>(rpt, col_in, vi, perm, inv, srl, cl, cs,
                                                           A.nrows, Np, C, (__nv_bfloat16 *)val, col);
            break;
    }
    SELL_CUDA_TRY(cudaGetLastError());
    return SELL_OK;
}

int bits_for(unsigned long long v) {  // bits needed to hold 0..v
    int b = 0;
    while (b < 64 && (v >> b) != 0) ++b;
    return b;
}

sell_status sort_windows(const int32_t *rl, int64_t N, int64_t sigma, int max_rl, int32_t *perm,
                         const Allocator &al, cudaStream_t s) {
    const int64_t W = std::min<int64_t>(sigma, N);
    if (W <= kWindowSortMax) {
        int wpb = (int)std::max<int64_t>(1, kWindowSortMax / W);
        int64_t tile = wpb * W;
        int P = 1;
        while (P < tile) P <<= 1;
        int64_t nblk = (N + tile - 1) / tile;
        size_t smem = (size_t)P * sizeof(unsigned long long);
        k_window_sort<<<(unsigned)nblk, 1024, smem, s>>>(rl, N, W, wpb, P, perm);
        SELL_CUDA_TRY(cudaGetLastError());
        return SELL_OK;
    }
    // LSD radix sort on (window, max_rl - rowLen), stable, values = row ids
    int64_t nwin = (N + sigma - 1) / sigma;
    int lbits = std::max(1, bits_for((unsigned long long)max_rl));
    int wbits = bits_for((unsigned long long)(nwin - 1));
    int total = lbits + wbits;
    if (total > 64) return fail(SELL_EUNSUPPORTED, "sort key wider than 64 bits");
    int passes = (total + 7) / 8;
    int64_t ntiles = (N + kRadixTile - 1) / kRadixTile;
    DevBuf k0, k1, v1, hist, off;
    SELL_TRY(k0.alloc(al, N * sizeof(unsigned long long), s));
    SELL_TRY(k1.alloc(al, N * sizeof(unsigned long long), s));
    SELL_TRY(v1.alloc(al, N * sizeof(int32_t), s));
    SELL_TRY(hist.alloc(al, 256 * ntiles * sizeof(uint32_t), s));
    SELL_TRY(off.alloc(al, (256 * ntiles + 1) * sizeof(int64_t), s));
    unsigned long long *ka = k0.as<unsigned long long>(), *kb = k1.as<unsigned long long>();
    // the values ping-pong between perm and v1; an odd pass count ends in v1
    int32_t *va = (passes % 2 == 0) ? perm : v1.as<int32_t>();
    int32_t *vb = (passes % 2 == 0) ? v1.as<int32_t>() : perm;
    k_radix_init<<<grid_for(N, 256), 256, 0, s>>>(rl, N, sigma, lbits, max_rl, ka, va);
    SELL_CUDA_TRY(cudaGetLastError());
    for (int p = 0; p < passes; ++p) {
        int shift = 8 * p;
        k_radix_hist<<<(unsigned)ntiles, kRadixThreads, 0, s>>>(ka, N, shift, ntiles,
                                                               hist.as<uint32_t>());
        SELL_CUDA_TRY(cudaGetLastError());
        SELL_TRY(scan_exclusive<uint32_t>(hist.as<uint32_t>(), 1, 256 * ntiles, off.as<int64_t>(),
                                          al, s));
        k_radix_scatter<<<(unsigned)ntiles, kRadixThreads, 0, s>>>(ka, va, kb, vb, N, shift, ntiles,
                                                                   off.as<int64_t>());
        SELL_CUDA_TRY(cudaGetLastError());
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    // after the last swap `va` holds the result and is `perm` by construction
    return SELL_OK;
}

sell_status validate(const sell_csr *A, const sell_opts *o) {
    if (!A || !o) return fail(SELL_EINVAL, "sell_build: NULL matrix or options");
    if (o->C < 1) return fail(SELL_EINVAL, "sell_build: C must be >= 1");
    if (o->sigma < 1) return fail(SELL_EINVAL, "sell_build: sigma must be >= 1");
    if (o->store_type != SELL_F64 && o->store_type != SELL_F32 && o->store_type != SELL_BF16)
        return fail(SELL_EINVAL, "sell_build: unknown store_type");
    if (o->reserved != 0) return fail(SELL_EINVAL, "sell_build: reserved must be 0");
    if (o->flags & ~SELL_BUILD_PERMUTE_COLS) return fail(SELL_EINVAL, "sell_build: unknown flags");
    if (A->nrows < 0 || A->ncols < 0 || A->nnz < 0)
        return fail(SELL_EINVAL, "sell_build: negative size");
    if (A->nrows > 0x7FFFFFFFll || A->ncols > 0x7FFFFFFFll)
        return fail(SELL_EINVAL, "sell_build: nrows and ncols must be below 2^31");
    if (A->val_type != SELL_F64 && A->val_type != SELL_F32)
        return fail(SELL_EINVAL, "sell_build: val_type must be SELL_F64 or SELL_F32");
    if (!A->rpt) return fail(SELL_EINVAL, "sell_build: NULL rpt");
    if (A->nnz > 0 && (!A->col || !A->val)) return fail(SELL_EINVAL, "sell_build: NULL col/val");
    if ((o->flags & SELL_BUILD_PERMUTE_COLS) && A->nrows != A->ncols)
        return fail(SELL_EINVAL, "sell_build: column permutation needs a square matrix");
    int64_t np = (A->nrows + o->C - 1) / o->C * (int64_t)o->C;
    if (np > 0x7FFFFFFFll) return fail(SELL_EINVAL, "sell_build: padded row count exceeds 2^31");
    return SELL_OK;
}

}  // namespace

sell_status build_format(const sell_csr *A, const sell_opts *o, cudaStream_t s, sell_matrix *h) {
    SELL_TRY(validate(A, o));
    const Allocator al = current_allocator();
    const int64_t N = A->nrows, nnz = A->nnz;
    const int C = o->C;
    const int64_t Nc = (N + C - 1) / C, Np = Nc * C;
    const size_t vin = A->val_type == SELL_F64 ? 8 : 4;

    // 1. the CRS arrays on the device
    DevBuf drpt, dcol, dval;
    const int64_t *rpt = A->rpt;
    const int32_t *col_in = A->col;
    const void *val_in = A->val;
    if (!A->on_device) {
        if (A->rpt[0] != 0 || A->rpt[N] != nnz)
            return fail(SELL_EINVAL, "sell_build: rpt[0] must be 0 and rpt[nrows] must be nnz");
        SELL_TRY(drpt.alloc(al, (N + 1) * sizeof(int64_t), s));
        SELL_CUDA_TRY(cudaMemcpyAsync(drpt.p, A->rpt, (N + 1) * sizeof(int64_t),
                                      cudaMemcpyHostToDevice, s));
        if (nnz > 0) {
            SELL_TRY(dcol.alloc(al, nnz * sizeof(int32_t), s));
            SELL_TRY(dval.alloc(al, nnz * vin, s));
            SELL_CUDA_TRY(cudaMemcpyAsync(dcol.p, A->col, nnz * sizeof(int32_t),
                                          cudaMemcpyHostToDevice, s));
            SELL_CUDA_TRY(cudaMemcpyAsync(dval.p, A->val, nnz * vin, cudaMemcpyHostToDevice, s));
        }
        rpt = drpt.as<int64_t>();
        col_in = dcol.as<int32_t>();
        val_in = dval.p;
    }

    // 2. row lengths + validation
    DevBuf rl, stats;
    SELL_TRY(stats.alloc(al, sizeof(BuildStats), s));
    SELL_CUDA_TRY(cudaMemsetAsync(stats.p, 0, sizeof(BuildStats), s));
    if (N > 0) {
        SELL_TRY(rl.alloc(al, N * sizeof(int32_t), s));
        k_rowlen<<<grid_for(N, 256, 152 * 16), 256, 0, s>>>(rpt, N, nnz, rl.as<int32_t>(),
                                                            stats.as<BuildStats>());
        SELL_CUDA_TRY(cudaGetLastError());
    }
    if (nnz > 0) {
        k_colcheck<<<grid_for(nnz, 256, 152 * 16), 256, 0, s>>>(col_in, nnz, A->ncols,
                                                                stats.as<BuildStats>());
        SELL_CUDA_TRY(cudaGetLastError());
    }
    BuildStats hs;
    SELL_CUDA_TRY(cudaMemcpyAsync(&hs, stats.p, sizeof(hs), cudaMemcpyDeviceToHost, s));
    SELL_CUDA_TRY(cudaStreamSynchronize(s));
    if (N == 0 && nnz != 0) hs.err |= kErrRptEnd;
    if (hs.err) {
        std::string m = "sell_build: malformed CRS:";
        if (hs.err & kErrRpt0) m += " rpt[0] != 0;";
        if (hs.err & kErrRptOrder) m += " rpt decreasing;";
        if (hs.err & kErrRptEnd) m += " rpt[nrows] != nnz;";
        if (hs.err & kErrRowLong) m += " row longer than 2^31-1;";
        if (hs.err & kErrCol) m += " column index out of range;";
        return fail(SELL_EINVAL, m);
    }

    // 3. sorting scope
    DevBuf perm;
    const bool sorted = o->sigma > 1 && N > 1;
    if (sorted) {
        SELL_TRY(perm.alloc(al, N * sizeof(int32_t), s));
        SELL_TRY(sort_windows(rl.as<int32_t>(), N, o->sigma, hs.max_rl, perm.as<int32_t>(), al, s));
    }

    // 4. chunk lengths (Eq. "max") and sorted row lengths
    DevBuf srl, cl, cs, inv;
    if (Np > 0) {
        SELL_TRY(srl.alloc(al, Np * sizeof(int32_t), s));
        SELL_TRY(cl.alloc(al, Nc * sizeof(int32_t), s));
        SELL_CUDA_TRY(cudaMemsetAsync(cl.p, 0, Nc * sizeof(int32_t), s));
    }
    const bool permute_cols = (o->flags & SELL_BUILD_PERMUTE_COLS) != 0;
    if (permute_cols && N > 0) SELL_TRY(inv.alloc(al, N * sizeof(int32_t), s));
    if (Np > 0) {
        int g = grid_for(Np, 256);
        k_chunk_len<<<g, 256, 0, s>>>(rl.as<int32_t>(), sorted ? perm.as<int32_t>() : nullptr, N, Np,
                                      C, srl.as<int32_t>(), cl.as<int32_t>(),
                                      permute_cols ? inv.as<int32_t>() : nullptr);
        SELL_CUDA_TRY(cudaGetLastError());
    }
    // 5. chunk offsets, and the chunks that hold rows longer than kSeg
    SELL_TRY(cs.alloc(al, (Nc + 1) * sizeof(int64_t), s));
    SELL_TRY(scan_exclusive<int32_t>(cl.as<int32_t>(), C, Nc, cs.as<int64_t>(), al, s));
    DevBuf lflag, lpos;
    if (Nc > 0) {
        SELL_TRY(lflag.alloc(al, Nc * sizeof(int32_t), s));
        SELL_TRY(lpos.alloc(al, (Nc + 1) * sizeof(int64_t), s));
        k_long_flags<<<grid_for(Nc, 256), 256, 0, s>>>(cl.as<int32_t>(), Nc, lflag.as<int32_t>());
        SELL_CUDA_TRY(cudaGetLastError());
        SELL_TRY(scan_exclusive<int32_t>(lflag.as<int32_t>(), 1, Nc, lpos.as<int64_t>(), al, s));
    }
    int64_t stored = 0, nlong = 0;
    SELL_CUDA_TRY(cudaMemcpyAsync(&stored, cs.as<int64_t>() + Nc, sizeof(int64_t),
                                  cudaMemcpyDeviceToHost, s));
    if (Nc > 0)
        SELL_CUDA_TRY(cudaMemcpyAsync(&nlong, lpos.as<int64_t>() + Nc, sizeof(int64_t),
                                      cudaMemcpyDeviceToHost, s));
    SELL_CUDA_TRY(cudaStreamSynchronize(s));
    DevBuf lchunk, lnseg, lubase, lunit, cnt, cnt2, part, lrow, lmeta;
    int64_t nunits = 0;
    if (nlong > 0) {
        SELL_TRY(lchunk.alloc(al, nlong * sizeof(int32_t), s));
        k_long_compact<<<grid_for(Nc, 256), 256, 0, s>>>(cl.as<int32_t>(), lpos.as<int64_t>(), Nc,
                                                         lchunk.as<int32_t>());
        SELL_CUDA_TRY(cudaGetLastError());
        SELL_TRY(lnseg.alloc(al, nlong * sizeof(int32_t), s));
        SELL_TRY(lubase.alloc(al, (nlong + 1) * sizeof(int64_t), s));
        k_long_nseg<<<grid_for(nlong, 256), 256, 0, s>>>(cl.as<int32_t>(), lchunk.as<int32_t>(), nlong,
                                                         lnseg.as<int32_t>());
        SELL_CUDA_TRY(cudaGetLastError());
        SELL_TRY(scan_exclusive<int32_t>(lnseg.as<int32_t>(), 1, nlong, lubase.as<int64_t>(), al, s));
        SELL_CUDA_TRY(cudaMemcpyAsync(&nunits, lubase.as<int64_t>() + nlong, sizeof(int64_t),
                                      cudaMemcpyDeviceToHost, s));
        SELL_CUDA_TRY(cudaStreamSynchronize(s));
        SELL_TRY(lunit.alloc(al, nunits * sizeof(int2), s));
        k_long_units<<<grid_for(nlong, 256), 256, 0, s>>>(lnseg.as<int32_t>(), lubase.as<int64_t>(), nlong,
                                                          lunit.as<int2>());
        SELL_CUDA_TRY(cudaGetLastError());
        SELL_TRY(lrow.alloc(al, (size_t)nlong * C * sizeof(int32_t), s));
        SELL_TRY(lmeta.alloc(al, (size_t)nlong * sizeof(int4), s));
        k_long_rows<<<grid_for(nlong, 256), 256, 0, s>>>(srl.as<int32_t>(), N, C, lchunk.as<int32_t>(),
                                                         lnseg.as<int32_t>(), nlong, lrow.as<int32_t>(),
                                                         lmeta.as<int4>());
        SELL_CUDA_TRY(cudaGetLastError());
        SELL_TRY(cnt.alloc(al, nlong * C * sizeof(int32_t), s));
        SELL_CUDA_TRY(cudaMemsetAsync(cnt.p, 0, nlong * C * sizeof(int32_t), s));
        SELL_TRY(cnt2.alloc(al, (size_t)nunits * C * sizeof(int32_t), s));
        SELL_CUDA_TRY(cudaMemsetAsync(cnt2.p, 0, (size_t)nunits * C * sizeof(int32_t), s));
        SELL_TRY(part.alloc(al, (size_t)nunits * C * 8, s));
    }

    // 6. values and columns
    DevBuf val, col;
    const size_t vs = value_size(o->store_type);
    if (stored > 0) {
        SELL_TRY(val.alloc(al, stored * vs, s));
        SELL_TRY(col.alloc(al, stored * sizeof(int32_t), s));
        if (A->val_type == SELL_F64)
            SELL_TRY(launch_scatter<double>(*A, rpt, col_in, val_in, sorted ? perm.as<int32_t>() : nullptr,
                                            permute_cols ? inv.as<int32_t>() : nullptr,
                                            srl.as<int32_t>(), cl.as<int32_t>(), cs.as<int64_t>(), Np, C,
                                            o->store_type, val.p, col.as<int32_t>(), s));
        else
            SELL_TRY(launch_scatter<float>(*A, rpt, col_in, val_in, sorted ? perm.as<int32_t>() : nullptr,
                                           permute_cols ? inv.as<int32_t>() : nullptr,
                                           srl.as<int32_t>(), cl.as<int32_t>(), cs.as<int64_t>(), Np, C,
                                           o->store_type, val.p, col.as<int32_t>(), s));
    }
    SELL_CUDA_TRY(cudaStreamSynchronize(s));

    // 7. hand the arrays to the handle
    h->nrows = N;
    h->ncols = A->ncols;
    h->nnz = nnz;
    h->nchunks = Nc;
    h->stored = stored;
    h->sigma = o->sigma;
    h->max_rl = hs.max_rl;
    h->C = C;
    h->store_type = o->store_type;
    h->flags = o->flags;
    h->beta = stored > 0 ? (double)nnz / (double)stored : 1.0;
    if (N > 0 && nnz > 0) {
        double mean = (double)nnz / (double)N;
        double var = (double)hs.sumsq / (double)N - mean * mean;
        h->zeta = var > 0 ? std::sqrt(var) / mean : 0.0;
    } else {
        h->zeta = 0.0;
    }
    h->al = al;
    h->nlong = nlong;
    h->nunits = nunits;
    h->part_k = nunits > 0 ? 1 : 0;
    h->device_bytes = val.bytes + col.bytes + cs.bytes + cl.bytes + srl.bytes + perm.bytes + lchunk.bytes +
                      lunit.bytes + cnt.bytes + cnt2.bytes + part.bytes + lrow.bytes + lmeta.bytes;
    h->lchunk = (int32_t *)lchunk.release_ownership();
    h->lunit = (int2 *)lunit.release_ownership();
    h->lrow = (int32_t *)lrow.release_ownership();
    h->lmeta = (int4 *)lmeta.release_ownership();
    h->cnt = (int32_t *)cnt.release_ownership();
    h->cnt2 = (int32_t *)cnt2.release_ownership();
    h->part = part.release_ownership();
    h->val = val.release_ownership();
    h->col = (int32_t *)col.release_ownership();
    h->cs = (int64_t *)cs.release_ownership();
    h->cl = (int32_t *)cl.release_ownership();
    h->srl = (int32_t *)srl.release_ownership();
    h->perm = (int32_t *)perm.release_ownership();
    return SELL_OK;
}

// The per-warp work split of the bulk-staged SpMV for nw warps (the per-chunk
// staged columns are computed on the first call).  Synchronises s.
sell_status bulk_plan(sell_matrix *h, int64_t nw, cudaStream_t s) {
    const int64_t Nc = h->nchunks;
    if (Nc >= INT32_MAX || nw >= (1 << 20)) return fail(SELL_EUNSUPPORTED, "bulk-staged SpMV: plan too large");
    const Allocator &al = h->al;
    if (!h->dstat) {
        void *p = al.get(sizeof(int32_t), s);
        if (!p) return fail(SELL_ENOMEM, "bulk plan allocation failed");
        h->dstat = static_cast<int32_t *>(p);
        SELL_CUDA_TRY(cudaMemsetAsync(h->dstat, 0, sizeof(int32_t), s));
    }
    DevBuf bss, bw;
    if (h->wsplit_n != nw && Nc > 0) {
        SELL_TRY(bw.alloc(al, Nc * sizeof(int32_t), s));
        if (!h->bsc) {
            void *p = al.get(Nc * sizeof(int32_t), s);
            if (!p) return fail(SELL_ENOMEM, "bulk plan allocation failed");
            h->bsc = static_cast<int32_t *>(p);
        }
        k_bulk_cols<<<grid_for(Nc * 32, 256, 152 * 16), 256, 0, s>>>(h->srl, h->nrows, Nc, h->C, h->bsc,
                                                                      bw.as<int32_t>());
        SELL_CUDA_TRY(cudaGetLastError());
    }
    if (h->wsplit_n != nw) {
        if (h->wsplit) {
            al.put(h->wsplit, s);
            h->wsplit = nullptr;
            h->wsplit_n = 0;
        }
        void *p = al.get((nw + 1) * sizeof(int32_t), s);
        if (!p) return fail(SELL_ENOMEM, "bulk plan allocation failed");
        h->wsplit = static_cast<int32_t *>(p);
        SELL_TRY(bss.alloc(al, (Nc + 1) * sizeof(int64_t), s));
        if (Nc > 0) {
            SELL_TRY(scan_exclusive<int32_t>(bw.as<int32_t>(), 1, Nc, bss.as<int64_t>(), al, s));
        } else {
            SELL_CUDA_TRY(cudaMemsetAsync(bss.p, 0, sizeof(int64_t), s));
        }
        k_bulk_split<<<grid_for(nw + 1, 256), 256, 0, s>>>(bss.as<int64_t>(), Nc, nw, h->wsplit);
        SELL_CUDA_TRY(cudaGetLastError());
        h->wsplit_n = nw;
    }
    SELL_CUDA_TRY(cudaStreamSynchronize(s));
    return SELL_OK;
}

}  // namespace sell
