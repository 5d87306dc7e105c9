/*
 * sell_oracle.c -- plain, slow, obviously correct CPU oracle for SELL-C-sigma.
 *
 * TEST INFRASTRUCTURE ONLY.  This file exists to check the CUDA library; it is
 * not part of the product path.  Only the test suite, the smoke check in
 * __graft_entry__.py and the CPU-baseline leg of bench.py may load it.  It
 * shares no code, header, table or constant with the CUDA library.
 *
 * Source of every function: Kreutzer, Hager, Wellein, Fehske, Bishop,
 * "A unified sparse matrix data format for efficient general sparse
 * matrix-vector multiply on modern processors with wide SIMD units"
 * (arXiv:1307.6209).
 *
 * Arithmetic: IEEE binary64, compiled with -ffp-contract=off so that every
 * product and every sum is rounded separately (no fused multiply-add).  The
 * summation order inside a row is the CRS order of Listing "crs".
 *
 * Parity pins (all in tests/test_oracle_pins.py):
 *   orc_csr_spmv / orc_csr_spmmv / orc_csr_spmv_rows : exact rational
 *       arithmetic on tiny matrices (error within n*u*sum|a||x|), dense
 *       brute force, Laplacian row sums with x = 1.
 *   orc_sell_plan / orc_sell_fill : SELL-1-1 == CRS, SELL-N-1 == ELLPACK,
 *       sigma >= N == pJDS (sort invariants), beta closed forms of Sec. 3.4
 *       (Eq. "betaworst", sigma = C^2 gives beta = 1, constant chunk row
 *       length gives beta = 1, sigma dividing C leaves beta unchanged).
 *   orc_sell_spmv : bitwise equal to orc_csr_spmv for finite x, for every
 *       (C, sigma).
 *   orc_round : f32 leg equals the C cast; bf16 leg checked on hand-derived
 *       ties, overflow and subnormal boundaries.
 *   orc_zeta : closed form on constant and two-valued length profiles.
 * The pins are themselves tested: tests/test_oracle_mutants.py plants one
 * plausible mistake at a time in a copy of this file and checks that a named
 * pin fails; tests/test_oracle_properties.py checks the same facts on random
 * small matrices (hypothesis).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Sec. 3.1, Listing "crs": y_i = sum_{j=rpt[i]}^{rpt[i+1]-1} val[j] x[col[j]].
 * accumulate = 0 : y = A x   (sum starts at +0.0)
 * accumulate = 1 : y = y + A x (sum starts at the old y_i, as in the listing)
 * The row loop may run on several OpenMP threads; each row is summed by one
 * thread in CRS order, so the result does not depend on the thread count.
 * schedule_guided selects GUIDED,1 instead of STATIC, the heuristic of Sec. 5
 * (Eq. "cv"). */
void orc_csr_spmv(int64_t nrows, const int64_t *rpt, const int32_t *col,
                  const double *val, const double *x, double *y,
                  int accumulate, int nthreads, int schedule_guided)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
    omp_set_schedule(schedule_guided ? omp_sched_guided : omp_sched_static,
                     schedule_guided ? 1 : 0);
#pragma omp parallel for schedule(runtime)
#endif
    for (int64_t i = 0; i < nrows; ++i) {
        double s = accumulate ? y[i] : 0.0;
        for (int64_t j = rpt[i]; j < rpt[i + 1]; ++j) {
            double p = val[j] * x[col[j]];
            s = s + p;
        }
        y[i] = s;
    }
    (void)nthreads;
    (void)schedule_guided;
}

/* The same definition evaluated for a list of rows only (used to check
 * sampled outputs of very large products one row at a time). */
void orc_csr_spmv_rows(const int64_t *rpt, const int32_t *col,
                       const double *val, const double *x,
                       const int64_t *rows, int64_t nsel, double *out,
                       double *absout)
{
    for (int64_t t = 0; t < nsel; ++t) {
        int64_t i = rows[t];
        double s = 0.0, a = 0.0;
        for (int64_t j = rpt[i]; j < rpt[i + 1]; ++j) {
            double p = val[j] * x[col[j]];
            s = s + p;
            a = a + fabs(p);
        }
        out[t] = s;
        if (absout) absout[t] = a;
    }
}

/* Multiple right-hand sides: Y[:, c] = A X[:, c] for c < k, with X (ncols x k)
 * and Y (nrows x k) row-major with leading dimensions ldx, ldy.  Each column
 * is the definition above; nothing else. */
void orc_csr_spmmv(int64_t nrows, const int64_t *rpt, const int32_t *col,
                   const double *val, int32_t k, const double *X, int64_t ldx,
                   double *Y, int64_t ldy, int accumulate)
{
    for (int64_t i = 0; i < nrows; ++i) {
        for (int32_t c = 0; c < k; ++c) {
            double s = accumulate ? Y[i * ldy + c] : 0.0;
            for (int64_t j = rpt[i]; j < rpt[i + 1]; ++j) {
                double p = val[j] * X[(int64_t)col[j] * ldx + c];
                s = s + p;
            }
            Y[i * ldy + c] = s;
        }
    }
}

/* Row-wise sum of |a_ij x_j| (the scale of the rounding-error bound). */
void orc_csr_absdot(int64_t nrows, const int64_t *rpt, const int32_t *col,
                    const double *val, const double *x, double *out)
{
    for (int64_t i = 0; i < nrows; ++i) {
        double a = 0.0;
        for (int64_t j = rpt[i]; j < rpt[i + 1]; ++j)
            a = a + fabs(val[j] * x[col[j]]);
        out[i] = a;
    }
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.3 / 3.4: the SELL-C-sigma format, built step by step.
 *
 * Step 1  rowLen[i] = rpt[i+1] - rpt[i].
 * Step 2  rows are sorted by rowLen in descending order inside each window of
 *         sigma consecutive rows [w*sigma, min((w+1)*sigma, N)); equal lengths
 *         keep their original order (stable).  perm[new] = old.  sigma <= 1
 *         sorts nothing; sigma >= N sorts globally (pJDS).
 * Step 3  Nc = ceil(N / C); cl[c] = max of rowLen over the rows c*C..c*C+C-1
 *         of the sorted order (Eq. "max"); rows past N have length 0.
 * Step 4  cs[0] = 0, cs[c+1] = cs[c] + C * cl[c]   (cl[i] = (cs[i+1]-cs[i])/C).
 * Step 5  entry j of sorted row r = c*C + l is stored at cs[c] + j*C + l
 *         (column-major inside the chunk, Listing "sell"); padding has
 *         val = 0 and col = 0 (Sec. 4).
 */
typedef struct {
    int32_t len;
    int64_t row;
} orc_key;

static int orc_key_cmp(const void *pa, const void *pb)
{
    const orc_key *a = (const orc_key *)pa, *b = (const orc_key *)pb;
    if (a->len != b->len) return (a->len > b->len) ? -1 : 1; /* longer first */
    if (a->row != b->row) return (a->row < b->row) ? -1 : 1; /* stable ties */
    return 0;
}

/* Steps 1-4.  Outputs: rl[N] (original order), perm[N], cl[Nc], cs[Nc+1].
 * Returns 0, or -1 for invalid parameters / a row longer than INT32_MAX,
 * or -2 when out of memory. */
int orc_sell_plan(int64_t nrows, const int64_t *rpt, int32_t C, int64_t sigma,
                  int32_t *rl, int32_t *perm, int32_t *cl, int64_t *cs)
{
    if (nrows < 0 || C < 1 || sigma < 1) return -1;
    for (int64_t i = 0; i < nrows; ++i) {
        int64_t len = rpt[i + 1] - rpt[i];
        if (len < 0 || len > INT32_MAX) return -1;
        rl[i] = (int32_t)len;
    }
    int64_t win = (sigma > nrows) ? nrows : sigma;
    if (win <= 1) {
        for (int64_t i = 0; i < nrows; ++i) perm[i] = (int32_t)i;
    } else {
        orc_key *keys = (orc_key *)malloc(sizeof(orc_key) * (size_t)win);
        if (!keys) return -2;
        for (int64_t w0 = 0; w0 < nrows; w0 += sigma) {
            int64_t w1 = w0 + sigma < nrows ? w0 + sigma : nrows;
            for (int64_t i = w0; i < w1; ++i) {
                keys[i - w0].len = rl[i];
                keys[i - w0].row = i;
            }
            qsort(keys, (size_t)(w1 - w0), sizeof(orc_key), orc_key_cmp);
            for (int64_t i = w0; i < w1; ++i) perm[i] = (int32_t)keys[i - w0].row;
        }
        free(keys);
    }
    int64_t nc = (nrows + C - 1) / C;
    cs[0] = 0;
    for (int64_t c = 0; c < nc; ++c) {
        int32_t m = 0;
        for (int32_t l = 0; l < C; ++l) {
            int64_t r = c * C + l;
            int32_t len = (r < nrows) ? rl[perm[r]] : 0;
            if (len > m) m = len;
        }
        cl[c] = m;
        cs[c + 1] = cs[c] + (int64_t)C * m;
    }
    return 0;
}

/* Step 5, plus the per-sorted-row length array srl[Nc*C] (rows past N get 0).
 * permute_cols = 1 renumbers columns into the sorted order (square matrices
 * only): col' = invperm[col], the symmetric permutation of Sec. 3.4. */
int orc_sell_fill(int64_t nrows, int64_t ncols, const int64_t *rpt,
                  const int32_t *col, const double *val, int32_t C,
                  const int32_t *rl, const int32_t *perm, const int32_t *cl,
                  const int64_t *cs, int permute_cols, double *sval,
                  int32_t *scol, int32_t *srl)
{
    int64_t nc = (nrows + C - 1) / C;
    int32_t *inv = NULL;
    if (permute_cols) {
        if (ncols != nrows) return -1;
        inv = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nrows > 0 ? nrows : 1));
        if (!inv) return -2;
        for (int64_t r = 0; r < nrows; ++r) inv[perm[r]] = (int32_t)r;
    }
    for (int64_t c = 0; c < nc; ++c) {
        for (int32_t l = 0; l < C; ++l) {
            int64_t r = c * C + l;
            int64_t old = (r < nrows) ? perm[r] : -1;
            int32_t len = (old >= 0) ? rl[old] : 0;
            srl[r] = len;
            for (int32_t j = 0; j < cl[c]; ++j) {
                int64_t pos = cs[c] + (int64_t)j * C + l;
                if (j < len) {
                    int64_t src = rpt[old] + j;
                    sval[pos] = val[src];
                    scol[pos] = inv ? inv[col[src]] : col[src];
                } else {
                    sval[pos] = 0.0;
                    scol[pos] = 0;
                }
            }
        }
    }
    free(inv);
    return 0;
}

/* Listing "sell" generalised from C = 4 to any C: loop over chunks, over the
 * chunk length cl[c] (padding included), over the C rows of the chunk.  The
 * sorted-order results are then put back in original order, y[perm[r]], or
 * left in sorted order when permuted_io = 1 (x is then in sorted order too). */
void orc_sell_spmv(int64_t nrows, int32_t C, const int32_t *perm,
                   const int32_t *cl, const int64_t *cs, const double *sval,
                   const int32_t *scol, const double *x, double *y,
                   int accumulate, int permuted_io)
{
    int64_t nc = (nrows + C - 1) / C;
    double *tmp = (double *)malloc(sizeof(double) * (size_t)(nc * C > 0 ? nc * C : 1));
    if (!tmp) return;
    for (int64_t r = 0; r < nc * C; ++r) {
        double init = 0.0;
        if (accumulate && r < nrows) init = permuted_io ? y[r] : y[perm[r]];
        tmp[r] = init;
    }
    for (int64_t c = 0; c < nc; ++c) {
        for (int32_t j = 0; j < cl[c]; ++j) {
            for (int32_t l = 0; l < C; ++l) {
                int64_t pos = cs[c] + (int64_t)j * C + l;
                double p = sval[pos] * x[scol[pos]];
                tmp[c * C + l] = tmp[c * C + l] + p;
            }
        }
    }
    for (int64_t r = 0; r < nrows; ++r) {
        if (permuted_io) y[r] = tmp[r];
        else y[perm[r]] = tmp[r];
    }
    free(tmp);
}

/* Eq. "beta": chunk occupancy = Nnz / sum_{c<Nc} C * cl[c]. */
double orc_beta(int64_t nnz, int64_t nchunks, int32_t C, const int32_t *cl)
{
    int64_t stored = 0;
    for (int64_t c = 0; c < nchunks; ++c) stored += (int64_t)C * cl[c];
    return stored > 0 ? (double)nnz / (double)stored : 1.0;
}

/* Eq. "cv": zeta = sqrt( sum_i (rowLen_i - Nnzr)^2 / N ) / Nnzr, Nnzr = Nnz/N
 * (the sum runs over the N rows i = 0..N-1). */
double orc_zeta(int64_t nrows, const int32_t *rl)
{
    if (nrows <= 0) return 0.0;
    double sum = 0.0;
    for (int64_t i = 0; i < nrows; ++i) sum += rl[i];
    double mean = sum / (double)nrows;
    if (mean == 0.0) return 0.0;
    double sq = 0.0;
    for (int64_t i = 0; i < nrows; ++i) {
        double d = rl[i] - mean;
        sq += d * d;
    }
    return sqrt(sq / (double)nrows) / mean;
}

/* ------------------------------------------------------------------------ */
/* Reduced-precision storage of the values (an extension; the paper stores
 * binary64 only, Sec. 5).  Each value is rounded once, to nearest with ties to
 * even, straight from binary64 to the target format:
 *   to = 1 : IEEE binary32   (8 exponent bits, 24-bit significand)
 *   to = 2 : bfloat16        (8 exponent bits,  8-bit significand)
 * Both share the binary32 exponent range: normal numbers down to 2^-126 and
 * subnormals with the fixed spacing 2^(-126-(p-1)).  The value is rounded by
 * scaling with the spacing q of its binade (a power of two, so the scaling is
 * exact), rounding to an integer with ties to even and scaling back; a result
 * at or above 2^128 overflows to infinity.  The rounded binary64 value is then
 * exactly representable and is written out in the target encoding. */
static double orc_round_to(double d, int p)
{
    if (d == 0.0 || isnan(d) || isinf(d)) return d;
    double a = fabs(d);
    int e;
    frexp(a, &e);        /* a = m * 2^e, m in [0.5, 1): binade exponent e-1 */
    int E = e - 1;
    if (E < -126) E = -126; /* subnormal range: fixed spacing */
    double q = ldexp(1.0, E - (p - 1));
    double r = nearbyint(a / q) * q; /* default rounding mode: ties to even */
    if (r >= ldexp(1.0, 128)) r = INFINITY;
    return d < 0 ? -r : r;
}

void orc_round(int64_t n, const double *in, int to, void *out)
{
    for (int64_t i = 0; i < n; ++i) {
        double r;
        if (isnan(in[i])) {
            float f = NAN;
            r = f;
        } else {
            r = orc_round_to(in[i], to == 1 ? 24 : 8);
        }
        float f = (float)r; /* exact: r is representable in binary32 */
        if (to == 1) {
            ((float *)out)[i] = f;
        } else {
            uint32_t bits;
            memcpy(&bits, &f, 4);
            ((uint16_t *)out)[i] = (uint16_t)(bits >> 16); /* exact by construction */
        }
    }
}

/* bfloat16 bit pattern -> binary64 (exact). */
void orc_bf16_to_f64(int64_t n, const uint16_t *in, double *out)
{
    for (int64_t i = 0; i < n; ++i) {
        uint32_t bits = (uint32_t)in[i] << 16;
        float f;
        memcpy(&f, &bits, 4);
        out[i] = f;
    }
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
