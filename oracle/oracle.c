/*
 * oracle.c -- plain, slow, obviously-correct CPU reference for the
 * Faugere-Lachartre (FL) reduction over GF(p), p < 2^16.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file: only the tests, the package smoke check and the CPU
 * baseline leg of the benchmark do.  It shares no code, header, table or
 * helper with the CUDA library.
 *
 * Arithmetic: exact integers.  Residues are kept in [0,p); working rows are
 * uint64 accumulators that are only reduced with the C `%` operator when a
 * value is read as a multiplier or stored (delayed reduction; every term
 * added is < p^2 < 2^32, and no entry receives more than 2^31 additions, so
 * no accumulator can overflow 2^64).  For a prime p >= 2^16 (oracle_rref32,
 * p < 2^31) a term is < 2^62, so there every addition is reduced at once.
 *
 * Functions and the passages they follow (GBLA paper, arXiv 1602.06097):
 *   oracle_rref     -- textbook Gauss-Jordan on the WHOLE matrix, rows taken
 *                      in input order: FL steps 4-5 plus the reduced-echelon
 *                      pass (Sec. 4.1, the RREF remark after step 5), and
 *                      the "normalize, reduce by matching head" rule of
 *                      Alg. 3 (Sec. 4.4).  Output: the unique reduced row
 *                      echelon form of M, rows sorted by pivot column.
 *   oracle_pivots   -- FL step 1 pivot choice (Sec. 3.1, Sec. 4.1 step 1):
 *                      the leading (leftmost) nonzero of a row is its pivot
 *                      candidate; among rows with the same candidate column
 *                      the one keeping A sparsest is chosen.  The paper does
 *                      not fix the tie-break; this oracle reads it as
 *                      (fewest nonzeros, then smallest input row index).
 *   oracle_rref32, oracle_echelon32
 *                   -- oracle_rref and oracle_echelon for primes p < 2^31
 *                      with 32-bit values (the paper's uint32 coefficient
 *                      type, Sec. 2): the same steps, each addition reduced.
 *   oracle_echelon  -- the "new order of operations" (Alg. 2, Sec. 4.3) in
 *                      plain row form: every non-pivot row is reduced by the
 *                      normalised pivot rows in ascending pivot column order
 *                      (this is C <- C*A^-1 with D <- D - C*A^-1*B applied on
 *                      the fly), then the leftover rows (the Schur complement
 *                      D') are brought to reduced echelon form by the same
 *                      textbook Gauss-Jordan (Sec. 4.1 step 4).  Output: the
 *                      normalised pivot rows plus RREF(D'), merged in pivot
 *                      column order (the canonical non-reduced echelon form).
 *
 * Parity pins live in tests/test_oracle.py (brute-force row spaces over
 * GF(7), Leibniz-determinant ranks, closed-form special cases, invariants).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

static double ora_now(void)
{
    struct timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

#define ORA_OK 0
#define ORA_E_INVAL 1
#define ORA_E_NOMEM 2

/* Compile-time planted mistakes, used only by the mutation test that shows
 * the pins are sensitive.  0 = the real oracle. */
#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0
#endif

/* Modular inverse by the extended Euclidean algorithm (a != 0 mod p). */
static uint64_t ora_inv(uint64_t a, uint64_t p)
{
    int64_t t = 0, newt = 1;
    int64_t r = (int64_t)p, newr = (int64_t)(a % p);
    while (newr != 0) {
        int64_t q = r / newr, tmp;
        tmp = t - q * newt; t = newt; newt = tmp;
        tmp = r - q * newr; r = newr; newr = tmp;
    }
    if (t < 0) t += (int64_t)p;
    return (uint64_t)t;
}

/* Validate a CSR matrix: row_ptr monotone from 0, columns strictly increasing
 * inside a row and in [0,n), values in [1,p).  p must be a prime below pmax
 * (2^16, or 2^31 for the 32-bit entry point; primality checked by trial
 * division).  Values come as uint16 (val) or uint32 (val32). */
static int ora_validate_w(int64_t m, int64_t n, uint32_t p, uint32_t pmax, const int64_t *row_ptr,
                          const int32_t *col, const uint16_t *val, const uint32_t *val32)
{
    if (m < 0 || n < 0 || p < 2 || p >= pmax) return ORA_E_INVAL;
    for (uint64_t d = 2; d * d <= p; ++d)
        if (p % d == 0) return ORA_E_INVAL;
    if (m > 0 && !row_ptr) return ORA_E_INVAL;
    if (m > 0 && row_ptr[0] != 0) return ORA_E_INVAL;
    for (int64_t i = 0; i < m; ++i) {
        if (row_ptr[i + 1] < row_ptr[i]) return ORA_E_INVAL;
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            if (col[e] < 0 || col[e] >= n) return ORA_E_INVAL;
            if (e > row_ptr[i] && col[e] <= col[e - 1]) return ORA_E_INVAL;
            const uint32_t v = val32 ? val32[e] : val[e];
            if (v == 0 || v >= p) return ORA_E_INVAL;
        }
    }
    return ORA_OK;
}

static int ora_validate(int64_t m, int64_t n, uint32_t p, const int64_t *row_ptr, const int32_t *col,
                        const uint16_t *val)
{
    return ora_validate_w(m, n, p, 65536u, row_ptr, col, val, NULL);
}

/* A growing list of reduced dense rows (entries in [0,p)), each with the
 * column of its pivot (leading 1). */
typedef struct {
    int64_t n, count, cap;
    uint32_t *rows;   /* count x n */
    int64_t *pcol;    /* pivot column of each row */
    int64_t *nz;      /* nonzero entries of each row */
} ora_rows;

static int ora_rows_push(ora_rows *R, const uint64_t *w, int64_t pc)
{
    if (R->count == R->cap) {
        int64_t nc = R->cap ? 2 * R->cap : 16;
        uint32_t *nr = (uint32_t *)realloc(R->rows, (size_t)nc * (size_t)(R->n ? R->n : 1) * sizeof(uint32_t));
        if (!nr) return ORA_E_NOMEM;
        R->rows = nr;
        int64_t *np = (int64_t *)realloc(R->pcol, (size_t)nc * sizeof(int64_t));
        if (!np) return ORA_E_NOMEM;
        R->pcol = np;
        int64_t *nzp = (int64_t *)realloc(R->nz, (size_t)nc * sizeof(int64_t));
        if (!nzp) return ORA_E_NOMEM;
        R->nz = nzp;
        R->cap = nc;
    }
    uint32_t *dst = R->rows + (size_t)R->count * (size_t)R->n;
    int64_t nz = 0;
    for (int64_t k = 0; k < R->n; ++k) {
        dst[k] = (uint32_t)w[k];
        nz += dst[k] != 0;
    }
    R->pcol[R->count] = pc;
    R->nz[R->count] = nz;
    R->count++;
    return ORA_OK;
}

/*
 * Textbook Gauss-Jordan over GF(p) on dense rows.
 *
 * Forward pass (Sec. 4.1 step 4, Alg. 3): each row in turn is scattered into
 * a dense accumulator; scanning its columns left to right, every nonzero
 * entry whose column already owns a pivot row is cancelled by subtracting
 * that multiple of the pivot row; the first nonzero entry whose column owns
 * no pivot makes the row (normalised to a leading 1) the pivot of that
 * column.  Rows that cancel completely are zero reductions and are dropped.
 *
 * Backward pass (the RREF remark after FL step 5): pivot rows are taken in
 * descending pivot column order; each one subtracts from itself the final
 * rows of all larger pivot columns, which clears every pivot column except
 * its own.
 *
 * `in` holds `m_in` dense input rows of width n with entries in [0,p).
 * Result rows (sorted by pivot column, entries in [0,p)) go to *out.
 *
 * Work counter (optional): *ops is increased by the number of modular
 * multiply-adds with a nonzero pivot-row entry, pivot entry excluded: one
 * subtraction of a multiple of row P adds nnz(P) - 1, in the forward pass
 * and in the backward pass alike.
 */
static int ora_gauss_jordan(int64_t n, uint32_t p, int64_t m_in,
                            const uint32_t *in, ora_rows *out, double *ops)
{
    double work = 0;
    int rc = ORA_OK;
    int64_t *pivot_of = (int64_t *)malloc((size_t)(n ? n : 1) * sizeof(int64_t));
    uint64_t *w = (uint64_t *)malloc((size_t)(n ? n : 1) * sizeof(uint64_t));
    ora_rows E = {n, 0, 0, NULL, NULL, NULL};
    if (!pivot_of || !w) { rc = ORA_E_NOMEM; goto done; }
    for (int64_t j = 0; j < n; ++j) pivot_of[j] = -1;

    for (int64_t i = 0; i < m_in; ++i) {
        const uint32_t *src = in + (size_t)i * (size_t)n;
        for (int64_t k = 0; k < n; ++k) w[k] = src[k];
        for (int64_t j = 0; j < n; ++j) {
            uint64_t f = w[j] % p;
            if (f == 0) continue;
            if (pivot_of[j] >= 0) {
                const uint32_t *P = E.rows + (size_t)pivot_of[j] * (size_t)n;
                work += (double)(E.nz[pivot_of[j]] - 1);
                uint64_t g = p - f;            /* subtract f * P */
#if ORACLE_MUTANT == 1
                g = f;                          /* planted: wrong sign */
#endif
                for (int64_t k = j; k < n; ++k) {
                    w[k] += g * P[k];
                    if (p >= 65536u) w[k] %= p;   /* terms up to 2^62: reduce each addition */
                }
            } else {
                uint64_t inv = ora_inv(f, p);
                for (int64_t k = 0; k < j; ++k) w[k] = 0;
                for (int64_t k = j; k < n; ++k) w[k] = (w[k] % p) * inv % p;
                pivot_of[j] = E.count;
                if ((rc = ora_rows_push(&E, w, j)) != ORA_OK) goto done;
                break;
            }
        }
    }

    /* Backward pass, descending pivot columns. */
    {
        int64_t r = E.count;
        int64_t *order = (int64_t *)malloc((size_t)(r ? r : 1) * sizeof(int64_t));
        if (!order) { rc = ORA_E_NOMEM; goto done; }
        int64_t t = 0;
        for (int64_t j = 0; j < n; ++j)
            if (pivot_of[j] >= 0) order[t++] = pivot_of[j]; /* ascending columns */
        for (int64_t a = r - 1; a >= 0; --a) {
            uint32_t *Q = E.rows + (size_t)order[a] * (size_t)n;
            int64_t qc = E.pcol[order[a]];
            for (int64_t k = 0; k < n; ++k) w[k] = Q[k];
            for (int64_t b = a + 1; b < r; ++b) {
                int64_t c = E.pcol[order[b]];
                uint64_t f = w[c] % p;
                if (f == 0) continue;
                const uint32_t *P = E.rows + (size_t)order[b] * (size_t)n;
                work += (double)(E.nz[order[b]] - 1);
                uint64_t g = p - f;
#if ORACLE_MUTANT == 2
                if (b == a + 1) continue;       /* planted: dropped term */
#endif
                for (int64_t k = c; k < n; ++k) {
                    w[k] += g * P[k];
                    if (p >= 65536u) w[k] %= p;
                }
            }
            int64_t nz = 0;
            for (int64_t k = qc; k < n; ++k) {
                Q[k] = (uint32_t)(w[k] % p);
                nz += Q[k] != 0;
            }
            E.nz[order[a]] = nz;
        }
        /* Emit in ascending pivot column order. */
        for (int64_t a = 0; a < r; ++a) {
            const uint32_t *Q = E.rows + (size_t)order[a] * (size_t)n;
            for (int64_t k = 0; k < n; ++k) w[k] = Q[k];
            if ((rc = ora_rows_push(out, w, E.pcol[order[a]])) != ORA_OK) { free(order); goto done; }
        }
        free(order);
    }
done:
    if (ops) *ops += work;
    free(pivot_of);
    free(w);
    free(E.rows);
    free(E.pcol);
    free(E.nz);
    return rc;
}

/* Convert reduced dense rows to a freshly malloc'ed CSR (zeros dropped). */
static int ora_rows_to_csr(const ora_rows *R, int64_t **rp, int32_t **cl, uint16_t **vl)
{
    int64_t nnz = 0;
    for (int64_t a = 0; a < R->count; ++a)
        for (int64_t k = 0; k < R->n; ++k)
            if (R->rows[(size_t)a * (size_t)R->n + (size_t)k]) nnz++;
    int64_t *row_ptr = (int64_t *)malloc((size_t)(R->count + 1) * sizeof(int64_t));
    int32_t *col = (int32_t *)malloc((size_t)(nnz ? nnz : 1) * sizeof(int32_t));
    uint16_t *val = (uint16_t *)malloc((size_t)(nnz ? nnz : 1) * sizeof(uint16_t));
    if (!row_ptr || !col || !val) { free(row_ptr); free(col); free(val); return ORA_E_NOMEM; }
    int64_t e = 0;
    row_ptr[0] = 0;
    for (int64_t a = 0; a < R->count; ++a) {
        const uint32_t *Q = R->rows + (size_t)a * (size_t)R->n;
        for (int64_t k = 0; k < R->n; ++k)
            if (Q[k]) { col[e] = (int32_t)k; val[e] = (uint16_t)Q[k]; ++e; }
        row_ptr[a + 1] = e;
    }
    *rp = row_ptr; *cl = col; *vl = val;
    return ORA_OK;
}

void oracle_free(void *ptr) { free(ptr); }

/*
 * RREF(M) over GF(p), M given as CSR (m x n).  On success *rank is the number
 * of rows of the result and *out_* are malloc'ed (release with oracle_free).
 */
int oracle_rref(int64_t m, int64_t n, uint32_t p, const int64_t *row_ptr,
                const int32_t *col, const uint16_t *val, int64_t *rank,
                int64_t **out_row_ptr, int32_t **out_col, uint16_t **out_val)
{
    int rc = ora_validate(m, n, p, row_ptr, col, val);
    if (rc) return rc;
    uint32_t *dense = (uint32_t *)calloc((size_t)(m ? m : 1) * (size_t)(n ? n : 1), sizeof(uint32_t));
    if (!dense) return ORA_E_NOMEM;
    for (int64_t i = 0; i < m; ++i)
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e)
            dense[(size_t)i * (size_t)n + (size_t)col[e]] = val[e];
    ora_rows R = {n, 0, 0, NULL, NULL, NULL};
    rc = ora_gauss_jordan(n, p, m, dense, &R, NULL);
    free(dense);
    if (rc == ORA_OK) rc = ora_rows_to_csr(&R, out_row_ptr, out_col, out_val);
    if (rc == ORA_OK) *rank = R.count;
    free(R.rows);
    free(R.pcol);
    free(R.nz);
    return rc;
}

/*
 * RREF(M) over GF(p) for a prime p < 2^31, values as uint32 (the paper's
 * 32-bit coefficient type, Sec. 2): the Gauss-Jordan of oracle_rref with
 * every addition reduced.  Output as oracle_rref, values uint32.
 */
int oracle_rref32(int64_t m, int64_t n, uint32_t p, const int64_t *row_ptr,
                  const int32_t *col, const uint32_t *val, int64_t *rank,
                  int64_t **out_row_ptr, int32_t **out_col, uint32_t **out_val)
{
    int rc = ora_validate_w(m, n, p, 2147483648u, row_ptr, col, NULL, val);
    if (rc) return rc;
    uint32_t *dense = (uint32_t *)calloc((size_t)(m ? m : 1) * (size_t)(n ? n : 1), sizeof(uint32_t));
    if (!dense) return ORA_E_NOMEM;
    for (int64_t i = 0; i < m; ++i)
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e)
            dense[(size_t)i * (size_t)n + (size_t)col[e]] = val[e];
    ora_rows R = {n, 0, 0, NULL, NULL, NULL};
    rc = ora_gauss_jordan(n, p, m, dense, &R, NULL);
    free(dense);
    if (rc == ORA_OK) {
        int64_t nnz = 0;
        for (int64_t i = 0; i < R.count; ++i) nnz += R.nz[i];
        int64_t *rp = (int64_t *)malloc((size_t)(R.count + 1) * sizeof(int64_t));
        int32_t *cl = (int32_t *)malloc((size_t)(nnz ? nnz : 1) * sizeof(int32_t));
        uint32_t *vl = (uint32_t *)malloc((size_t)(nnz ? nnz : 1) * sizeof(uint32_t));
        if (!rp || !cl || !vl) {
            free(rp); free(cl); free(vl);
            rc = ORA_E_NOMEM;
        } else {
            int64_t e = 0;
            rp[0] = 0;
            for (int64_t i = 0; i < R.count; ++i) {
                const uint32_t *Q = R.rows + (size_t)i * (size_t)n;
                for (int64_t k = 0; k < n; ++k)
                    if (Q[k]) { cl[e] = (int32_t)k; vl[e] = Q[k]; ++e; }
                rp[i + 1] = e;
            }
            *out_row_ptr = rp;
            *out_col = cl;
            *out_val = vl;
            *rank = R.count;
        }
    }
    free(R.rows);
    free(R.pcol);
    free(R.nz);
    return rc;
}

/*
 * FL step 1 pivot choice.  piv_row[c] = input row chosen as pivot for column
 * c, or -1 if no row leads at c.  Rows lead at their leftmost nonzero; among
 * rows sharing a leading column the one with the fewest nonzeros wins, ties
 * going to the smaller row index.  Returns the number of pivots.
 */
int64_t oracle_pivots(int64_t m, int64_t n, const int64_t *row_ptr, const int32_t *col,
                      int64_t *piv_row)
{
    int64_t npiv = 0;
    for (int64_t c = 0; c < n; ++c) piv_row[c] = -1;
    for (int64_t i = 0; i < m; ++i) {
        int64_t w = row_ptr[i + 1] - row_ptr[i];
        if (w == 0) continue;
        int64_t c = col[row_ptr[i]];
        int64_t cur = piv_row[c];
        if (cur < 0) { piv_row[c] = i; npiv++; continue; }
        int64_t wc = row_ptr[cur + 1] - row_ptr[cur];
#if ORACLE_MUTANT == 3
        if (w > wc) piv_row[c] = i;              /* planted: densest row wins */
#else
        if (w < wc) piv_row[c] = i;              /* strictly fewer: earlier index keeps ties */
#endif
    }
    return npiv;
}

/*
 * Canonical echelon form by the new order of operations (Alg. 2), plain row
 * form.  Output rows: the chosen pivot rows normalised to a leading 1, plus
 * RREF of the Schur complement, merged by pivot column.
 */
/* The new-order echelon for either value width: values come as uint16
 * (val16, p < 2^16, output out_val16) or uint32 (val32, p < 2^31, output
 * out_val32).  For p >= 2^16 every addition is reduced (terms reach 2^62). */
#define ORA_VAL(e) (val32 ? (uint64_t)val32[e] : (uint64_t)val16[e])
static int ora_echelon_w(int64_t m, int64_t n, uint32_t p, const int64_t *row_ptr,
                         const int32_t *col, const uint16_t *val16, const uint32_t *val32, int64_t *rank,
                         int64_t **out_row_ptr, int32_t **out_col, uint16_t **out_val16, uint32_t **out_val32,
                         int64_t *npiv_out, double *seconds, double *ops)
{
    /* seconds (optional, 2 entries): wall time of the row reduction by the
     * pivot rows, and of the Gauss-Jordan pass on the Schur complement.
     * ops (optional, 4 entries): modular multiply-adds with a nonzero operand
     * entry, counted as the work is done (one op = one multiply-add):
     *   [0] ops_b: a non-pivot row reduced by pivot row j (x_j != 0) does
     *       one per entry of that row at the other pivot columns -- the
     *       sparse C <- C*A^-1 (Alg. 2);
     *   [1] ops_c: ... and one per entry at the non-pivot columns -- the
     *       Schur update D <- D - X*B;
     *   [2] ops_d: the Gauss-Jordan pass on the Schur complement (forward
     *       and backward, nnz(P) - 1 per row subtraction);
     *   [3] ops_e: the back-substitution of the top block, 0 here (this
     *       form keeps the pivot rows as they are). */
    double t0 = ora_now(), t1 = t0;
    double ops_b = 0, ops_c = 0, ops_d = 0;
    int rc = ora_validate_w(m, n, p, val32 ? 2147483648u : 65536u, row_ptr, col, val16, val32);
    if (rc) return rc;
    int64_t *piv_row = (int64_t *)malloc((size_t)(n ? n : 1) * sizeof(int64_t));
    uint64_t *inv_lead = (uint64_t *)malloc((size_t)(n ? n : 1) * sizeof(uint64_t));
    char *is_piv_row = (char *)calloc((size_t)(m ? m : 1), 1);
    if (!piv_row || !inv_lead || !is_piv_row) { rc = ORA_E_NOMEM; goto fail0; }
    int64_t npiv = oracle_pivots(m, n, row_ptr, col, piv_row);
    for (int64_t c = 0; c < n; ++c)
        if (piv_row[c] >= 0) {
            is_piv_row[piv_row[c]] = 1;
            inv_lead[c] = ora_inv(ORA_VAL(row_ptr[piv_row[c]]), p);
        }
    /* entries of each pivot row at other pivot columns (na) and at the
     * non-pivot columns (nb), for the work counter */
    int64_t *na = (int64_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
    int64_t *nb = (int64_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
    if (!na || !nb) { free(na); free(nb); rc = ORA_E_NOMEM; goto fail0; }
    for (int64_t c = 0; c < n; ++c)
        if (piv_row[c] >= 0)
            for (int64_t e = row_ptr[piv_row[c]] + 1; e < row_ptr[piv_row[c] + 1]; ++e) {
                if (piv_row[col[e]] >= 0) na[c]++;
                else nb[c]++;
            }

    /* Non-pivot, non-empty rows in input order. */
    int64_t mcd = 0;
    for (int64_t i = 0; i < m; ++i)
        if (!is_piv_row[i] && row_ptr[i + 1] > row_ptr[i]) mcd++;
    int64_t *cd_rows = (int64_t *)malloc((size_t)(mcd ? mcd : 1) * sizeof(int64_t));
    uint32_t *left = (uint32_t *)calloc((size_t)(mcd ? mcd : 1) * (size_t)(n ? n : 1), sizeof(uint32_t));
    if (!cd_rows || !left) { free(cd_rows); free(left); free(na); free(nb); rc = ORA_E_NOMEM; goto fail0; }
    mcd = 0;
    for (int64_t i = 0; i < m; ++i)
        if (!is_piv_row[i] && row_ptr[i + 1] > row_ptr[i]) cd_rows[mcd++] = i;

    /* Reduce every non-pivot row by the pivot rows, pivot columns ascending
     * (Alg. 2: the multiplier dense_C[j] is final once all smaller pivot
     * columns are cleared, since the pivot rows are zero left of their
     * leading column).  Rows are independent of one another. */
    int fail = 0;
#pragma omp parallel reduction(+ : ops_b, ops_c)
    {
        uint64_t *w = (uint64_t *)malloc((size_t)(n ? n : 1) * sizeof(uint64_t));
        if (!w) {
#pragma omp atomic write
            fail = 1;
        }
#pragma omp for schedule(dynamic, 4)
        for (int64_t t = 0; t < mcd; ++t) {
            if (!w) continue;
            int64_t i = cd_rows[t];
            memset(w, 0, (size_t)n * sizeof(uint64_t));
            for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) w[col[e]] = ORA_VAL(e);
            for (int64_t j = 0; j < n; ++j) {
                if (piv_row[j] < 0) continue;
                uint64_t f = w[j] % p;
                if (f == 0) { w[j] = 0; continue; }
                /* multiplier of the normalised pivot row = f; the pivot row
                 * holds val * inv_lead, so subtract (f * inv_lead) * val. */
                int64_t r = piv_row[j];
                ops_b += (double)na[j];
                ops_c += (double)nb[j];
                uint64_t g = (p - f) * inv_lead[j] % p;
                for (int64_t e = row_ptr[r]; e < row_ptr[r + 1]; ++e) {
                    w[col[e]] += g * ORA_VAL(e);
                    if (p >= 65536u) w[col[e]] %= p;   /* terms up to 2^62 */
                }
            }
            uint32_t *dst = left + (size_t)t * (size_t)n;
            for (int64_t k = 0; k < n; ++k) dst[k] = (uint32_t)(w[k] % p);
        }
        free(w);
    }
    free(na);
    free(nb);
    if (fail) { free(cd_rows); free(left); rc = ORA_E_NOMEM; goto fail0; }

    t1 = ora_now();
    ora_rows B = {n, 0, 0, NULL, NULL, NULL};
    rc = ora_gauss_jordan(n, p, mcd, left, &B, &ops_d);
    if (ops) { ops[0] = ops_b; ops[1] = ops_c; ops[2] = ops_d; ops[3] = 0; }
    if (seconds) { seconds[0] = t1 - t0; seconds[1] = ora_now() - t1; }
    free(left);
    free(cd_rows);
    if (rc) { free(B.rows); free(B.pcol); free(B.nz); goto fail0; }

    /* Merge: top rows (pivot columns of A) and bottom rows (pivots of D'). */
    {
        int64_t r = npiv + B.count, nnz = 0;
        for (int64_t c = 0; c < n; ++c)
            if (piv_row[c] >= 0) nnz += row_ptr[piv_row[c] + 1] - row_ptr[piv_row[c]];
        for (int64_t a = 0; a < B.count; ++a)
            for (int64_t k = 0; k < n; ++k)
                if (B.rows[(size_t)a * (size_t)n + (size_t)k]) nnz++;
        int64_t *rp = (int64_t *)malloc((size_t)(r + 1) * sizeof(int64_t));
        int32_t *cl = (int32_t *)malloc((size_t)(nnz ? nnz : 1) * sizeof(int32_t));
        uint16_t *vl = val32 ? NULL : (uint16_t *)malloc((size_t)(nnz ? nnz : 1) * sizeof(uint16_t));
        uint32_t *vl32 = val32 ? (uint32_t *)malloc((size_t)(nnz ? nnz : 1) * sizeof(uint32_t)) : NULL;
        int64_t *bottom_of = (int64_t *)malloc((size_t)(n ? n : 1) * sizeof(int64_t));
        if (!rp || !cl || (!vl && !vl32) || !bottom_of) {
            free(rp); free(cl); free(vl); free(vl32); free(bottom_of); free(B.rows); free(B.pcol); free(B.nz);
            rc = ORA_E_NOMEM; goto fail0;
        }
        for (int64_t c = 0; c < n; ++c) bottom_of[c] = -1;
        for (int64_t a = 0; a < B.count; ++a) bottom_of[B.pcol[a]] = a;
        int64_t e = 0, a_out = 0;
        rp[0] = 0;
        for (int64_t c = 0; c < n; ++c) {
            if (piv_row[c] >= 0) {
                int64_t i = piv_row[c];
                for (int64_t s = row_ptr[i]; s < row_ptr[i + 1]; ++s) {
                    cl[e] = col[s];
                    const uint64_t v = ORA_VAL(s) * inv_lead[c] % p;
                    if (vl32) vl32[e] = (uint32_t)v;
                    else vl[e] = (uint16_t)v;
                    ++e;
                }
                rp[++a_out] = e;
            } else if (bottom_of[c] >= 0) {
                const uint32_t *Q = B.rows + (size_t)bottom_of[c] * (size_t)n;
                for (int64_t k = 0; k < n; ++k)
                    if (Q[k]) {
                        cl[e] = (int32_t)k;
                        if (vl32) vl32[e] = Q[k];
                        else vl[e] = (uint16_t)Q[k];
                        ++e;
                    }
                rp[++a_out] = e;
            }
        }
        free(bottom_of);
        free(B.rows);
        free(B.pcol);
        free(B.nz);
        *out_row_ptr = rp; *out_col = cl;
        if (vl32) *out_val32 = vl32;
        else *out_val16 = vl;
        *rank = r;
        if (npiv_out) *npiv_out = npiv;
    }
fail0:
    free(piv_row);
    free(inv_lead);
    free(is_piv_row);
    return rc;
}
#undef ORA_VAL

int oracle_echelon(int64_t m, int64_t n, uint32_t p, const int64_t *row_ptr,
                   const int32_t *col, const uint16_t *val, int64_t *rank,
                   int64_t **out_row_ptr, int32_t **out_col, uint16_t **out_val,
                   int64_t *npiv_out, double *seconds, double *ops)
{
    return ora_echelon_w(m, n, p, row_ptr, col, val, NULL, rank, out_row_ptr, out_col, out_val, NULL, npiv_out,
                         seconds, ops);
}

/*
 * The new-order echelon form (as oracle_echelon) for a prime p < 2^31 with
 * uint32 values (the paper's 32-bit coefficient type, Sec. 2).
 */
int oracle_echelon32(int64_t m, int64_t n, uint32_t p, const int64_t *row_ptr,
                     const int32_t *col, const uint32_t *val, int64_t *rank,
                     int64_t **out_row_ptr, int32_t **out_col, uint32_t **out_val, int64_t *npiv_out)
{
    return ora_echelon_w(m, n, p, row_ptr, col, NULL, val, rank, out_row_ptr, out_col, NULL, out_val, npiv_out,
                         NULL, NULL);
}

/*
 * Work counts of the row reduction of Alg. 2 alone (no Gauss-Jordan pass, no
 * output), for matrices whose Schur complement is too large for the textbook
 * pass: ops[0] = ops_b and ops[1] = ops_c exactly as oracle_echelon counts
 * them (every non-pivot row reduced by the normalised pivot rows in ascending
 * pivot column order, one op per entry of a pivot row with a nonzero
 * multiplier), *npiv_out the pivot count.  seconds (optional) receives the
 * wall time.
 */
int oracle_row_counts(int64_t m, int64_t n, uint32_t p, const int64_t *row_ptr, const int32_t *col,
                      const uint16_t *val, double *ops, int64_t *npiv_out, double *seconds)
{
    double t0 = ora_now();
    int rc = ora_validate(m, n, p, row_ptr, col, val);
    if (rc) return rc;
    int64_t *piv_row = (int64_t *)malloc((size_t)(n ? n : 1) * sizeof(int64_t));
    uint64_t *inv_lead = (uint64_t *)malloc((size_t)(n ? n : 1) * sizeof(uint64_t));
    char *is_piv_row = (char *)calloc((size_t)(m ? m : 1), 1);
    int64_t *na = (int64_t *)calloc((size_t)(n ? n : 1), sizeof(int64_t));
    int64_t *nb = (int64_t *)calloc((size_t)(n ? n : 1), sizeof(int64_t));
    double ops_b = 0, ops_c = 0;
    int fail = 0;
    if (!piv_row || !inv_lead || !is_piv_row || !na || !nb) { rc = ORA_E_NOMEM; goto done; }
    int64_t npiv = oracle_pivots(m, n, row_ptr, col, piv_row);
    for (int64_t c = 0; c < n; ++c)
        if (piv_row[c] >= 0) {
            is_piv_row[piv_row[c]] = 1;
            inv_lead[c] = ora_inv(val[row_ptr[piv_row[c]]], p);
            for (int64_t e = row_ptr[piv_row[c]] + 1; e < row_ptr[piv_row[c] + 1]; ++e) {
                if (piv_row[col[e]] >= 0) na[c]++;
                else nb[c]++;
            }
        }
#pragma omp parallel reduction(+ : ops_b, ops_c)
    {
        uint64_t *w = (uint64_t *)malloc((size_t)(n ? n : 1) * sizeof(uint64_t));
        if (!w) {
#pragma omp atomic write
            fail = 1;
        }
#pragma omp for schedule(dynamic, 4)
        for (int64_t i = 0; i < m; ++i) {
            if (!w || is_piv_row[i] || row_ptr[i + 1] == row_ptr[i]) continue;
            memset(w, 0, (size_t)n * sizeof(uint64_t));
            for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) w[col[e]] = val[e];
            for (int64_t j = 0; j < n; ++j) {
                if (piv_row[j] < 0) continue;
                uint64_t f = w[j] % p;
                if (f == 0) { w[j] = 0; continue; }
                int64_t r = piv_row[j];
                ops_b += (double)na[j];
                ops_c += (double)nb[j];
                uint64_t g = (p - f) * inv_lead[j] % p;
                for (int64_t e = row_ptr[r]; e < row_ptr[r + 1]; ++e) w[col[e]] += g * val[e];
            }
        }
        free(w);
    }
    if (fail) { rc = ORA_E_NOMEM; goto done; }
    ops[0] = ops_b;
    ops[1] = ops_c;
    if (npiv_out) *npiv_out = npiv;
    if (seconds) *seconds = ora_now() - t0;
done:
    free(piv_row);
    free(inv_lead);
    free(is_piv_row);
    free(na);
    free(nb);
    return rc;
}

