/*
 * gk_oracle.c - plain, slow, obviously correct FP64 CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path may
 * include, link or call this file; only the tests, the smoke check and the
 * benchmark's CPU-baseline leg use it.  It shares no code, header, table or
 * helper with the CUDA library.
 *
 * What it follows:
 *  - The linear-operator model of the paper (Section 4.2 "Ginkgo's Linear
 *    Operator Abstraction"): a matrix applied to b gives A b; a solver
 *    applied to (b, x) overwrites the initial guess x with the solution
 *    (Section 3.5 "pyGinkgo API", Listing 1).
 *  - Stopping criteria of the config solver (Section 3.5, Listing 2): an
 *    iteration cap OR a residual-norm reduction relative to the right-hand
 *    side norm ("baseline": "rhs_norm").
 *  - GMRES with Givens rotations and a residual check after every
 *    Hessenberg update (Section 6.2.1, the GMRES discussion).
 *  - CG (Hestenes-Stiefel), BiCGSTAB (van der Vorst 1992) and GMRES(m)
 *    (Saad-Schultz 1986) in their textbook forms; the paper prints no
 *    pseudo-code for them.
 *  - CSR / ELL / SELL-P layouts: the paper names "other matrix formats"
 *    (Section 3.1) without defining them; the layouts below are this
 *    library's stated readings (column-major padded slices, col = -1 and
 *    value = +0.0 for padding).
 *
 * Every floating-point operation is IEEE double with no contraction
 * (compile with -ffp-contract=off) so that results are identical on x86
 * and Arm hosts; the explicit fma() calls of ILU(0) are correctly rounded
 * fused multiply-adds on both.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* status codes, same meaning as the library's public ones */
#define OR_OK 0
#define OR_NOT_CONVERGED 1
#define OR_BREAKDOWN 2
#define OR_ERR_INVALID (-1)
#define OR_ERR_ZERO_DIAG (-5)
#define OR_ERR_NAN (-6)

/* ------------------------------------------------------------------ */
/* dense vector helpers (plain left-to-right loops)                    */
/* ------------------------------------------------------------------ */

static double dot(int32_t n, const double* u, const double* v)
{
    double s = 0.0;
    for (int32_t i = 0; i < n; ++i) s += u[i] * v[i];
    return s;
}

static double nrm2(int32_t n, const double* u) { return sqrt(dot(n, u, u)); }

/* ------------------------------------------------------------------ */
/* SpMV  y = alpha * A x + beta * y  (Section 4.2: a matrix LinOp's     */
/* apply is an SpMV; the advanced form adds alpha and beta)            */
/* ------------------------------------------------------------------ */

/* compensated = 1: Neumaier-compensated sum of a_ij * x_j over the row in
 * CSR order (the check mode).  compensated = 0: plain sequential sum.
 * beta == 0 means y is not read (BLAS convention), so NaN in y does not
 * propagate. */
void or_spmv_csr(int32_t n, const int32_t* rp, const int32_t* ci,
                 const double* va, const double* x, double alpha, double beta,
                 double* y, int compensated)
{
    for (int32_t i = 0; i < n; ++i) {
        double s = 0.0, c = 0.0;
        for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
            double p = va[k] * x[ci[k]];
            if (compensated) {
                double t = s + p;
                if (fabs(s) >= fabs(p)) c += (s - t) + p;
                else c += (p - t) + s;
                s = t;
            } else {
                s += p;
            }
        }
        s += c;
        y[i] = (beta == 0.0) ? alpha * s : alpha * s + beta * y[i];
    }
}

/* COO SpMV straight from the definition: every row sum starts at zero,
 * the triplets (row[k], col[k], val[k]) are visited in storage order and
 * each adds val * x[col] to its row's sum (Neumaier-compensated, as in the
 * CSR check mode, when compensated = 1); then y_i = alpha s_i + beta y_i
 * for every row, including rows without entries (beta == 0: y not read).
 * The paper benchmarks COO beside CSR (Section 6.1).  Returns -1 if a
 * triplet lies outside the matrix, else 0. */
int or_spmv_coo(int32_t n, int32_t ncols, int64_t nnz, const int32_t* row,
                const int32_t* col, const double* val, const double* x, double alpha,
                double beta, double* y, int compensated)
{
    double* s = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    double* c = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    for (int64_t k = 0; k < nnz; ++k) {
        if (row[k] < 0 || row[k] >= n || col[k] < 0 || col[k] >= ncols) {
            free(s);
            free(c);
            return -1;
        }
        const int32_t i = row[k];
        const double p = val[k] * x[col[k]];
        if (compensated) {
            const double t = s[i] + p;
            if (fabs(s[i]) >= fabs(p)) c[i] += (s[i] - t) + p;
            else c[i] += (p - t) + s[i];
            s[i] = t;
        } else {
            s[i] += p;
        }
    }
    for (int32_t i = 0; i < n; ++i) {
        const double si = s[i] + c[i];
        y[i] = (beta == 0.0) ? alpha * si : alpha * si + beta * y[i];
    }
    free(s);
    free(c);
    return 0;
}

/* Row-parallel version of the plain sum (bitwise identical to
 * or_spmv_csr with compensated = 0, since each row is summed by one
 * thread in the same order).  Returns the number of threads used. */
int or_spmv_csr_omp(int32_t n, const int32_t* rp, const int32_t* ci,
                    const double* va, const double* x, double alpha,
                    double beta, double* y, int threads)
{
    int used = 1;
#ifdef _OPENMP
    if (threads <= 0) threads = omp_get_max_threads();
#pragma omp parallel for schedule(static) num_threads(threads)
    for (int32_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int32_t k = rp[i]; k < rp[i + 1]; ++k) s += va[k] * x[ci[k]];
        y[i] = (beta == 0.0) ? alpha * s : alpha * s + beta * y[i];
    }
#pragma omp parallel num_threads(threads)
    {
#pragma omp single
        used = omp_get_num_threads();
    }
#else
    (void)threads;
    or_spmv_csr(n, rp, ci, va, x, alpha, beta, y, 0);
#endif
    return used;
}

/* ------------------------------------------------------------------ */
/* COO -> CSR (COO and CSR are the two formats the paper benchmarks,  */
/* Section 6.1)                                                        */
/* ------------------------------------------------------------------ */

typedef struct {
    int32_t col;
    int64_t pos; /* position in the COO input */
} or_entry;

static int cmp_entry(const void* a, const void* b)
{
    const or_entry* x = (const or_entry*)a;
    const or_entry* y = (const or_entry*)b;
    if (x->col != y->col) return x->col < y->col ? -1 : 1;
    if (x->pos != y->pos) return x->pos < y->pos ? -1 : 1;
    return 0;
}

/* Entries are ordered by (row, col); entries with equal (row, col) are
 * summed in their input order, left to right (in float arithmetic when
 * sum_f32 != 0, i.e. for FP32 matrices).  Explicit zeros are kept.
 * Returns the number of stored entries after merging, or -1 on an index
 * out of range.  out_col / out_val need room for nnz entries. */
int64_t or_coo_to_csr(int32_t n, int32_t ncols, int64_t nnz,
                      const int32_t* row, const int32_t* col,
                      const double* val, int sum_f32, int32_t* row_ptr,
                      int32_t* out_col, double* out_val)
{
    for (int64_t k = 0; k < nnz; ++k)
        if (row[k] < 0 || row[k] >= n || col[k] < 0 || col[k] >= ncols)
            return -1;
    /* bucket the entries by row, keeping input order inside each row */
    int64_t* start = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    for (int64_t k = 0; k < nnz; ++k) start[row[k] + 1]++;
    for (int32_t i = 0; i < n; ++i) start[i + 1] += start[i];
    int64_t* fill = (int64_t*)malloc(((size_t)n + 1) * sizeof(int64_t));
    memcpy(fill, start, ((size_t)n + 1) * sizeof(int64_t));
    or_entry* e = (or_entry*)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(or_entry));
    for (int64_t k = 0; k < nnz; ++k) {
        int64_t d = fill[row[k]]++;
        e[d].col = col[k];
        e[d].pos = k;
    }
    /* per row: sort by (col, input position), then merge equal columns */
    int64_t out = 0;
    row_ptr[0] = 0;
    for (int32_t i = 0; i < n; ++i) {
        int64_t a = start[i], b = start[i + 1];
        qsort(e + a, (size_t)(b - a), sizeof(or_entry), cmp_entry);
        int64_t k = a;
        while (k < b) {
            int32_t c = e[k].col;
            if (sum_f32) {
                float s = (float)val[e[k].pos];
                int64_t j = k + 1;
                while (j < b && e[j].col == c) { s = s + (float)val[e[j].pos]; ++j; }
                out_val[out] = (double)s;
                k = j;
            } else {
                double s = val[e[k].pos];
                int64_t j = k + 1;
                while (j < b && e[j].col == c) { s = s + val[e[j].pos]; ++j; }
                out_val[out] = s;
                k = j;
            }
            out_col[out] = c;
            ++out;
        }
        row_ptr[i + 1] = (int32_t)out;
    }
    free(e);
    free(fill);
    free(start);
    return out;
}

/* ------------------------------------------------------------------ */
/* CSR -> ELL and CSR -> SELL-P (layouts are this library's reading:   */
/* the paper plans further formats without defining them, Section 3.1)*/
/* ------------------------------------------------------------------ */

/* ELL width K = longest row. */
int32_t or_ell_width(int32_t n, const int32_t* rp)
{
    int32_t k = 0;
    for (int32_t i = 0; i < n; ++i)
        if (rp[i + 1] - rp[i] > k) k = rp[i + 1] - rp[i];
    return k;
}

/* ELL: entry j of row i at index j * stride + i (column-major), stride >= n.
 * Padding (j >= row length, and rows n..stride-1) is col -1, value +0.0. */
void or_csr_to_ell(int32_t n, const int32_t* rp, const int32_t* ci,
                   const double* va, int32_t K, int64_t stride,
                   int32_t* ecol, double* eval)
{
    for (int64_t t = 0; t < (int64_t)K * stride; ++t) { ecol[t] = -1; eval[t] = 0.0; }
    for (int32_t i = 0; i < n; ++i)
        for (int32_t j = 0; j < rp[i + 1] - rp[i]; ++j) {
            ecol[(int64_t)j * stride + i] = ci[rp[i] + j];
            eval[(int64_t)j * stride + i] = va[rp[i] + j];
        }
}

/* ELL -> CSR (drops padding; for round-trip pins). Returns nnz. */
int64_t or_ell_to_csr(int32_t n, int32_t K, int64_t stride, const int32_t* ecol,
                      const double* eval, int32_t* rp, int32_t* ci, double* va)
{
    int64_t out = 0;
    rp[0] = 0;
    for (int32_t i = 0; i < n; ++i) {
        for (int32_t j = 0; j < K; ++j) {
            int64_t t = (int64_t)j * stride + i;
            if (ecol[t] >= 0) { ci[out] = ecol[t]; va[out] = eval[t]; ++out; }
        }
        rp[i + 1] = (int32_t)out;
    }
    return out;
}

/* SELL-P sizes: slice s holds rows [s*S, s*S + S).  slice_lengths[s] =
 * longest row of the slice rounded up to a multiple of f; slice_sets is
 * the exclusive prefix sum of slice_lengths (nslices + 1 entries). */
void or_sellp_sizes(int32_t n, const int32_t* rp, int32_t S, int32_t f,
                    int32_t* slice_lengths, int64_t* slice_sets)
{
    int32_t ns = (n + S - 1) / S;
    slice_sets[0] = 0;
    for (int32_t s = 0; s < ns; ++s) {
        int32_t m = 0;
        for (int32_t i = s * S; i < s * S + S && i < n; ++i)
            if (rp[i + 1] - rp[i] > m) m = rp[i + 1] - rp[i];
        int32_t len = ((m + f - 1) / f) * f;
        slice_lengths[s] = len;
        slice_sets[s + 1] = slice_sets[s] + len;
    }
}

/* Entry j of row i = s*S + t is stored at (slice_sets[s] + j) * S + t.
 * Padding, including the virtual rows past n in the last slice, is
 * col -1, value +0.0. */
void or_csr_to_sellp(int32_t n, const int32_t* rp, const int32_t* ci,
                     const double* va, int32_t S, const int64_t* slice_sets,
                     int32_t* scol, double* sval)
{
    int32_t ns = (n + S - 1) / S;
    int64_t total = slice_sets[ns] * S;
    for (int64_t t = 0; t < total; ++t) { scol[t] = -1; sval[t] = 0.0; }
    for (int32_t i = 0; i < n; ++i) {
        int32_t s = i / S, t = i % S;
        for (int32_t j = 0; j < rp[i + 1] - rp[i]; ++j) {
            int64_t at = (slice_sets[s] + j) * S + t;
            scol[at] = ci[rp[i] + j];
            sval[at] = va[rp[i] + j];
        }
    }
}

/* SELL-P -> CSR (drops padding; for round-trip pins). Returns nnz. */
int64_t or_sellp_to_csr(int32_t n, int32_t S, const int32_t* slice_lengths,
                        const int64_t* slice_sets, const int32_t* scol,
                        const double* sval, int32_t* rp, int32_t* ci, double* va)
{
    int64_t out = 0;
    rp[0] = 0;
    for (int32_t i = 0; i < n; ++i) {
        int32_t s = i / S, t = i % S;
        for (int32_t j = 0; j < slice_lengths[s]; ++j) {
            int64_t at = (slice_sets[s] + j) * S + t;
            if (scol[at] >= 0) { ci[out] = scol[at]; va[out] = sval[at]; ++out; }
        }
        rp[i + 1] = (int32_t)out;
    }
    return out;
}

/* ------------------------------------------------------------------ */
/* Jacobi, block size 1 (Listing 2: "preconditioner::Jacobi",          */
/* "max_block_size": 1): z_i = r_i / a_ii                              */
/* ------------------------------------------------------------------ */

/* dinv[i] = 1 / a_ii.  A row without a stored diagonal, or with a zero
 * diagonal, is an error (OR_ERR_ZERO_DIAG). */
int or_jacobi_gen(int32_t n, const int32_t* rp, const int32_t* ci,
                  const double* va, double* dinv)
{
    for (int32_t i = 0; i < n; ++i) {
        double d = 0.0;
        int found = 0;
        for (int32_t k = rp[i]; k < rp[i + 1]; ++k)
            if (ci[k] == i) { d += va[k]; found = 1; }
        if (!found || d == 0.0) return OR_ERR_ZERO_DIAG;
        dinv[i] = 1.0 / d;
    }
    return OR_OK;
}

/* Block-Jacobi (the config solver's preconditioner with max_block_size > 1,
 * Listing 2): the diagonal blocks of A over bs consecutive rows (the last
 * block may be smaller), each inverted by Gauss-Jordan elimination with
 * partial pivoting on the dense block.  binv holds block b's inverse at
 * binv[b*bs*bs + i*bs + j] (unused slots of a short last block are 0).
 * A block with no nonzero pivot left is singular: OR_ERR_ZERO_DIAG. */
int or_block_jacobi_gen(int32_t n, const int32_t* rp, const int32_t* ci,
                        const double* va, int32_t bs, double* binv)
{
    if (bs < 1) return OR_ERR_INVALID;
    const int32_t nb = (n + bs - 1) / bs;
    double* a = (double*)malloc(sizeof(double) * (size_t)bs * bs);
    double* e = (double*)malloc(sizeof(double) * (size_t)bs * bs);
    int status = OR_OK;
    for (int32_t kb = 0; kb < nb && status == OR_OK; ++kb) {
        const int32_t r0 = kb * bs;
        const int32_t m = (n - r0 < bs) ? n - r0 : bs;
        for (int32_t i = 0; i < m * m; ++i) { a[i] = 0.0; e[i] = 0.0; }
        for (int32_t i = 0; i < m; ++i) {
            e[i * m + i] = 1.0;
            for (int32_t k = rp[r0 + i]; k < rp[r0 + i + 1]; ++k) {
                const int32_t j = ci[k] - r0;
                if (j >= 0 && j < m) a[i * m + j] += va[k];
            }
        }
        for (int32_t c = 0; c < m; ++c) {
            int32_t piv = c;
            for (int32_t r = c + 1; r < m; ++r)
                if (fabs(a[r * m + c]) > fabs(a[piv * m + c])) piv = r;
            if (a[piv * m + c] == 0.0) { status = OR_ERR_ZERO_DIAG; break; }
            if (piv != c)
                for (int32_t j = 0; j < m; ++j) {
                    double t = a[c * m + j]; a[c * m + j] = a[piv * m + j]; a[piv * m + j] = t;
                    t = e[c * m + j]; e[c * m + j] = e[piv * m + j]; e[piv * m + j] = t;
                }
            const double d = a[c * m + c];
            for (int32_t j = 0; j < m; ++j) { a[c * m + j] /= d; e[c * m + j] /= d; }
            for (int32_t r = 0; r < m; ++r) {
                if (r == c) continue;
                const double f = a[r * m + c];
                if (f == 0.0) continue;
                for (int32_t j = 0; j < m; ++j) {
                    a[r * m + j] -= f * a[c * m + j];
                    e[r * m + j] -= f * e[c * m + j];
                }
            }
        }
        double* out = binv + (size_t)kb * bs * bs;
        for (int32_t i = 0; i < bs * bs; ++i) out[i] = 0.0;
        for (int32_t i = 0; i < m; ++i)
            for (int32_t j = 0; j < m; ++j) out[i * bs + j] = e[i * m + j];
    }
    free(a);
    free(e);
    return status;
}

/* z = binv r block by block */
void or_block_jacobi_apply(int32_t n, int32_t bs, const double* binv, const double* r, double* z)
{
    for (int32_t i = 0; i < n; ++i) {
        const int32_t kb = i / bs, r0 = kb * bs, li = i - r0;
        const int32_t m = (n - r0 < bs) ? n - r0 : bs;
        const double* row = binv + (size_t)kb * bs * bs + (size_t)li * bs;
        double s = 0.0;
        for (int32_t j = 0; j < m; ++j) s += row[j] * r[r0 + j];
        z[i] = s;
    }
}

/* ILU(0), the incomplete LU factorisation without fill-in behind the
 * paper's Ilu preconditioner (Listing 1; Section 5 names ILU and IC among
 * the preconditioners pyGinkgo binds).  It follows the textbook IKJ form (Saad,
 * "Iterative Methods for Sparse Linear Systems", 2nd ed., Section 10.3.2,
 * the ILU(0) algorithm): for each row i in order, for each stored k < i in
 * ascending order, a_ik /= a_kk and then a_ij -= a_ik * a_kj for every
 * stored j > k of row k that is also stored in row i.  Entries outside the
 * pattern are dropped.  Each update a - l * u is one fused multiply-add
 * (C99 fma: the exact value rounded once).  lu[] (nnz) receives L's strictly lower part (unit
 * diagonal implied) and U (diagonal and above) in A's CSR order.
 * Rows need their columns strictly ascending (no duplicates): otherwise
 * OR_ERR_INVALID.  A row without a stored diagonal, or a zero pivot u_ii,
 * is OR_ERR_ZERO_DIAG. */
static int32_t diag_pos(const int32_t* rp, const int32_t* ci, int32_t i)
{
    for (int32_t p = rp[i]; p < rp[i + 1]; ++p)
        if (ci[p] == i) return p;
    return -1;
}

int or_ilu0(int32_t n, const int32_t* rp, const int32_t* ci, const double* va, double* lu)
{
    for (int32_t i = 0; i < n; ++i) {
        for (int32_t p = rp[i] + 1; p < rp[i + 1]; ++p)
            if (ci[p] <= ci[p - 1]) return OR_ERR_INVALID;
        if (diag_pos(rp, ci, i) < 0) return OR_ERR_ZERO_DIAG;
    }
    for (int64_t p = 0; p < (int64_t)rp[n]; ++p) lu[p] = va[p];
    for (int32_t i = 0; i < n; ++i) {
        for (int32_t p = rp[i]; p < rp[i + 1] && ci[p] < i; ++p) {
            const int32_t k = ci[p];
            const int32_t dk = diag_pos(rp, ci, k);
            lu[p] = lu[p] / lu[dk];
            for (int32_t q = dk + 1; q < rp[k + 1]; ++q) {
                const int32_t j = ci[q];
                for (int32_t t = p + 1; t < rp[i + 1]; ++t)
                    if (ci[t] == j) {
                        lu[t] = fma(-lu[p], lu[q], lu[t]);
                        break;
                    }
            }
        }
        if (lu[diag_pos(rp, ci, i)] == 0.0) return OR_ERR_ZERO_DIAG;
    }
    return OR_OK;
}

/* z = U^{-1} L^{-1} r with the factors of or_ilu0.  Forward substitution
 * in ascending row order, y_i = r_i - sum_{j<i} l_ij y_j with the terms
 * subtracted in ascending column order; back substitution in descending
 * row order, z_i = (y_i - sum_{j>i} u_ij z_j) * (1 / u_ii) with the terms
 * subtracted in descending column order (each unknown is used in the order
 * the substitution produced it), each subtraction of a product one fused
 * multiply-add (fma).  The paper does not fix the arithmetic of the
 * substitution; this reading scales by the pivot's reciprocal, rounded
 * once, as a preconditioner that stores inverted pivots does. */
void or_ilu0_apply(int32_t n, const int32_t* rp, const int32_t* ci, const double* lu,
                   const double* r, double* z)
{
    double* y = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (int32_t i = 0; i < n; ++i) {
        double s = r[i];
        for (int32_t p = rp[i]; p < rp[i + 1] && ci[p] < i; ++p) s = fma(-lu[p], y[ci[p]], s);
        y[i] = s;
    }
    for (int32_t i = n - 1; i >= 0; --i) {
        const int32_t d = diag_pos(rp, ci, i);
        double s = y[i];
        for (int32_t p = rp[i + 1] - 1; p > d; --p) s = fma(-lu[p], z[ci[p]], s);
        const double rd = 1.0 / lu[d];
        z[i] = s * rd;
    }
    free(y);
}

/* Sparse triangular solve with A's own lower (upper = 0) or upper triangle
 * (the triangular solvers pyGinkgo binds beside ILU and IC, Section 5):
 * T x = b by forward (lower) or back (upper) substitution, entries of the
 * other triangle ignored.  Row i's terms are subtracted in the order the
 * substitution produced the unknowns (lower: ascending columns, upper:
 * descending), each as one fused multiply-add, then scaled by the rounded
 * reciprocal 1 / a_ii (unit = 0) or taken as is (unit = 1: unit diagonal,
 * the stored diagonal ignored), the same arithmetic as or_ilu0_apply.
 * Every row must store its diagonal and have strictly ascending columns
 * (else OR_ERR_INVALID); unit = 0 with a zero diagonal is OR_ERR_ZERO_DIAG. */
int or_trsv(int32_t n, const int32_t* rp, const int32_t* ci, const double* va, int upper,
            int unit, const double* b, double* x)
{
    for (int32_t i = 0; i < n; ++i) {
        for (int32_t p = rp[i] + 1; p < rp[i + 1]; ++p)
            if (ci[p] <= ci[p - 1]) return OR_ERR_INVALID;
        const int32_t d = diag_pos(rp, ci, i);
        if (d < 0) return OR_ERR_INVALID;
        if (!unit && va[d] == 0.0) return OR_ERR_ZERO_DIAG;
    }
    for (int32_t t = 0; t < n; ++t) {
        const int32_t i = upper ? n - 1 - t : t;
        const int32_t d = diag_pos(rp, ci, i);
        double s = b[i];
        if (!upper)
            for (int32_t p = rp[i]; p < d; ++p) s = fma(-va[p], x[ci[p]], s);
        else
            for (int32_t p = rp[i + 1] - 1; p > d; --p) s = fma(-va[p], x[ci[p]], s);
        if (!unit) {
            const double rd = 1.0 / va[d];
            s = s * rd;
        }
        x[i] = s;
    }
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Solvers                                                             */
/* ------------------------------------------------------------------ */

typedef struct {
    int32_t method;     /* 0 CG, 1 BiCGSTAB, 2 GMRES, 3 CGS */
    int32_t precond;    /* 0 none, 1 Jacobi, 2 block-Jacobi, 3 ILU(0) */
    double tol;         /* relative to ||b||_2 ("rhs_norm" baseline) */
    int32_t max_iters;  /* CG: iterations; BiCGSTAB: iterations; GMRES: Arnoldi steps */
    int32_t krylov_dim; /* GMRES restart length m */
    int32_t block_size; /* block-Jacobi (precond 2): rows per diagonal block */
} or_opts;

typedef struct {
    int32_t status;
    int32_t iters;
    int32_t restarts;      /* GMRES cycles restarted; CG/BiCGSTAB residual replacements */
    double rel_res_rec;    /* last recurrence (or Givens) residual / ||b|| */
    double rel_res_true;   /* ||b - A x|| / ||b|| at exit */
} or_info;

typedef struct {
    int32_t n;
    const int32_t* rp;
    const int32_t* ci;
    const double* va;
} or_mat;

static void mv(const or_mat* A, const double* x, double* y)
{
    or_spmv_csr(A->n, A->rp, A->ci, A->va, x, 1.0, 0.0, y, 0);
}

/* r = b - A x */
static void resid(const or_mat* A, const double* b, const double* x, double* r)
{
    mv(A, x, r);
    for (int32_t i = 0; i < A->n; ++i) r[i] = b[i] - r[i];
}

/* z = M^{-1} r (identity without a preconditioner) */
/* Preconditioner M^{-1}: none (kind 0), Jacobi (1: data = 1/a_ii),
 * block-Jacobi (2: data = the inverted diagonal blocks of bs rows) or
 * ILU(0) (3: data = the factors of or_ilu0 in A's pattern). */
typedef struct {
    int32_t kind;
    int32_t bs;
    double* data;
    int32_t n;          /* ILU(0): the pattern the factors live in */
    const int32_t* rp;
    const int32_t* ci;
} or_prec;

static int prec_setup(int32_t n, const int32_t* rp, const int32_t* ci, const double* va,
                      const or_opts* o, or_prec* P)
{
    P->kind = o->precond;
    P->bs = o->block_size;
    P->data = NULL;
    P->n = n;
    P->rp = rp;
    P->ci = ci;
    if (P->kind == 3) {
        P->data = (double*)malloc(sizeof(double) * (size_t)(rp[n] > 0 ? rp[n] : 1));
        const int st = or_ilu0(n, rp, ci, va, P->data);
        if (st != OR_OK) {
            free(P->data);
            return st;
        }
        return OR_OK;
    }
    if (P->kind == 1) {
        P->data = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
        if (or_jacobi_gen(n, rp, ci, va, P->data) != OR_OK) {
            free(P->data);
            return OR_ERR_ZERO_DIAG;
        }
    } else if (P->kind == 2) {
        if (P->bs < 1) return OR_ERR_INVALID;
        const int64_t nb = ((int64_t)n + P->bs - 1) / P->bs;
        P->data = (double*)malloc(sizeof(double) * (size_t)(nb > 0 ? nb : 1) * P->bs * P->bs);
        const int st = or_block_jacobi_gen(n, rp, ci, va, P->bs, P->data);
        if (st != OR_OK) {
            free(P->data);
            return st;
        }
    }
    return OR_OK;
}

static void prec(int32_t n, const or_prec* P, const double* r, double* z)
{
    if (P->kind == 2) {
        or_block_jacobi_apply(n, P->bs, P->data, r, z);
        return;
    }
    if (P->kind == 3) {
        or_ilu0_apply(n, P->rp, P->ci, P->data, r, z);
        return;
    }
    for (int32_t i = 0; i < n; ++i) z[i] = P->kind == 1 ? P->data[i] * r[i] : r[i];
}

/* rec_hist (optional, max_iters + 1 entries): relative recurrence residual
 * after each iteration, entry 0 = initial residual. */

/* CG, Hestenes-Stiefel form with an optional left preconditioner M:
 *   r = b - A x; z = M^{-1} r; p = z; rho = <r, z>
 *   repeat: q = A p; alpha = rho / <p, q>; x += alpha p; r -= alpha q;
 *           test ||r||; z = M^{-1} r; rho' = <r, z>; beta = rho' / rho;
 *           p = z + beta p
 * <p, q> <= 0 means A is not SPD: OR_BREAKDOWN.  When the recurrence
 * residual passes the test, the true residual b - A x is computed; if it
 * fails, r is replaced by it and the iteration restarts from x. */
int or_cg(int32_t n, const int32_t* rp, const int32_t* ci, const double* va,
          const double* b, double* x, const or_opts* o, or_info* info,
          double* rec_hist)
{
    or_mat A = {n, rp, ci, va};
    memset(info, 0, sizeof(*info));
    or_prec P;
    {
        const int pst = prec_setup(n, rp, ci, va, o, &P);
        if (pst != OR_OK) return info->status = pst;
    }
    double bnorm = nrm2(n, b);
    if (bnorm == 0.0) {
        for (int32_t i = 0; i < n; ++i) x[i] = 0.0;
        free(P.data);
        return info->status = OR_OK;
    }
    double thr = o->tol * bnorm;
    size_t sz = sizeof(double) * (size_t)n;
    double *r = malloc(sz), *z = malloc(sz), *p = malloc(sz), *q = malloc(sz);
    resid(&A, b, x, r);
    double rn = nrm2(n, r);
    info->rel_res_rec = info->rel_res_true = rn / bnorm;
    if (rec_hist) rec_hist[0] = rn / bnorm;
    int status = OR_NOT_CONVERGED;
    if (!isfinite(rn)) status = OR_ERR_NAN;
    else if (rn <= thr) status = OR_OK;
    prec(n, &P, r, z);
    memcpy(p, z, sz);
    double rho = dot(n, r, z);
    int32_t k = 0;
    while (status == OR_NOT_CONVERGED && k < o->max_iters) {
        mv(&A, p, q);
        double pq = dot(n, p, q);
        if (!isfinite(pq)) { status = OR_ERR_NAN; break; }
        if (pq <= 0.0) { status = OR_BREAKDOWN; break; }
        double alpha = rho / pq;
        for (int32_t i = 0; i < n; ++i) x[i] += alpha * p[i];
        for (int32_t i = 0; i < n; ++i) r[i] -= alpha * q[i];
        ++k;
        rn = nrm2(n, r);
        info->rel_res_rec = rn / bnorm;
        if (rec_hist) rec_hist[k] = rn / bnorm;
        if (!isfinite(rn)) { status = OR_ERR_NAN; break; }
        if (rn <= thr) {
            resid(&A, b, x, r);
            double tn = nrm2(n, r);
            if (tn <= thr) { status = OR_OK; break; }
            /* residual replacement: restart from the current x */
            info->restarts++;
            prec(n, &P, r, z);
            memcpy(p, z, sz);
            rho = dot(n, r, z);
            continue;
        }
        prec(n, &P, r, z);
        double rho_new = dot(n, r, z);
        double beta = rho_new / rho;
        rho = rho_new;
        for (int32_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
    }
    info->iters = k;
    resid(&A, b, x, q);
    info->rel_res_true = nrm2(n, q) / bnorm;
    free(r); free(z); free(p); free(q); free(P.data);
    return info->status = status;
}

/* BiCGSTAB (van der Vorst 1992) with right preconditioning:
 *   r = b - A x; rhat = r; rho = alpha = omega = 1; v = p = 0
 *   repeat: rho' = <rhat, r> (0: breakdown); beta = (rho'/rho)(alpha/omega)
 *           p = r + beta (p - omega v); phat = M^{-1} p; v = A phat
 *           alpha = rho' / <rhat, v>; s = r - alpha v
 *           if ||s|| passes: x += alpha phat, stop (half-step exit)
 *           shat = M^{-1} s; t = A shat; omega = <t, s> / <t, t> (0: breakdown)
 *           x += alpha phat + omega shat; r = s - omega t; rho = rho'
 * A passed recurrence test whose true residual fails restarts from x
 * (r = rhat = b - A x, rho = alpha = omega = 1, v = p = 0).  Every started
 * iteration counts, including one left at the half step. */
int or_bicgstab(int32_t n, const int32_t* rp, const int32_t* ci,
                const double* va, const double* b, double* x,
                const or_opts* o, or_info* info, double* rec_hist)
{
    or_mat A = {n, rp, ci, va};
    memset(info, 0, sizeof(*info));
    or_prec P;
    {
        const int pst = prec_setup(n, rp, ci, va, o, &P);
        if (pst != OR_OK) return info->status = pst;
    }
    double bnorm = nrm2(n, b);
    if (bnorm == 0.0) {
        for (int32_t i = 0; i < n; ++i) x[i] = 0.0;
        free(P.data);
        return info->status = OR_OK;
    }
    double thr = o->tol * bnorm;
    size_t sz = sizeof(double) * (size_t)n;
    double *r = malloc(sz), *rh = malloc(sz), *p = malloc(sz), *ph = malloc(sz);
    double *v = malloc(sz), *s = malloc(sz), *sh = malloc(sz), *t = malloc(sz);
    resid(&A, b, x, r);
    double rn = nrm2(n, r);
    info->rel_res_rec = rn / bnorm;
    if (rec_hist) rec_hist[0] = rn / bnorm;
    int status = OR_NOT_CONVERGED;
    if (!isfinite(rn)) status = OR_ERR_NAN;
    else if (rn <= thr) status = OR_OK;
    memcpy(rh, r, sz);
    double rho = 1.0, alpha = 1.0, omega = 1.0;
    memset(v, 0, sz);
    memset(p, 0, sz);
    int32_t k = 0;
    while (status == OR_NOT_CONVERGED && k < o->max_iters) {
        double rho_new = dot(n, rh, r);
        if (!isfinite(rho_new)) { status = OR_ERR_NAN; break; }
        if (rho_new == 0.0) { status = OR_BREAKDOWN; break; }
        double beta = (rho_new / rho) * (alpha / omega);
        for (int32_t i = 0; i < n; ++i) p[i] = r[i] + beta * (p[i] - omega * v[i]);
        prec(n, &P, p, ph);
        mv(&A, ph, v);
        double rv = dot(n, rh, v);
        if (rv == 0.0) { status = OR_BREAKDOWN; break; }
        alpha = rho_new / rv;
        for (int32_t i = 0; i < n; ++i) s[i] = r[i] - alpha * v[i];
        ++k;
        double sn = nrm2(n, s);
        if (!isfinite(sn)) { status = OR_ERR_NAN; break; }
        if (sn <= thr) {
            for (int32_t i = 0; i < n; ++i) x[i] += alpha * ph[i];
            info->rel_res_rec = sn / bnorm;
            if (rec_hist) rec_hist[k] = sn / bnorm;
            resid(&A, b, x, r);
            double tn = nrm2(n, r);
            if (tn <= thr) { status = OR_OK; break; }
            info->restarts++;
            memcpy(rh, r, sz);
            rho = alpha = omega = 1.0;
            memset(v, 0, sz);
            memset(p, 0, sz);
            continue;
        }
        prec(n, &P, s, sh);
        mv(&A, sh, t);
        double tt = dot(n, t, t);
        double ts = dot(n, t, s);
        if (tt == 0.0) { status = OR_BREAKDOWN; break; }
        omega = ts / tt;
        if (omega == 0.0) { status = OR_BREAKDOWN; break; }
        for (int32_t i = 0; i < n; ++i) x[i] += alpha * ph[i] + omega * sh[i];
        for (int32_t i = 0; i < n; ++i) r[i] = s[i] - omega * t[i];
        rho = rho_new;
        rn = nrm2(n, r);
        info->rel_res_rec = rn / bnorm;
        if (rec_hist) rec_hist[k] = rn / bnorm;
        if (!isfinite(rn)) { status = OR_ERR_NAN; break; }
        if (rn <= thr) {
            resid(&A, b, x, r);
            double tn = nrm2(n, r);
            if (tn <= thr) { status = OR_OK; break; }
            info->restarts++;
            memcpy(rh, r, sz);
            rho = alpha = omega = 1.0;
            memset(v, 0, sz);
            memset(p, 0, sz);
        }
    }
    info->iters = k;
    resid(&A, b, x, t);
    info->rel_res_true = nrm2(n, t) / bnorm;
    free(r); free(rh); free(p); free(ph); free(v); free(s); free(sh); free(t);
    free(P.data);
    return info->status = status;
}

/* CGS (conjugate gradient squared, Sonneveld 1989), preconditioned form
 * with M^{-1} applied to the search directions: the paper benchmarks it
 * against CuPy's CGS (Section 6.2.1).  With shadow residual rt = r_0:
 *   rho = <rt, r>  (0: breakdown)
 *   first step after a (re)start: u = r, p = u
 *   else: beta = rho / rho_old; u = r + beta q; p = u + beta (q + beta p)
 *   ph = M^{-1} p; vh = A ph; sigma = <rt, vh> (0: breakdown); alpha = rho / sigma
 *   q = u - alpha vh; uh = M^{-1} (u + q); x += alpha uh; r -= alpha A uh
 * Two SpMVs per iteration.  The stopping test and the residual replacement
 * (restart from the true residual when the recurrence passes but the true
 * residual does not) are those of the other solvers here. */
int or_cgs(int32_t n, const int32_t* rp, const int32_t* ci,
           const double* va, const double* b, double* x,
           const or_opts* o, or_info* info, double* rec_hist)
{
    or_mat A = {n, rp, ci, va};
    memset(info, 0, sizeof(*info));
    or_prec P;
    {
        const int pst = prec_setup(n, rp, ci, va, o, &P);
        if (pst != OR_OK) return info->status = pst;
    }
    double bnorm = nrm2(n, b);
    if (bnorm == 0.0) {
        for (int32_t i = 0; i < n; ++i) x[i] = 0.0;
        free(P.data);
        return info->status = OR_OK;
    }
    double thr = o->tol * bnorm;
    size_t sz = sizeof(double) * (size_t)n;
    double *r = malloc(sz), *rt = malloc(sz), *u = malloc(sz), *p = malloc(sz);
    double *q = malloc(sz), *ph = malloc(sz), *vh = malloc(sz), *t = malloc(sz);
    double *uh = malloc(sz);
    resid(&A, b, x, r);
    double rn = nrm2(n, r);
    info->rel_res_rec = rn / bnorm;
    if (rec_hist) rec_hist[0] = rn / bnorm;
    int status = OR_NOT_CONVERGED;
    if (!isfinite(rn)) status = OR_ERR_NAN;
    else if (rn <= thr) status = OR_OK;
    memcpy(rt, r, sz);
    double rho_old = 1.0;
    int first = 1;
    int32_t k = 0;
    while (status == OR_NOT_CONVERGED && k < o->max_iters) {
        double rho = dot(n, rt, r);
        if (!isfinite(rho)) { status = OR_ERR_NAN; break; }
        if (rho == 0.0) { status = OR_BREAKDOWN; break; }
        if (first) {
            memcpy(u, r, sz);
            memcpy(p, u, sz);
            first = 0;
        } else {
            double beta = rho / rho_old;
            for (int32_t i = 0; i < n; ++i) u[i] = r[i] + beta * q[i];
            for (int32_t i = 0; i < n; ++i) p[i] = u[i] + beta * (q[i] + beta * p[i]);
        }
        prec(n, &P, p, ph);
        mv(&A, ph, vh);
        double sigma = dot(n, rt, vh);
        if (!isfinite(sigma)) { status = OR_ERR_NAN; break; }
        if (sigma == 0.0) { status = OR_BREAKDOWN; break; }
        double alpha = rho / sigma;
        for (int32_t i = 0; i < n; ++i) q[i] = u[i] - alpha * vh[i];
        for (int32_t i = 0; i < n; ++i) t[i] = u[i] + q[i];
        prec(n, &P, t, uh);
        for (int32_t i = 0; i < n; ++i) x[i] += alpha * uh[i];
        mv(&A, uh, t);
        for (int32_t i = 0; i < n; ++i) r[i] -= alpha * t[i];
        rho_old = rho;
        ++k;
        rn = nrm2(n, r);
        info->rel_res_rec = rn / bnorm;
        if (rec_hist) rec_hist[k] = rn / bnorm;
        if (!isfinite(rn)) { status = OR_ERR_NAN; break; }
        if (rn <= thr) {
            resid(&A, b, x, r);
            double tn = nrm2(n, r);
            if (tn <= thr) { status = OR_OK; break; }
            info->restarts++;
            memcpy(rt, r, sz);
            first = 1;
        }
    }
    info->iters = k;
    resid(&A, b, x, t);
    info->rel_res_true = nrm2(n, t) / bnorm;
    free(r); free(rt); free(u); free(p); free(q); free(ph); free(vh); free(t); free(uh);
    free(P.data);
    return info->status = status;
}

/* GMRES(m), right-preconditioned (A M^{-1} u = b, x = M^{-1} u), modified
 * Gram-Schmidt Arnoldi, Givens rotations on the Hessenberg matrix with the
 * residual estimate |g_{k+1}| checked after every column (the GMRES
 * discussion in Section 6.2.1).  One cycle:
 *   r = b - A x; beta0 = ||r||; v_1 = r / beta0; g = beta0 e_1
 *   for k = 1..m: w = A M^{-1} v_k; MGS against v_1..v_k -> h_{1..k,k};
 *     h_{k+1,k} = ||w||; apply the k-1 earlier rotations to column k;
 *     new rotation c = h_kk / d, s = h_{k+1,k} / d, d = hypot(h_kk, h_{k+1,k});
 *     g_{k+1} = -s g_k, g_k = c g_k; stop the cycle when |g_{k+1}| passes,
 *     when h_{k+1,k} = 0 (happy breakdown) or at k = m; else v_{k+1} = w / h_{k+1,k}
 *   solve the upper-triangular H y = g (back substitution); x += M^{-1} V y
 * A new cycle starts from the true residual, which also decides
 * convergence.  max_iters counts Arnoldi steps over all cycles.
 * rec_hist (optional) receives |g_{k+1}| / ||b|| after every step. */
int or_gmres(int32_t n, const int32_t* rp, const int32_t* ci,
             const double* va, const double* b, double* x, const or_opts* o,
             or_info* info, double* rec_hist)
{
    or_mat A = {n, rp, ci, va};
    memset(info, 0, sizeof(*info));
    int32_t m = o->krylov_dim > 0 ? o->krylov_dim : 30;
    or_prec P;
    {
        const int pst = prec_setup(n, rp, ci, va, o, &P);
        if (pst != OR_OK) return info->status = pst;
    }
    double bnorm = nrm2(n, b);
    if (bnorm == 0.0) {
        for (int32_t i = 0; i < n; ++i) x[i] = 0.0;
        free(P.data);
        return info->status = OR_OK;
    }
    double thr = o->tol * bnorm;
    size_t sz = sizeof(double) * (size_t)n;
    double* V = malloc(sz * (size_t)(m + 1));
    double *w = malloc(sz), *z = malloc(sz), *r = malloc(sz);
    double* H = calloc((size_t)(m + 1) * (size_t)m, sizeof(double)); /* H[i*m + j] */
    double *cs = calloc((size_t)m, sizeof(double)), *sn = calloc((size_t)m, sizeof(double));
    double *g = calloc((size_t)m + 1, sizeof(double)), *y = calloc((size_t)m, sizeof(double));
    int status = OR_NOT_CONVERGED;
    int32_t total = 0;
    int first = 1;
    for (;;) {
        resid(&A, b, x, r);
        double beta0 = nrm2(n, r);
        info->rel_res_true = beta0 / bnorm;
        if (first) {
            info->rel_res_rec = beta0 / bnorm;
            if (rec_hist) rec_hist[0] = beta0 / bnorm;
        }
        if (!isfinite(beta0)) { status = OR_ERR_NAN; break; }
        if (beta0 <= thr) { status = OR_OK; break; }
        if (total >= o->max_iters) break;
        if (!first) info->restarts++;
        first = 0;
        for (int32_t i = 0; i < n; ++i) V[i] = r[i] / beta0;
        memset(g, 0, sizeof(double) * (size_t)(m + 1));
        memset(H, 0, sizeof(double) * (size_t)(m + 1) * (size_t)m);
        g[0] = beta0;
        int32_t k = 0;
        while (k < m && total < o->max_iters) {
            prec(n, &P, V + (size_t)k * n, z);
            mv(&A, z, w);
            for (int32_t j = 0; j <= k; ++j) {
                double h = dot(n, w, V + (size_t)j * n);
                H[j * m + k] = h;
                for (int32_t i = 0; i < n; ++i) w[i] -= h * V[(size_t)j * n + i];
            }
            double hk1 = nrm2(n, w);
            H[(k + 1) * m + k] = hk1;
            for (int32_t j = 0; j < k; ++j) {
                double a = H[j * m + k], bb = H[(j + 1) * m + k];
                H[j * m + k] = cs[j] * a + sn[j] * bb;
                H[(j + 1) * m + k] = -sn[j] * a + cs[j] * bb;
            }
            double a = H[k * m + k], bb = H[(k + 1) * m + k];
            double d = hypot(a, bb);
            if (d == 0.0) { status = OR_BREAKDOWN; break; }
            cs[k] = a / d;
            sn[k] = bb / d;
            H[k * m + k] = d;
            H[(k + 1) * m + k] = 0.0;
            g[k + 1] = -sn[k] * g[k];
            g[k] = cs[k] * g[k];
            ++k;
            ++total;
            double est = fabs(g[k]);
            info->rel_res_rec = est / bnorm;
            if (rec_hist) rec_hist[total] = est / bnorm;
            if (!isfinite(est)) { status = OR_ERR_NAN; break; }
            if (hk1 == 0.0 || est <= thr) break;
            for (int32_t i = 0; i < n; ++i) V[(size_t)k * n + i] = w[i] / hk1;
        }
        if (status != OR_NOT_CONVERGED) break;
        /* back substitution H(0:k,0:k) y = g(0:k) */
        for (int32_t i = k - 1; i >= 0; --i) {
            double s = g[i];
            for (int32_t j = i + 1; j < k; ++j) s -= H[i * m + j] * y[j];
            y[i] = s / H[i * m + i];
        }
        /* x += M^{-1} (V y) */
        for (int32_t i = 0; i < n; ++i) {
            double u = 0.0;
            for (int32_t j = 0; j < k; ++j) u += V[(size_t)j * n + i] * y[j];
            w[i] = u;
        }
        prec(n, &P, w, z);
        for (int32_t i = 0; i < n; ++i) x[i] += z[i];
    }
    info->iters = total;
    if (status != OR_OK) {
        resid(&A, b, x, r);
        info->rel_res_true = nrm2(n, r) / bnorm;
    }
    free(V); free(w); free(z); free(r); free(H); free(cs); free(sn); free(g); free(y);
    free(P.data);
    return info->status = status;
}
