/*
 * gk.h - C ABI of the GB300 sparse operator library.
 *
 * The calls follow the paper's linear-operator model (Section 4.2,
 * "Ginkgo's Linear Operator Abstraction"): a matrix is created once, then
 * "applied" to a vector (an SpMV), and a solver is "applied" to a
 * right-hand side b and an initial guess x, which it overwrites with the
 * solution (Section 3.5 "pyGinkgo API", Listing 1).  Stopping follows the
 * config solver's criteria (Listing 2): an iteration cap or a residual
 * reduction relative to ||b||_2.
 *
 * General rules for every call:
 *  - Return value: a gk_status.  No call aborts or throws; on an error the
 *    outputs are left unspecified unless stated otherwise.
 *  - Memory: a gk_matrix owns device copies of its arrays; the caller keeps
 *    its own inputs.  Vector pointers are borrowed for the duration of the
 *    call only.  Indices are int32, zero-based.
 *  - Value types: GK_F64 uses double for values, vectors and scalars;
 *    GK_F32 uses float; GK_BF16 stores matrix values as bfloat16 and uses
 *    float vectors with float accumulation.
 *  - Streams: `stream` is a cudaStream_t (NULL = legacy default stream).
 *    Device-pointer calls are stream-ordered and return without waiting,
 *    unless documented otherwise.  Calls given host pointers copy through
 *    library-owned device buffers and return after the result is back on
 *    the host.
 *  - One GPU: a matrix lives on the device that was current when it was
 *    created; every later call on it must run with that device current.
 *  - Thread safety: calls on different matrices may run concurrently from
 *    different host threads; calls on the same matrix must be serialised
 *    by the caller (the handle caches workspace and solver state).
 */
#ifndef GK_H
#define GK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GK_VERSION 1

typedef struct gk_matrix_s* gk_matrix;

/* Value types.  F64 and F32 store and compute in their type; BF16 and F16
 * store matrix values as bfloat16 / IEEE half (F16: |a_ij| <= 65504, larger
 * values become infinite) and compute in FP32 with FP32 vectors. */
typedef enum { GK_F64 = 0, GK_F32 = 1, GK_BF16 = 2, GK_F16 = 3 } gk_dtype;

/* Storage formats.
 * GK_CSR  : row_ptr[n+1], col_idx[nnz], values[nnz]; columns ascending
 *           within a row is NOT required for SpMV.
 * GK_COO  : row[nnz], col[nnz], values[nnz] in CSR order (sorted by row).
 *           A COO handle also keeps the CSR row pointer it was converted
 *           from: apply runs the COO kernel, the solvers use the CSR view.
 * GK_ELL  : K = longest row, stride = n rounded up to 32; entry j of row i
 *           at j*stride + i; padding col = -1, value = +0.0.
 * GK_SELLP: slices of S consecutive rows; slice_lengths[s] = longest row
 *           of slice s rounded up to a multiple of the stride factor f;
 *           slice_sets = exclusive prefix sum of slice_lengths
 *           (num_slices + 1 entries); entry j of row i = s*S + t at
 *           (slice_sets[s] + j)*S + t; padding col = -1, value = +0.0,
 *           including the virtual rows past n in the last slice.
 * The paper plans formats beyond CSR and COO (Section 3.1)
 * without defining them; these layouts are this library's definition. */
typedef enum { GK_CSR = 0, GK_ELL = 1, GK_SELLP = 2, GK_COO = 3 } gk_format;

/* Krylov methods: CG (Hestenes-Stiefel), BiCGSTAB (van der Vorst), GMRES(m),
 * and CGS (Sonneveld's conjugate gradient squared, the solver the paper
 * benchmarks beside CG and GMRES in Section 6.2.1). */
typedef enum { GK_CG = 0, GK_BICGSTAB = 1, GK_GMRES = 2, GK_CGS = 3 } gk_method;
/* Preconditioners: the config solver's Jacobi (Listing 2) as point Jacobi
 * (max_block_size 1) and block-Jacobi over diagonal blocks of block_size
 * consecutive rows (max_block_size > 1; each block inverted by Gauss-Jordan
 * with partial pivoting, a singular block is GK_ERR_ZERO_DIAG), and
 * ILU(0), the Ilu preconditioner of Listing 1: incomplete LU without
 * fill-in (A's pattern; the IKJ form, each update one fused
 * multiply-add) applied as z = U^-1 (L^-1 r) by exact forward and backward
 * substitution (the pivots applied as reciprocals rounded once).  ILU(0) needs every row's columns strictly ascending (what
 * gk_matrix_create_coo and the conversions produce; otherwise
 * GK_ERR_INVALID) and a stored diagonal with nonzero pivots (otherwise
 * GK_ERR_ZERO_DIAG).  For a symmetric matrix its U equals D L^T in exact
 * arithmetic, so it is also the IC(0) preconditioner L D L^T and suits CG.
 * The factors are built on first use and kept with the handle. */
typedef enum {
    GK_PRECOND_NONE = 0,
    GK_PRECOND_JACOBI = 1,
    GK_PRECOND_BLOCK_JACOBI = 2,
    GK_PRECOND_ILU = 3
} gk_precond;
typedef enum { GK_MEM_HOST = 0, GK_MEM_DEVICE = 1 } gk_memory;

typedef enum {
    GK_OK = 0,
    GK_NOT_CONVERGED = 1,  /* iteration cap reached; x holds the last iterate */
    GK_BREAKDOWN = 2,      /* CG: <p,Ap> <= 0; BiCGSTAB: rho, <rhat,v>, omega = 0;
                              CGS: <rt,r> or <rt,A M^-1 p> = 0;
                              GMRES: zero Givens denominator */
    GK_ERR_INVALID = -1,   /* bad argument or malformed matrix */
    GK_ERR_OOM = -2,       /* device allocation failed */
    GK_ERR_CUDA = -3,      /* a CUDA runtime call failed */
    GK_ERR_TIMEOUT = -4,   /* a bounded device-side wait ran out */
    GK_ERR_ZERO_DIAG = -5, /* Jacobi: missing or zero diagonal entry */
    GK_ERR_NAN = -6,       /* NaN or Inf met in a residual norm */
    GK_ERR_UNSUPPORTED = -7 /* combination not provided (e.g. wrong device) */
} gk_status;

/* Shape and layout of a matrix handle (all counts in entries). */
typedef struct {
    int32_t n;             /* rows */
    int32_t ncols;         /* columns */
    int64_t nnz;           /* stored nonzeros, padding excluded */
    gk_format format;
    gk_dtype dtype;
    int32_t max_row;       /* longest row */
    int32_t ell_width;     /* ELL: K */
    int64_t ell_stride;    /* ELL: stride */
    int32_t slice_size;    /* SELL-P: S */
    int32_t stride_factor; /* SELL-P: f */
    int32_t num_slices;    /* SELL-P: ceil(n / S) */
    int64_t stored;        /* entries held in col/values incl. padding */
    int64_t device_bytes;  /* bytes of the format arrays on the device */
    int32_t spmv_kernel;   /* SpMV kernel apply uses: 0 CSR vector, 1 CSR row-tile,
                              2 CSR merge-path, 3 ELL, 4 SELL-P, 5 COO,
                              6 CSR warp-tile */
    int32_t spmv_launches; /* kernel launches per apply */
    int32_t device_error;  /* nonzero if a kernel on this matrix gave up a
                              bounded device-side wait, so its results are
                              invalid: bit 0 the CSR row-tile SpMV (since the
                              last gk_solve began, which clears it), bit 1 the
                              last ILU(0) application, bit 2 the last
                              gk_triangular_solve */
    int32_t solve_format;  /* layout the solvers' SpMV uses on this matrix: -1
                              until the first gk_solve picks it (CSR matrices
                              may solve on an ELL or SELL-P copy), else a
                              gk_format */
} gk_matrix_desc;

/* ---------------------------------------------------------------------
 * Matrix creation and conversion
 * ------------------------------------------------------------------- */

/* Create a CSR matrix (the paper's default format: `format="Csr"` in
 * Listing 1).  row_ptr has n+1 entries, col_idx and values nnz entries;
 * `values` holds double (GK_F64), float (GK_F32) or uint16 bfloat16 bits
 * (GK_BF16).  `mem` says whether the three arrays are host or device
 * pointers; they are copied, the caller keeps ownership.  The copy is
 * validated on the device: row_ptr[0] = 0, non-decreasing, row_ptr[n] =
 * nnz, 0 <= col < ncols; otherwise GK_ERR_INVALID.  n = 0 and nnz = 0 are
 * valid.  Synchronises `stream`. */
gk_status gk_matrix_create_csr(int32_t n, int32_t ncols, int64_t nnz,
                               const int32_t* row_ptr, const int32_t* col_idx,
                               const void* values, gk_dtype dtype,
                               gk_memory mem, void* stream, gk_matrix* out);

/* Create a CSR matrix from COO triplets (COO is the paper's second
 * benchmarked format, Section 6).  Entries may come in any order; they are
 * ordered by (row, col) on the device, entries with equal (row, col) are
 * summed in their input order (float arithmetic for GK_F32/GK_BF16 input,
 * double for GK_F64), explicit zeros are kept.  Result is bit-for-bit the
 * same for any thread schedule.  Index out of range: GK_ERR_INVALID.
 * GK_BF16 values are summed as float and rounded to bfloat16 once.
 * Synchronises `stream`. */
gk_status gk_matrix_create_coo(int32_t n, int32_t ncols, int64_t nnz,
                               const int32_t* row, const int32_t* col,
                               const void* values, gk_dtype dtype,
                               gk_memory mem, void* stream, gk_matrix* out);

/* New handle holding A in format `fmt` with value type `dtype` (values
 * rounded to nearest even when narrowing; no arithmetic otherwise).
 * slice_size (S, 1..1024) and stride_factor (f >= 1) apply to GK_SELLP;
 * pass 0 for the defaults S = 32, f = 1.  A is unchanged.  Converting to
 * GK_CSR from any format is allowed.  Synchronises `stream`. */
gk_status gk_matrix_convert(gk_matrix A, gk_format fmt, gk_dtype dtype,
                            int32_t slice_size, int32_t stride_factor,
                            void* stream, gk_matrix* out);

/* Shape and layout of A; blocking (reads the device error word). */
gk_status gk_matrix_describe(gk_matrix A, gk_matrix_desc* out);

/* Copy the format arrays to caller-owned HOST buffers (any pointer may be
 * NULL to skip that array):
 *   CSR  : idx_a = row_ptr[n+1], col = col_idx[nnz], values[nnz]
 *   COO  : idx_a = row[nnz], col[nnz], values[nnz]
 *   ELL  : col[K*stride], values[K*stride]              (idx_a, sets unused)
 *   SELLP: idx_a = slice_lengths[num_slices], sets = slice_sets[num_slices+1],
 *          col[stored], values[stored]
 * values are in the matrix dtype (bfloat16 as uint16 bits).  Blocking. */
gk_status gk_matrix_export(gk_matrix A, int32_t* idx_a, int64_t* sets,
                           int32_t* col, void* values);

/* Frees the handle and everything it owns (after a device synchronise). */
gk_status gk_matrix_destroy(gk_matrix A);

/* ---------------------------------------------------------------------
 * Apply (SpMV)
 * ------------------------------------------------------------------- */

/* x = A b  (a matrix LinOp's apply, Section 4.2; the paper's SpMV
 * benchmark computes x = A b, Section 6.1).  b has ncols entries, x has n.
 * Both device pointers (stream-ordered, asynchronous) or both host
 * pointers (staged, blocking).  b and x must not overlap. */
gk_status gk_apply(gk_matrix A, const void* b, void* x, void* stream);

/* x = alpha * A b + beta * x  (the advanced apply).  When beta == 0, x is
 * not read, so NaN/Inf already in x does not propagate.  alpha and beta
 * are rounded to the vector type. */
gk_status gk_apply_adv(gk_matrix A, double alpha, const void* b, double beta,
                       void* x, void* stream);

/* ---------------------------------------------------------------------
 * Solve
 * ------------------------------------------------------------------- */

typedef struct {
    gk_method method;
    gk_precond precond;   /* none, Jacobi, block-Jacobi (block_size below) or ILU(0) */
    double tol;           /* stop when ||b - A x||_2 <= tol * ||b||_2 */
    int32_t max_iters;    /* CG/BiCGSTAB iterations; GMRES Arnoldi steps (all cycles) */
    int32_t krylov_dim;   /* GMRES restart length m (0 = 30, the paper's value); <= 64 */
    int32_t mixed;        /* 0: plain; 1: FP32 inner solves in FP64 iterative
                             refinement; 2: BF16-stored FP32 inner solves;
                             3: FP16-stored FP32 inner solves */
    double inner_tol;     /* refinement: inner reduction (0 = 1e-2 with BF16- or
                             FP16-stored values and for GMRES, else 1e-5); an
                             inner solve confirms its true residual but gives up
                             after two residual replacements.  A correction that
                             raises the FP64 true residual above 4x the best
                             so far, or whose inner solve broke down or met a
                             NaN, and three outer steps that together gain less
                             than 2x, end the refinement: the solve finishes in
                             FP64 from the best iterate (counted as one
                             restart; its iterations count in iters, within
                             max_iters) */
    int32_t max_outer;    /* refinement: outer cap (0 = 50) */
    const double* batch_tols; /* gk_solve_batched only: per-system tolerances
                             (host array of `count`), NULL = tol for all */
    int32_t engine;       /* 0 automatic; 1 multi-kernel (any n, any format);
                             2 single-block (CSR, CG/BiCGSTAB, n <= 16384);
                             3 cluster of up to 16 blocks (CSR, CG, n <= 16384).
                             Automatic picks 3 for CSR CG with n <= 16384 when a
                             cluster can be scheduled, else 1.  Block-Jacobi,
                             ILU(0) and CGS run on engine 1 only. */
    int32_t block_size;   /* block-Jacobi rows per diagonal block, 1..32 */
    int64_t wait_budget_ns; /* longest a device-side wait of this solve may last
                             (the ILU(0) substitutions' polls on values other
                             warps produce, or the window mode's waits on its
                             copies of row records; the CSR row-tile kernel's
                             waits on its staged copies) before it gives up: the solve
                             then returns GK_ERR_TIMEOUT and x holds no valid
                             iterate.  0 = the default of 2 s; negative values
                             are GK_ERR_INVALID */
} gk_solve_opts;

typedef struct {
    gk_status status;
    int32_t iters;            /* iterations (refinement: inner, summed) */
    int32_t restarts;         /* GMRES restarts; CG/BiCGSTAB residual replacements */
    int32_t outer_iters;      /* refinement steps (0 without refinement) */
    double rel_res_recurrence;/* last recurrence / Givens estimate over ||b|| */
    double rel_res_true;      /* ||b - A x||_2 / ||b||_2 recomputed at exit */
    float device_ms;          /* device time of the solve (CUDA events) */
    int32_t spmv_format;      /* layout the solve's SpMV ran on (GK_CSR, GK_ELL or
                                 GK_SELLP; refinement: the FP64 residual's) */
    int32_t slice_size;       /* SELL-P slice size of that layout, else 0 */
    int32_t block_threads;    /* threads per block of the single-block engine and
                                 of gk_solve_batched (autotuned), else 0 */
} gk_solve_info;

/* Solve A x = b for square A (Listing 1: solver.apply(b, x) overwrites
 * the initial guess).  CG (Hestenes-Stiefel), BiCGSTAB (van der Vorst,
 * right-preconditioned), CGS (Sonneveld, M^-1 on the search directions,
 * multi-kernel engine only) or GMRES(m) (right-preconditioned, Givens
 * rotations, residual estimate checked after every Arnoldi step as in
 * Section 6.2.1).  GK_OK is returned only when the recomputed true
 * residual meets tol; when the recurrence residual passes but the true
 * one does not, the residual is replaced by the true one and the method
 * restarts from x.  b = 0 gives x = 0 and GK_OK after 0 iterations.
 * b, x: device pointers of n entries (x in/out, the initial guess).
 * info may be NULL.  Blocks until the solve is finished (one stream
 * synchronise); everything is enqueued on `stream`.
 * On the multi-kernel engine the Krylov loop runs on the device: one CUDA
 * graph (built on the first solve with a given method, preconditioner and
 * Krylov dimension, then kept with the handle) repeats chunks of iterations
 * in a conditional loop node, with the confirmation of a passed recurrence
 * residual and the residual replacement decided by kernels; the host only
 * reads the outcome (GK_SOLVE_LOOP=host launches one graph per pass from
 * the host instead, two in flight; same results).  The solve works on the
 * handle's own copies of b and x.
 * SpMV layout (multi-kernel engine and refinement on a CSR matrix): a matrix
 * of at least 2^24 entries whose apply uses the CSR warp-tile kernel
 * (gk_matrix_desc.spmv_kernel 6) solves on its own arrays; otherwise the
 * first solve keeps an ELL copy of A
 * when ELL stores at most 1.2 x nnz entries, else a SELL-P(32) copy under the
 * same bound, else uses the CSR kernels; the copy lives with the handle
 * (gk_matrix_desc.solve_format reports the pick).
 * The rule reads only the sparsity pattern, so results are reproducible
 * across handles.  Environment GK_SOLVE_FORMAT=csr|ell|sellp forces a layout,
 * =timed picks the fastest of three timed SpMVs per admissible layout. */
gk_status gk_solve(gk_matrix A, const void* b, void* x,
                   const gk_solve_opts* opts, gk_solve_info* info,
                   void* stream);

/* The same solve as gk_solve, enqueued on `stream` without waiting for it:
 * the call returns once the work is enqueued and the outcome arrives in
 * `info`, a DEVICE pointer to one gk_solve_info the caller owns, when the
 * solve's work on the stream completes (device_ms is 0; read info after
 * synchronising the stream or an event recorded after the call).  x holds
 * the solution at the same point.  This is the serving form of the solver
 * LinOp (Listing 1): a thread can enqueue many solves and never wait on any.
 * The whole Krylov loop runs on the device (one CUDA graph whose
 * conditional loop node repeats the iterations and the stopping test, see
 * gk_solve), on the multi-kernel engine for every matrix size.  The first
 * solve of a matrix builds what it needs (preconditioner, solver layout,
 * the graph) and synchronises `stream` while doing so; later solves with
 * the same method, preconditioner and Krylov dimension only enqueue.
 * Solves on one matrix must be ordered (the same stream, or synchronised):
 * the handle's workspace serves one solve at a time.  Refinement (mixed != 0)
 * is GK_ERR_UNSUPPORTED here: its outer loop runs on the host.  Argument
 * errors are returned at once like gk_solve's; the solve's own status
 * (convergence, breakdown, a timed-out wait) is in info->status. */
gk_status gk_solve_async(gk_matrix A, const void* b, void* x,
                         const gk_solve_opts* opts, gk_solve_info* info, void* stream);

/* Solve `count` independent systems As[i] x_i = b_i in one launch, one
 * thread block per system, whole iteration inside the kernel.  Each system's
 * SpMV runs on a layout built for the call (one conversion launch for the
 * whole batch): its CSR arrays, an ELL copy (where ELL stores at most 1.2 x
 * its nonzeros) or a SELL-P copy with slices of S rows; every layout sums a
 * row in CSR order, so the layout never changes a result.  The layout
 * policy (CSR, ELL, SELL-P with S = 8, 16 or 32) and the block size
 * (128/256/512 threads) are autotuned per batch shape on the first call for
 * that shape (value type, method, preconditioner, log2 of the largest n and
 * of the count): each candidate runs the batch capped at 30 iterations from
 * the callers' initial guesses, which are restored afterwards; the choice
 * is cached for the process and reported per system in infos (spmv_format,
 * slice_size, block_threads).  Batches of fewer than 64 systems, or with
 * GK_AUTOTUNE=0, use CSR and 256 threads;
 * GK_BATCH_LAYOUT (csr | ell | sellp8 | sellp16 | sellp32 | sellp64) and
 * GK_BATCH_THREADS force either choice.  All
 * matrices must be CSR, square, of the same dtype, with n <= 16384; CG
 * and BiCGSTAB (GMRES: GK_ERR_UNSUPPORTED).  infos has count entries
 * (may be NULL).  bs / xs: arrays of device pointers (host arrays of
 * pointers).  Blocking. */
gk_status gk_solve_batched(int32_t count, const gk_matrix* As,
                           const void* const* bs, void* const* xs,
                           const gk_solve_opts* opts, gk_solve_info* infos,
                           void* stream);

/* ---------------------------------------------------------------------
 * Preconditioner as an operator
 * ------------------------------------------------------------------- */

/* z = M^-1 r for the preconditioner `kind` of the square matrix A (a
 * preconditioner is a LinOp whose apply transforms a vector, Section 4.2):
 * GK_PRECOND_NONE copies, JACOBI scales by 1 / a_ii, BLOCK_JACOBI applies
 * the inverted diagonal blocks of block_size (1..32) rows, ILU solves
 * L y = r then U z = y.  r and z: distinct device vectors of n entries in
 * the vector type (double for GK_F64, float otherwise).  The
 * preconditioner is built on first use and cached with A (errors as for
 * gk_solve).  Stream-ordered on `stream`; kinds NONE to BLOCK_JACOBI
 * return without waiting, ILU waits for the result and returns
 * GK_ERR_TIMEOUT if a substitution's bounded wait ran out (z is then
 * wrong, and gk_matrix_describe reports device_error until the next ILU
 * application).  The substitutions run sync-free: each warp solves a chunk
 * of consecutive rows and waits, bounded by wait_budget_ns (0 = 2 s;
 * negative: GK_ERR_INVALID), for the values its rows depend on.  On
 * stencil-like matrices (at most 4 terms a row per triangle, dependencies
 * at most 2 levels back, levels of at most 12,288 rows) setup may pick the
 * window mode instead, when it is faster: one cluster of 16 blocks solves
 * a triangle level by level through distributed shared memory, and its
 * only waits, for its own copies of the next level's row records, take the
 * same budget.  Every mode gives the same bits. */
gk_status gk_precond_apply(gk_matrix A, gk_precond kind, int32_t block_size,
                           const void* r, void* z, int64_t wait_budget_ns, void* stream);

/* The ILU(0) factors of A, built on first use, copied to the host array
 * lu (nnz entries in the vector type) in A's CSR order (for a padded
 * format, the order of its CSR conversion): entries left of the diagonal
 * hold L (unit diagonal implied), the rest U.  Blocking. */
gk_status gk_ilu_factors(gk_matrix A, void* lu, void* stream);

/* Sparse triangular solve T x = b with the lower (upper = 0) or upper
 * (upper = 1) triangle of the square matrix A, diagonal included; entries
 * of the other triangle are ignored (the triangular solvers pyGinkgo binds
 * beside ILU and IC, Section 5).  unit_diagonal = 1 takes the diagonal as
 * 1 (the stored values are then ignored, zeros allowed).  Every row must
 * store its diagonal and have strictly ascending columns (GK_ERR_INVALID
 * otherwise); a zero diagonal value without unit_diagonal is
 * GK_ERR_ZERO_DIAG.  Arithmetic: row i's terms subtracted in the order the
 * substitution produced the unknowns (lower: ascending columns; upper:
 * descending), each as one fused multiply-add, then scaled by 1 / a_ii
 * rounded once.  b, x: distinct device vectors of n entries in the vector
 * type.  The pattern analysis (dependency levels, the claim order, the
 * timed chunk shape) is built on first use and kept with A; the solve is
 * the sync-free substitution kernel of ILU(0).  Blocks until x is written;
 * GK_ERR_TIMEOUT if a wait ran past wait_budget_ns (0 = 2 s; negative:
 * GK_ERR_INVALID). */
gk_status gk_triangular_solve(gk_matrix A, int upper, int unit_diagonal, const void* b,
                              void* x, int64_t wait_budget_ns, void* stream);

/* ---------------------------------------------------------------------
 * SpMV without device allocation
 * ------------------------------------------------------------------- */

/* Largest n + nnz that gk_spmv_csr_f64_noalloc accepts. */
#define GK_NOALLOC_MAX_ITEMS 134217728

/* x = alpha * A b + beta * x for an FP64 CSR matrix given as raw DEVICE
 * arrays (row_ptr[n+1], col_idx[nnz], values[nnz]; b has ncols entries,
 * x has n), without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc - code
 * whose device memory is owned by a framework's pool allocator that must
 * not see foreign allocations, or code in a loop where an allocation,
 * which can synchronise the device, is not allowed.
 *
 * It runs the merge-path kernels that gk_apply uses for skewed CSR
 * matrices, with the per-block carry scratch held in a fixed file-scope
 * device array of 768 KB that every GPU loading this library keeps until
 * the process exits.  No cudaMalloc, cudaFree or allocating library call
 * is made.  The first call on each device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current; make that
 * first call before any stream capture.
 *
 * All calls share the one scratch array: calls that overlap on the GPU
 * (for example on two streams) race and give wrong results; serialise
 * them.  Each call rewrites every scratch entry it reads, so nothing
 * carries over from the previous call.
 *
 * Errors: GK_ERR_INVALID for negative sizes, null pointers, or
 * n + nnz > GK_NOALLOC_MAX_ITEMS (the scratch holds the carries of at most
 * GK_NOALLOC_MAX_ITEMS / 2048 blocks); GK_ERR_UNSUPPORTED on a device
 * ordinal >= 64.  The arrays are not validated: they must form a valid
 * CSR matrix (row_ptr non-decreasing from 0 to nnz, 0 <= col < ncols).
 * beta == 0 does not read x.  Stream-ordered on `stream`, asynchronous. */
gk_status gk_spmv_csr_f64_noalloc(int32_t n, int32_t ncols, int64_t nnz,
                                  const int32_t* row_ptr, const int32_t* col_idx,
                                  const double* values, double alpha, const double* b,
                                  double beta, double* x, void* stream);

/* Static English text for a status code. */
const char* gk_status_string(gk_status s);

/* GK_VERSION of the built library. */
int32_t gk_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GK_H */
