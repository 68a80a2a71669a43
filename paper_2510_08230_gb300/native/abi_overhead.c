/* abi_overhead.c - native driver for the binding-overhead experiment.
 *
 * The paper measures what its Python binding costs against calling the
 * library from native code (Section 6.3): P_overhead, the relative loss of
 * SpMV performance, and T_overhead, the extra time per SpMV.  This driver is
 * the native side: it loads a CSR matrix from a file, builds the handle
 * (optionally its COO form), and times `reps` calls of gk_apply on device
 * vectors with a device synchronisation after each call, on a monotonic host
 * clock, the same protocol bench.py applies to the Python binding.
 *
 * File layout (little endian): int32 n, int32 ncols, int64 nnz,
 * int32 row_ptr[n+1], int32 col[nnz], float64 values[nnz].
 * Usage: abi_overhead FILE csr|coo REPS  ->  prints "seconds_per_apply".
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

#include <cuda_runtime.h>

#include "gk.h"

static double now_s(void) {
    struct timespec t;
    clock_gettime(CLOCK_MONOTONIC, &t);
    return (double)t.tv_sec + 1e-9 * (double)t.tv_nsec;
}

static int fail(const char* what) {
    fprintf(stderr, "abi_overhead: %s\n", what);
    return 1;
}

int main(int argc, char** argv) {
    if (argc != 4) return fail("usage: abi_overhead FILE csr|coo REPS");
    const int coo = strcmp(argv[2], "coo") == 0;
    const int reps = atoi(argv[3]);
    if (reps < 1) return fail("REPS must be >= 1");
    FILE* f = fopen(argv[1], "rb");
    if (!f) return fail("cannot open the matrix file");
    int32_t n = 0, ncols = 0;
    int64_t nnz = 0;
    if (fread(&n, 4, 1, f) != 1 || fread(&ncols, 4, 1, f) != 1 || fread(&nnz, 8, 1, f) != 1 ||
        n < 0 || ncols < 0 || nnz < 0) {
        fclose(f);
        return fail("bad header");
    }
    int32_t* rp = (int32_t*)malloc(4 * ((size_t)n + 1));
    int32_t* ci = (int32_t*)malloc(4 * (size_t)(nnz > 0 ? nnz : 1));
    double* va = (double*)malloc(8 * (size_t)(nnz > 0 ? nnz : 1));
    if (!rp || !ci || !va) return fail("out of host memory");
    if (fread(rp, 4, (size_t)n + 1, f) != (size_t)n + 1 || fread(ci, 4, (size_t)nnz, f) != (size_t)nnz ||
        fread(va, 8, (size_t)nnz, f) != (size_t)nnz) {
        fclose(f);
        return fail("short file");
    }
    fclose(f);
    gk_matrix A = NULL, B = NULL;
    if (gk_matrix_create_csr(n, ncols, nnz, rp, ci, va, GK_F64, GK_MEM_HOST, NULL, &A) != GK_OK)
        return fail("gk_matrix_create_csr failed");
    if (coo) {
        if (gk_matrix_convert(A, GK_COO, GK_F64, 0, 0, NULL, &B) != GK_OK)
            return fail("gk_matrix_convert failed");
        gk_matrix_destroy(A);
        A = B;
    }
    double *b = NULL, *x = NULL;
    if (cudaMalloc((void**)&b, 8 * (size_t)(ncols > 0 ? ncols : 1)) != cudaSuccess ||
        cudaMalloc((void**)&x, 8 * (size_t)(n > 0 ? n : 1)) != cudaSuccess)
        return fail("cudaMalloc failed");
    cudaMemset(b, 0, 8 * (size_t)(ncols > 0 ? ncols : 1));
    for (int r = 0; r < 10; ++r) {  // warm-up (plans, attributes)
        if (gk_apply(A, b, x, NULL) != GK_OK) return fail("gk_apply failed");
        cudaDeviceSynchronize();
    }
    const double t0 = now_s();
    for (int r = 0; r < reps; ++r) {
        gk_apply(A, b, x, NULL);
        cudaDeviceSynchronize();
    }
    const double t1 = now_s();
    printf("%.9e\n", (t1 - t0) / reps);
    cudaFree(b);
    cudaFree(x);
    gk_matrix_destroy(A);
    free(rp);
    free(ci);
    free(va);
    return 0;
}
