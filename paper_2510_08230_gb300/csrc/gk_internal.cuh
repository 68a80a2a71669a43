// gk_internal.cuh - internal types and helpers of the GB300 sparse library.
//
// Value types: F64 stores and computes in double; F32 in float; BF16 and F16
// store matrix values as bfloat16 / IEEE half and compute in float (vectors
// are float).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>
#include <stdio.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <mutex>
#include <string>

#include "gk.h"

namespace gk {

// ------------------------------------------------------------------ types
template <gk_dtype D> struct Types;
template <> struct Types<GK_F64> { using V = double; using T = double; };
template <> struct Types<GK_F32> { using V = float; using T = float; };
template <> struct Types<GK_BF16> { using V = __nv_bfloat16; using T = float; };
template <> struct Types<GK_F16> { using V = __half; using T = float; };

inline size_t value_bytes(gk_dtype d) { return d == GK_F64 ? 8 : d == GK_F32 ? 4 : 2; }
inline size_t vector_bytes(gk_dtype d) { return d == GK_F64 ? 8 : 4; }
inline bool valid_dtype(int d) { return d == GK_F64 || d == GK_F32 || d == GK_BF16 || d == GK_F16; }

__device__ __forceinline__ double to_t(double v, double) { return v; }
__device__ __forceinline__ float to_t(float v, float) { return v; }
__device__ __forceinline__ float to_t(__nv_bfloat16 v, float) { return __bfloat162float(v); }
__device__ __forceinline__ float to_t(__half v, float) { return __half2float(v); }

// conversions between value types (round to nearest even when narrowing)
template <typename O> struct Cvt;
template <> struct Cvt<double> {
    static __device__ __forceinline__ double f(double v) { return v; }
    static __device__ __forceinline__ double f(float v) { return (double)v; }
    static __device__ __forceinline__ double f(__nv_bfloat16 v) { return (double)__bfloat162float(v); }
    static __device__ __forceinline__ double f(__half v) { return (double)__half2float(v); }
};
template <> struct Cvt<float> {
    static __device__ __forceinline__ float f(double v) { return __double2float_rn(v); }
    static __device__ __forceinline__ float f(float v) { return v; }
    static __device__ __forceinline__ float f(__nv_bfloat16 v) { return __bfloat162float(v); }
    static __device__ __forceinline__ float f(__half v) { return __half2float(v); }
};
template <> struct Cvt<__nv_bfloat16> {
    static __device__ __forceinline__ __nv_bfloat16 f(double v) { return __double2bfloat16(v); }
    static __device__ __forceinline__ __nv_bfloat16 f(float v) { return __float2bfloat16_rn(v); }
    static __device__ __forceinline__ __nv_bfloat16 f(__nv_bfloat16 v) { return v; }
    static __device__ __forceinline__ __nv_bfloat16 f(__half v) {
        return __float2bfloat16_rn(__half2float(v));
    }
};
// IEEE half: values beyond +-65504 round to +-inf (the caller's range)
template <> struct Cvt<__half> {
    static __device__ __forceinline__ __half f(double v) { return __double2half(v); }
    static __device__ __forceinline__ __half f(float v) { return __float2half_rn(v); }
    static __device__ __forceinline__ __half f(__half v) { return v; }
    static __device__ __forceinline__ __half f(__nv_bfloat16 v) {
        return __float2half_rn(__bfloat162float(v));
    }
};
template <typename O, typename I>
__device__ __forceinline__ O cvt(I v) { return Cvt<O>::f(v); }

// accumulation type used when merging duplicate COO entries
template <typename V> struct AccOf;
template <> struct AccOf<double> { using type = double; };
template <> struct AccOf<float> { using type = float; };
template <> struct AccOf<__nv_bfloat16> { using type = float; };
template <> struct AccOf<__half> { using type = float; };
__device__ __forceinline__ double to_acc(double v) { return v; }
__device__ __forceinline__ float to_acc(float v) { return v; }
__device__ __forceinline__ float to_acc(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_acc(__half v) { return __half2float(v); }
template <typename O, typename A>
__device__ __forceinline__ O from_acc(A v) { return Cvt<O>::f(v); }

// fused multiply-add with one rounding
__device__ __forceinline__ double fmadd(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fmadd(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// read-only, L1-cached load of a matrix value / index
__device__ __forceinline__ double ldv(const double* p) { return __ldg(p); }
__device__ __forceinline__ float ldv(const float* p) { return __ldg(p); }
__device__ __forceinline__ float ldv(const __nv_bfloat16* p) {
    return __bfloat162float(__ldg(p));
}
__device__ __forceinline__ float ldv(const __half* p) { return __half2float(__ldg(p)); }

// streaming loads for data touched once (do not keep in L1)
__device__ __forceinline__ double ld_stream(const double* p) { return __ldcs(p); }
__device__ __forceinline__ float ld_stream(const float* p) { return __ldcs(p); }
__device__ __forceinline__ float ld_stream(const __nv_bfloat16* p) {
    unsigned short u = __ldcs(reinterpret_cast<const unsigned short*>(p));
    return __bfloat162float(__ushort_as_bfloat16(u));
}
__device__ __forceinline__ float ld_stream(const __half* p) {
    unsigned short u = __ldcs(reinterpret_cast<const unsigned short*>(p));
    return __half2float(__ushort_as_half(u));
}
__device__ __forceinline__ int32_t ld_stream(const int32_t* p) { return __ldcs(p); }

// ------------------------------------------------------------------ errors
void set_error(const char* where, cudaError_t e);
const char* last_error();

#define GK_CUDA(...)                                   \
    do {                                               \
        cudaError_t e_ = (__VA_ARGS__);                \
        if (e_ != cudaSuccess) {                       \
            ::gk::set_error(#__VA_ARGS__, e_);         \
            return e_ == cudaErrorMemoryAllocation     \
                       ? GK_ERR_OOM                    \
                       : GK_ERR_CUDA;                  \
        }                                              \
    } while (0)

#define GK_TRY(...)                                    \
    do {                                               \
        gk_status s_ = (__VA_ARGS__);                  \
        if (s_ != GK_OK) return s_;                    \
    } while (0)

// Allocation padded by 64 bytes so that 16-byte vector loads rounded out
// to alignment at either end of an array stay inside the allocation.
cudaError_t dmalloc(void** p, size_t bytes);
template <typename X>
cudaError_t dmalloc_t(X** p, size_t count) {
    return dmalloc(reinterpret_cast<void**>(p), count * sizeof(X));
}
void dfree(void* p);

// Device buffer that only grows (workspace cache).
struct DevBuf {
    void* ptr = nullptr;
    size_t bytes = 0;
    gk_status ensure(size_t want);
    void release();
};

// ------------------------------------------------------------------ matrix
// CSR launch plan.  Row tiles: tile c covers the rows starting in nonzero
// chunk c; tile_desc[c] = {first row, end row, aligned first nonzero,
// staged entries}, staged entries <= tile_cap.  Merge path: block_row[b] =
// first row of merge block b (n_blocks + 1 entries).
constexpr int WT_WARPS = 8;  // warps per block of the warp-tile kernel (CSR kind 3)
constexpr int WT_SMEM_CAP = 208 * 1024;  // largest ring of one warp-tile block (the
                                         // epilogues' static shared memory fits beside it)

struct CsrPlan {
    int kind = 0;            // 0 vector (G lanes / row), 1 row-tile, 2 merge, 3 warp-tile
    int lanes = 1;           // vector kernel lanes per row
    int32_t ntiles = 0;
    int32_t chunk = 0;       // nnz per chunk used to cut tiles
    int32_t tile_cap = 0;    // staged entries per tile (row-tile: >= chunk + max_row + 14;
                             // warp-tile: >= 32 * wt_rpl * max_row + 14)
    int32_t stages = 0;      // row-tile pipeline depth (0 = as many as fit, max 3);
                             // warp-tile: stages per warp
    int4* tile_desc = nullptr;
    int32_t wt_rpl = 2;      // warp-tile: rows per lane (tiles of 32 * wt_rpl rows)
    int32_t merge_blocks = 0;
    int32_t merge_e = 8;     // merge-path items per lane (4, 6 or 8)
    int32_t merge_warp = 2;  // merge units: 1 one warp (32*E items, operands staged in
                             // shared memory), 2 one warp (operands in registers),
                             // 0 one block (256*E items)
    int32_t* block_row = nullptr;
    int32_t* err = nullptr;  // device word set by a kernel whose bounded wait ran out
};

struct SolverCache;  // solve.cu

// Two triangular factors sharing one CSR pattern: the ILU(0) factors, or a
// matrix's own lower and upper triangles (gk_triangular_solve), with what
// the substitution kernels need.  Built on first use and owned by the
// handle (ilu.cu).
struct TriStore {
    int state = 0;                  // 1 built, < 0 the gk_status of a failed build
    int zero_diag = 0;              // some diagonal value is zero
    int32_t* rp = nullptr;          // row_ptr / col copies of the pattern
    int32_t* ci = nullptr;
    int32_t* dpos = nullptr;        // position of each row's diagonal
    void* lu = nullptr;             // values in CSR order (vector type)
    void* rdiag = nullptr;          // 1 / diagonal (vector type)
    int32_t* ord = nullptr;         // chunks in claim (level) order: L, then U
    int32_t nord[2] = {0, 0};       // claim-order lengths (L at ord, U after it)
    int32_t warps[2] = {0, 0};      // warps per substitution launch (L, U)
    int32_t cs = 32;                // rows per substitution chunk
    int32_t cpw = 1;                // substitution chunks per warp
    void* sync = nullptr;           // claim, exit and error words of both directions
    // level-synchronous substitution (lvl = 1: picked): rows of L then U in
    // level order (2n), each triangle's level starts (nlev + 1 each)
    int32_t lvl = 0;
    int32_t* lrows = nullptr;
    int32_t* lstart = nullptr;
    int32_t nlev[2] = {0, 0};
    // window mode (win = 1: picked): one record per level-ordered row of L
    // then U (WinRec of the vector type), the deepest dependency in levels
    // of each triangle, and the level-ordered input scratch (n values)
    int32_t win = 0;
    int32_t wdist[2] = {1, 1};
    void* wrec = nullptr;
    void* wperm = nullptr;
    DevBuf w;                       // scratch of one application
    void release() {
        dfree(lrows);
        dfree(lstart);
        dfree(wrec);
        dfree(wperm);
        lrows = lstart = nullptr;
        wrec = wperm = nullptr;
        dfree(rp);
        dfree(ci);
        dfree(dpos);
        dfree(lu);
        dfree(rdiag);
        dfree(ord);
        dfree(sync);
        rp = ci = dpos = ord = nullptr;
        lu = rdiag = sync = nullptr;
        w.release();
    }
    ~TriStore() { release(); }
};

// result of one solve (either engine)
struct SolveOut {
    gk_status status = GK_OK;
    int32_t iters = 0, restarts = 0;
    double rec = 0.0, tru = 0.0;
    int32_t layout = GK_CSR, slice = 0, threads = 0;  // the SpMV layout and block size used
};

}  // namespace gk

struct gk_matrix_s {
    int device = 0;
    int32_t n = 0, ncols = 0;
    int64_t nnz = 0;
    gk_format fmt = GK_CSR;
    gk_dtype dtype = GK_F64;
    int32_t max_row = 0;
    double mean_row = 0.0;
    // CSR
    int32_t* row_ptr = nullptr;
    int32_t* col = nullptr;
    void* val = nullptr;
    // COO view (apply runs the COO kernel; fmt stays GK_CSR for everything else)
    int coo = 0;
    int32_t* coo_row = nullptr;     // row of every entry
    int32_t* empty_rows = nullptr;  // rows without entries
    int32_t n_empty = 0;
    int coo_e = 4;                  // entries per lane of the COO kernel (4, 8, 12 or 16)
    // ELL
    int32_t K = 0;
    int64_t stride = 0;
    // SELL-P
    int32_t S = 0, f = 0, nslices = 0;
    int32_t* slice_len = nullptr;
    int64_t* slice_set = nullptr;
    int64_t stored = 0;
    // launch plan for CSR SpMV
    gk::CsrPlan plan;
    // derived data, built on first use
    void* dinv = nullptr;         // Jacobi inverse diagonal (vector type)
    int dinv_state = 0;           // 0 not built, 1 ok, -1 zero diagonal
    void* binv = nullptr;         // block-Jacobi inverses (vector type, column-major blocks)
    int32_t binv_bs = 0;          // their block size (0 none, -bs singular)
    // ILU(0) factors, and A's own triangles for gk_triangular_solve, built on
    // first use (ilu.cu)
    gk::TriStore* ilu = nullptr;
    gk::TriStore* tri = nullptr;
    gk_matrix_s* lowp[3] = {nullptr, nullptr, nullptr};  // same layout, other dtype
    gk_matrix_s* solve_fmt = nullptr;  // SpMV layout picked for solves (null: not tuned)
    int solve_fmt_tuned = 0;
    gk::SolverCache* solver = nullptr;
    gk::DevBuf stage_in, stage_out;  // host-pointer apply staging
    gk::DevBuf carry;                // merge-path block carries
    cudaStream_t side = nullptr;     // library streams for graph capture (the second
    cudaStream_t side2 = nullptr;    // captures the body of a solve's loop)
    uint64_t wait_ns = 2000000000ull;  // budget of the row-tile kernel's waits (a solve's
                                       // wait_budget_ns while it runs, else 2 s)
    std::mutex mu;
};

namespace gk {
gk_status build_csr_plan(gk_matrix A, cudaStream_t s);
gk_status ensure_jacobi(gk_matrix A, cudaStream_t s);
gk_status get_lowp(gk_matrix A, gk_dtype d, cudaStream_t s, gk_matrix* out);
void free_solver_cache(gk_matrix A);
gk_status spmv_dispatch(gk_matrix A, double alpha, const void* b, double beta,
                        void* x, cudaStream_t s);
int num_sms();
// CUDA graph capture excludes the library's device-wide driver calls in
// other host threads.  On GB300 with driver 580, cuStreamEndCapture crashed
// when another thread freed device memory or synchronised the device while
// the capture was open (serving workers uploading, evicting and building
// solve graphs at once), even with captures serialised.  So a capture holds
// the gate exclusively (GateCapture: one capture at a time), and every
// allocation, free and device synchronisation holds it shared (GateShared;
// re-entrant within a thread, and a no-op inside the thread's own capture).
struct GateShared {
    GateShared();
    ~GateShared();
    bool held;
};
struct GateCapture {
    GateCapture();
    ~GateCapture();
};
}  // namespace gk
