// matrix.cu - matrix handles: creation (CSR, COO), validation, format and
// value-type conversion, export, launch planning.
//
// COO -> CSR follows the ordering rule of the library's COO entry point:
// entries sorted by (row, col); equal (row, col) entries summed in input
// order; explicit zeros kept.  The device algorithm is: count rows, scan,
// scatter (row, col, input position) keys into row buckets in any order,
// sort each bucket by (col, input position) - a total order, so the result
// does not depend on the scatter order - then merge equal columns left to
// right.
#include <algorithm>
#include <cstring>
#include <vector>

#include <shared_mutex>

#include "prims.cuh"

namespace gk {

static thread_local std::string g_last_error;

void set_error(const char* where, cudaError_t e) {
    g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
}
const char* last_error() { return g_last_error.c_str(); }

static std::shared_mutex g_gate;
static thread_local int g_gate_depth = 0;   // shared holds of this thread
static thread_local bool g_in_capture = false;

GateShared::GateShared() : held(false) {
    if (g_in_capture) return;
    if (g_gate_depth++ == 0) {
        g_gate.lock_shared();
        held = true;
    }
}
GateShared::~GateShared() {
    if (g_in_capture) return;
    if (--g_gate_depth == 0 && held) g_gate.unlock_shared();
}
GateCapture::GateCapture() {
    g_gate.lock();
    g_in_capture = true;
}
GateCapture::~GateCapture() {
    g_in_capture = false;
    g_gate.unlock();
}

cudaError_t dmalloc(void** p, size_t bytes) {
    GateShared gate;
    *p = nullptr;
    return cudaMalloc(p, bytes + 64);
}
void dfree(void* p) {
    GateShared gate;
    if (p) cudaFree(p);
}

gk_status DevBuf::ensure(size_t want) {
    if (want <= bytes && ptr) return GK_OK;
    GateShared gate;
    if (ptr) {
        cudaFree(ptr);
        ptr = nullptr;
        bytes = 0;
    }
    size_t b = std::max<size_t>(want, 256);
    GK_CUDA(dmalloc(&ptr, b));
    bytes = b;
    return GK_OK;
}
void DevBuf::release() {
    GateShared gate;
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    bytes = 0;
}

int num_sms() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

__global__ void k_scan_blocksums(int64_t* __restrict__ bsum, int64_t nb) {
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < nb; base += SCAN_TILE) {
        int64_t v[SCAN_ITEMS];
        const int64_t my = base + (int64_t)threadIdx.x * SCAN_ITEMS;
#pragma unroll
        for (int i = 0; i < SCAN_ITEMS; ++i) v[i] = (my + i < nb) ? bsum[my + i] : 0;
        int64_t tot = block_excl_scan(v);
        const int64_t c = carry;
#pragma unroll
        for (int i = 0; i < SCAN_ITEMS; ++i)
            if (my + i < nb) bsum[my + i] = v[i] + c;
        __syncthreads();
        if (threadIdx.x == 0) carry = c + tot;
        __syncthreads();
    }
}

// ---------------------------------------------------------------- kernels

// Validation of a CSR copy.  err bits: 1 row_ptr[0] != 0, 2 decreasing,
// 4 row_ptr[n] != nnz, 8 column out of range.  Also max row length.
__global__ void k_validate_rowptr(int32_t n, int64_t nnz, const int32_t* __restrict__ rp,
                                  unsigned int* err, int32_t* max_row) {
    int32_t local_max = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t a = rp[i], b = rp[i + 1];
        if (b < a) atomicOr(err, 2u);
        else local_max = max(local_max, b - a);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (rp[0] != 0) atomicOr(err, 1u);
        if ((int64_t)rp[n] != nnz) atomicOr(err, 4u);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) local_max = max(local_max, __shfl_xor_sync(0xffffffffu, local_max, o));
    if ((threadIdx.x & 31) == 0 && local_max > 0) atomicMax(max_row, local_max);
}

__global__ void k_validate_cols(int64_t nnz, int32_t ncols, const int32_t* __restrict__ ci,
                                unsigned int* err) {
    bool bad = false;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz;
         k += (int64_t)gridDim.x * blockDim.x) {
        int32_t c = ci[k];
        bad |= (c < 0) | (c >= ncols);
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(err, 8u);
}

__global__ void k_coo_count(int64_t nnz, int32_t n, int32_t ncols, const int32_t* __restrict__ row,
                            const int32_t* __restrict__ col, int32_t* __restrict__ cnt,
                            unsigned int* err) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz;
         k += (int64_t)gridDim.x * blockDim.x) {
        int32_t r = row[k], c = col[k];
        if (r < 0 || r >= n || c < 0 || c >= ncols) {
            atomicOr(err, 8u);
            continue;
        }
        atomicAdd(cnt + r, 1);
    }
}

__global__ void k_coo_scatter(int64_t nnz, const int32_t* __restrict__ row,
                              const int32_t* __restrict__ col, const int64_t* __restrict__ start,
                              int32_t* __restrict__ cursor, uint64_t* __restrict__ keys) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz;
         k += (int64_t)gridDim.x * blockDim.x) {
        int32_t r = row[k];
        int64_t pos = start[r] + atomicAdd(cursor + r, 1);
        keys[pos] = ((uint64_t)(uint32_t)col[k] << 32) | (uint64_t)(uint32_t)k;
    }
}

// Sort rows of length in (W/2, W] (W <= 32) with W-lane bitonic networks.
template <int W>
__global__ void k_sort_rows_sub(int32_t n, const int64_t* __restrict__ start,
                                uint64_t* __restrict__ keys) {
    const int lane = threadIdx.x & (W - 1);
    const int64_t g = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / W;
    const int64_t ng = ((int64_t)gridDim.x * blockDim.x) / W;
    // the loop trip count is uniform across the warp (groups advance together)
    const int64_t warp_first = g - (threadIdx.x & 31) / W;
    for (int64_t base = warp_first; base < n; base += ng) {
        const int64_t r = base + (threadIdx.x & 31) / W;
        int64_t a = 0, L = 0;
        if (r < n) {
            a = start[r];
            L = start[r + 1] - a;
        }
        const bool mine = (L > W / 2) && (L <= W);
        uint64_t v = (mine && lane < L) ? keys[a + lane] : ~0ull;
#pragma unroll
        for (int k = 2; k <= W; k <<= 1) {
#pragma unroll
            for (int j = k >> 1; j > 0; j >>= 1) {
                uint64_t o = __shfl_xor_sync(0xffffffffu, v, j, W);
                bool up = ((lane & k) == 0);
                bool lower = ((lane & j) == 0);
                uint64_t mn = v < o ? v : o, mx = v < o ? o : v;
                v = (lower == up) ? mn : mx;
            }
        }
        if (mine && lane < L) keys[a + lane] = v;
    }
}

// Sort rows of length in (lo, hi] with one block per row, keys padded to a
// power of two in shared memory (dynamic smem of cap keys).
__global__ void k_sort_rows_block(int32_t n, const int64_t* __restrict__ start,
                                  uint64_t* __restrict__ keys, int64_t lo, int64_t hi, int cap) {
    extern __shared__ uint64_t sk[];
    for (int64_t r = blockIdx.x; r < n; r += gridDim.x) {
        const int64_t a = start[r], L = start[r + 1] - a;
        if (L <= lo || L > hi) continue;
        int P = 1;
        while (P < L) P <<= 1;
        for (int i = threadIdx.x; i < P; i += blockDim.x) sk[i] = i < L ? keys[a + i] : ~0ull;
        __syncthreads();
        for (int k = 2; k <= P; k <<= 1) {
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int i = threadIdx.x; i < P; i += blockDim.x) {
                    int p = i ^ j;
                    if (p > i) {
                        bool up = ((i & k) == 0);
                        uint64_t x = sk[i], y = sk[p];
                        if ((x > y) == up) {
                            sk[i] = y;
                            sk[p] = x;
                        }
                    }
                }
                __syncthreads();
            }
        }
        for (int i = threadIdx.x; i < L; i += blockDim.x) keys[a + i] = sk[i];
        __syncthreads();
        (void)cap;
    }
}

// Rows longer than the shared-memory sorter: bitonic sort in a global
// scratch area of P keys per block.
__global__ void k_sort_rows_global(int32_t n, const int64_t* __restrict__ start,
                                   uint64_t* __restrict__ keys, int64_t lo,
                                   uint64_t* __restrict__ scratch, int64_t P) {
    uint64_t* sk = scratch + (int64_t)blockIdx.x * P;
    for (int64_t r = blockIdx.x; r < n; r += gridDim.x) {
        const int64_t a = start[r], L = start[r + 1] - a;
        if (L <= lo) continue;
        int64_t Q = 1;
        while (Q < L) Q <<= 1;
        for (int64_t i = threadIdx.x; i < Q; i += blockDim.x) sk[i] = i < L ? keys[a + i] : ~0ull;
        __syncthreads();
        for (int64_t k = 2; k <= Q; k <<= 1) {
            for (int64_t j = k >> 1; j > 0; j >>= 1) {
                for (int64_t i = threadIdx.x; i < Q; i += blockDim.x) {
                    int64_t p = i ^ j;
                    if (p > i) {
                        bool up = ((i & k) == 0);
                        uint64_t x = sk[i], y = sk[p];
                        if ((x > y) == up) {
                            sk[i] = y;
                            sk[p] = x;
                        }
                    }
                }
                __syncthreads();
            }
        }
        for (int64_t i = threadIdx.x; i < L; i += blockDim.x) keys[a + i] = sk[i];
        __syncthreads();
    }
}

__global__ void k_count_unique(int32_t n, const int64_t* __restrict__ start,
                               const uint64_t* __restrict__ keys, int64_t* __restrict__ ucnt) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x) {
        int64_t a = start[r], b = start[r + 1], c = 0;
        uint32_t prev = 0;
        for (int64_t k = a; k < b; ++k) {
            uint32_t col = (uint32_t)(keys[k] >> 32);
            if (k == a || col != prev) ++c;
            prev = col;
        }
        ucnt[r] = c;
    }
}

template <typename VIn, typename VOut, typename Acc>
__global__ void k_merge_unique(int32_t n, const int64_t* __restrict__ start,
                               const uint64_t* __restrict__ keys, const int64_t* __restrict__ uoff,
                               const VIn* __restrict__ val, int32_t* __restrict__ out_col,
                               VOut* __restrict__ out_val) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x) {
        int64_t a = start[r], b = start[r + 1], o = uoff[r];
        int64_t k = a;
        while (k < b) {
            uint32_t c = (uint32_t)(keys[k] >> 32);
            Acc s = (Acc)to_acc(val[(uint32_t)keys[k]]);
            int64_t j = k + 1;
            while (j < b && (uint32_t)(keys[j] >> 32) == c) {
                s = s + (Acc)to_acc(val[(uint32_t)keys[j]]);
                ++j;
            }
            out_col[o] = (int32_t)c;
            out_val[o] = from_acc<VOut>(s);
            ++o;
            k = j;
        }
    }
}

__global__ void k_i64_to_i32(int64_t m, const int64_t* __restrict__ in, int32_t* __restrict__ out,
                             unsigned int* err) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t v = in[i];
        if (v > INT32_MAX) atomicOr(err, 16u);
        out[i] = (int32_t)v;
    }
}

// value conversion (round to nearest even on narrowing)
template <typename VIn, typename VOut>
__global__ void k_convert_values(int64_t m, const VIn* __restrict__ in, VOut* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = cvt<VOut>(in[i]);
}

template <typename VIn, typename VOut>
__global__ void k_csr_to_ell(int32_t n, int64_t stride, int32_t K, const int32_t* __restrict__ rp,
                             const int32_t* __restrict__ ci, const VIn* __restrict__ va,
                             int32_t* __restrict__ ecol, VOut* __restrict__ eval) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < stride;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t a = 0, L = 0;
        if (i < n) {
            a = rp[i];
            L = rp[i + 1] - a;
        }
        for (int32_t j = 0; j < K; ++j) {
            int64_t at = (int64_t)j * stride + i;
            if (j < L) {
                ecol[at] = ci[a + j];
                eval[at] = cvt<VOut>(va[a + j]);
            } else {
                ecol[at] = -1;
                eval[at] = cvt<VOut>(0.0);
            }
        }
    }
}

__global__ void k_slice_lengths(int32_t n, int32_t S, int32_t f, int32_t nslices,
                                const int32_t* __restrict__ rp, int32_t* __restrict__ slen) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nslices;
         s += (int64_t)gridDim.x * blockDim.x) {
        int32_t m = 0;
        int64_t lo = s * S, hi = lo + S < (int64_t)n ? lo + S : (int64_t)n;
        for (int64_t i = lo; i < hi; ++i) m = max(m, rp[i + 1] - rp[i]);
        slen[s] = ((m + f - 1) / f) * f;
    }
}

template <typename VIn, typename VOut>
__global__ void k_csr_to_sellp(int32_t n, int32_t S, int32_t nslices, const int32_t* __restrict__ rp,
                               const int32_t* __restrict__ ci, const VIn* __restrict__ va,
                               const int32_t* __restrict__ slen, const int64_t* __restrict__ sset,
                               int32_t* __restrict__ scol, VOut* __restrict__ sval) {
    const int64_t slots = (int64_t)nslices * S;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < slots;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = i / S, t = i - s * S;
        int32_t a = 0, L = 0;
        if (i < n) {
            a = rp[i];
            L = rp[i + 1] - a;
        }
        const int64_t base = sset[s];
        const int32_t len = slen[s];
        for (int32_t j = 0; j < len; ++j) {
            int64_t at = (base + j) * S + t;
            if (j < L) {
                scol[at] = ci[a + j];
                sval[at] = cvt<VOut>(va[a + j]);
            } else {
                scol[at] = -1;
                sval[at] = cvt<VOut>(0.0);
            }
        }
    }
}

// ELL / SELL-P back to CSR: count stored (col >= 0) entries per row ...
__global__ void k_padded_row_counts(int32_t n, int fmt, int64_t stride, int32_t K, int32_t S,
                                    const int32_t* __restrict__ slen,
                                    const int64_t* __restrict__ sset,
                                    const int32_t* __restrict__ pcol, int32_t* __restrict__ cnt) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t c = 0;
        if (fmt == GK_ELL) {
            for (int32_t j = 0; j < K; ++j) c += pcol[(int64_t)j * stride + i] >= 0;
        } else {
            const int64_t s = i / S, t = i - s * S;
            for (int32_t j = 0; j < slen[s]; ++j) c += pcol[(sset[s] + j) * S + t] >= 0;
        }
        cnt[i] = c;
    }
}

// ... then copy them in order.
template <typename VIn, typename VOut>
__global__ void k_padded_to_csr(int32_t n, int fmt, int64_t stride, int32_t K, int32_t S,
                                const int32_t* __restrict__ slen, const int64_t* __restrict__ sset,
                                const int32_t* __restrict__ pcol, const VIn* __restrict__ pval,
                                const int32_t* __restrict__ rp, int32_t* __restrict__ ci,
                                VOut* __restrict__ va) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t o = rp[i];
        if (fmt == GK_ELL) {
            for (int32_t j = 0; j < K; ++j) {
                int64_t at = (int64_t)j * stride + i;
                if (pcol[at] >= 0) {
                    ci[o] = pcol[at];
                    va[o] = cvt<VOut>(pval[at]);
                    ++o;
                }
            }
        } else {
            const int64_t s = i / S, t = i - s * S;
            for (int32_t j = 0; j < slen[s]; ++j) {
                int64_t at = (sset[s] + j) * S + t;
                if (pcol[at] >= 0) {
                    ci[o] = pcol[at];
                    va[o] = cvt<VOut>(pval[at]);
                    ++o;
                }
            }
        }
    }
}

__device__ __forceinline__ int32_t rows_before_nnz(int32_t n, const int32_t* __restrict__ rp,
                                                   int64_t target) {
    int32_t lo = 0, hi = n;  // first row r with row_ptr[r] >= target
    while (lo < hi) {
        const int32_t mid = lo + ((hi - lo) >> 1);
        if ((int64_t)rp[mid] < target) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Row-tile plan: tile c holds the rows whose first nonzero lies in
// [c * chunk, (c + 1) * chunk); its staged range is rounded out to 8 entries.
__global__ void k_tile_desc(int32_t n, const int32_t* __restrict__ rp, int32_t chunk,
                            int32_t ntiles, int4* __restrict__ desc) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ntiles;
         c += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r0 = rows_before_nnz(n, rp, c * (int64_t)chunk);
        const int32_t r1 = (c + 1 == ntiles) ? n : rows_before_nnz(n, rp, (c + 1) * (int64_t)chunk);
        const int32_t e0 = r0 < r1 ? rp[r0] : 0, e1 = r0 < r1 ? rp[r1] : 0;
        const int32_t a0 = e0 & ~7;
        const int32_t w = (e1 > e0) ? (((e1 + 7) & ~7) - a0) : 0;
        desc[c] = make_int4(r0, r1, a0, w);
    }
}

// Merge plan: block b starts at path item b * items; its first row is the
// number of rows whose end item lies before that point.
__global__ void k_merge_rows(int32_t n, int64_t nnz, const int32_t* __restrict__ rp,
                             int32_t items, int32_t nblocks, int32_t* __restrict__ mrow) {
    const int64_t N = (int64_t)n + nnz;
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b <= nblocks;
         b += (int64_t)gridDim.x * blockDim.x) {
        const int64_t d = min(b * (int64_t)items, N);
        int32_t lo = 0, hi = n;
        while (lo < hi) {
            const int32_t mid = lo + ((hi - lo) >> 1);
            if ((int64_t)rp[mid + 1] + mid + 1 > d) hi = mid;
            else lo = mid + 1;
        }
        mrow[b] = lo;
    }
}

// ------------------------------------------------------------ host helpers

static unsigned grid_for(int64_t work, int threads = 256) {
    int64_t b = (work + threads - 1) / threads;
    int64_t cap = (int64_t)num_sms() * 16;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (unsigned)b;
}

template <class F>
static gk_status dispatch_dtype(gk_dtype d, F&& f) {
    switch (d) {
        case GK_F64: return f(Types<GK_F64>{});
        case GK_F32: return f(Types<GK_F32>{});
        case GK_BF16: return f(Types<GK_BF16>{});
        case GK_F16: return f(Types<GK_F16>{});
    }
    return GK_ERR_INVALID;
}

static gk_status read_err(unsigned int* derr, cudaStream_t s, unsigned int* herr) {
    GK_CUDA(cudaMemcpyAsync(herr, derr, sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
    GK_CUDA(cudaStreamSynchronize(s));
    return GK_OK;
}

static gk_matrix new_handle() {
    gk_matrix A = new (std::nothrow) gk_matrix_s();
    if (A) cudaGetDevice(&A->device);
    return A;
}

static void free_arrays(gk_matrix A) {
    dfree(A->row_ptr);
    dfree(A->col);
    dfree(A->val);
    dfree(A->slice_len);
    dfree(A->slice_set);
    dfree(A->plan.tile_desc);
    dfree(A->plan.block_row);
    dfree(A->plan.err);
    dfree(A->dinv);
    dfree(A->binv);
    A->binv = nullptr;
    A->binv_bs = 0;
    dfree(A->coo_row);
    dfree(A->empty_rows);
    A->coo_row = A->empty_rows = nullptr;
    delete A->ilu;
    delete A->tri;
    A->ilu = A->tri = nullptr;
    A->row_ptr = A->col = nullptr;
    A->val = nullptr;
    A->slice_len = nullptr;
    A->slice_set = nullptr;
    A->plan.tile_desc = nullptr;
    A->plan.block_row = A->plan.err = nullptr;
    A->dinv = nullptr;
}

static void destroy_handle(gk_matrix A) {
    if (!A) return;
    for (int i = 0; i < 3; ++i) destroy_handle(A->lowp[i]);
    if (A->solve_fmt != A) destroy_handle(A->solve_fmt);
    free_solver_cache(A);
    free_arrays(A);
    A->stage_in.release();
    A->stage_out.release();
    A->carry.release();
    if (A->side) cudaStreamDestroy(A->side);
    if (A->side2) cudaStreamDestroy(A->side2);
    delete A;
}

// COO view of a CSR handle: the row of every entry, and the list of rows
// without entries (the COO kernel never visits them).
__global__ void k_coo_rows(int32_t n, const int32_t* __restrict__ rp, int32_t* __restrict__ rows,
                           int32_t* __restrict__ empty, unsigned int* __restrict__ n_empty) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = rp[i], b = rp[i + 1];
        for (int32_t k = a; k < b; ++k) rows[k] = (int32_t)i;
        if (a == b) empty[atomicAdd(n_empty, 1u)] = (int32_t)i;  // order of the list is free
    }
}

static gk_status build_coo_view(gk_matrix A, cudaStream_t s) {
    DevBuf cnt, tmp_empty;
    GK_TRY(cnt.ensure(16));
    GK_CUDA(cudaMemsetAsync(cnt.ptr, 0, 16, s));
    GK_CUDA(dmalloc_t(&A->coo_row, (size_t)std::max<int64_t>(A->nnz, 1)));
    GK_TRY(tmp_empty.ensure(4 * (size_t)std::max(A->n, 1)));
    if (A->n > 0)
        k_coo_rows<<<grid_for(A->n), 256, 0, s>>>(A->n, A->row_ptr, A->coo_row,
                                                   (int32_t*)tmp_empty.ptr, (unsigned int*)cnt.ptr);
    GK_CUDA(cudaGetLastError());
    unsigned int ne = 0;
    GK_CUDA(cudaMemcpyAsync(&ne, cnt.ptr, 4, cudaMemcpyDeviceToHost, s));
    GK_CUDA(cudaStreamSynchronize(s));
    A->n_empty = (int32_t)ne;
    if (ne) {
        GK_CUDA(dmalloc_t(&A->empty_rows, (size_t)ne));
        GK_CUDA(cudaMemcpyAsync(A->empty_rows, tmp_empty.ptr, 4 * (size_t)ne, cudaMemcpyDeviceToDevice, s));
        GK_CUDA(cudaStreamSynchronize(s));
    }
    A->coo = 1;
    // triplets per lane: 8 in FP64 (fewer FP64 carry adds per nonzero; 343 us
    // against 366 us for 4 on the 4M-row Zipf matrix), 4 in FP32 (279 us
    // against 291 us)
    A->coo_e = A->dtype == GK_F64 ? 8 : 4;
    if (const char* e = getenv("GK_COO_E")) {
        const int v = atoi(e);
        A->coo_e = (v == 8 || v == 12 || v == 16) ? v : 4;
    }
    return GK_OK;
}

// CSR launch plan: row tiles when rows are short, merge path otherwise.
gk_status build_csr_plan(gk_matrix A, cudaStream_t s) {
    CsrPlan& P = A->plan;
    dfree(P.tile_desc);
    dfree(P.block_row);
    dfree(P.err);
    P = CsrPlan();
    GK_CUDA(dmalloc_t(&P.err, 4));
    GK_CUDA(cudaMemsetAsync(P.err, 0, 4, s));
    if (A->fmt != GK_CSR || A->n == 0) return GK_OK;
    const double mean = A->mean_row;
    int lanes = 1;
    while (lanes < 32 && lanes < mean) lanes <<= 1;
    P.lanes = lanes;
    // row tiles of ~rows_per_tile rows of mean length; staged capacity
    // covers the chunk plus the longest row plus alignment slack
    // measured on GB300 (256^3 stencil): one staged tile per block with
    // 512-row tiles beats deeper per-block pipelines, because more resident
    // blocks hide the x-gather latency better than prefetching does
    int rows_per_tile = 512;
    if (const char* e = getenv("GK_TILE_ROWS")) rows_per_tile = std::max(32, atoi(e));
    int32_t chunk = (int32_t)std::min<double>(
        8192.0, std::max<double>(512.0, rows_per_tile * std::ceil(std::max(mean, 1.0))));
    chunk = (chunk + 7) & ~7;
    const int64_t cap = (int64_t)chunk + A->max_row + 16;
    // warp tiles (kind 3): 32 * wt_rpl rows per warp, staged capacity of the
    // longest possible tile, one stage per warp by default (measured on
    // GB300, 3D 7-point 256^3 FP64: 1 stage 279 us, 2 stages 367 us, 3 644 us:
    // a smaller ring lets more warps reside, which hides the copy latency
    // better than prefetching within a warp); chosen for short rows of
    // near-uniform length when 8 warps' rings leave room for two blocks per SM
    const int64_t vb = (int64_t)value_bytes(A->dtype);
    int wt_rpl = 2;
    if (const char* e = getenv("GK_WT_RPL")) {
        const int v = atoi(e);
        wt_rpl = (v == 1 || v == 4) ? v : 2;
    }
    const int64_t wt_cap = ((int64_t)32 * wt_rpl * A->max_row + 14 + 7) & ~(int64_t)7;
    int wt_nst = 1;
    if (const char* e = getenv("GK_WT_STAGES")) wt_nst = std::max(1, std::min(4, atoi(e)));
    auto wt_block_bytes = [&](int nst) {
        return (int64_t)WT_WARPS * (((int64_t)nst * wt_cap * (4 + vb) + 8 * nst + 127) & ~(int64_t)127);
    };
    const bool wt_fits = wt_block_bytes(wt_nst) <= WT_SMEM_CAP;
    int kind = (A->max_row <= 1024) ? 1 : 2;
    if (wt_fits && wt_block_bytes(wt_nst) <= 112 * 1024 && A->max_row <= 2.0 * mean + 1.0)
        kind = 3;
    if (const char* force = getenv("GK_CSR_KERNEL")) kind = atoi(force);
    if (kind == 3 && !wt_fits) kind = 1;
    // a single staged tile must fit in shared memory
    if (kind == 1 && ((cap + 7) & ~7) * (int64_t)(4 + value_bytes(A->dtype)) > 200 * 1024) kind = 2;
    P.kind = kind;
    P.stages = 1;
    if (const char* e = getenv("GK_ROWTILE_STAGES")) P.stages = std::max(1, std::min(3, atoi(e)));
    if (kind == 3) {
        P.stages = wt_nst;
        P.wt_rpl = wt_rpl;
        P.tile_cap = (int32_t)wt_cap;
    } else if (kind == 1) {
        P.chunk = chunk;
        P.tile_cap = (int32_t)((cap + 7) & ~7);
        P.ntiles = (int32_t)std::max<int64_t>(1, (A->nnz + chunk - 1) / chunk);
        GK_CUDA(dmalloc_t(&P.tile_desc, (size_t)P.ntiles));
        k_tile_desc<<<grid_for(P.ntiles), 256, 0, s>>>(A->n, A->row_ptr, chunk, P.ntiles,
                                                       P.tile_desc);
        GK_CUDA(cudaGetLastError());
    } else if (kind == 2) {
        // Merge-path units: 32*E items per warp.  Default: operands in
        // registers (k_csr_merge_reg), E = 8 -- measured fastest on the 4M-row
        // Zipf(1.8) matrix (FP64 424 us; E = 4, 6, 12, 16 and the kernel that
        // stages operands in shared memory were slower).  GK_MERGE_E and
        // GK_MERGE_UNIT (reg | warp | block) select the other instances.
        int E = 8;
        if (const char* e = getenv("GK_MERGE_E")) E = atoi(e);
        if (E != 4 && E != 6 && E != 8) E = 8;
        P.merge_warp = 2;
        if (const char* w = getenv("GK_MERGE_UNIT"))
            P.merge_warp = !strcmp(w, "block") ? 0 : !strcmp(w, "warp") ? 1 : 2;
        P.merge_e = E;
        const int64_t items = (P.merge_warp ? 32 : 256) * (int64_t)E;  // path items per unit
        const int64_t N = (int64_t)A->n + A->nnz;
        P.merge_blocks = (int32_t)std::max<int64_t>(1, (N + items - 1) / items);
        GK_CUDA(dmalloc_t(&P.block_row, (size_t)P.merge_blocks + 1));
        k_merge_rows<<<grid_for(P.merge_blocks + 1), 256, 0, s>>>(A->n, A->nnz, A->row_ptr,
                                                                  (int32_t)items, P.merge_blocks,
                                                                  P.block_row);
        GK_CUDA(cudaGetLastError());
    }
    return GK_OK;
}

// Validates a CSR handle's arrays, computes max/mean row length and plans.
static gk_status finish_csr(gk_matrix A, cudaStream_t s) {
    DevBuf flags;
    GK_TRY(flags.ensure(16));
    unsigned int* derr = reinterpret_cast<unsigned int*>(flags.ptr);
    int32_t* dmax = reinterpret_cast<int32_t*>(derr + 1);
    GK_CUDA(cudaMemsetAsync(flags.ptr, 0, 16, s));
    if (A->n > 0)
        k_validate_rowptr<<<grid_for(A->n), 256, 0, s>>>(A->n, A->nnz, A->row_ptr, derr, dmax);
    if (A->nnz > 0)
        k_validate_cols<<<grid_for(A->nnz), 256, 0, s>>>(A->nnz, A->ncols, A->col, derr);
    GK_CUDA(cudaGetLastError());
    unsigned int h[2] = {0, 0};
    GK_CUDA(cudaMemcpyAsync(h, flags.ptr, 8, cudaMemcpyDeviceToHost, s));
    GK_CUDA(cudaStreamSynchronize(s));
    flags.release();
    if (h[0]) return GK_ERR_INVALID;
    A->max_row = (int32_t)h[1];
    A->mean_row = A->n ? (double)A->nnz / A->n : 0.0;
    GK_TRY(build_csr_plan(A, s));
    GK_CUDA(cudaStreamSynchronize(s));
    return GK_OK;
}

static gk_status copy_in(void* dst, const void* src, size_t bytes, gk_memory mem, cudaStream_t s) {
    if (bytes == 0) return GK_OK;
    if (!src) return GK_ERR_INVALID;
    GK_CUDA(cudaMemcpyAsync(dst, src, bytes,
                            mem == GK_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                            s));
    return GK_OK;
}

}  // namespace gk

using namespace gk;

extern "C" {

const char* gk_status_string(gk_status s) {
    switch (s) {
        case GK_OK: return "ok";
        case GK_NOT_CONVERGED: return "not converged: iteration cap reached";
        case GK_BREAKDOWN: return "breakdown of the Krylov recurrence";
        case GK_ERR_INVALID: return "invalid argument or malformed matrix";
        case GK_ERR_OOM: return "device memory allocation failed";
        case GK_ERR_CUDA: return "CUDA runtime error";
        case GK_ERR_TIMEOUT: return "device-side wait timed out";
        case GK_ERR_ZERO_DIAG: return "zero or missing diagonal entry (Jacobi)";
        case GK_ERR_NAN: return "NaN or Inf in a residual norm";
        case GK_ERR_UNSUPPORTED: return "unsupported combination";
    }
    return "unknown status";
}

int32_t gk_version(void) { return GK_VERSION; }

gk_status gk_matrix_create_csr(int32_t n, int32_t ncols, int64_t nnz, const int32_t* row_ptr,
                               const int32_t* col_idx, const void* values, gk_dtype dtype,
                               gk_memory mem, void* stream, gk_matrix* out) {
    if (!out) return GK_ERR_INVALID;
    *out = nullptr;
    if (n < 0 || ncols < 0 || nnz < 0 || nnz > INT32_MAX || !valid_dtype(dtype) || !row_ptr ||
        (mem != GK_MEM_HOST && mem != GK_MEM_DEVICE))
        return GK_ERR_INVALID;
    if (nnz > 0 && (!col_idx || !values)) return GK_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    gk_matrix A = new_handle();
    if (!A) return GK_ERR_OOM;
    A->n = n;
    A->ncols = ncols;
    A->nnz = nnz;
    A->fmt = GK_CSR;
    A->dtype = dtype;
    gk_status st = GK_OK;
    auto fail = [&](gk_status e) {
        destroy_handle(A);
        return e;
    };
    if (dmalloc_t(&A->row_ptr, (size_t)n + 1) != cudaSuccess ||
        dmalloc_t(&A->col, (size_t)std::max<int64_t>(nnz, 1)) != cudaSuccess ||
        dmalloc(&A->val, value_bytes(dtype) * (size_t)std::max<int64_t>(nnz, 1)) != cudaSuccess)
        return fail(GK_ERR_OOM);
    if ((st = copy_in(A->row_ptr, row_ptr, sizeof(int32_t) * ((size_t)n + 1), mem, s)) != GK_OK ||
        (st = copy_in(A->col, col_idx, sizeof(int32_t) * (size_t)nnz, mem, s)) != GK_OK ||
        (st = copy_in(A->val, values, value_bytes(dtype) * (size_t)nnz, mem, s)) != GK_OK)
        return fail(st);
    if ((st = finish_csr(A, s)) != GK_OK) return fail(st);
    *out = A;
    return GK_OK;
}

gk_status gk_matrix_create_coo(int32_t n, int32_t ncols, int64_t nnz, const int32_t* row,
                               const int32_t* col, const void* values, gk_dtype dtype,
                               gk_memory mem, void* stream, gk_matrix* out) {
    if (!out) return GK_ERR_INVALID;
    *out = nullptr;
    if (n < 0 || ncols < 0 || nnz < 0 || nnz > INT32_MAX || !valid_dtype(dtype) ||
        (mem != GK_MEM_HOST && mem != GK_MEM_DEVICE))
        return GK_ERR_INVALID;
    if (nnz > 0 && (!row || !col || !values)) return GK_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t vb = value_bytes(dtype);
    // device staging of the triplets
    DevBuf drow, dcol, dval, cnt, start, cursor, keys, ucnt, uoff, tmp, flags, scratch;
    auto cleanup = [&]() {
        drow.release(); dcol.release(); dval.release(); cnt.release(); start.release();
        cursor.release(); keys.release(); ucnt.release(); uoff.release(); tmp.release();
        flags.release(); scratch.release();
    };
    gk_matrix A = nullptr;
    auto fail = [&](gk_status e) {
        cleanup();
        destroy_handle(A);
        return e;
    };
    const size_t nz1 = (size_t)std::max<int64_t>(nnz, 1);
    if (drow.ensure(4 * nz1) || dcol.ensure(4 * nz1) || dval.ensure(vb * nz1) ||
        cnt.ensure(4 * ((size_t)n + 1)) || start.ensure(8 * ((size_t)n + 1)) ||
        cursor.ensure(4 * ((size_t)n + 1)) || keys.ensure(8 * nz1) ||
        ucnt.ensure(8 * ((size_t)n + 1)) || uoff.ensure(8 * ((size_t)n + 1)) || flags.ensure(16))
        return fail(GK_ERR_OOM);
    gk_status st;
    if ((st = copy_in(drow.ptr, row, 4 * (size_t)nnz, mem, s)) != GK_OK ||
        (st = copy_in(dcol.ptr, col, 4 * (size_t)nnz, mem, s)) != GK_OK ||
        (st = copy_in(dval.ptr, values, vb * (size_t)nnz, mem, s)) != GK_OK)
        return fail(st);
    unsigned int* derr = reinterpret_cast<unsigned int*>(flags.ptr);
    int32_t* dcnt = reinterpret_cast<int32_t*>(cnt.ptr);
    int64_t* dstart = reinterpret_cast<int64_t*>(start.ptr);
    int32_t* dcur = reinterpret_cast<int32_t*>(cursor.ptr);
    uint64_t* dkeys = reinterpret_cast<uint64_t*>(keys.ptr);
    if (cudaMemsetAsync(flags.ptr, 0, 16, s) || cudaMemsetAsync(dcnt, 0, 4 * ((size_t)n + 1), s) ||
        cudaMemsetAsync(dcur, 0, 4 * ((size_t)n + 1), s))
        return fail(GK_ERR_CUDA);
    if (nnz > 0)
        k_coo_count<<<grid_for(nnz), 256, 0, s>>>(nnz, n, ncols, (const int32_t*)drow.ptr,
                                                  (const int32_t*)dcol.ptr, dcnt, derr);
    unsigned int herr = 0;
    if ((st = read_err(derr, s, &herr)) != GK_OK) return fail(st);
    if (herr) return fail(GK_ERR_INVALID);
    if ((st = scan_exclusive<int32_t, int64_t>(dcnt, dstart, n, tmp, s)) != GK_OK) return fail(st);
    if (nnz > 0)
        k_coo_scatter<<<grid_for(nnz), 256, 0, s>>>(nnz, (const int32_t*)drow.ptr,
                                                    (const int32_t*)dcol.ptr, dstart, dcur, dkeys);
    // longest row, for choosing the sorters
    std::vector<int32_t> hcnt((size_t)n + 1, 0);
    if (n > 0 && cudaMemcpyAsync(hcnt.data(), dcnt, 4 * (size_t)n, cudaMemcpyDeviceToHost, s))
        return fail(GK_ERR_CUDA);
    if (cudaStreamSynchronize(s)) return fail(GK_ERR_CUDA);
    int64_t maxL = 0;
    for (int32_t i = 0; i < n; ++i) maxL = std::max<int64_t>(maxL, hcnt[i]);
    if (n > 0 && maxL > 1) {
        const unsigned gs = grid_for((int64_t)n * 8);
        k_sort_rows_sub<2><<<gs, 256, 0, s>>>(n, dstart, dkeys);
        if (maxL > 2) k_sort_rows_sub<4><<<gs, 256, 0, s>>>(n, dstart, dkeys);
        if (maxL > 4) k_sort_rows_sub<8><<<gs, 256, 0, s>>>(n, dstart, dkeys);
        if (maxL > 8) k_sort_rows_sub<16><<<gs, 256, 0, s>>>(n, dstart, dkeys);
        if (maxL > 16) k_sort_rows_sub<32><<<gs, 256, 0, s>>>(n, dstart, dkeys);
        if (maxL > 32) {
            const int cap = 16384;  // keys in shared memory (128 KB)
            cudaFuncSetAttribute(k_sort_rows_block, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 cap * 8);
            const int64_t hi = std::min<int64_t>(maxL, cap);
            int P = 1;
            while (P < hi) P <<= 1;
            k_sort_rows_block<<<(unsigned)std::min<int64_t>(n, num_sms() * 4), 512, (size_t)P * 8,
                                s>>>(n, dstart, dkeys, 32, cap, P);
            if (maxL > cap) {
                int64_t Q = 1;
                while (Q < maxL) Q <<= 1;
                const int nb = 4;
                if (scratch.ensure((size_t)nb * Q * 8)) return fail(GK_ERR_OOM);
                k_sort_rows_global<<<nb, 1024, 0, s>>>(n, dstart, dkeys, cap,
                                                       (uint64_t*)scratch.ptr, Q);
            }
        }
    }
    int64_t* ducnt = reinterpret_cast<int64_t*>(ucnt.ptr);
    int64_t* duoff = reinterpret_cast<int64_t*>(uoff.ptr);
    if (n > 0) k_count_unique<<<grid_for(n), 256, 0, s>>>(n, dstart, dkeys, ducnt);
    if ((st = scan_exclusive<int64_t, int64_t>(ducnt, duoff, n, tmp, s)) != GK_OK) return fail(st);
    int64_t nnz_out = 0;
    if (cudaMemcpyAsync(&nnz_out, duoff + n, 8, cudaMemcpyDeviceToHost, s) ||
        cudaStreamSynchronize(s))
        return fail(GK_ERR_CUDA);
    A = new_handle();
    if (!A) return fail(GK_ERR_OOM);
    A->n = n;
    A->ncols = ncols;
    A->nnz = nnz_out;
    A->fmt = GK_CSR;
    A->dtype = dtype;
    if (dmalloc_t(&A->row_ptr, (size_t)n + 1) || dmalloc_t(&A->col, (size_t)std::max<int64_t>(nnz_out, 1)) ||
        dmalloc(&A->val, vb * (size_t)std::max<int64_t>(nnz_out, 1)))
        return fail(GK_ERR_OOM);
    k_i64_to_i32<<<grid_for((int64_t)n + 1), 256, 0, s>>>((int64_t)n + 1, duoff, A->row_ptr, derr);
    if (n > 0) {
        st = dispatch_dtype(dtype, [&](auto tp) -> gk_status {
            using V = typename decltype(tp)::V;
            using Acc = typename AccOf<V>::type;
            k_merge_unique<V, V, Acc><<<grid_for(n), 256, 0, s>>>(
                n, dstart, dkeys, duoff, (const V*)dval.ptr, A->col, (V*)A->val);
            return GK_OK;
        });
        if (st != GK_OK) return fail(st);
    }
    if (cudaGetLastError()) return fail(GK_ERR_CUDA);
    if ((st = finish_csr(A, s)) != GK_OK) return fail(st);
    cleanup();
    *out = A;
    return GK_OK;
}

gk_status gk_matrix_convert(gk_matrix A, gk_format fmt, gk_dtype dtype, int32_t slice_size,
                            int32_t stride_factor, void* stream, gk_matrix* out) {
    if (!A || !out || !valid_dtype(dtype)) return GK_ERR_INVALID;
    if (fmt != GK_CSR && fmt != GK_ELL && fmt != GK_SELLP && fmt != GK_COO) return GK_ERR_INVALID;
    *out = nullptr;
    const bool to_coo = fmt == GK_COO;
    if (to_coo) fmt = GK_CSR;  // the COO handle is a CSR handle plus the row of every entry
    cudaStream_t s = (cudaStream_t)stream;
    const int32_t S = slice_size ? slice_size : 32;
    const int32_t f = stride_factor ? stride_factor : 1;
    if (fmt == GK_SELLP && (S < 1 || S > 1024 || f < 1)) return GK_ERR_INVALID;
    // Step 1: a CSR source in the source dtype (A itself, or rebuilt from padding).
    gk_matrix C = A;
    gk_matrix tmpC = nullptr;
    auto fail = [&](gk_status e) {
        destroy_handle(tmpC);
        return e;
    };
    if (A->fmt != GK_CSR) {
        tmpC = new_handle();
        if (!tmpC) return GK_ERR_OOM;
        tmpC->n = A->n;
        tmpC->ncols = A->ncols;
        tmpC->nnz = A->nnz;
        tmpC->dtype = A->dtype;
        DevBuf cnt, tmp;
        if (cnt.ensure(4 * ((size_t)A->n + 1)) || dmalloc_t(&tmpC->row_ptr, (size_t)A->n + 1) ||
            dmalloc_t(&tmpC->col, (size_t)std::max<int64_t>(A->nnz, 1)) ||
            dmalloc(&tmpC->val, value_bytes(A->dtype) * (size_t)std::max<int64_t>(A->nnz, 1)))
            return fail(GK_ERR_OOM);
        if (A->n > 0)
            k_padded_row_counts<<<grid_for(A->n), 256, 0, s>>>(A->n, A->fmt, A->stride, A->K, A->S,
                                                               A->slice_len, A->slice_set, A->col,
                                                               (int32_t*)cnt.ptr);
        gk_status st = scan_exclusive<int32_t, int32_t>((int32_t*)cnt.ptr, tmpC->row_ptr, A->n, tmp, s);
        if (st != GK_OK) return fail(st);
        if (A->n > 0) {
            st = dispatch_dtype(A->dtype, [&](auto tp) -> gk_status {
                using V = typename decltype(tp)::V;
                k_padded_to_csr<V, V><<<grid_for(A->n), 256, 0, s>>>(
                    A->n, A->fmt, A->stride, A->K, A->S, A->slice_len, A->slice_set, A->col,
                    (const V*)A->val, tmpC->row_ptr, tmpC->col, (V*)tmpC->val);
                return GK_OK;
            });
            if (st != GK_OK) return fail(st);
        }
        if (cudaStreamSynchronize(s)) return fail(GK_ERR_CUDA);
        cnt.release();
        tmp.release();
        tmpC->max_row = A->max_row;
        C = tmpC;
    }
    gk_matrix B = new_handle();
    if (!B) return fail(GK_ERR_OOM);
    auto failB = [&](gk_status e) {
        destroy_handle(B);
        return fail(e);
    };
    B->n = A->n;
    B->ncols = A->ncols;
    B->nnz = A->nnz;
    B->fmt = fmt;
    B->dtype = dtype;
    B->max_row = A->max_row;
    B->mean_row = A->n ? (double)A->nnz / A->n : 0.0;
    const int64_t n = A->n;
    gk_status st = GK_OK;
    auto run = [&](auto src_tp, auto dst_tp) -> gk_status {
        using VI = typename decltype(src_tp)::V;
        using VO = typename decltype(dst_tp)::V;
        if (fmt == GK_CSR) {
            B->stored = C->nnz;
            GK_CUDA(dmalloc_t(&B->row_ptr, (size_t)n + 1));
            GK_CUDA(dmalloc_t(&B->col, (size_t)std::max<int64_t>(C->nnz, 1)));
            GK_CUDA(dmalloc(&B->val, sizeof(VO) * (size_t)std::max<int64_t>(C->nnz, 1)));
            GK_CUDA(cudaMemcpyAsync(B->row_ptr, C->row_ptr, 4 * ((size_t)n + 1), cudaMemcpyDeviceToDevice, s));
            if (C->nnz) {
                GK_CUDA(cudaMemcpyAsync(B->col, C->col, 4 * (size_t)C->nnz, cudaMemcpyDeviceToDevice, s));
                k_convert_values<VI, VO><<<grid_for(C->nnz), 256, 0, s>>>(C->nnz, (const VI*)C->val,
                                                                         (VO*)B->val);
            }
        } else if (fmt == GK_ELL) {
            B->K = C->max_row;
            B->stride = ((n + 31) / 32) * 32;
            B->stored = (int64_t)B->K * B->stride;
            GK_CUDA(dmalloc_t(&B->col, (size_t)std::max<int64_t>(B->stored, 1)));
            GK_CUDA(dmalloc(&B->val, sizeof(VO) * (size_t)std::max<int64_t>(B->stored, 1)));
            if (B->stored)
                k_csr_to_ell<VI, VO><<<grid_for(B->stride), 256, 0, s>>>(
                    (int32_t)n, B->stride, B->K, C->row_ptr, C->col, (const VI*)C->val, B->col,
                    (VO*)B->val);
        } else {
            B->S = S;
            B->f = f;
            B->nslices = (int32_t)((n + S - 1) / S);
            GK_CUDA(dmalloc_t(&B->slice_len, (size_t)std::max(B->nslices, 1)));
            GK_CUDA(dmalloc_t(&B->slice_set, (size_t)B->nslices + 1));
            if (B->nslices)
                k_slice_lengths<<<grid_for(B->nslices), 256, 0, s>>>((int32_t)n, S, f, B->nslices,
                                                                    C->row_ptr, B->slice_len);
            DevBuf tmp;
            GK_TRY(scan_exclusive<int32_t, int64_t>(B->slice_len, B->slice_set, B->nslices, tmp, s));
            int64_t total = 0;
            GK_CUDA(cudaMemcpyAsync(&total, B->slice_set + B->nslices, 8, cudaMemcpyDeviceToHost, s));
            GK_CUDA(cudaStreamSynchronize(s));
            tmp.release();
            B->stored = total * S;
            GK_CUDA(dmalloc_t(&B->col, (size_t)std::max<int64_t>(B->stored, 1)));
            GK_CUDA(dmalloc(&B->val, sizeof(VO) * (size_t)std::max<int64_t>(B->stored, 1)));
            if (B->nslices)
                k_csr_to_sellp<VI, VO><<<grid_for((int64_t)B->nslices * S), 256, 0, s>>>(
                    (int32_t)n, S, B->nslices, C->row_ptr, C->col, (const VI*)C->val,
                    B->slice_len, B->slice_set, B->col, (VO*)B->val);
        }
        GK_CUDA(cudaGetLastError());
        return GK_OK;
    };
    st = dispatch_dtype(C->dtype, [&](auto src) {
        return dispatch_dtype(dtype, [&](auto dst) { return run(src, dst); });
    });
    if (st != GK_OK) return failB(st);
    if (fmt == GK_CSR && (st = build_csr_plan(B, s)) != GK_OK) return failB(st);
    if (to_coo && (st = build_coo_view(B, s)) != GK_OK) return failB(st);
    if (cudaStreamSynchronize(s)) return failB(GK_ERR_CUDA);
    destroy_handle(tmpC);
    *out = B;
    return GK_OK;
}

gk_status gk_matrix_describe(gk_matrix A, gk_matrix_desc* d) {
    if (!A || !d) return GK_ERR_INVALID;
    std::memset(d, 0, sizeof(*d));
    d->n = A->n;
    d->ncols = A->ncols;
    d->nnz = A->nnz;
    d->format = A->coo ? GK_COO : A->fmt;
    d->dtype = A->dtype;
    d->max_row = A->max_row;
    d->ell_width = A->K;
    d->ell_stride = A->stride;
    d->slice_size = A->S;
    d->stride_factor = A->f;
    d->num_slices = A->nslices;
    d->spmv_kernel = A->coo ? 5
                     : A->fmt == GK_CSR ? (A->plan.kind == 3 ? 6 : A->plan.kind)
                     : A->fmt == GK_ELL ? 3 : 4;
    if (A->plan.err) {
        int32_t e = 0;
        if (cudaMemcpy(&e, A->plan.err, 4, cudaMemcpyDeviceToHost) == cudaSuccess && e)
            d->device_error |= 1;
    }
    // the substitution kernels' sticky error words (TriStore::sync: four
    // words per direction, the third is the error flag)
    const gk::TriStore* tri[2] = {A->ilu, A->tri};
    for (int k = 0; k < 2; ++k) {
        if (!tri[k] || tri[k]->state != 1 || !tri[k]->sync) continue;
        uint32_t w[8] = {};
        if (cudaMemcpy(w, tri[k]->sync, sizeof(w), cudaMemcpyDeviceToHost) == cudaSuccess &&
            (w[2] | w[6]))
            d->device_error |= 2 << k;
    }
    d->spmv_launches = A->coo ? (A->n_empty ? 3 : 2)
                       : (A->fmt == GK_CSR && A->plan.kind == 2) ? 2 : 1;
    d->solve_format = A->fmt != GK_CSR ? (int32_t)A->fmt
                      : !A->solve_fmt_tuned ? -1
                      : A->solve_fmt ? (int32_t)A->solve_fmt->fmt : (int32_t)GK_CSR;
    const size_t vb = value_bytes(A->dtype);
    if (A->fmt == GK_CSR) {
        d->stored = A->nnz;
        d->device_bytes = (int64_t)(4 * ((size_t)A->n + 1) + (4 + vb) * (size_t)A->nnz);
        if (A->coo) d->device_bytes += (int64_t)(4 * (size_t)A->nnz + 4 * (size_t)A->n_empty);
    } else if (A->fmt == GK_ELL) {
        d->stored = A->stored;
        d->device_bytes = (int64_t)((4 + vb) * (size_t)A->stored);
    } else {
        d->stored = A->stored;
        d->device_bytes = (int64_t)((4 + vb) * (size_t)A->stored + 4 * (size_t)A->nslices +
                                    8 * ((size_t)A->nslices + 1));
    }
    return GK_OK;
}

gk_status gk_matrix_export(gk_matrix A, int32_t* idx_a, int64_t* sets, int32_t* col, void* values) {
    if (!A) return GK_ERR_INVALID;
    GateShared gate;
    GK_CUDA(cudaDeviceSynchronize());
    const size_t vb = value_bytes(A->dtype);
    if (A->coo) {
        if (idx_a && A->nnz) GK_CUDA(cudaMemcpy(idx_a, A->coo_row, 4 * (size_t)A->nnz, cudaMemcpyDeviceToHost));
        if (col && A->nnz) GK_CUDA(cudaMemcpy(col, A->col, 4 * (size_t)A->nnz, cudaMemcpyDeviceToHost));
        if (values && A->nnz) GK_CUDA(cudaMemcpy(values, A->val, vb * (size_t)A->nnz, cudaMemcpyDeviceToHost));
    } else if (A->fmt == GK_CSR) {
        if (idx_a) GK_CUDA(cudaMemcpy(idx_a, A->row_ptr, 4 * ((size_t)A->n + 1), cudaMemcpyDeviceToHost));
        if (col && A->nnz) GK_CUDA(cudaMemcpy(col, A->col, 4 * (size_t)A->nnz, cudaMemcpyDeviceToHost));
        if (values && A->nnz) GK_CUDA(cudaMemcpy(values, A->val, vb * (size_t)A->nnz, cudaMemcpyDeviceToHost));
    } else {
        if (A->fmt == GK_SELLP) {
            if (idx_a && A->nslices)
                GK_CUDA(cudaMemcpy(idx_a, A->slice_len, 4 * (size_t)A->nslices, cudaMemcpyDeviceToHost));
            if (sets) GK_CUDA(cudaMemcpy(sets, A->slice_set, 8 * ((size_t)A->nslices + 1), cudaMemcpyDeviceToHost));
        }
        if (col && A->stored) GK_CUDA(cudaMemcpy(col, A->col, 4 * (size_t)A->stored, cudaMemcpyDeviceToHost));
        if (values && A->stored)
            GK_CUDA(cudaMemcpy(values, A->val, vb * (size_t)A->stored, cudaMemcpyDeviceToHost));
    }
    return GK_OK;
}

gk_status gk_matrix_destroy(gk_matrix A) {
    if (!A) return GK_ERR_INVALID;
    GateShared gate;  // streams, graphs, events and memory go: no capture meanwhile
    cudaDeviceSynchronize();
    destroy_handle(A);
    return GK_OK;
}

}  // extern "C"
