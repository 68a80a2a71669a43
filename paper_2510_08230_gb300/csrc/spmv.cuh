// spmv.cuh - SpMV kernels (CSR row-tile, CSR merge-path, CSR vector, ELL,
// SELL-P) with fused epilogues.
//
// A matrix LinOp's apply is an SpMV (Section 3.4); the advanced form adds
// alpha and beta.  Every kernel produces, for each row i, the sum
// s_i = sum_j a_ij b_j and passes (i, s_i) to an epilogue, which writes the
// output and may accumulate per-thread partial dot products; the kernel's
// last act is epi.finish(acc), which reduces those partials across the grid
// deterministically (fixed order, last block finishes).
//
// FP64 note for GB300: the FP64 pipe runs about 2 lane-FMAs per SM cycle,
// close to the rate at which HBM delivers FP64 nonzeros (12 B each).  The
// kernels therefore spend exactly one FMA per stored nonzero and reduce a
// row sum within one thread (row-tile, ELL, SELL-P) or with carries between
// threads (merge-path); no FP64 shuffle trees on the per-row path.
#pragma once

#include "prims.cuh"

namespace gk {

// ------------------------------------------------------------ epilogues

// x_i = s (mode 0), alpha s (mode 1) or alpha s + beta x_i (mode 2).
template <typename T>
struct EpiStore {
    T* __restrict__ y;
    T alpha, beta;
    int mode;
    static constexpr int NA = 0;
    __device__ __forceinline__ bool skip() const { return false; }
    __device__ __forceinline__ void row(int64_t i, T s, double*) const {
        if (mode == 0) y[i] = s;
        else if (mode == 1) y[i] = alpha * s;
        else y[i] = fmadd(beta, y[i], alpha * s);
    }
    __device__ __forceinline__ void finish(double*) const {}
};

template <class Epi>
struct AccArr {
    double v[Epi::NA > 0 ? Epi::NA : 1];
};

// ------------------------------------------------------------ kernels

// CSR row-tile kernel.  Tile c = rows [tile_row[c], tile_row[c+1]) whose
// nonzeros fit in `cap` entries.  The block copies the tile's col/val
// range into shared memory with 16-byte streaming loads (range rounded out
// to 8-entry alignment; allocations carry 64 bytes of slack), then one
// thread per row accumulates its row sequentially from shared memory.
template <typename V, typename T, class Epi>
__global__ void __launch_bounds__(256)
k_csr_rowtile(int32_t ntiles, const int32_t* __restrict__ tile_row,
              const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
              const V* __restrict__ va, const T* __restrict__ x, int32_t cap, Epi epi) {
    extern __shared__ __align__(16) unsigned char smem[];
    int32_t* s_col = reinterpret_cast<int32_t*>(smem);
    V* s_val = reinterpret_cast<V*>(smem + (size_t)cap * 4);
    if (epi.skip()) return;
    AccArr<Epi> acc{};
    for (int32_t c = blockIdx.x; c < ntiles; c += gridDim.x) {
        const int32_t r0 = __ldg(tile_row + c), r1 = __ldg(tile_row + c + 1);
        if (r0 >= r1) continue;  // uniform over the block
        const int32_t e0 = __ldg(rp + r0), e1 = __ldg(rp + r1);
        const int32_t a0 = e0 & ~7;
        const int32_t cnt = ((e1 + 7) & ~7) - a0;
        {
            const int4* gc = reinterpret_cast<const int4*>(ci + a0);
            int4* sc = reinterpret_cast<int4*>(s_col);
            for (int k = threadIdx.x; k < (cnt >> 2); k += blockDim.x) sc[k] = __ldcs(gc + k);
            const int nv = (int)((cnt * sizeof(V)) >> 4);
            const int4* gv = reinterpret_cast<const int4*>(va + a0);
            int4* sv = reinterpret_cast<int4*>(s_val);
            for (int k = threadIdx.x; k < nv; k += blockDim.x) sv[k] = __ldcs(gv + k);
        }
        __syncthreads();
        for (int32_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
            const int32_t ks = __ldg(rp + r) - a0, ke = __ldg(rp + r + 1) - a0;
            T s = T(0);
            for (int32_t k = ks; k < ke; ++k)
                s = fmadd(cvt<T>(s_val[k]), __ldg(x + s_col[k]), s);
            epi.row(r, s, acc.v);
        }
        __syncthreads();
    }
    epi.finish(acc.v);
}

// CSR merge-path kernel (apply only).  The path of n row ends and nnz
// nonzeros is cut into equal pieces of 256*E items per block and E items
// per thread; each thread walks its piece sequentially (one FMA per
// nonzero).  A row whose end lies in a thread's piece is finished there,
// adding the carries of earlier threads of the block whose pieces ended
// inside the same row.  The row open at the end of a block is handed to
// k_csr_merge_fixup as (carry_row, carry_val).
template <int E, typename V, typename T>
__global__ void __launch_bounds__(256)
k_csr_merge(int32_t n, int64_t nnz, const int32_t* __restrict__ rp,
            const int32_t* __restrict__ ci, const V* __restrict__ va,
            const T* __restrict__ x, EpiStore<T> epi, int32_t* __restrict__ carry_row,
            T* __restrict__ carry_val) {
    constexpr int TI = 256 * E;
    __shared__ int32_t s_rowend[TI + 1];
    __shared__ int32_t s_col[TI];
    __shared__ V s_val[TI];
    __shared__ int32_t s_trow[256];
    __shared__ T s_tcarry[256];
    __shared__ int32_t s_bounds[2];
    const int64_t N = (int64_t)n + nnz;
    const int64_t d0 = (int64_t)blockIdx.x * TI;
    const int64_t d1 = min(d0 + TI, N);
    if (threadIdx.x < 2) {
        const int64_t d = threadIdx.x == 0 ? d0 : d1;
        int32_t lo = 0, hi = n;  // rows whose end item lies before d
        while (lo < hi) {
            const int32_t mid = lo + ((hi - lo) >> 1);
            if ((int64_t)__ldg(rp + mid + 1) + mid + 1 > d) hi = mid;
            else lo = mid + 1;
        }
        s_bounds[threadIdx.x] = lo;
    }
    __syncthreads();
    const int32_t i0 = s_bounds[0], i1 = s_bounds[1];
    const int64_t j0 = d0 - i0, j1 = d1 - i1;
    const int32_t nloc = min(i1 - i0 + 1, n - i0);  // staged row ends
    for (int k = threadIdx.x; k < nloc; k += blockDim.x) s_rowend[k] = __ldg(rp + i0 + k + 1);
    for (int k = threadIdx.x; k < (int)(j1 - j0); k += blockDim.x) {
        s_col[k] = __ldcs(ci + j0 + k);
        s_val[k] = va[j0 + k];
    }
    __syncthreads();
    // this thread's start on the path
    const int64_t dt = min(d0 + (int64_t)threadIdx.x * E, d1);
    int32_t lo = 0, hi = max(0, nloc);
    while (lo < hi) {
        const int32_t mid = (lo + hi) >> 1;
        if ((int64_t)s_rowend[mid] + i0 + mid + 1 > dt) hi = mid;
        else lo = mid + 1;
    }
    int32_t i = i0 + lo;
    int64_t j = dt - i;
    const int64_t dend = min(dt + E, d1);
    T acc = T(0);
    int32_t head_row = -1;
    T head_val = T(0);
    int64_t rend = (i < n) ? (int64_t)s_rowend[i - i0] : 0;
    for (int64_t d = dt; d < dend; ++d) {
        if (i < n && j < rend) {
            acc = fmadd(cvt<T>(s_val[j - j0]), __ldg(x + s_col[j - j0]), acc);
            ++j;
        } else {
            if (head_row < 0) {
                head_row = i;
                head_val = acc;
            } else {
                epi.row(i, acc, nullptr);
            }
            acc = T(0);
            ++i;
            rend = (i < n && i - i0 < nloc) ? (int64_t)s_rowend[i - i0] : 0;
        }
    }
    s_trow[threadIdx.x] = (dt < d1) ? i : -1;
    s_tcarry[threadIdx.x] = acc;
    __syncthreads();
    if (head_row >= 0) {
        T v = head_val;
        for (int t = (int)threadIdx.x - 1; t >= 0 && s_trow[t] == head_row; --t) v = s_tcarry[t] + v;
        epi.row(head_row, v, nullptr);
    }
    if (threadIdx.x == blockDim.x - 1) {
        // open row at the end of the block: sum the trailing carries
        int t = (int)blockDim.x - 1;
        while (t >= 0 && s_trow[t] < 0) --t;
        int32_t r = t >= 0 ? s_trow[t] : -1;
        T v = T(0);
        for (; t >= 0 && s_trow[t] == r; --t) v = s_tcarry[t] + v;
        carry_row[blockIdx.x] = (r >= 0 && r < n) ? r : -1;
        carry_val[blockIdx.x] = v;
    }
}

// Adds the block carries to the rows they belong to: the first block of
// every run of blocks sharing a carry row sums the run in block order.
template <typename T>
__global__ void k_csr_merge_fixup(int32_t nblocks, const int32_t* __restrict__ carry_row,
                                  const T* __restrict__ carry_val, T* __restrict__ y, T alpha,
                                  int mode) {
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nblocks;
         b += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = carry_row[b];
        if (r < 0 || (b > 0 && carry_row[b - 1] == r)) continue;
        T v = carry_val[b];
        for (int64_t c = b + 1; c < nblocks && carry_row[c] == r; ++c) v = v + carry_val[c];
        y[r] = mode == 0 ? y[r] + v : fmadd(alpha, v, y[r]);
    }
}

// CSR vector kernel: G lanes per row (warp = 32/G rows per step), lane
// partial sums combined with shuffles.
template <int G, typename V, typename T, class Epi>
__global__ void __launch_bounds__(256)
k_csr_vector(int32_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
             const V* __restrict__ va, const T* __restrict__ x, Epi epi) {
    if (epi.skip()) return;
    AccArr<Epi> acc{};
    constexpr int RPW = 32 / G;
    const int lane = threadIdx.x & 31;
    const int sub = lane / G, gl = lane & (G - 1);
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = warp * RPW; base < n; base += nwarp * RPW) {
        const int64_t r = base + sub;
        T s = T(0);
        if (r < n) {
            const int32_t a = __ldg(rp + r), b = __ldg(rp + r + 1);
            for (int32_t k = a + gl; k < b; k += G) s = fmadd(ld_stream(va + k), __ldg(x + ld_stream(ci + k)), s);
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, G);
        if (gl == 0 && r < n) epi.row(r, s, acc.v);
    }
    epi.finish(acc.v);
}

// ELL: one thread per row, column-major coalesced loads; padding skipped.
template <typename V, typename T, class Epi>
__global__ void __launch_bounds__(256)
k_ell(int32_t n, int64_t stride, int32_t K, const int32_t* __restrict__ ec,
      const V* __restrict__ ev, const T* __restrict__ x, Epi epi) {
    if (epi.skip()) return;
    AccArr<Epi> acc{};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        T s = T(0);
        const int32_t* cp = ec + i;
        const V* vp = ev + i;
#pragma unroll 4
        for (int32_t j = 0; j < K; ++j) {
            const int32_t c = ld_stream(cp + (int64_t)j * stride);
            const T v = ld_stream(vp + (int64_t)j * stride);
            if (c >= 0) s = fmadd(v, __ldg(x + c), s);
        }
        epi.row(i, s, acc.v);
    }
    epi.finish(acc.v);
}

// SELL-P: one thread per row; the rows of a slice read consecutive
// addresses for every stored column position.
template <typename V, typename T, class Epi>
__global__ void __launch_bounds__(256)
k_sellp(int32_t n, int32_t S, const int32_t* __restrict__ slen, const int64_t* __restrict__ sset,
        const int32_t* __restrict__ sc, const V* __restrict__ sv, const T* __restrict__ x, Epi epi) {
    if (epi.skip()) return;
    AccArr<Epi> acc{};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t sl = i / S, t = i - sl * S;
        const int32_t len = __ldg(slen + sl);
        const int64_t base = __ldg(sset + sl) * S + t;
        T s = T(0);
#pragma unroll 4
        for (int32_t j = 0; j < len; ++j) {
            const int32_t c = ld_stream(sc + base + (int64_t)j * S);
            const T v = ld_stream(sv + base + (int64_t)j * S);
            if (c >= 0) s = fmadd(v, __ldg(x + c), s);
        }
        epi.row(i, s, acc.v);
    }
    epi.finish(acc.v);
}

// ------------------------------------------------------------ launcher

template <typename K>
static int occupancy_blocks(K kernel, int threads, size_t smem) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, threads, smem) != cudaSuccess || b < 1)
        b = 1;
    return b;
}

// Grid of a kernel family for matrix A: deterministic for a given matrix
// and device, so that the partial-sum layout of fused reductions is fixed.
struct Launch {
    unsigned grid = 1;
    size_t smem = 0;
};

// Launches the row-complete SpMV of A (row-tile / vector CSR, ELL, SELL-P)
// with epilogue epi.  For epilogues with NA > 0, the caller provides
// partials (NA * max_grid doubles) and a zeroed ticket through epi.
template <typename V, typename T, class Epi>
gk_status launch_spmv_rows(gk_matrix A, const T* x, const Epi& epi, cudaStream_t s,
                           unsigned* grid_out = nullptr) {
    const int sms = num_sms();
    unsigned grid = 1;
    if (A->fmt == GK_CSR && A->plan.kind == 1) {
        const size_t smem = (size_t)A->plan.tile_cap * (4 + sizeof(V));
        auto k = k_csr_rowtile<V, T, Epi>;
        static thread_local int occ_cache = 0;
        static thread_local size_t occ_smem = 0;
        if (occ_smem != smem || !occ_cache) {
            if (smem > 48 * 1024)
                cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
            occ_cache = occupancy_blocks(k, 256, smem);
            occ_smem = smem;
        }
        grid = (unsigned)std::min<int64_t>(A->plan.ntiles, (int64_t)sms * occ_cache);
        if (grid < 1) grid = 1;
        k<<<grid, 256, smem, s>>>(A->plan.ntiles, A->plan.tile_row, A->row_ptr, A->col,
                                  (const V*)A->val, x, A->plan.tile_cap, epi);
    } else if (A->fmt == GK_CSR) {
        const int G = A->plan.lanes;
        const int64_t rows_per_block = 256 / G;
        int64_t need = (A->n + rows_per_block - 1) / rows_per_block;
        grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)sms * 8));
        const int32_t n = A->n;
        const V* va = (const V*)A->val;
        switch (G) {
            case 1: k_csr_vector<1, V, T, Epi><<<grid, 256, 0, s>>>(n, A->row_ptr, A->col, va, x, epi); break;
            case 2: k_csr_vector<2, V, T, Epi><<<grid, 256, 0, s>>>(n, A->row_ptr, A->col, va, x, epi); break;
            case 4: k_csr_vector<4, V, T, Epi><<<grid, 256, 0, s>>>(n, A->row_ptr, A->col, va, x, epi); break;
            case 8: k_csr_vector<8, V, T, Epi><<<grid, 256, 0, s>>>(n, A->row_ptr, A->col, va, x, epi); break;
            case 16: k_csr_vector<16, V, T, Epi><<<grid, 256, 0, s>>>(n, A->row_ptr, A->col, va, x, epi); break;
            default: k_csr_vector<32, V, T, Epi><<<grid, 256, 0, s>>>(n, A->row_ptr, A->col, va, x, epi); break;
        }
    } else if (A->fmt == GK_ELL) {
        int64_t need = (A->n + 255) / 256;
        grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)sms * 8));
        k_ell<V, T, Epi><<<grid, 256, 0, s>>>(A->n, A->stride, A->K, A->col, (const V*)A->val, x, epi);
    } else {
        int64_t need = (A->n + 255) / 256;
        grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)sms * 8));
        k_sellp<V, T, Epi><<<grid, 256, 0, s>>>(A->n, A->S, A->slice_len, A->slice_set, A->col,
                                                (const V*)A->val, x, epi);
    }
    if (grid_out) *grid_out = grid;
    GK_CUDA(cudaGetLastError());
    return GK_OK;
}

// Upper bound of the grid launch_spmv_rows uses for A (sizes partials).
inline unsigned max_grid_rows(gk_matrix A) { return (unsigned)num_sms() * 8; }

}  // namespace gk
