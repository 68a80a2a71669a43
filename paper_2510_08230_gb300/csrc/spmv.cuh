// spmv.cuh - SpMV kernels (CSR row-tile, CSR merge-path, CSR vector, ELL,
// SELL-P) with fused epilogues.
//
// A matrix LinOp's apply is an SpMV (Section 4.2); the advanced form adds
// alpha and beta.  Every kernel produces, for each row i, the sum
// s_i = sum_j a_ij b_j and passes (i, s_i) to an epilogue, which writes the
// output and may accumulate per-thread partial dot products; the kernel's
// last act is epi.finish(acc), which reduces those partials across the grid
// deterministically (fixed order, last block finishes).  A thread keeps its
// partials in the vector type (FP32 in FP32 solves, so no FP64 instruction
// sits on their per-row path) and the grid reduction adds them in FP64.
//
// FP64 note for GB300: the FP64 pipe retires about 2 lane-FMAs per SM cycle
// (a warp instruction occupies it ~16 SM cycles whatever its active mask),
// close to the rate at which HBM delivers FP64 nonzeros (12 B each).  The
// kernels therefore spend one FMA per stored nonzero, keep warps converged
// in the FMA loops, and reduce a row within one thread (row-tile, ELL,
// SELL-P) or with carries between threads (merge-path); no FP64 shuffle
// trees on the per-row path.  Loads that feed the FMAs are issued in
// batches of 8 before the first FMA so that their latencies overlap.
#pragma once

#include "prims.cuh"
#include "tma.cuh"

namespace gk {

// ------------------------------------------------------------ epilogues

// x_i = s (mode 0), alpha s (mode 1) or alpha s + beta x_i (mode 2).
template <typename T>
struct EpiStore {
    T* __restrict__ y;
    T alpha, beta;
    int mode;
    static constexpr int NA = 0;
    using acc_t = T;
    __device__ __forceinline__ bool skip() const { return false; }
    __device__ __forceinline__ void row(int64_t i, T s, T*) const {
        if (mode == 0) y[i] = s;
        else if (mode == 1) y[i] = alpha * s;
        else y[i] = fmadd(beta, y[i], alpha * s);
    }
    __device__ __forceinline__ void finish(T*) const {}
    __device__ __forceinline__ void timed_out() const {}
};

template <class Epi>
struct AccArr {
    typename Epi::acc_t v[Epi::NA > 0 ? Epi::NA : 1];
};

constexpr int GATHER = 8;  // loads issued ahead of the FMAs that use them

// sum_{k in [ks, ke)} val[k] * x[col[k]] with values/columns in shared memory
template <typename T, typename V>
__device__ __forceinline__ T row_sum_staged(const int32_t* s_col, const V* s_val,
                                            const T* __restrict__ x, int32_t ks, int32_t ke) {
    T s = T(0);
    for (int32_t k0 = ks; k0 < ke; k0 += GATHER) {
        const int32_t m = min(GATHER, ke - k0);
        T vv[GATHER], xv[GATHER];
#pragma unroll
        for (int u = 0; u < GATHER; ++u) {
            if (u < m) {
                vv[u] = cvt<T>(s_val[k0 + u]);
                xv[u] = __ldg(x + s_col[k0 + u]);
            }
        }
#pragma unroll
        for (int u = 0; u < GATHER; ++u) {
            if (u >= m) break;
            s = fmadd(vv[u], xv[u], s);
        }
    }
    return s;
}

// Two rows [ks0, ke0) and [ks1, ke1) of a staged tile at once: the loads
// and gathers of both rows are issued before either FMA chain.
template <typename T, typename V>
__device__ __forceinline__ void row_pair_staged(const int32_t* s_col, const V* s_val,
                                                const T* __restrict__ x, int32_t ks0, int32_t ke0,
                                                int32_t ks1, int32_t ke1, T& s0, T& s1) {
    constexpr int B = 4;
    s0 = T(0);
    s1 = T(0);
    const int32_t l0 = ke0 - ks0, l1 = ke1 - ks1;
    const int32_t lmax = max(l0, l1);
    for (int32_t k0 = 0; k0 < lmax; k0 += B) {
        T v0[B], x0[B], v1[B], x1[B];
#pragma unroll
        for (int u = 0; u < B; ++u) {
            if (k0 + u < l0) {
                v0[u] = cvt<T>(s_val[ks0 + k0 + u]);
                x0[u] = __ldg(x + s_col[ks0 + k0 + u]);
            }
            if (k0 + u < l1) {
                v1[u] = cvt<T>(s_val[ks1 + k0 + u]);
                x1[u] = __ldg(x + s_col[ks1 + k0 + u]);
            }
        }
#pragma unroll
        for (int u = 0; u < B; ++u) {
            if (k0 + u < l0) s0 = fmadd(v0[u], x0[u], s0);
            if (k0 + u < l1) s1 = fmadd(v1[u], x1[u], s1);
        }
    }
}

// ------------------------------------------------------------ row-tile CSR

// Tile descriptor: rows [x, y), staged nonzero range [z, z + w) with z a
// multiple of 8 and w a multiple of 8 (16-byte aligned bulk copies).
//
// Persistent blocks take tiles c = blockIdx.x + k * gridDim.x.  Thread 0
// keeps NST (1..3) tiles in flight: for each it issues two cp.async.bulk copies
// (columns, values) into a shared-memory stage and arms the stage's
// mbarrier with the byte count.  All threads wait on the barrier (bounded),
// then one thread per row runs its row from shared memory; after a block
// barrier the stage is refilled with the tile NST steps ahead.
template <typename V, typename T, class Epi>
__global__ void __launch_bounds__(256)
k_csr_rowtile(int32_t ntiles, const int4* __restrict__ tdesc, const int32_t* __restrict__ rp,
              const int32_t* __restrict__ ci, const V* __restrict__ va,
              const T* __restrict__ x, int32_t cap, int NST, Epi epi, int32_t* __restrict__ err,
              uint64_t wait_ns) {
    extern __shared__ __align__(128) unsigned char smem[];
    const uint32_t cbytes = (uint32_t)cap * 4u;
    const uint32_t sbytes = (uint32_t)cap * (4u + (uint32_t)sizeof(V));
    if (epi.skip()) return;
    AccArr<Epi> acc{};
    const uint32_t bar0 = smem_addr(smem + (size_t)NST * sbytes);
    const uint32_t buf0 = smem_addr(smem);
    if (threadIdx.x == 0) {
        for (int s = 0; s < NST; ++s) mbar_init(bar0 + 8u * s, 1u);
        fence_mbar_init();
    }
    __syncthreads();
    const int32_t stride = (int32_t)gridDim.x;
    auto issue = [&](int32_t c, int s) {
        const int4 d = __ldg(tdesc + c);
        const uint32_t nc = (uint32_t)d.w * 4u, nv = (uint32_t)d.w * (uint32_t)sizeof(V);
        const uint32_t bar = bar0 + 8u * s;
        mbar_arrive_expect_tx(bar, nc + nv);
        if (d.w > 0) {
            bulk_g2s(buf0 + s * sbytes, ci + d.z, nc, bar);
            bulk_g2s(buf0 + s * sbytes + cbytes, va + d.z, nv, bar);
        }
    };
    if (threadIdx.x == 0)
        for (int s = 0; s < NST; ++s) {
            const int32_t c = (int32_t)blockIdx.x + s * stride;
            if (c < ntiles) issue(c, s);
        }
    int it = 0;
    bool timed_out = false;
    for (int32_t c = blockIdx.x; c < ntiles; c += stride, ++it) {
        const int s = it % NST;
        const bool ok = mbar_wait_bounded(bar0 + 8u * s, (uint32_t)(it / NST) & 1u, wait_ns);
        if (__syncthreads_or(!ok)) {
            timed_out = true;
            break;
        }
        const int4 d = __ldg(tdesc + c);
        const int32_t* s_col = reinterpret_cast<const int32_t*>(smem + (size_t)s * sbytes);
        const V* s_val = reinterpret_cast<const V*>(smem + (size_t)s * sbytes + cbytes);
        // two rows per thread per pass (r and r + blockDim), interleaved
        for (int32_t r = d.x + (int32_t)threadIdx.x; r < d.y; r += 2 * (int32_t)blockDim.x) {
            const int32_t r2 = r + (int32_t)blockDim.x;
            const bool has2 = r2 < d.y;
            const int32_t ks = __ldg(rp + r) - d.z, ke = __ldg(rp + r + 1) - d.z;
            const int32_t ks2 = has2 ? __ldg(rp + r2) - d.z : 0;
            const int32_t ke2 = has2 ? __ldg(rp + r2 + 1) - d.z : 0;
            T s0, s1;
            row_pair_staged<T, V>(s_col, s_val, x, ks, ke, ks2, ke2, s0, s1);
            epi.row(r, s0, acc.v);
            if (has2) epi.row(r2, s1, acc.v);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            const int32_t cn = c + NST * stride;
            if (cn < ntiles) {
                fence_proxy_async_smem();
                issue(cn, s);
            }
        }
    }
    if (timed_out) {
        if (threadIdx.x == 0) atomicExch(err, 1);
        epi.timed_out();
        // let the copies already issued land before the block exits (bounded
        // by the default limit, not the caller's budget: the shared memory
        // they write must outlive them)
        for (int k = 0; k < NST; ++k) {
            const int32_t c = (int32_t)blockIdx.x + (it + k) * stride;
            if (c >= ntiles) break;
            mbar_wait_bounded(bar0 + 8u * ((it + k) % NST), (uint32_t)((it + k) / NST) & 1u);
        }
    }
    epi.finish(acc.v);
}

// ------------------------------------------------------------ warp-tile CSR

// Tiles of 32 * RPL consecutive rows, one warp each, for short rows of
// near-uniform length (stencils, diffusion operators).  A warp owns a ring
// of NST shared-memory stages with one mbarrier each; lane 0 stages a tile's
// column and value range there with two bulk copies (the range rounded out
// to 8 entries: 16-byte aligned sources, sizes and destinations), NST - 1
// tiles ahead of the one the warp computes.  Lane l runs rows r0 + l,
// r0 + l + 32, ... of the tile from shared memory (two rows' loads issued
// before either FMA chain).  The warps of a block never wait for one another
// on the streaming path: a stage is refilled as soon as its own warp has
// read it.  Tile t holds rows [t * 32 RPL, (t + 1) * 32 RPL); warp g of the
// grid takes tiles g, g + W, g + 2W, ... (W warps in all).  With NST = 1 the
// warp waits for each tile's copy: the other resident warps cover the
// latency (measured fastest on the 3D stencils, where the small ring allows
// more resident warps).  Every wait is bounded by wait_ns; a warp whose
// wait runs out sets *err, lets its copies in flight land (default limit)
// and stops; the other warps finish, and the epilogue's reductions still run.
template <typename V>
__host__ __device__ constexpr uint32_t wt_stage_bytes(int32_t cap) {
    return (uint32_t)cap * (4u + (uint32_t)sizeof(V));
}
// one warp's ring: NST stages, then NST mbarriers; 128-byte multiple
template <typename V>
__host__ __device__ constexpr uint32_t wt_warp_bytes(int32_t cap, int nst) {
    return ((uint32_t)nst * wt_stage_bytes<V>(cap) + 8u * (uint32_t)nst + 127u) & ~127u;
}

template <int RPL, typename V, typename T, class Epi>
__global__ void __launch_bounds__(WT_WARPS * 32)
k_csr_warptile(int32_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
               const V* __restrict__ va, const T* __restrict__ x, int32_t cap, int NST, Epi epi,
               int32_t* __restrict__ err, uint64_t wait_ns) {
    extern __shared__ __align__(128) unsigned char smem[];
    constexpr unsigned FULL = 0xffffffffu;
    constexpr int ROWS = 32 * RPL;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint32_t cbytes = (uint32_t)cap * 4u;
    const uint32_t sbytes = wt_stage_bytes<V>(cap);
    unsigned char* ring = smem + (size_t)wid * wt_warp_bytes<V>(cap, NST);
    const uint32_t buf0 = smem_addr(ring);
    const uint32_t bar0 = smem_addr(ring + (size_t)NST * sbytes);
    AccArr<Epi> acc{};
    if (epi.skip()) return;
    const int32_t ntiles = (n + ROWS - 1) / ROWS;
    const int32_t W = (int32_t)gridDim.x * WT_WARPS;
    const int32_t g = (int32_t)blockIdx.x * WT_WARPS + wid;
    if (lane == 0) {
        for (int s = 0; s < NST; ++s) mbar_init(bar0 + 8u * s, 1u);
        fence_mbar_init();
    }
    __syncwarp();
    auto issue = [&](int32_t t, int s) {  // lane 0 only
        const int32_t r0 = t * ROWS, r1 = min(r0 + ROWS, n);
        const int32_t e0 = __ldg(rp + r0), e1 = __ldg(rp + r1);
        const int32_t a0 = e0 & ~7;
        const int32_t w = e1 > e0 ? ((e1 + 7) & ~7) - a0 : 0;
        const uint32_t bar = bar0 + 8u * s;
        mbar_arrive_expect_tx(bar, (uint32_t)w * (4u + (uint32_t)sizeof(V)));
        if (w > 0) {
            bulk_g2s(buf0 + s * sbytes, ci + a0, (uint32_t)w * 4u, bar);
            bulk_g2s(buf0 + s * sbytes + cbytes, va + a0, (uint32_t)w * (uint32_t)sizeof(V), bar);
        }
    };
    if (lane == 0)
        for (int s = 0; s < NST; ++s) {
            const int32_t t = g + s * W;
            if (t < ntiles) issue(t, s);
        }
    int it = 0;
    bool timed_out = false;
    for (int32_t t = g; t < ntiles; t += W, ++it) {
        const int s = it % NST;
        const int32_t r0 = t * ROWS;
        // row bounds first: their loads overlap the wait for the tile
        int32_t ks[RPL], ke[RPL];
        const int32_t a0 = __ldg(rp + r0) & ~7;
#pragma unroll
        for (int q = 0; q < RPL; ++q) {
            const int32_t r = r0 + lane + 32 * q;
            ks[q] = r < n ? __ldg(rp + r) - a0 : 0;
            ke[q] = r < n ? __ldg(rp + r + 1) - a0 : 0;
        }
        const bool ok = mbar_wait_bounded(bar0 + 8u * s, (uint32_t)(it / NST) & 1u, wait_ns);
        if (!__all_sync(FULL, ok)) {
            timed_out = true;
            break;
        }
        const int32_t* s_col = reinterpret_cast<const int32_t*>(ring + (size_t)s * sbytes);
        const V* s_val = reinterpret_cast<const V*>(ring + (size_t)s * sbytes + cbytes);
        if constexpr (RPL == 1) {
            const T sa = row_sum_staged<T, V>(s_col, s_val, x, ks[0], ke[0]);
            if (r0 + lane < n) epi.row(r0 + lane, sa, acc.v);
        } else {
#pragma unroll
            for (int q = 0; q < RPL; q += 2) {
                T sa, sb;
                row_pair_staged<T, V>(s_col, s_val, x, ks[q], ke[q], ks[q + 1], ke[q + 1], sa, sb);
                const int32_t ra = r0 + lane + 32 * q, rb = ra + 32;
                if (ra < n) epi.row(ra, sa, acc.v);
                if (rb < n) epi.row(rb, sb, acc.v);
            }
        }
        __syncwarp();  // every lane has read stage s
        if (lane == 0) {
            const int32_t tn = t + NST * W;
            if (tn < ntiles) {
                fence_proxy_async_smem();
                issue(tn, s);
            }
        }
    }
    if (timed_out) {
        if (lane == 0) {
            atomicExch(err, 1);
            // the copies already issued land before the warp stops (default limit)
            for (int k = 0; k < NST; ++k) {
                const int32_t t = g + (it + k) * W;
                if (t >= ntiles) break;
                mbar_wait_bounded(bar0 + 8u * ((it + k) % NST), (uint32_t)((it + k) / NST) & 1u);
            }
        }
        epi.timed_out();
        __syncwarp();
    }
    epi.finish(acc.v);
}

// ------------------------------------------------------------ carry scan

// Inclusive segmented scan over the warp: lanes holding the same key in a
// run of consecutive lanes add their values in a fixed tree order (at level
// o, a lane adds the partial of the lane o places before it if that lane has
// its key).  Only levels below the longest run of equal keys in the warp can
// add anything, so the scan stops there: the sums are the same as with all
// five levels, with fewer FP64 adds (runs are short on skewed matrices with
// short rows).  Key INT32_MAX marks a lane without an open row; such lanes
// are runs of their own (their sums are never used).
template <typename T>
__device__ __forceinline__ T warp_seg_scan(int32_t key, T v) {
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int32_t pkey = __shfl_up_sync(FULL, key, 1);
    const bool start = lane == 0 || pkey != key || key == INT32_MAX;
    const unsigned starts = __ballot_sync(FULL, start) & (0xffffffffu >> (31 - lane));
    const int run = (int)__reduce_max_sync(FULL, (unsigned)(lane - (31 - __clz(starts)) + 1));
    for (int o = 1; o < run; o <<= 1) {
        const int32_t okey = __shfl_up_sync(FULL, key, o);
        const T ov = __shfl_up_sync(FULL, v, o);
        if (lane >= o && okey == key) v = ov + v;
    }
    return v;
}

// ------------------------------------------------------------ merge-path CSR

// Shared-memory index with one pad slot per 8, so that threads walking
// consecutive 8-entry segments hit different banks.
__device__ __forceinline__ int mpad(int k) { return k + (k >> 3); }

constexpr size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }

// Shared-memory layout of the merge kernel; every array starts on a
// 16-byte boundary: values, gathered x, row ends, thread rows, carry scan.
template <int E, typename V, typename T>
struct MergeShape {
    static constexpr int TI = 256 * E;            // path items per block
    static constexpr int PADN = TI + TI / 8 + 8;  // padded entries
    static constexpr size_t OFF_XV = align16((size_t)PADN * sizeof(V));
    static constexpr size_t OFF_RE = align16(OFF_XV + (size_t)PADN * sizeof(T));
    static constexpr size_t OFF_TR = align16(OFF_RE + (size_t)(TI + 1) * 4);
    static constexpr size_t OFF_SC = align16(OFF_TR + 256 * 4);
    static constexpr size_t BYTES = align16(OFF_SC + 256 * sizeof(T));
};

template <int E, typename V, typename T>
constexpr size_t merge_smem_bytes() {
    return MergeShape<E, V, T>::BYTES;
}

// CSR merge-path kernel (apply only).  The path of n row ends and nnz
// nonzeros is cut into equal pieces of 256*E items per block and E items
// per thread.  Phase 1: the block stages its row ends, values and the
// gathered x values (all gathers independent, so many are in flight).
// Phase 2: each thread walks its piece sequentially from shared memory (one
// FMA per nonzero).  A row whose end lies in a thread's piece is finished
// there, adding the carries of earlier threads of the block whose pieces
// ended inside the same row.  The row open at the end of a block is handed
// to k_csr_merge_fixup as (carry_row, carry_val).  block_row (n_blocks + 1
// entries) gives each block's first row; when null the block finds it by
// binary search.
template <int E, typename V, typename T>
__global__ void __launch_bounds__(256)
k_csr_merge(int32_t n, int64_t nnz, const int32_t* __restrict__ rp,
            const int32_t* __restrict__ ci, const V* __restrict__ va,
            const T* __restrict__ x, EpiStore<T> epi, const int32_t* __restrict__ block_row,
            int32_t* __restrict__ carry_row, T* __restrict__ carry_val) {
    using Sh = MergeShape<E, V, T>;
    constexpr int TI = Sh::TI;
    extern __shared__ __align__(128) unsigned char smem[];
    V* s_val = reinterpret_cast<V*>(smem);
    T* s_xv = reinterpret_cast<T*>(smem + Sh::OFF_XV);
    int32_t* s_rowend = reinterpret_cast<int32_t*>(smem + Sh::OFF_RE);
    int32_t* s_trow = reinterpret_cast<int32_t*>(smem + Sh::OFF_TR);
    T* s_scan = reinterpret_cast<T*>(smem + Sh::OFF_SC);
    __shared__ int32_t s_bounds[2];
    const int64_t N = (int64_t)n + nnz;
    const int64_t d0 = (int64_t)blockIdx.x * TI;
    const int64_t d1 = min(d0 + TI, N);
    if (threadIdx.x < 2) {
        if (block_row) {
            s_bounds[threadIdx.x] = __ldg(block_row + blockIdx.x + threadIdx.x);
        } else {
            const int64_t d = threadIdx.x == 0 ? d0 : d1;
            int32_t lo = 0, hi = n;  // rows whose end item lies before d
            while (lo < hi) {
                const int32_t mid = lo + ((hi - lo) >> 1);
                if ((int64_t)__ldg(rp + mid + 1) + mid + 1 > d) hi = mid;
                else lo = mid + 1;
            }
            s_bounds[threadIdx.x] = lo;
        }
    }
    __syncthreads();
    const int32_t i0 = s_bounds[0], i1 = s_bounds[1];
    const int64_t j0 = d0 - i0, j1 = d1 - i1;
    const int32_t nloc = min(i1 - i0 + 1, n - i0);  // staged row ends
    const int32_t cnt = (int32_t)(j1 - j0);
    for (int k = threadIdx.x; k < nloc; k += blockDim.x) s_rowend[k] = __ldg(rp + i0 + k + 1);
    constexpr int G = E < GATHER ? E : GATHER;  // loads in flight per thread
    for (int k0 = threadIdx.x; k0 < cnt; k0 += G * blockDim.x) {
        int32_t c[G];
        V v[G];
        T xv[G];
#pragma unroll
        for (int u = 0; u < G; ++u) {
            const int k = k0 + u * (int)blockDim.x;
            if (k < cnt) {
                c[u] = __ldcs(ci + j0 + k);
                v[u] = va[j0 + k];
            }
        }
#pragma unroll
        for (int u = 0; u < G; ++u) {
            const int k = k0 + u * (int)blockDim.x;
            if (k < cnt) xv[u] = __ldg(x + c[u]);
        }
#pragma unroll
        for (int u = 0; u < G; ++u) {
            const int k = k0 + u * (int)blockDim.x;
            if (k < cnt) {
                s_val[mpad(k)] = v[u];
                s_xv[mpad(k)] = xv[u];
            }
        }
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
            const int k = mpad((int)(j - j0));
            acc = fmadd(cvt<T>(s_val[k]), s_xv[k], acc);
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
    // Carries: thread t ends its piece inside row s_trow[t] with partial sum
    // acc.  A segmented inclusive scan over the threads (log steps, fixed
    // order) gives S[t] = sum of the carries of the run of threads ending
    // at t that share its row; rows are non-decreasing over valid threads.
    const bool valid = dt < d1;
    const int32_t myrow = valid ? i : INT32_MAX;
    s_trow[threadIdx.x] = myrow;
    T sc = acc;
    s_scan[threadIdx.x] = sc;
    __syncthreads();
    for (int o = 1; o < (int)blockDim.x; o <<= 1) {
        const bool take = (int)threadIdx.x >= o && s_trow[threadIdx.x - o] == myrow;
        const T other = take ? s_scan[threadIdx.x - o] : T(0);
        __syncthreads();
        if (take) sc = other + sc;
        s_scan[threadIdx.x] = sc;
        __syncthreads();
    }
    if (head_row >= 0) {
        T v = head_val;
        if (threadIdx.x > 0 && s_trow[threadIdx.x - 1] == head_row) v = s_scan[threadIdx.x - 1] + v;
        epi.row(head_row, v, nullptr);
    }
    // the row open at the end of the block: carried by the last valid thread
    if (valid && (threadIdx.x == blockDim.x - 1 || s_trow[threadIdx.x + 1] == INT32_MAX)) {
        carry_row[blockIdx.x] = (i < n) ? i : -1;
        carry_val[blockIdx.x] = sc;
    }
}

// Merge path with register operands (apply only): the same 32*E-item warp
// units and lane pieces as k_csr_merge_warp, but a lane loads the values and
// columns of its (at most E, contiguous) nonzeros straight from global
// memory and gathers their x into registers; only the unit's row ends are
// staged in shared memory (for the lane's binary search and the row ends it
// meets).  The walk visits the lane's nonzero slots k = 0..E-1 in order and
// closes every row that ends before slot k first, so each nonzero costs one
// FMA on registers indexed at compile time.
template <int E>
struct MergeRegShape {
    static constexpr int WI = 32 * E;
    static constexpr size_t WARP_BYTES = align16((size_t)(WI + 1) * 4);
    static constexpr size_t BYTES = 8 * WARP_BYTES;
};

template <int E, typename V, typename T>
__global__ void __launch_bounds__(256)
k_csr_merge_reg(int32_t n, int64_t nnz, const int32_t* __restrict__ rp,
                const int32_t* __restrict__ ci, const V* __restrict__ va,
                const T* __restrict__ x, EpiStore<T> epi, const int32_t* __restrict__ unit_row,
                int64_t nunits, int32_t* __restrict__ carry_row, T* __restrict__ carry_val) {
    constexpr int WI = MergeRegShape<E>::WI;
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t u = (int64_t)blockIdx.x * 8 + warp;
    if (u >= nunits) return;  // the whole warp; no block barrier follows
    int32_t* s_rowend = reinterpret_cast<int32_t*>(smem + (size_t)warp * MergeRegShape<E>::WARP_BYTES);
    const int64_t N = (int64_t)n + nnz;
    const int64_t d0 = u * WI;
    const int64_t d1 = min(d0 + WI, N);
    int32_t bnd = 0;
    if (lane < 2) bnd = __ldg(unit_row + u + lane);
    const int32_t i0 = __shfl_sync(FULL, bnd, 0), i1 = __shfl_sync(FULL, bnd, 1);
    const int32_t nloc = min(i1 - i0 + 1, n - i0);  // staged row ends
    for (int k = lane; k < nloc; k += 32) s_rowend[k] = __ldg(rp + i0 + k + 1);
    __syncwarp();
    // this lane's start on the path: row i, nonzero j
    const int64_t dt = min(d0 + (int64_t)lane * E, d1);
    const int64_t dend = min(dt + E, d1);
    int32_t lo = 0, hi = max(0, nloc);
    while (lo < hi) {
        const int32_t mid = (lo + hi) >> 1;
        if ((int64_t)s_rowend[mid] + i0 + mid + 1 > dt) hi = mid;
        else lo = mid + 1;
    }
    int32_t i = i0 + lo;
    const int64_t j0 = dt - i;
    // the lane's end on the path: row iend, nonzero jend (its nonzeros are [j0, jend))
    lo = 0;
    hi = max(0, nloc);
    while (lo < hi) {
        const int32_t mid = (lo + hi) >> 1;
        if ((int64_t)s_rowend[mid] + i0 + mid + 1 > dend) hi = mid;
        else lo = mid + 1;
    }
    const int32_t iend = i0 + lo;
    const int64_t jend = dend - iend;
    const int cnt = (int)(jend - j0);  // nonzeros of this lane, 0..E
    V v[E];
    T xv[E];
    {
        int32_t c[E];
#pragma unroll
        for (int k = 0; k < E; ++k)
            if (k < cnt) {
                c[k] = __ldcs(ci + j0 + k);
                v[k] = va[j0 + k];
            }
#pragma unroll
        for (int k = 0; k < E; ++k)
            if (k < cnt) xv[k] = __ldg(x + c[k]);
    }
    T acc = T(0);
    int32_t head_row = -1;
    T head_val = T(0);
    int64_t rend = (i < n) ? (int64_t)s_rowend[i - i0] : 0;
    // close the rows that end at nonzero position p (before its slot)
    auto close_until = [&](int64_t p) {
        while (i < iend && rend <= p) {
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
    };
#pragma unroll
    for (int k = 0; k < E; ++k) {
        if (k < cnt) {
            close_until(j0 + k);
            acc = fmadd(cvt<T>(v[k]), xv[k], acc);
        }
    }
    close_until(jend);  // row ends after the last nonzero of the piece
    // carries: as in k_csr_merge_warp
    const bool valid = dt < d1;
    const int32_t myrow = valid ? i : INT32_MAX;
    const T sc = warp_seg_scan(myrow, acc);
    const int32_t prow = __shfl_up_sync(FULL, myrow, 1);
    const T psc = __shfl_up_sync(FULL, sc, 1);
    const int32_t nrow = __shfl_down_sync(FULL, myrow, 1);
    if (head_row >= 0) {
        T vv = head_val;
        if (lane > 0 && prow == head_row) vv = psc + vv;
        epi.row(head_row, vv, nullptr);
    }
    if (valid && (lane == 31 || nrow == INT32_MAX)) {
        carry_row[u] = (i < n) ? i : -1;
        carry_val[u] = sc;
    }
}

// Shared-memory layout of the warp-level merge kernel, per warp (8 warps a
// block): values, gathered x, row ends; every array on a 16-byte boundary.
template <int E, typename V, typename T>
struct MergeWarpShape {
    static constexpr int WI = 32 * E;             // path items per warp
    static constexpr int PADN = WI + WI / 8 + 8;  // padded entries
    static constexpr size_t OFF_XV = align16((size_t)PADN * sizeof(V));
    static constexpr size_t OFF_RE = align16(OFF_XV + (size_t)PADN * sizeof(T));
    static constexpr size_t WARP_BYTES = align16(OFF_RE + (size_t)(WI + 1) * 4);
    static constexpr size_t BYTES = 8 * WARP_BYTES;
};

// CSR merge-path kernel at warp granularity (apply only).  The path of n
// row ends and nnz nonzeros is cut into units of 32*E items, one unit per
// warp and E items per lane; the 8 warps of a block share nothing but the
// block's shared memory, so the kernel has no block barrier and a warp
// never waits for another.  A warp stages its row ends, values and the
// gathered x values (E independent gathers per lane in flight), each lane
// walks its piece (one FMA per nonzero), and the carries of lanes whose
// pieces end inside a row are combined with a 5-level segmented shuffle
// scan (a level's add runs only in warps where some run is that long).  The
// row open at the end of a unit goes to k_csr_merge_fixup as (carry_row,
// carry_val).  unit_row (nunits + 1 entries) gives each unit's first row;
// when null the warp finds it by binary search.
template <int E, typename V, typename T>
__global__ void __launch_bounds__(256)
k_csr_merge_warp(int32_t n, int64_t nnz, const int32_t* __restrict__ rp,
                 const int32_t* __restrict__ ci, const V* __restrict__ va,
                 const T* __restrict__ x, EpiStore<T> epi, const int32_t* __restrict__ unit_row,
                 int64_t nunits, int32_t* __restrict__ carry_row, T* __restrict__ carry_val) {
    using Sh = MergeWarpShape<E, V, T>;
    constexpr int WI = Sh::WI;
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t u = (int64_t)blockIdx.x * 8 + warp;
    if (u >= nunits) return;  // the whole warp; no block barrier follows
    unsigned char* base = smem + (size_t)warp * Sh::WARP_BYTES;
    V* s_val = reinterpret_cast<V*>(base);
    T* s_xv = reinterpret_cast<T*>(base + Sh::OFF_XV);
    int32_t* s_rowend = reinterpret_cast<int32_t*>(base + Sh::OFF_RE);
    const int64_t N = (int64_t)n + nnz;
    const int64_t d0 = u * WI;
    const int64_t d1 = min(d0 + WI, N);
    int32_t bnd = 0;
    if (unit_row) {
        if (lane < 2) bnd = __ldg(unit_row + u + lane);
    } else if (lane < 2) {
        const int64_t d = lane == 0 ? d0 : d1;
        int32_t lo = 0, hi = n;  // rows whose end item lies before d
        while (lo < hi) {
            const int32_t mid = lo + ((hi - lo) >> 1);
            if ((int64_t)__ldg(rp + mid + 1) + mid + 1 > d) hi = mid;
            else lo = mid + 1;
        }
        bnd = lo;
    }
    const int32_t i0 = __shfl_sync(FULL, bnd, 0), i1 = __shfl_sync(FULL, bnd, 1);
    const int64_t j0 = d0 - i0, j1 = d1 - i1;
    const int32_t nloc = min(i1 - i0 + 1, n - i0);  // staged row ends
    const int32_t cnt = (int32_t)(j1 - j0);
    for (int k = lane; k < nloc; k += 32) s_rowend[k] = __ldg(rp + i0 + k + 1);
    {
        int32_t c[E];
        V v[E];
        T xv[E];
#pragma unroll
        for (int q = 0; q < E; ++q) {
            const int k = lane + 32 * q;
            if (k < cnt) {
                c[q] = __ldcs(ci + j0 + k);
                v[q] = va[j0 + k];
            }
        }
#pragma unroll
        for (int q = 0; q < E; ++q) {
            const int k = lane + 32 * q;
            if (k < cnt) xv[q] = __ldg(x + c[q]);
        }
#pragma unroll
        for (int q = 0; q < E; ++q) {
            const int k = lane + 32 * q;
            if (k < cnt) {
                s_val[mpad(k)] = v[q];
                s_xv[mpad(k)] = xv[q];
            }
        }
    }
    __syncwarp();
    // this lane's start on the path
    const int64_t dt = min(d0 + (int64_t)lane * E, d1);
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
            const int k = mpad((int)(j - j0));
            acc = fmadd(cvt<T>(s_val[k]), s_xv[k], acc);
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
    // Carries: lane l ends its piece inside row myrow with partial sum acc;
    // rows are non-decreasing over the valid lanes, so a segmented inclusive
    // scan (fixed order) gives each lane the sum over its run of lanes.
    const bool valid = dt < d1;
    const int32_t myrow = valid ? i : INT32_MAX;
    const T sc = warp_seg_scan(myrow, acc);
    const int32_t prow = __shfl_up_sync(FULL, myrow, 1);
    const T psc = __shfl_up_sync(FULL, sc, 1);
    const int32_t nrow = __shfl_down_sync(FULL, myrow, 1);
    if (head_row >= 0) {
        T vv = head_val;
        if (lane > 0 && prow == head_row) vv = psc + vv;
        epi.row(head_row, vv, nullptr);
    }
    // the row open at the end of the unit: carried by the last valid lane
    if (valid && (lane == 31 || nrow == INT32_MAX)) {
        carry_row[u] = (i < n) ? i : -1;
        carry_val[u] = sc;
    }
}

// COO SpMV (apply only): triplets sorted by (row, col).  The nonzeros are
// cut into units of 32*4H per warp, 4H consecutive triplets per lane, read
// in groups of 4 with 16-byte loads (no shared-memory staging: the row index
// comes with every entry).  A lane sums each run of equal rows; a row ends where the next
// triplet (in this lane, the next lane, the next unit, or none) has another
// row.  The first row a lane ends may have begun in earlier lanes: it adds
// their carries, combined with the 5-level segmented shuffle scan used by
// the merge kernel; the run open at the end of a unit goes to
// k_csr_merge_fixup.  Rows without entries are written by k_coo_empty.

// E consecutive entries starting at k (k % E == 0): 16-byte loads when the
// group is whole (the arrays start on 256-byte boundaries), else one by one.
template <int E, typename V>
__device__ __forceinline__ void load_group(const V* __restrict__ p, int64_t k, int64_t nnz,
                                           bool full, V (&v)[E]) {
    constexpr int PER = 16 / (int)sizeof(V) < E ? 16 / (int)sizeof(V) : E;  // per 16 B
    struct alignas(PER * sizeof(V)) Q { V e[PER]; };
    if (full) {
#pragma unroll
        for (int h = 0; h < E / PER; ++h) {
            const Q q = *reinterpret_cast<const Q*>(p + k + h * PER);
#pragma unroll
            for (int c = 0; c < PER; ++c) v[h * PER + c] = q.e[c];
        }
    } else {
#pragma unroll
        for (int c = 0; c < E; ++c) v[c] = k + c < nnz ? p[k + c] : V{};
    }
}

template <int H, typename V, typename T>
__global__ void __launch_bounds__(256)
k_coo_warp(int32_t n, int64_t nnz, const int32_t* __restrict__ rows,
           const int32_t* __restrict__ ci, const V* __restrict__ va, const T* __restrict__ x,
           EpiStore<T> epi, int64_t nunits, int32_t* __restrict__ carry_row,
           T* __restrict__ carry_val) {
    constexpr unsigned FULL = 0xffffffffu;
    constexpr int G = 4;           // triplets per 16-byte group load
    constexpr int EPL = G * H;     // triplets per lane
    constexpr int WI = 32 * EPL;   // triplets per warp unit
    const int lane = threadIdx.x & 31;
    const int64_t u = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (u >= nunits) return;  // the whole warp
    const int64_t k0 = u * WI + (int64_t)lane * EPL;
    T acc = T(0);
    int32_t head_row = -1;
    T head_val = T(0);
    bool begun_here = false;  // the open run began after a row end in this lane
    bool open = false;
    int32_t last = -1;
    // groups of 4 triplets, one after the other (few registers live), the
    // walk state carried across groups
#pragma unroll 1
    for (int g = 0; g < H; ++g) {
        const int64_t kg = k0 + (int64_t)g * G;
        if (kg >= nnz) break;
        const bool full = kg + G <= nnz;
        int32_t r[G], c[G];
        V v[G];
        load_group<G>(rows, kg, nnz, full, r);
        load_group<G>(ci, kg, nnz, full, c);
        load_group<G>(va, kg, nnz, full, v);
        const int32_t rnext = kg + G < nnz ? __ldg(rows + kg + G) : INT32_MAX;
        // x gathers at uniformly random columns reuse nothing in L1: read
        // them through L2 only (.cg), leaving L1 to the streamed triplets
        T xv[G];
#pragma unroll
        for (int q = 0; q < G; ++q) xv[q] = kg + q < nnz ? __ldcg(x + c[q]) : T(0);
#pragma unroll
        for (int q = 0; q < G; ++q) {
            if (kg + q < nnz) {
                acc = fmadd(cvt<T>(v[q]), xv[q], acc);
                open = true;
                last = r[q];
                const int32_t nr = (q + 1 < G) ? (kg + q + 1 < nnz ? r[q + 1] : INT32_MAX) : rnext;
                if (nr != r[q]) {  // row r[q] ends here
                    if (!begun_here) {
                        head_row = r[q];
                        head_val = acc;
                    } else {
                        epi.row(r[q], acc, nullptr);
                    }
                    acc = T(0);
                    begun_here = true;
                    open = false;
                }
            }
        }
    }
    // the lane's open run (a row that continues in the next lane) is its carry
    const int32_t myrow = open ? last : INT32_MAX;
    const T sc = warp_seg_scan(myrow, acc);
    const int32_t prow = __shfl_up_sync(FULL, myrow, 1);
    const T psc = __shfl_up_sync(FULL, sc, 1);
    if (head_row >= 0) {
        T vv = head_val;
        if (lane > 0 && prow == head_row) vv = psc + vv;
        epi.row(head_row, vv, nullptr);
    }
    // the unit's open run: carried by its last lane holding entries
    const bool has = k0 < nnz;
    const bool next_has = __shfl_down_sync(FULL, has ? 1 : 0, 1) != 0;
    if (has && (lane == 31 || !next_has)) {
        carry_row[u] = myrow != INT32_MAX ? myrow : -1;
        carry_val[u] = sc;
    }
}

// Rows without entries: x_i = 0 (modes 0, 1) or beta x_i (mode 2).
template <typename T>
__global__ void k_coo_empty(int32_t count, const int32_t* __restrict__ idx, EpiStore<T> epi) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < count;
         k += (int64_t)gridDim.x * blockDim.x)
        epi.row(idx[k], T(0), nullptr);
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

// ------------------------------------------------------------ vector CSR

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

// ------------------------------------------------------------ ELL / SELL-P

// One row: `len` stored entries at base, base + step, ... (column-major
// padded layouts).  Padding has col -1 and value 0 and adds nothing.
template <typename T, typename V>
__device__ __forceinline__ T row_sum_padded(const int32_t* __restrict__ pc,
                                            const V* __restrict__ pv, const T* __restrict__ x,
                                            int64_t base, int64_t step, int32_t len) {
    T s = T(0);
#pragma unroll 4
    for (int32_t j = 0; j < len; ++j) {
        const int64_t at = base + (int64_t)j * step;
        const int32_t c = ld_stream(pc + at);
        const T v = ld_stream(pv + at);
        if (c >= 0) s = fmadd(v, __ldg(x + c), s);
    }
    return s;
}

// Paired value type for two adjacent rows (16-byte loads for FP64).
template <typename V> struct Pair2;
template <> struct Pair2<double> { using type = double2; };
template <> struct Pair2<float> { using type = float2; };
template <> struct Pair2<__nv_bfloat16> { using type = __nv_bfloat162; };
template <> struct Pair2<__half> { using type = __half2; };

template <typename T, typename P>
__device__ __forceinline__ void unpack2(const P& p, T& a, T& b) {
    a = cvt<T>(p.x);
    b = cvt<T>(p.y);
}

// Two adjacent rows i, i+1 (i even) stored column-major with `step`
// between entries of a row: one 8-byte column load and one paired value
// load per entry position serve both rows.
template <typename T, typename V>
__device__ __forceinline__ void row_pair_padded(const int32_t* __restrict__ pc,
                                                const V* __restrict__ pv,
                                                const T* __restrict__ x, int64_t base,
                                                int64_t step, int32_t len, T& s0, T& s1) {
    using P = typename Pair2<V>::type;
    s0 = T(0);
    s1 = T(0);
#pragma unroll 4
    for (int32_t j = 0; j < len; ++j) {
        const int64_t at = base + (int64_t)j * step;
        const int2 c = __ldcs(reinterpret_cast<const int2*>(pc + at));
        const P pvv = *reinterpret_cast<const P*>(pv + at);
        T v0, v1;
        unpack2<T>(pvv, v0, v1);
        const T x0 = c.x >= 0 ? __ldg(x + c.x) : T(0);
        const T x1 = c.y >= 0 ? __ldg(x + c.y) : T(0);
        s0 = fmadd(v0, x0, s0);
        s1 = fmadd(v1, x1, s1);
    }
}

// Two pairs of adjacent rows (a0, a0+1) and (b0, b0+1), their loads issued
// together: twice the bytes in flight of row_pair_padded.
template <typename T, typename V>
__device__ __forceinline__ void row_quad_padded(const int32_t* __restrict__ pc,
                                                const V* __restrict__ pv,
                                                const T* __restrict__ x, int64_t a0, int64_t b0,
                                                int64_t step, int32_t len, T (&s)[4]) {
    using P = typename Pair2<V>::type;
    s[0] = s[1] = s[2] = s[3] = T(0);
#pragma unroll 2
    for (int32_t j = 0; j < len; ++j) {
        const int64_t ja = a0 + (int64_t)j * step, jb = b0 + (int64_t)j * step;
        const int2 ca = __ldcs(reinterpret_cast<const int2*>(pc + ja));
        const int2 cb = __ldcs(reinterpret_cast<const int2*>(pc + jb));
        const P pa = *reinterpret_cast<const P*>(pv + ja);
        const P pb = *reinterpret_cast<const P*>(pv + jb);
        T v0, v1, v2, v3;
        unpack2<T>(pa, v0, v1);
        unpack2<T>(pb, v2, v3);
        const T x0 = ca.x >= 0 ? __ldg(x + ca.x) : T(0);
        const T x1 = ca.y >= 0 ? __ldg(x + ca.y) : T(0);
        const T x2 = cb.x >= 0 ? __ldg(x + cb.x) : T(0);
        const T x3 = cb.y >= 0 ? __ldg(x + cb.y) : T(0);
        s[0] = fmadd(v0, x0, s[0]);
        s[1] = fmadd(v1, x1, s[1]);
        s[2] = fmadd(v2, x2, s[2]);
        s[3] = fmadd(v3, x3, s[3]);
    }
}

// ELL: one thread per pair of adjacent rows (stride is a multiple of 32,
// so pairs never straddle it), column-major coalesced paired loads.  With
// QUAD a thread takes pairs q and q + G (G = grid threads) together while
// both exist: more loads in flight when a thread has few pairs to do.
template <typename V, typename T, class Epi, bool QUAD = false>
__global__ void __launch_bounds__(256)
k_ell(int32_t n, int64_t stride, int32_t K, const int32_t* __restrict__ ec,
      const V* __restrict__ ev, const T* __restrict__ x, Epi epi) {
    if (epi.skip()) return;
    AccArr<Epi> acc{};
    const int64_t npairs = ((int64_t)n + 1) / 2;
    const int64_t G = (int64_t)gridDim.x * blockDim.x;
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (QUAD) {
        for (; q + G < npairs; q += 2 * G) {
            const int64_t i = 2 * q, k = 2 * (q + G);
            T sq[4];
            row_quad_padded<T, V>(ec, ev, x, i, k, stride, K, sq);
            epi.row(i, sq[0], acc.v);
            epi.row(i + 1, sq[1], acc.v);
            epi.row(k, sq[2], acc.v);
            if (k + 1 < n) epi.row(k + 1, sq[3], acc.v);
        }
    }
    for (; q < npairs; q += G) {
        const int64_t i = 2 * q;
        T s0, s1;
        row_pair_padded<T, V>(ec, ev, x, i, stride, K, s0, s1);
        epi.row(i, s0, acc.v);
        if (i + 1 < n) epi.row(i + 1, s1, acc.v);
    }
    epi.finish(acc.v);
}

// SELL-P: one thread per row; the rows of a slice read consecutive
// addresses for every stored column position.  The slice metadata of the
// thread's next row is loaded before the current row is processed.  With
// an even slice size, a thread takes two adjacent rows of one slice and
// uses paired loads (k_sellp_pairs).
template <typename V, typename T, class Epi>
__global__ void __launch_bounds__(256)
k_sellp(int32_t n, int32_t S, const int32_t* __restrict__ slen, const int64_t* __restrict__ sset,
        const int32_t* __restrict__ sc, const V* __restrict__ sv, const T* __restrict__ x, Epi epi) {
    if (epi.skip()) return;
    AccArr<Epi> acc{};
    // row indices fit in 32 bits; S is a power of two in the common case
    const int sh = (S & (S - 1)) == 0 ? __ffs(S) - 1 : -1;
    auto slice_of = [&](uint32_t r) -> uint32_t { return sh >= 0 ? (r >> sh) : r / (uint32_t)S; };
    const int64_t G = (int64_t)gridDim.x * blockDim.x;
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int32_t len = 0;
    int64_t base = 0;
    if (i < n) {
        const uint32_t sl = slice_of((uint32_t)i);
        len = __ldg(slen + sl);
        base = __ldg(sset + sl) * S + ((int64_t)i - (int64_t)sl * S);
    }
    while (i < n) {
        const int64_t in = i + G;
        int32_t len_n = 0;
        int64_t base_n = 0;
        if (in < n) {
            const uint32_t sl = slice_of((uint32_t)in);
            len_n = __ldg(slen + sl);
            base_n = __ldg(sset + sl) * S + (in - (int64_t)sl * S);
        }
        epi.row(i, row_sum_padded<T, V>(sc, sv, x, base, S, len), acc.v);
        i = in;
        len = len_n;
        base = base_n;
    }
    epi.finish(acc.v);
}

template <typename V, typename T, class Epi>
__global__ void __launch_bounds__(256)
k_sellp_pairs(int32_t n, int32_t S, const int32_t* __restrict__ slen,
              const int64_t* __restrict__ sset, const int32_t* __restrict__ sc,
              const V* __restrict__ sv, const T* __restrict__ x, Epi epi) {
    if (epi.skip()) return;
    AccArr<Epi> acc{};
    const int sh = (S & (S - 1)) == 0 ? __ffs(S) - 1 : -1;
    auto slice_of = [&](uint32_t r) -> uint32_t { return sh >= 0 ? (r >> sh) : r / (uint32_t)S; };
    const int64_t npairs = ((int64_t)n + 1) / 2;
    const int64_t G = (int64_t)gridDim.x * blockDim.x;
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int32_t len = 0;
    int64_t base = 0;
    if (q < npairs) {
        const uint32_t r = (uint32_t)(2 * q), sl = slice_of(r);
        len = __ldg(slen + sl);
        base = __ldg(sset + sl) * S + ((int64_t)r - (int64_t)sl * S);
    }
    while (q < npairs) {
        const int64_t qn = q + G;
        int32_t len_n = 0;
        int64_t base_n = 0;
        if (qn < npairs) {
            const uint32_t r = (uint32_t)(2 * qn), sl = slice_of(r);
            len_n = __ldg(slen + sl);
            base_n = __ldg(sset + sl) * S + ((int64_t)r - (int64_t)sl * S);
        }
        T s0, s1;
        row_pair_padded<T, V>(sc, sv, x, base, S, len, s0, s1);
        const int64_t i = 2 * q;
        epi.row(i, s0, acc.v);
        if (i + 1 < n) epi.row(i + 1, s1, acc.v);
        q = qn;
        len = len_n;
        base = base_n;
    }
    epi.finish(acc.v);
}

// ------------------------------------------------------------ launcher

// Lets `kernel` take the device's opt-in shared memory per block minus its
// own static shared memory as dynamic shared memory (a constant per kernel).
template <typename K>
static gk_status allow_max_dynamic_smem(K kernel) {
    cudaFuncAttributes fa;
    GK_CUDA(cudaFuncGetAttributes(&fa, kernel));
    int dev = 0, optin = 0;
    GK_CUDA(cudaGetDevice(&dev));
    GK_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    GK_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 optin - (int)fa.sharedSizeBytes));
    return GK_OK;
}

template <typename K>
static int occupancy_blocks(K kernel, int threads, size_t smem) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, threads, smem) != cudaSuccess || b < 1)
        b = 1;
    return b;
}

constexpr int ROWTILE_MAX_STAGES = 3;
constexpr size_t ROWTILE_SMEM_BUDGET = 200 * 1024;

// stages of the row-tile pipeline that fit the shared-memory budget
inline int rowtile_stages(const gk_matrix A, size_t vbytes) {
    const size_t stage = (size_t)A->plan.tile_cap * (4 + vbytes);
    int nst = A->plan.stages > 0 ? A->plan.stages : ROWTILE_MAX_STAGES;
    while (nst > 1 && (size_t)nst * stage + 8 * nst > ROWTILE_SMEM_BUDGET) --nst;
    return nst;
}

inline size_t rowtile_smem(const gk_matrix A, size_t vbytes) {
    const int nst = rowtile_stages(A, vbytes);
    return (size_t)nst * (size_t)A->plan.tile_cap * (4 + vbytes) + 8 * (size_t)nst;
}

// Launches the row-complete SpMV of A (row-tile / vector CSR, ELL, SELL-P)
// with epilogue epi.  For epilogues with NA > 0, the caller provides
// partials (NA * num_sms() * 8 doubles) and a zeroed ticket through epi.
// The grid depends only on the matrix and the device, so the partial-sum
// layout of fused reductions is fixed.
template <typename V, typename T, class Epi>
gk_status launch_spmv_rows(gk_matrix A, const T* x, const Epi& epi, cudaStream_t s,
                           unsigned* grid_out = nullptr) {
    const int sms = num_sms();
    unsigned grid = 1;
    if (A->fmt == GK_CSR && A->plan.kind == 1) {
        const size_t smem = rowtile_smem(A, sizeof(V));
        const int nst = rowtile_stages(A, sizeof(V));
        auto k = k_csr_rowtile<V, T, Epi>;
        static thread_local int occ_cache = 0;
        static thread_local size_t occ_smem = 0;
        if (occ_smem != smem || !occ_cache) {
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
            occ_cache = std::min(occupancy_blocks(k, 256, smem), 8);
            occ_smem = smem;
        }
        grid = (unsigned)std::min<int64_t>(A->plan.ntiles, (int64_t)sms * occ_cache);
        if (grid < 1) grid = 1;
        k<<<grid, 256, smem, s>>>(A->plan.ntiles, A->plan.tile_desc, A->row_ptr, A->col,
                                  (const V*)A->val, x, A->plan.tile_cap, nst, epi, A->plan.err,
                                  A->wait_ns);
    } else if (A->fmt == GK_CSR && A->plan.kind == 3) {
        const int nst = A->plan.stages, rpl = A->plan.wt_rpl;
        const int32_t cap = A->plan.tile_cap;
        const size_t smem = (size_t)WT_WARPS * wt_warp_bytes<V>(cap, nst);
        auto launch = [&](auto k) -> gk_status {
            // one fixed cap for every launch (the most this kernel may take):
            // host threads launching it for matrices of different tile sizes
            // must not lower each other's limit between setting it and
            // launching
            static thread_local int occ_cache = 0;
            static thread_local size_t occ_smem = 0;
            if (occ_smem != smem || !occ_cache) {
                GK_TRY(allow_max_dynamic_smem(k));
                occ_cache = std::min(occupancy_blocks(k, WT_WARPS * 32, smem), 8);
                occ_smem = smem;
            }
            const int64_t rows = 32 * (int64_t)rpl;
            const int64_t ntiles = ((int64_t)A->n + rows - 1) / rows;
            grid = (unsigned)std::max<int64_t>(
                1, std::min<int64_t>((ntiles + WT_WARPS - 1) / WT_WARPS, (int64_t)sms * occ_cache));
            k<<<grid, WT_WARPS * 32, smem, s>>>(A->n, A->row_ptr, A->col, (const V*)A->val, x,
                                                cap, nst, epi, A->plan.err, A->wait_ns);
            return GK_OK;
        };
        if (rpl == 1) GK_TRY(launch(k_csr_warptile<1, V, T, Epi>));
        else if (rpl == 4) GK_TRY(launch(k_csr_warptile<4, V, T, Epi>));
        else GK_TRY(launch(k_csr_warptile<2, V, T, Epi>));
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
        // grid-stride kernels: one full wave of resident blocks, no ragged second wave
        static const int quad = [] {
            const char* e = getenv("GK_ELL_QUAD");
            return e ? atoi(e) : 1;
        }();
        if (quad) {
            static thread_local int occ = 0;
            if (!occ) occ = std::min(occupancy_blocks(k_ell<V, T, Epi, true>, 256, 0), 8);
            int64_t need = ((A->n + 1) / 2 + 255) / 256;
            grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)sms * occ));
            k_ell<V, T, Epi, true><<<grid, 256, 0, s>>>(A->n, A->stride, A->K, A->col,
                                                        (const V*)A->val, x, epi);
        } else {
            static thread_local int occ = 0;
            if (!occ) occ = std::min(occupancy_blocks(k_ell<V, T, Epi>, 256, 0), 8);
            int64_t need = ((A->n + 1) / 2 + 255) / 256;
            grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)sms * occ));
            k_ell<V, T, Epi><<<grid, 256, 0, s>>>(A->n, A->stride, A->K, A->col, (const V*)A->val,
                                                  x, epi);
        }
    } else if (A->S % 2 == 0) {
        static thread_local int occ = 0;
        if (!occ) occ = std::min(occupancy_blocks(k_sellp_pairs<V, T, Epi>, 256, 0), 8);
        int64_t need = ((A->n + 1) / 2 + 255) / 256;
        grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)sms * occ));
        k_sellp_pairs<V, T, Epi><<<grid, 256, 0, s>>>(A->n, A->S, A->slice_len, A->slice_set,
                                                      A->col, (const V*)A->val, x, epi);
    } else {
        static thread_local int occ = 0;
        if (!occ) occ = std::min(occupancy_blocks(k_sellp<V, T, Epi>, 256, 0), 8);
        int64_t need = (A->n + 255) / 256;
        grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)sms * occ));
        k_sellp<V, T, Epi><<<grid, 256, 0, s>>>(A->n, A->S, A->slice_len, A->slice_set, A->col,
                                                (const V*)A->val, x, epi);
    }
    if (grid_out) *grid_out = grid;
    GK_CUDA(cudaGetLastError());
    return GK_OK;
}

// Upper bound of the grid launch_spmv_rows uses for A (sizes partials).
inline unsigned max_grid_rows(gk_matrix A) { return (unsigned)num_sms() * 8; }

// merge-path items per thread for a value type
template <typename V>
struct MergeE {
    static constexpr int value = 8;
};

}  // namespace gk
