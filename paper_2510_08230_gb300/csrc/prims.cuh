// prims.cuh - device building blocks: exclusive scan, fixed-order block
// reductions and the "last block finishes" pattern used for deterministic
// two-stage reductions.
#pragma once

#include "gk_internal.cuh"

namespace gk {

constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

template <typename X>
__device__ __forceinline__ X warp_incl_scan(X v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        X t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Exclusive scan of a block's SCAN_TILE items held SCAN_ITEMS per thread;
// returns the block total.  All threads must call.
template <typename X>
__device__ X block_excl_scan(X (&v)[SCAN_ITEMS]) {
    __shared__ X warp_tot[32];
    X run = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) { X t = v[i]; v[i] = run; run += t; }
    X incl = warp_incl_scan(run);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        X w = (lane < (int)(blockDim.x >> 5)) ? warp_tot[lane] : X(0);
        X wi = warp_incl_scan(w);
        warp_tot[lane] = wi - w;  // exclusive
    }
    __syncthreads();
    X off = warp_tot[warp] + (incl - run);
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) v[i] += off;
    __shared__ X tot_sh;
    if (threadIdx.x == blockDim.x - 1) tot_sh = off + run;
    __syncthreads();
    X t = tot_sh;
    __syncthreads();
    return t;
}

template <typename In>
__global__ void k_scan_reduce(const In* __restrict__ in, int64_t m, int64_t* __restrict__ bsum) {
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    int64_t s = 0;
    for (int i = threadIdx.x; i < SCAN_TILE; i += blockDim.x) {
        int64_t k = base + i;
        if (k < m) s += (int64_t)in[k];
    }
    __shared__ int64_t sh[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        int64_t w = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
        if (threadIdx.x == 0) bsum[blockIdx.x] = w;
    }
}

// single block: in-place exclusive scan of nb block sums
__global__ void k_scan_blocksums(int64_t* __restrict__ bsum, int64_t nb);

template <typename In, typename Out>
__global__ void k_scan_apply(const In* __restrict__ in, int64_t m,
                             const int64_t* __restrict__ boff, Out* __restrict__ out) {
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    int64_t v[SCAN_ITEMS];
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) v[i] = (base + i < m) ? (int64_t)in[base + i] : 0;
    int64_t tot = block_excl_scan(v);
    const int64_t off = boff[blockIdx.x];
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i)
        if (base + i < m) out[base + i] = (Out)(v[i] + off);
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[m] = (Out)(off + tot);
}

// out[0..m] = exclusive prefix sum of in[0..m), out[m] = total.
template <typename In, typename Out>
gk_status scan_exclusive(const In* in, Out* out, int64_t m, DevBuf& tmp, cudaStream_t s) {
    if (m <= 0) {
        GK_CUDA(cudaMemsetAsync(out, 0, sizeof(Out), s));
        return GK_OK;
    }
    const int64_t nb = (m + SCAN_TILE - 1) / SCAN_TILE;
    GK_TRY(tmp.ensure(sizeof(int64_t) * (size_t)nb));
    int64_t* bs = reinterpret_cast<int64_t*>(tmp.ptr);
    k_scan_reduce<In><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, m, bs);
    k_scan_blocksums<<<1, SCAN_THREADS, 0, s>>>(bs, nb);
    k_scan_apply<In, Out><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, m, bs, out);
    GK_CUDA(cudaGetLastError());
    return GK_OK;
}

// ---------------------------------------------------------------- reductions
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Fixed-order sum of NA per-thread values over the block (blockDim <= 512);
// the result is valid in every lane of warp 0.  All threads must call.
// FP64 warp instructions are expensive on this part (~16 SM cycles each),
// so threads only store their values and warp 0 adds them: lane l sums
// sh[l], sh[l+32], ... in two interleaved chains (even and odd slots),
// then a 5-level shuffle tree combines the lanes.  Few registers stay live,
// so the reduction does not lower the occupancy of the kernel calling it.
template <int NA>
__device__ __forceinline__ void block_sum(double (&v)[NA]) {
    __shared__ double sh[NA > 0 ? NA : 1][512];
#pragma unroll
    for (int a = 0; a < NA; ++a) sh[a][threadIdx.x] = v[a];
    __syncthreads();
    if (threadIdx.x < 32) {
        const unsigned nb = blockDim.x;
#pragma unroll
        for (int a = 0; a < NA; ++a) {
            double s0 = 0.0, s1 = 0.0;
            unsigned idx = threadIdx.x;
            for (; idx + 32u < nb; idx += 64u) {
                s0 += sh[a][idx];
                s1 += sh[a][idx + 32u];
            }
            if (idx < nb) s0 += sh[a][idx];
            v[a] = warp_sum(s0 + s1);
        }
    }
    __syncthreads();
}

// block_sum with the result broadcast to every thread of the block.
template <int NA>
__device__ __forceinline__ void block_allsum_bcast(double (&v)[NA]) {
    __shared__ double tot[NA > 0 ? NA : 1];
    block_sum<NA>(v);
    if (threadIdx.x == 0)
#pragma unroll
        for (int a = 0; a < NA; ++a) tot[a] = v[a];
    __syncthreads();
#pragma unroll
    for (int a = 0; a < NA; ++a) v[a] = tot[a];
    __syncthreads();
}

// Two-stage deterministic reduction: every block writes its NA partial
// sums to partials[a * gridDim.x + blockIdx.x]; the last block to arrive
// (atomic ticket, no waiting) sums all partials in block order and calls
// fin(totals) from thread 0, then re-arms the ticket.  The result does not
// depend on which block arrives last.
template <int NA, class Fin>
__device__ void grid_reduce_finish(double (&v)[NA], double* partials,
                                   unsigned int* ticket, const Fin& fin) {
    __shared__ bool am_last;
    block_sum<NA>(v);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int a = 0; a < NA; ++a) partials[(size_t)a * gridDim.x + blockIdx.x] = v[a];
        __threadfence();
        unsigned t = atomicAdd(ticket, 1u);
        am_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    double tot[NA];
#pragma unroll
    for (int a = 0; a < NA; ++a) {
        double s = 0.0;
        for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x)
            s += __ldcg(partials + (size_t)a * gridDim.x + b);
        tot[a] = s;
    }
    block_sum<NA>(tot);
    if (threadIdx.x == 0) {
        fin(tot);
        *ticket = 0u;
    }
}

}  // namespace gk
