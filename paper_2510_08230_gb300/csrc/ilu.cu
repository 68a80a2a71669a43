// ilu.cu - ILU(0) factorisation on the device, the preconditioner entry
// points (gk_precond_apply, gk_ilu_factors) and sparse triangular solves
// with a matrix's own triangles (gk_triangular_solve), which reuse the same
// setup (without the factorisation) and substitution kernels.
//
// Setup, once per matrix:
//  1. k_ilu_prep: strictly ascending columns, diagonal positions.
//  2. k_chunk_levels (L and U): the level of every chunk of rows in the
//     dependency graph of each substitution; a counting sort by level
//     (k_level_hist, k_level_scan, k_level_scatter) gives the claim order
//     of the substitution kernels and the widest level (their grid cap).
//  3. k_ilu_factor: the factorisation (the IKJ form of ILU(0): for every
//     row i, for every stored k < i in ascending order, l_ik = a_ik / u_kk,
//     then a_ij -= l_ik u_kj for every stored j > k of row k that row i
//     also stores) runs sync-free: one warp per row, rows claimed chunk by
//     chunk in the L claim order of 32-row chunks and in ascending order
//     inside a chunk (a topological order), so a row only waits (bounded) on
//     rows claimed before it.  Row i waits for row k to be final before it
//     reads u_kk and row k's upper part; the lanes then update row i's
//     entries for row k's columns in parallel (each entry is hit at most
//     once per k, and the k steps run in ascending order), so every entry
//     sees exactly the oracle's sequence of roundings.  Each update
//     a_ij - l_ik u_kj is one fused multiply-add.
//  4. k_ilu_store: factors rounded to the vector type, 1 / u_ii.
//  5. tune_chunks: the substitutions' chunk size and chunks per warp, timed.
//
// The factors are computed in double from the stored values and rounded
// once to the vector type (double for GK_F64, float otherwise).
#include "ilu.cuh"
#include "solve_engine.cuh"

namespace gk {

// strictly ascending columns, diagonal position, values widened to double
template <typename V>
__global__ void k_ilu_prep(int32_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                           const V* __restrict__ va, double* __restrict__ fac,
                           int32_t* __restrict__ dpos, unsigned* bad) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t d = -1;
        const int32_t b = rp[i], e = rp[i + 1];
        for (int32_t k = b; k < e; ++k) {
            const int32_t c = ci[k];
            if (k > b && c <= ci[k - 1]) atomicOr(bad, 1u);
            if (c == (int32_t)i) d = k;
            fac[k] = cvt<double>(va[k]);
        }
        if (d < 0) atomicOr(bad, 2u);
        dpos[i] = d;
    }
}

// Spin until *p != 0 (bounded as wait_flag); returns the value, 0 after a
// time-out.
__device__ __forceinline__ unsigned wait_nonzero(const unsigned* p, unsigned* err) {
    unsigned v = ld_acquire_u32(p);
    if (v) return v;
    const uint64_t t0 = globaltimer_ns();
    unsigned ns = 32;
    for (;;) {
        __nanosleep(ns);
        if (ns < 256) ns <<= 1;
        v = ld_relaxed_u32(p);
        if (v) return ld_acquire_u32(p);
        if (ld_relaxed_u32(err) != 0u) return 0u;
        if (globaltimer_ns() - t0 > WAIT_LIMIT_NS) {
            atomicExch(err, 1u);
            return 0u;
        }
    }
}

// lev[c] = 1 + the highest level among the chunks (of cs rows) chunk c
// depends on (L: columns left of the chunk; U: right of it); chunks claimed
// in solve order.  misc[0] claim counter, misc[1] wait ran out, misc[3] the
// highest level.
template <bool UP>
__global__ void __launch_bounds__(256)
k_chunk_levels(int32_t n, int32_t nch, int32_t cs, const int32_t* __restrict__ rp,
               const int32_t* __restrict__ ci, const int32_t* __restrict__ dpos, unsigned* lev,
               unsigned* misc) {
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    for (;;) {
        int c = 0;
        if (lane == 0) c = (int)atomicAdd(&misc[0], 1u);
        c = __shfl_sync(FULL, c, 0);
        if (c >= nch) break;
        const int32_t cc = UP ? nch - 1 - c : c;
        const int32_t c0 = cc * cs, c1 = min(c0 + cs, n);
        const int32_t i = c0 + lane;
        unsigned mx = 0;
        if (lane < cs && i < n) {
            const int32_t d = dpos[i];
            int32_t last = -1;
            if (!UP) {
                for (int32_t k = rp[i]; k < d; ++k) {
                    const int32_t j = ci[k];
                    if (j >= c0) break;
                    const int32_t cj = j / cs;
                    if (cj != last) {
                        mx = max(mx, wait_nonzero(lev + cj, &misc[1]));
                        last = cj;
                    }
                }
            } else {
                for (int32_t k = rp[i + 1] - 1; k > d; --k) {
                    const int32_t j = ci[k];
                    if (j < c1) break;
                    const int32_t cj = j / cs;
                    if (cj != last) {
                        mx = max(mx, wait_nonzero(lev + cj, &misc[1]));
                        last = cj;
                    }
                }
            }
        }
        mx = __reduce_max_sync(FULL, mx);
        if (lane == 0) {
            st_release_u32(lev + cc, mx + 1);
            atomicMax(&misc[3], mx + 1);
        }
    }
}

// cnt[l] = chunks on level l (levels 1..nch)
__global__ void k_level_hist(int32_t nch, const unsigned* __restrict__ lev, unsigned* cnt) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nch;
         c += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&cnt[lev[c]], 1u);
}

// In place exclusive scan of cnt[0, len), each count first rounded up to a
// multiple of pad, by one block of 1024 threads; *maxw = the largest
// (rounded) count, *total = the sum.
__global__ void __launch_bounds__(1024)
k_level_scan(int32_t len, int32_t pad, unsigned* cnt, unsigned* maxw, unsigned* total) {
    __shared__ unsigned wsum[32];
    __shared__ unsigned carry;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) carry = 0;
    unsigned mx = 0;
    __syncthreads();
    for (int32_t base = 0; base < len; base += 1024) {
        const int32_t k = base + tid;
        const unsigned v = k < len ? (cnt[k] + pad - 1) / pad * pad : 0u;
        mx = max(mx, v);
        unsigned incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) wsum[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            unsigned w = wsum[lane], wi = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned t = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += t;
            }
            wsum[lane] = wi - w;  // exclusive warp offsets
        }
        __syncthreads();
        const unsigned excl = carry + wsum[wid] + incl - v;
        if (k < len) cnt[k] = excl;
        __syncthreads();
        if (tid == 1023) carry = excl + v;
        __syncthreads();
    }
    mx = __reduce_max_sync(0xffffffffu, mx);
    if (lane == 0) atomicMax(maxw, mx);
    if (tid == 0) *total = carry;
}

// ord[start[lev[c]]++] = c (order inside a level is immaterial: no chunk
// depends on another of its level; the padding slots keep -1)
__global__ void k_level_scatter(int32_t nch, const unsigned* __restrict__ lev, unsigned* cursor,
                                int32_t* __restrict__ ord) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nch;
         c += (int64_t)gridDim.x * blockDim.x)
        ord[atomicAdd(&cursor[lev[c]], 1u)] = (int32_t)c;
}

// misc[0] claim counter, misc[1] wait ran out, misc[2] zero pivot
__global__ void __launch_bounds__(256)
k_ilu_factor(int32_t n, int32_t nch, int32_t cs, const int32_t* __restrict__ rp,
             const int32_t* __restrict__ ci, const int32_t* __restrict__ dpos,
             const int32_t* __restrict__ ord, double* fac, unsigned* done, unsigned* misc) {
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int64_t nclaim = (int64_t)nch * cs;
    for (;;) {
        int64_t c = 0;
        if (lane == 0) c = (int64_t)atomicAdd(&misc[0], 1u);
        c = __shfl_sync(FULL, c, 0);
        if (c >= nclaim) break;
        const int32_t i = ord[c / cs] * cs + (int32_t)(c % cs);
        if (i >= n) continue;  // past the last row of the last chunk
        const int32_t p1 = rp[i + 1], d = dpos[i];
        int ok = 1;
        for (int32_t pk = rp[i]; pk < d; ++pk) {
            const int32_t k = ci[pk];
            if (lane == 0 && ok) ok = wait_flag(done + k, 1u, &misc[1]) ? 1 : 0;
            ok = __shfl_sync(FULL, ok, 0);
            __syncwarp();  // row k's values, released by its warp, are read after the acquire
            const int32_t dk = dpos[k], ek = rp[k + 1];
            const double l = __ddiv_rn(__ldcg(fac + pk), __ldcg(fac + dk));
            for (int32_t q = dk + 1 + lane; q < ek; q += 32) {
                const int32_t j = ci[q];
                int32_t lo = pk + 1, hi = p1;  // j in row i's columns after k
                while (lo < hi) {
                    const int32_t mid = (lo + hi) >> 1;
                    if (ci[mid] < j) lo = mid + 1;
                    else hi = mid;
                }
                if (lo < p1 && ci[lo] == j)
                    fac[lo] = __fma_rn(-l, __ldcg(fac + q), __ldcg(fac + lo));
            }
            if (lane == 0) fac[pk] = l;
            __threadfence_block();
            __syncwarp();
        }
        if (lane == 0 && __ldcg(fac + d) == 0.0) atomicOr(&misc[2], 1u);
        __threadfence();
        __syncwarp();
        if (lane == 0) st_release_u32(done + i, 1u);
    }
}

// factors rounded to the vector type; the pivots' reciprocals 1 / u_ii
// computed in double and rounded once
// (*zero set when a diagonal value is 0)
template <typename T>
__global__ void k_ilu_store(int32_t n, int64_t nnz, const double* __restrict__ fac,
                            const int32_t* __restrict__ dpos, T* __restrict__ lu,
                            T* __restrict__ rdiag, unsigned* zero) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz;
         k += (int64_t)gridDim.x * blockDim.x)
        lu[k] = cvt<T>(fac[k]);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double d = fac[dpos[i]];
        if (d == 0.0) atomicOr(zero, 1u);
        rdiag[i] = cvt<T>(__ddiv_rn(1.0, d));
    }
}

static size_t ilu_sync_bytes() { return 2 * sizeof(TrsvSync); }


// Grid of `kernel` (256 threads) when each of `items` needs one warp, at
// most the resident blocks.
template <typename K>
static unsigned resident_grid(K kernel, int64_t items) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, 256, 0) != cudaSuccess || b < 1)
        b = 1;
    const int64_t need = (items + 7) / 8;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)num_sms() * b));
}

// Dependency levels of the L (up = false) or U graph of cs-row chunks into
// lev (nch entries); *nlev = the number of levels.
static gk_status chunk_levels(const TriStore* S, int32_t n, int32_t cs, bool up, DevBuf& lev,
                              unsigned* nlev, cudaStream_t s) {
    const int32_t nch = (n + cs - 1) / cs;
    DevBuf misc;
    GK_TRY(lev.ensure(sizeof(unsigned) * (size_t)nch));
    GK_TRY(misc.ensure(64));
    GK_CUDA(cudaMemsetAsync(lev.ptr, 0, sizeof(unsigned) * (size_t)nch, s));
    GK_CUDA(cudaMemsetAsync(misc.ptr, 0, 64, s));
    unsigned* mp = (unsigned*)misc.ptr;
    if (up)
        k_chunk_levels<true><<<resident_grid(k_chunk_levels<true>, nch), 256, 0, s>>>(
            n, nch, cs, S->rp, S->ci, S->dpos, (unsigned*)lev.ptr, mp);
    else
        k_chunk_levels<false><<<resident_grid(k_chunk_levels<false>, nch), 256, 0, s>>>(
            n, nch, cs, S->rp, S->ci, S->dpos, (unsigned*)lev.ptr, mp);
    GK_CUDA(cudaGetLastError());
    unsigned h[4] = {0, 0, 0, 0};
    GK_CUDA(cudaMemcpyAsync(h, mp, sizeof(h), cudaMemcpyDeviceToHost, s));
    GK_CUDA(cudaStreamSynchronize(s));
    misc.release();
    if (h[1]) return GK_ERR_TIMEOUT;
    *nlev = h[3];
    return GK_OK;
}

// The claim order of nch chunks with levels lev: sorted by level into ord,
// each level's run padded to a multiple of pad with -1 (at most
// nch + (pad - 1) * levels entries; ord holds cap entries, at least that);
// *nord = its length, *maxw = the widest padded level.
static gk_status level_order(int32_t nch, int32_t pad, const DevBuf& lev, int32_t* ord,
                             size_t cap, unsigned* maxw, unsigned* nord, cudaStream_t s) {
    DevBuf cnt, misc;
    GK_TRY(cnt.ensure(sizeof(unsigned) * ((size_t)nch + 2)));
    GK_TRY(misc.ensure(64));
    GK_CUDA(cudaMemsetAsync(cnt.ptr, 0, sizeof(unsigned) * ((size_t)nch + 2), s));
    GK_CUDA(cudaMemsetAsync(misc.ptr, 0, 64, s));
    unsigned* mp = (unsigned*)misc.ptr;
    const unsigned g = ew_grid(nch);
    k_level_hist<<<g, 256, 0, s>>>(nch, (const unsigned*)lev.ptr, (unsigned*)cnt.ptr);
    k_level_scan<<<1, 1024, 0, s>>>(nch + 2, pad, (unsigned*)cnt.ptr, mp + 2, mp + 4);
    GK_CUDA(cudaMemsetAsync(ord, 0xFF, sizeof(int32_t) * std::min(cap, (size_t)pad * nch), s));
    k_level_scatter<<<g, 256, 0, s>>>(nch, (const unsigned*)lev.ptr, (unsigned*)cnt.ptr, ord);
    GK_CUDA(cudaGetLastError());
    unsigned h[5] = {0, 0, 0, 0, 0};
    GK_CUDA(cudaMemcpyAsync(h, mp, sizeof(h), cudaMemcpyDeviceToHost, s));
    GK_CUDA(cudaStreamSynchronize(s));
    cnt.release();
    misc.release();
    *maxw = h[2];
    *nord = h[4];
    return GK_OK;
}

// Chunk levels of both triangles for the two chunk sizes (32 and 8 rows),
// computed once per matrix and shared by the factorisation order and every
// substitution candidate.
struct IluLevels {
    DevBuf l32, u32, l8, u8, l1, u1;
    unsigned nl32 = 0, nu32 = 0, nl8 = 0, nu8 = 0, nl1 = 0, nu1 = 0;
    const DevBuf& get(int cs, bool up) const {
        return cs == 32 ? (up ? u32 : l32) : cs == 8 ? (up ? u8 : l8) : (up ? u1 : l1);
    }
    unsigned levels(int cs, bool up) const {
        return cs == 32 ? (up ? nu32 : nl32) : cs == 8 ? (up ? nu8 : nl8) : (up ? nu1 : nl1);
    }
    ~IluLevels() {
        for (DevBuf* b : {&l32, &u32, &l8, &u8, &l1, &u1}) b->release();
    }
};

// Level-synchronous mode: the rows of each triangle in level order (the
// counting sort of their row levels, no padding) and the first position of
// every level.  Levels are numbered 1..nlev (every level holds a row);
// level l starts at start[l - 1], and start[nlev] = n.
__global__ void k_level_starts(int32_t n, const int32_t* __restrict__ rows,
                               const unsigned* __restrict__ lev, int32_t* __restrict__ start,
                               int32_t nlev) {
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const unsigned l = lev[rows[idx]];
        if (idx == 0 || lev[rows[idx - 1]] != l) start[l - 1] = (int32_t)idx;
        if (idx == n - 1) start[nlev] = n;
    }
}

// ---------------------------------------------------- window-mode records
__global__ void k_scatter_pos(int32_t n, const int32_t* __restrict__ rows, int32_t* __restrict__ pos) {
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
         idx += (int64_t)gridDim.x * blockDim.x)
        pos[rows[idx]] = (int32_t)idx;
}

// most terms of a row and deepest dependency (in levels) of one triangle
template <bool UP>
__global__ void k_win_check(int32_t n, const unsigned* __restrict__ lev,
                            const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                            const int32_t* __restrict__ dpos, unsigned* out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t d = dpos[i];
        const int32_t k0 = UP ? d + 1 : rp[i], k1 = UP ? rp[i + 1] : d;
        unsigned md = 0;
        for (int32_t k = k0; k < k1; ++k) md = max(md, lev[i] - lev[ci[k]]);
        atomicMax(out, (unsigned)(k1 - k0));
        atomicMax(out + 1, md);
    }
}

// record of level-ordered row idx: its terms in substitution order, each
// with the block that owns its source row in the source's level, how many
// levels back that is, and the source's index in the block's share
template <typename T, bool UP>
__global__ void k_win_rec(int32_t n, const int32_t* __restrict__ rows,
                          const unsigned* __restrict__ lev, const int32_t* __restrict__ pos,
                          const int32_t* __restrict__ start, const int32_t* __restrict__ rp,
                          const int32_t* __restrict__ ci, const int32_t* __restrict__ dpos,
                          const T* __restrict__ lu, const T* __restrict__ rdiag,
                          WinRec<T>* __restrict__ rec) {
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int32_t i = rows[idx];
        const int32_t d = dpos[i];
        WinRec<T> R;
        R.rd = rdiag[i];
        for (int t = 0; t < WIN_MAXT; ++t) {
            R.co[t] = -1;
            R.v[t] = T(0);
        }
        // L: ascending from the row start; U: descending from the row end
        const int32_t nt = UP ? rp[i + 1] - 1 - d : d - rp[i];
        for (int32_t t = 0; t < nt && t < WIN_MAXT; ++t) {
            const int32_t k = UP ? rp[i + 1] - 1 - t : rp[i] + t;
            const int32_t j = ci[k];
            const int32_t lj = (int32_t)lev[j] - 1;  // levels are 1-based
            const int32_t s0 = start[lj], len = start[lj + 1] - s0;
            const int32_t per = (len + WIN_BLOCKS - 1) / WIN_BLOCKS;
            const int32_t q = pos[j] - s0, r = q / per;
            R.co[t] = (int16_t)((r << (WIN_IDX_BITS + 1)) |
                                ((int32_t)(lev[i] - lev[j] - 1) << WIN_IDX_BITS) | (q - r * per));
            R.v[t] = lu[k];
        }
        rec[idx] = R;
    }
}

// Builds the window-mode data when the matrix qualifies (at most WIN_MAXT
// terms a row and dependencies at most WIN_MAXD levels back in each
// triangle, at most WIN_CAP rows of a level per block); *ok = false
// otherwise.  Needs the row levels (build_row_levels).
template <typename T>
static gk_status build_win(TriStore* S, int32_t n, const IluLevels& lv, cudaStream_t s, bool* ok) {
    *ok = false;
    if (n == 0) return GK_OK;
    {  // the cluster must fit: WIN_BLOCKS blocks with their shared memory
        auto k = k_ilu_trsv_win<T, false, IluOutStore<T>, IluSkipNever, IluNoErr>;
        GK_TRY(win_attributes<T>(k));
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(WIN_BLOCKS, 1, 1);
        cfg.blockDim = dim3(WIN_THREADS, 1, 1);
        cfg.dynamicSmemBytes = WinSmem<T>::bytes;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = WIN_BLOCKS;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int nc = 0;
        if (cudaOccupancyMaxActiveClusters(&nc, k, &cfg) != cudaSuccess || nc < 1) {
            (void)cudaGetLastError();
            return GK_OK;
        }
    }
    const unsigned* lev[2] = {(const unsigned*)lv.l1.ptr, (const unsigned*)lv.u1.ptr};
    // shares per block: from the level starts
    for (int u = 0; u < 2; ++u) {
        std::vector<int32_t> h((size_t)S->nlev[u] + 1);
        const int32_t* st = S->lstart + (u ? S->nlev[0] + 1 : 0);
        GK_CUDA(cudaMemcpyAsync(h.data(), st, sizeof(int32_t) * h.size(), cudaMemcpyDeviceToHost, s));
        GK_CUDA(cudaStreamSynchronize(s));
        for (int32_t L = 0; L < S->nlev[u]; ++L)
            if ((h[L + 1] - h[L] + WIN_BLOCKS - 1) / WIN_BLOCKS > WIN_CAP) return GK_OK;
    }
    DevBuf chk;
    GK_TRY(chk.ensure(16));
    GK_CUDA(cudaMemsetAsync(chk.ptr, 0, 16, s));
    unsigned* cp = (unsigned*)chk.ptr;
    const unsigned g = ew_grid(n);
    k_win_check<false><<<g, 256, 0, s>>>(n, lev[0], S->rp, S->ci, S->dpos, cp);
    k_win_check<true><<<g, 256, 0, s>>>(n, lev[1], S->rp, S->ci, S->dpos, cp + 2);
    GK_CUDA(cudaGetLastError());
    unsigned h[4];
    GK_CUDA(cudaMemcpyAsync(h, cp, sizeof(h), cudaMemcpyDeviceToHost, s));
    GK_CUDA(cudaStreamSynchronize(s));
    chk.release();
    if (h[0] > WIN_MAXT || h[2] > WIN_MAXT || h[1] > WIN_MAXD || h[3] > WIN_MAXD) return GK_OK;
    if (!S->wrec) GK_CUDA(dmalloc(&S->wrec, 2 * sizeof(WinRec<T>) * (size_t)n));
    // the kernel's input copies are widened to 16-byte boundaries
    if (!S->wperm) GK_CUDA(dmalloc(&S->wperm, sizeof(T) * ((size_t)n + WinSmem<T>::AL)));
    DevBuf pos;
    GK_TRY(pos.ensure(sizeof(int32_t) * (size_t)n));
    int32_t* pp = (int32_t*)pos.ptr;
    WinRec<T>* rec = static_cast<WinRec<T>*>(S->wrec);
    for (int u = 0; u < 2; ++u) {
        const int32_t* rows = S->lrows + (u ? n : 0);
        const int32_t* st = S->lstart + (u ? S->nlev[0] + 1 : 0);
        k_scatter_pos<<<g, 256, 0, s>>>(n, rows, pp);
        if (u)
            k_win_rec<T, true><<<g, 256, 0, s>>>(n, rows, lev[1], pp, st, S->rp, S->ci, S->dpos,
                                                (const T*)S->lu, (const T*)S->rdiag, rec + n);
        else
            k_win_rec<T, false><<<g, 256, 0, s>>>(n, rows, lev[0], pp, st, S->rp, S->ci, S->dpos,
                                                 (const T*)S->lu, (const T*)S->rdiag, rec);
    }
    GK_CUDA(cudaGetLastError());
    GK_CUDA(cudaStreamSynchronize(s));
    pos.release();
    S->wdist[0] = (int32_t)std::max(1u, h[1]);
    S->wdist[1] = (int32_t)std::max(1u, h[3]);
    *ok = true;
    return GK_OK;
}

static gk_status build_row_levels(TriStore* S, int32_t n, const IluLevels& lv, cudaStream_t s) {
    if (S->lrows) return GK_OK;
    const size_t nl = lv.nl1, nu = lv.nu1;
    GK_CUDA(dmalloc_t(&S->lrows, 2 * (size_t)std::max(n, 1)));
    GK_CUDA(dmalloc_t(&S->lstart, nl + nu + 2));
    unsigned mw = 0, no = 0;
    GK_TRY(level_order(n, 1, lv.l1, S->lrows, (size_t)n, &mw, &no, s));
    if (no != (unsigned)n) return GK_ERR_CUDA;
    GK_TRY(level_order(n, 1, lv.u1, S->lrows + n, (size_t)n, &mw, &no, s));
    if (no != (unsigned)n) return GK_ERR_CUDA;
    const unsigned g = ew_grid(n);
    k_level_starts<<<g, 256, 0, s>>>(n, S->lrows, (const unsigned*)lv.l1.ptr, S->lstart, (int32_t)nl);
    k_level_starts<<<g, 256, 0, s>>>(n, S->lrows + n, (const unsigned*)lv.u1.ptr, S->lstart + nl + 1,
                                     (int32_t)nu);
    GK_CUDA(cudaGetLastError());
    S->nlev[0] = (int32_t)nl;
    S->nlev[1] = (int32_t)nu;
    return GK_OK;
}

// claim-order entries S->ord holds (both directions)
static size_t ord_capacity(int32_t n) { return 2 * 4 * (size_t)std::max((n + 7) / 8, 1); }

template <typename T>
static IluDev<T> tri_view(const TriStore* S, int32_t n) {
    IluDev<T> f;
    f.n = n;
    f.cs = S->cs;
    f.cpw = S->cpw;
    f.nch = (n + f.cs - 1) / f.cs;
    f.rp = S->rp;
    f.ci = S->ci;
    f.dpos = S->dpos;
    f.lu = (const T*)S->lu;
    f.rdiag = (const T*)S->rdiag;
    f.ord_l = S->ord;
    f.ord_u = S->ord + S->nord[0];
    f.nord[0] = S->nord[0];
    f.nord[1] = S->nord[1];
    f.warps[0] = S->warps[0];
    f.warps[1] = S->warps[1];
    f.sy = (TrsvSync*)S->sync;
    if (const char* e = getenv("GK_ILU_PAUSE")) f.pause_max = (unsigned)std::max(32, atoi(e));
    f.lvl = S->lvl;
    f.lrows[0] = S->lrows;
    f.lrows[1] = S->lrows ? S->lrows + n : nullptr;
    f.lstart[0] = S->lstart;
    f.lstart[1] = S->lstart ? S->lstart + S->nlev[0] + 1 : nullptr;
    f.nlev[0] = S->nlev[0];
    f.nlev[1] = S->nlev[1];
    f.win = S->win;
    f.wdist[0] = S->wdist[0];
    f.wdist[1] = S->wdist[1];
    f.wrec[0] = S->wrec;
    f.wrec[1] = S->wrec ? static_cast<const char*>(S->wrec) + sizeof(WinRec<T>) * (size_t)n : nullptr;
    f.wperm = static_cast<T*>(S->wperm);
    return f;
}

template <typename T>
IluDev<T> ilu_view(gk_matrix A) {
    return tri_view<T>(A->ilu, A->n);
}
template IluDev<double> ilu_view<double>(gk_matrix);
template IluDev<float> ilu_view<float>(gk_matrix);

// Rows per substitution chunk and chunks per warp, timed per matrix:
// 32-row chunks need the fewest dependency levels, 8-row chunks the
// shortest chain inside a chunk; four 8-row chunks to a warp need 4x fewer
// warps but move in step.  Single-row chunks, 32 to a warp (rows of one
// dependency level, so a warp's rows never wait on each other), remove the
// chain inside a chunk altogether: a level costs one hand-off; they are a
// candidate when the row levels are wide enough (the padded claim order at
// most twice n).  Which wins depends on the pattern (measured on GB300,
// FP64: the 128^3 diffusion matrix 3.05 ms with 32 rows, 3.26 with four
// 8-row chunks a warp; the 2D 5-point Laplacian 1024^2 17.4 ms, 10.4 with
// one 8-row chunk a warp, 12.5 with four).  Each candidate gets its claim
// orders, grid caps and one timed application (after a warm-up one) of
// z = M^-1 d with d = 1/u_ii; the fastest is kept.  GK_ILU_CHUNK (8 or 32,
// one chunk a warp; 1: single rows, 32 a warp; lvl: the level-synchronous
// cluster kernel) forces a shape.  Results never depend on the choice,
// only the time does.
template <typename T>
static gk_status tune_chunks(TriStore* S, int32_t n, const IluLevels& lv, cudaStream_t s) {
    int forced = 0;
    bool forced_lvl = false, forced_win = false;
    if (const char* e = getenv("GK_ILU_CHUNK")) {
        const int v = atoi(e);
        if (v == 1 || v == 8 || v == 32) forced = v;
        // the chunk state stays valid under a forced level-synchronous mode
        if (!strcmp(e, "lvl")) forced_lvl = true, forced = 32;
        if (!strcmp(e, "win")) forced_win = true, forced = 32;
    }
    int64_t mult = 2;
    if (const char* e = getenv("GK_ILU_WARPS")) mult = std::max(1, atoi(e));
    const int all_cs[4] = {32, 8, 8, 1}, all_cpw[4] = {1, 1, 4, 32};
    // single-row chunks only when their padded claim orders stay within 2n
    const bool rows_ok = (size_t)n + 31 * (size_t)std::max(lv.nl1, lv.nu1) <= 2 * (size_t)n;
    const int ncand = forced ? 1 : rows_ok ? 4 : 3;
    DevBuf ordb[4], tmp;
    int32_t warps[4][2] = {}, nord[4][2] = {};
    GK_TRY(tmp.ensure(2 * sizeof(T) * (size_t)n));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    GK_CUDA(cudaEventCreate(&e0));
    GK_CUDA(cudaEventCreate(&e1));
    gk_status st = GK_OK;
    float best = 0.f;
    int pick = 0;
    for (int k = 0; k < ncand && st == GK_OK; ++k) {
        const int32_t cs = forced ? forced : all_cs[k];
        const int32_t cpw = forced ? (forced == 1 ? 32 : 1) : all_cpw[k];
        const int32_t nch = (n + cs - 1) / cs;
        // claim-order entries at most, per direction: every level padded
        const size_t cap = std::min((size_t)cpw * nch,
                                    (size_t)nch + (size_t)(cpw - 1) *
                                                      std::max(lv.levels(cs, false),
                                                               lv.levels(cs, true)));
        unsigned wl = 0, wu = 0, nl = 0, nu = 0;
        st = ordb[k].ensure(2 * sizeof(int32_t) * cap);
        int32_t* ob = (int32_t*)ordb[k].ptr;
        if (st == GK_OK) st = level_order(nch, cpw, lv.get(cs, false), ob, cap, &wl, &nl, s);
        if (st == GK_OK)
            st = level_order(nch, cpw, lv.get(cs, true), ob + nl, cap, &wu, &nu, s);
        if (st != GK_OK) break;
        nord[k][0] = (int32_t)nl;
        nord[k][1] = (int32_t)nu;
        // warps: a few times the widest level, in warps of cpw chunks
        warps[k][0] = (int32_t)std::min<int64_t>(std::max<int64_t>(64, mult * (int64_t)wl / cpw), nl / cpw);
        warps[k][1] = (int32_t)std::min<int64_t>(std::max<int64_t>(64, mult * (int64_t)wu / cpw), nu / cpw);
        if (ncand == 1) break;
        IluDev<T> f = tri_view<T>(S, n);
        f.cs = cs;
        f.cpw = cpw;
        f.nch = nch;
        f.ord_l = ob;
        f.ord_u = ob + nl;
        f.nord[0] = nord[k][0];
        f.nord[1] = nord[k][1];
        f.warps[0] = warps[k][0];
        f.warps[1] = warps[k][1];
        T* w = (T*)tmp.ptr;
        const IluSrc<T> src{(const T*)S->rdiag};
        float ms = 0.f;
        st = ilu_apply<T>(f, src, w, IluOutStore<T>{w + n}, IluSkipNever{}, IluNoErr{}, s);
        if (st == GK_OK && cudaEventRecord(e0, s) != cudaSuccess) st = GK_ERR_CUDA;
        if (st == GK_OK)
            st = ilu_apply<T>(f, src, w, IluOutStore<T>{w + n}, IluSkipNever{}, IluNoErr{}, s);
        if (st == GK_OK && (cudaEventRecord(e1, s) != cudaSuccess ||
                            cudaEventSynchronize(e1) != cudaSuccess ||
                            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
            st = GK_ERR_CUDA;
        if (st == GK_OK && (k == 0 || ms < best)) {
            best = ms;
            pick = k;
        }
    }
    // the level-synchronous mode (one cluster, a barrier per row level):
    // only when forced -- it measured slower than the chunked kernel on
    // every matrix tried (GB300, FP64: 128^3 diffusion 4.70 against 2.81 ms
    // per application, 2D Laplacian 1024^2 13.2 against 9.5 ms, power-law
    // n = 2^21 with a dominant diagonal 76 against 12 ms): a level costs
    // ~6 us, the L2 round trips of its row data and unknowns plus the
    // barrier's release of its stores
    bool lvl = false;
    if (st == GK_OK && forced_lvl) {
        gk_status ls = build_row_levels(S, n, lv, s);
        float ms = 0.f;
        if (ls == GK_OK) {
            IluDev<T> f = tri_view<T>(S, n);
            f.lvl = 1;
            T* w = (T*)tmp.ptr;
            const IluSrc<T> src{(const T*)S->rdiag};
            ls = ilu_apply<T>(f, src, w, IluOutStore<T>{w + n}, IluSkipNever{}, IluNoErr{}, s);
            if (ls == GK_OK && cudaEventRecord(e0, s) != cudaSuccess) ls = GK_ERR_CUDA;
            if (ls == GK_OK)
                ls = ilu_apply<T>(f, src, w, IluOutStore<T>{w + n}, IluSkipNever{}, IluNoErr{}, s);
            if (ls == GK_OK && (cudaEventRecord(e1, s) != cudaSuccess ||
                                cudaEventSynchronize(e1) != cudaSuccess ||
                                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
                ls = GK_ERR_CUDA;
        }
        if (ls != GK_OK) {
            cudaGetLastError();  // a cluster that cannot be scheduled: keep the chunks
            if (forced_lvl) st = ls;
        } else {
            lvl = forced_lvl || ms < best;
        }
    }
    // the window mode (stencil-like matrices, see k_ilu_trsv_win): timed
    // against the chunks when the matrix qualifies
    bool win = false;
    if (st == GK_OK && !lvl && (forced_win || !forced)) {
        bool ok = false;
        gk_status ws = build_row_levels(S, n, lv, s);
        if (ws == GK_OK) ws = build_win<T>(S, n, lv, s, &ok);
        float ms = 0.f;
        if (ws == GK_OK && ok) {
            IluDev<T> f = tri_view<T>(S, n);
            f.win = 1;
            T* w = (T*)tmp.ptr;
            const IluSrc<T> src{(const T*)S->rdiag};
            ws = ilu_apply<T>(f, src, w, IluOutStore<T>{w + n}, IluSkipNever{}, IluNoErr{}, s);
            if (ws == GK_OK && cudaEventRecord(e0, s) != cudaSuccess) ws = GK_ERR_CUDA;
            if (ws == GK_OK)
                ws = ilu_apply<T>(f, src, w, IluOutStore<T>{w + n}, IluSkipNever{}, IluNoErr{}, s);
            if (ws == GK_OK && (cudaEventRecord(e1, s) != cudaSuccess ||
                                cudaEventSynchronize(e1) != cudaSuccess ||
                                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
                ws = GK_ERR_CUDA;
        }
        if (ws != GK_OK) {
            cudaGetLastError();  // a cluster that cannot be scheduled: keep the chunks
            if (forced_win) st = ws;
        } else if (ok) {
            win = forced_win || ms < best;
        }
        if (!win) {  // not picked: its records go
            dfree(S->wrec);
            dfree(S->wperm);
            S->wrec = S->wperm = nullptr;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != GK_OK) return st;
    S->lvl = lvl ? 1 : 0;
    S->win = win ? 1 : 0;
    TrsvSync h[2];
    GK_CUDA(cudaMemcpyAsync(h, S->sync, sizeof(h), cudaMemcpyDeviceToHost, s));
    GK_CUDA(cudaStreamSynchronize(s));
    if (h[0].err | h[1].err) return GK_ERR_TIMEOUT;
    const int32_t cs = forced ? forced : all_cs[pick];
    const int32_t cpw = forced ? (forced == 1 ? 32 : 1) : all_cpw[pick];
    const size_t need = (size_t)nord[pick][0] + nord[pick][1];
    if (need > ord_capacity(n)) {  // single-row chunks: a longer claim order
        dfree(S->ord);
        S->ord = nullptr;
        GK_CUDA(dmalloc_t(&S->ord, need));
    }
    GK_CUDA(cudaMemcpyAsync(S->ord, ordb[pick].ptr,
                            sizeof(int32_t) * ((size_t)nord[pick][0] + nord[pick][1]),
                            cudaMemcpyDeviceToDevice, s));
    GK_CUDA(cudaStreamSynchronize(s));
    S->cs = cs;
    S->cpw = cpw;
    S->nord[0] = nord[pick][0];
    S->nord[1] = nord[pick][1];
    S->warps[0] = std::max(1, warps[pick][0]);
    S->warps[1] = std::max(1, warps[pick][1]);
    return GK_OK;
}

// Builds S for the CSR matrix C with values rounded to the vector type of
// vdt.  factorize: the ILU(0) factors (a missing diagonal or zero pivot is
// GK_ERR_ZERO_DIAG); otherwise C's own values, for triangular solves (a
// missing diagonal is GK_ERR_INVALID, a zero one is recorded in
// S->zero_diag).
static gk_status tri_build(TriStore* S, gk_dtype vdt, gk_matrix C, bool factorize,
                           cudaStream_t s) {
    const int32_t n = C->n;
    const int64_t nnz = C->nnz;
    const size_t vb = vector_bytes(vdt);
    GK_CUDA(dmalloc_t(&S->rp, (size_t)n + 1));
    GK_CUDA(dmalloc_t(&S->ci, (size_t)std::max<int64_t>(nnz, 1)));
    GK_CUDA(dmalloc_t(&S->dpos, (size_t)std::max(n, 1)));
    GK_CUDA(dmalloc(&S->lu, vb * (size_t)std::max<int64_t>(nnz, 1)));
    GK_CUDA(dmalloc(&S->rdiag, vb * (size_t)std::max(n, 1)));
    GK_CUDA(dmalloc(&S->sync, ilu_sync_bytes()));
    // claim orders: at most 4 entries per 8-row chunk and direction (single-
    // row chunks, when picked, reallocate it)
    GK_CUDA(dmalloc_t(&S->ord, ord_capacity(n)));
    GK_CUDA(cudaMemcpyAsync(S->rp, C->row_ptr, sizeof(int32_t) * ((size_t)n + 1),
                            cudaMemcpyDeviceToDevice, s));
    if (nnz > 0)
        GK_CUDA(cudaMemcpyAsync(S->ci, C->col, sizeof(int32_t) * (size_t)nnz,
                                cudaMemcpyDeviceToDevice, s));
    // claim counters, exit counters and error flags start at 0
    GK_CUDA(cudaMemsetAsync(S->sync, 0, ilu_sync_bytes(), s));

    DevBuf fac, done, misc;
    GK_TRY(fac.ensure(sizeof(double) * (size_t)std::max<int64_t>(nnz, 1)));
    GK_TRY(done.ensure(sizeof(unsigned) * (size_t)std::max(n, 1)));
    GK_TRY(misc.ensure(64));
    GK_CUDA(cudaMemsetAsync(done.ptr, 0, sizeof(unsigned) * (size_t)std::max(n, 1), s));
    GK_CUDA(cudaMemsetAsync(misc.ptr, 0, 64, s));
    unsigned* mp = (unsigned*)misc.ptr;
    unsigned h[4] = {0, 0, 0, 0};
    if (n > 0) {
        const unsigned g = ew_grid(n);
        auto prep = [&](auto vt) {
            using V = decltype(vt);
            k_ilu_prep<V><<<g, 256, 0, s>>>(n, S->rp, S->ci, (const V*)C->val,
                                           (double*)fac.ptr, S->dpos, mp + 3);
        };
        if (C->dtype == GK_F64) prep(double());
        else if (C->dtype == GK_F32) prep(float());
        else if (C->dtype == GK_F16) prep(__half());
        else prep(__nv_bfloat16());
        GK_CUDA(cudaGetLastError());
        GK_CUDA(cudaMemcpyAsync(h, mp, sizeof(h), cudaMemcpyDeviceToHost, s));
        GK_CUDA(cudaStreamSynchronize(s));
        if (h[3] & 1u) return GK_ERR_INVALID;
        if (h[3] & 2u) return factorize ? GK_ERR_ZERO_DIAG : GK_ERR_INVALID;
        // chunk levels for both sizes and directions, once
        IluLevels lv;
        GK_TRY(chunk_levels(S, n, 32, false, lv.l32, &lv.nl32, s));
        GK_TRY(chunk_levels(S, n, 32, true, lv.u32, &lv.nu32, s));
        GK_TRY(chunk_levels(S, n, 8, false, lv.l8, &lv.nl8, s));
        GK_TRY(chunk_levels(S, n, 8, true, lv.u8, &lv.nu8, s));
        GK_TRY(chunk_levels(S, n, 1, false, lv.l1, &lv.nl1, s));
        GK_TRY(chunk_levels(S, n, 1, true, lv.u1, &lv.nu1, s));
        if (factorize) {
            // rows claimed chunk by chunk in the L level order of 32-row chunks
            const int32_t cs = 32, nch = (n + cs - 1) / cs;
            unsigned wl = 0, nl = 0;
            GK_TRY(level_order(nch, 1, lv.l32, S->ord, (size_t)nch, &wl, &nl, s));
            k_ilu_factor<<<resident_grid(k_ilu_factor,
                                         std::min<int64_t>(n, 2 * (int64_t)cs * wl + 256)),
                           256, 0, s>>>(n, nch, cs, S->rp, S->ci, S->dpos, S->ord,
                                        (double*)fac.ptr, (unsigned*)done.ptr, mp);
            GK_CUDA(cudaGetLastError());
            GK_CUDA(cudaMemcpyAsync(h, mp, sizeof(h), cudaMemcpyDeviceToHost, s));
            GK_CUDA(cudaStreamSynchronize(s));
            if (h[1]) return GK_ERR_TIMEOUT;
            if (h[2]) return GK_ERR_ZERO_DIAG;
        }
        GK_CUDA(cudaMemsetAsync(mp + 2, 0, sizeof(unsigned), s));
        if (vdt == GK_F64)
            k_ilu_store<double><<<ew_grid(nnz), 256, 0, s>>>(n, nnz, (const double*)fac.ptr,
                                                             S->dpos, (double*)S->lu,
                                                             (double*)S->rdiag, mp + 2);
        else
            k_ilu_store<float><<<ew_grid(nnz), 256, 0, s>>>(n, nnz, (const double*)fac.ptr,
                                                            S->dpos, (float*)S->lu,
                                                            (float*)S->rdiag, mp + 2);
        GK_CUDA(cudaGetLastError());
        GK_CUDA(cudaMemcpyAsync(h, mp, sizeof(h), cudaMemcpyDeviceToHost, s));
        GK_CUDA(cudaStreamSynchronize(s));
        S->zero_diag = h[2] != 0;
        GK_TRY(vdt == GK_F64 ? tune_chunks<double>(S, n, lv, s) : tune_chunks<float>(S, n, lv, s));
    }
    GK_CUDA(cudaStreamSynchronize(s));
    return GK_OK;
}

// The TriStore *slot of A (ILU factors or raw triangles), built on first use.
static gk_status ensure_store(gk_matrix A, TriStore** slot, bool factorize, cudaStream_t s) {
    if (*slot && (*slot)->state == 1) return GK_OK;
    if (*slot && (*slot)->state < 0) return (gk_status)(*slot)->state;
    if (A->n != A->ncols) return GK_ERR_INVALID;
    if (!*slot) {
        *slot = new (std::nothrow) TriStore();
        if (!*slot) return GK_ERR_OOM;
    }
    TriStore* S = *slot;
    gk_matrix C = A, tmp = nullptr;
    if (A->fmt != GK_CSR) {
        GK_TRY(gk_matrix_convert(A, GK_CSR, A->dtype, 0, 0, s, &tmp));
        C = tmp;
    }
    const gk_status st = tri_build(S, A->dtype, C, factorize, s);
    if (tmp) gk_matrix_destroy(tmp);
    if (st != GK_OK) {
        cudaStreamSynchronize(s);
        S->release();
        // a malformed or singular pattern stays so; other failures may be retried
        if (st == GK_ERR_INVALID || st == GK_ERR_ZERO_DIAG) S->state = (int)st;
        return st;
    }
    S->state = 1;
    return GK_OK;
}

gk_status ensure_ilu(gk_matrix A, cudaStream_t s) { return ensure_store(A, &A->ilu, true, s); }

template <typename T>
__global__ void EW_BOUNDS k_scale_by(int32_t n, const T* __restrict__ d, const T* __restrict__ r,
                                     T* __restrict__ z) {
    GRID_LOOP(i, n) z[i] = d[i] * r[i];
}

template <typename T>
static gk_status precond_apply_t(gk_matrix A, int kind, int32_t bs, const T* r, T* z,
                                 uint64_t wait_ns, cudaStream_t s) {
    const int32_t n = A->n;
    if (kind == GK_PRECOND_NONE) {
        if (n > 0 && z != r)
            GK_CUDA(cudaMemcpyAsync(z, r, sizeof(T) * (size_t)n, cudaMemcpyDeviceToDevice, s));
        return GK_OK;
    }
    if (kind == GK_PRECOND_JACOBI) {
        GK_TRY(ensure_jacobi(A, s));
        if (n > 0) k_scale_by<T><<<ewg(k_scale_by<T>, n), 256, 0, s>>>(n, (const T*)A->dinv, r, z);
        GK_CUDA(cudaGetLastError());
        return GK_OK;
    }
    if (kind == GK_PRECOND_BLOCK_JACOBI) {
        GK_TRY(ensure_block_jacobi(A, bs, s));
        if (n > 0)
            k_bj_apply<T, EpiStoreHalt<T>><<<ewg(k_bj_apply<T, EpiStoreHalt<T>>, n), 256, 0, s>>>(
                n, bs, (const T*)A->binv, r, EpiStoreHalt<T>{z, nullptr});
        GK_CUDA(cudaGetLastError());
        return GK_OK;
    }
    GK_TRY(ensure_ilu(A, s));
    if (n == 0) return GK_OK;
    GK_TRY(A->ilu->w.ensure(sizeof(T) * (size_t)n));
    IluDev<T> f = ilu_view<T>(A);
    f.wait_ns = wait_ns;
    GK_TRY(ilu_clear_err(f, s));
    GK_TRY(ilu_apply<T>(f, IluSrc<T>{r}, (T*)A->ilu->w.ptr, IluOutStore<T>{z}, IluSkipNever{},
                        IluNoErr{}, s));
    TrsvSync h[2];
    GK_CUDA(cudaMemcpyAsync(h, f.sy, sizeof(h), cudaMemcpyDeviceToHost, s));
    GK_CUDA(cudaStreamSynchronize(s));
    if (h[0].err | h[1].err) return GK_ERR_TIMEOUT;
    return GK_OK;
}

// T x = b with A's lower (upper = 0) or upper triangle; unit: unit diagonal.
template <typename T>
static gk_status tri_solve_t(gk_matrix A, int upper, int unit, const T* b, T* x,
                             uint64_t wait_ns, cudaStream_t s) {
    GK_TRY(ensure_store(A, &A->tri, false, s));
    if (!unit && A->tri->zero_diag) return GK_ERR_ZERO_DIAG;
    if (A->n == 0) return GK_OK;
    IluDev<T> f = tri_view<T>(A->tri, A->n);
    f.wait_ns = wait_ns;
    f.ldiag = (!upper && !unit) ? 1 : 0;
    f.udiag = unit ? 0 : 1;
    GK_TRY(ilu_clear_err(f, s));
    GK_TRY(tri_apply<T>(f, upper != 0, b, x, s));
    TrsvSync h[2];
    GK_CUDA(cudaMemcpyAsync(h, f.sy, sizeof(h), cudaMemcpyDeviceToHost, s));
    GK_CUDA(cudaStreamSynchronize(s));
    if (h[0].err | h[1].err) return GK_ERR_TIMEOUT;
    return GK_OK;
}

}  // namespace gk

using namespace gk;

extern "C" gk_status gk_triangular_solve(gk_matrix A, int upper, int unit_diagonal, const void* b,
                                         void* x, int64_t wait_budget_ns, void* stream) {
    if (!A || ((!b || !x) && A->n > 0)) return GK_ERR_INVALID;
    if (wait_budget_ns < 0) return GK_ERR_INVALID;
    const uint64_t wb = wait_budget_ns > 0 ? (uint64_t)wait_budget_ns : WAIT_LIMIT_NS;
    if (A->n != A->ncols) return GK_ERR_INVALID;
    if (A->n > 0 && b == x) return GK_ERR_INVALID;
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != A->device) return GK_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(A->mu);
    cudaStream_t s = (cudaStream_t)stream;
    if (A->dtype == GK_F64)
        return tri_solve_t<double>(A, upper, unit_diagonal, (const double*)b, (double*)x, wb, s);
    return tri_solve_t<float>(A, upper, unit_diagonal, (const float*)b, (float*)x, wb, s);
}

extern "C" gk_status gk_precond_apply(gk_matrix A, gk_precond kind, int32_t block_size,
                                      const void* r, void* z, int64_t wait_budget_ns,
                                      void* stream) {
    if (!A || (!r && A->n > 0) || (!z && A->n > 0)) return GK_ERR_INVALID;
    if (wait_budget_ns < 0) return GK_ERR_INVALID;
    const uint64_t wb = wait_budget_ns > 0 ? (uint64_t)wait_budget_ns : WAIT_LIMIT_NS;
    if (A->n != A->ncols) return GK_ERR_INVALID;
    if (kind < GK_PRECOND_NONE || kind > GK_PRECOND_ILU) return GK_ERR_INVALID;
    if (kind == GK_PRECOND_ILU && A->n > 0 && r == z) return GK_ERR_INVALID;
    if (kind == GK_PRECOND_BLOCK_JACOBI && (block_size < 1 || block_size > BJ_MAX))
        return GK_ERR_INVALID;
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != A->device) return GK_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(A->mu);
    cudaStream_t s = (cudaStream_t)stream;
    if (A->dtype == GK_F64)
        return precond_apply_t<double>(A, (int)kind, block_size, (const double*)r, (double*)z,
                                       wb, s);
    return precond_apply_t<float>(A, (int)kind, block_size, (const float*)r, (float*)z, wb, s);
}

extern "C" gk_status gk_ilu_factors(gk_matrix A, void* lu, void* stream) {
    if (!A || (!lu && A->nnz > 0)) return GK_ERR_INVALID;
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != A->device) return GK_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(A->mu);
    cudaStream_t s = (cudaStream_t)stream;
    GK_TRY(ensure_ilu(A, s));
    if (A->nnz > 0)
        GK_CUDA(cudaMemcpyAsync(lu, A->ilu->lu, vector_bytes(A->dtype) * (size_t)A->nnz,
                                cudaMemcpyDeviceToHost, s));
    GK_CUDA(cudaStreamSynchronize(s));
    return GK_OK;
}
