// ilu.cuh - ILU(0) preconditioner: device factors and the two triangular
// substitutions z = U^-1 (L^-1 r) that apply it.
//
// ILU(0) keeps A's sparsity pattern (the paper's first usage example pairs
// GMRES(30) with an Ilu preconditioner, Listing 1; Section 5 lists ILU and
// IC among the bound preconditioners).  The factors live in one value
// array lu[] in the CSR order of A (unit-lower L strictly below the
// diagonal, U on and above it), beside private copies of row_ptr / col,
// the position of every row's diagonal and the pivots' reciprocals.
//
// Substitution is a dependency problem: row i of L^-1 r needs every y_j
// with l_ij != 0.  The kernel is sync-free (no level-by-level launches, one
// launch per triangle):
//  - Rows are cut into chunks of cs consecutive rows (cs = 32, 16 or 8,
//    timed per matrix at setup: shorter chunks shorten the serial chain
//    inside a chunk, longer ones cut the number of dependency levels when
//    rows depend on their neighbours); a warp solves cpw chunks at once
//    (cpw = 1, or 32 / cs to fill the warp, also timed), a group of cs lanes
//    per chunk and one lane per row.  A warp always takes chunks of one
//    level (each level's run in the claim order is padded to a multiple of
//    cpw with empty entries), so the chunks sharing a warp never depend on
//    one another.  Warps claim chunks from an atomic counter in
//    a topological order of the chunk dependency graph (by level: a
//    chunk's level is one more than the highest level it depends on,
//    computed once per matrix), so a chunk only ever waits on chunks
//    claimed before it by running warps: no deadlock.  Claiming by level
//    also keeps warps from spinning on chunks far ahead of the wavefront,
//    and the grid is capped at a few times the widest level.
//  - The values are their own ready signal: before a launch every slot of
//    the output holds a signalling-NaN sentinel (k_ilu_mark), which no
//    arithmetic produces; a lane polls the slot of each value it needs
//    (relaxed loads at GPU scope, a few issued together) until it holds a
//    number.  Inputs are multiplied by 1 on load, which turns any
//    signalling NaN into a quiet one and leaves every other value as it is,
//    so a copied input cannot look like the sentinel either.
//  - A lane first subtracts its row's terms outside the chunk, in the
//    order the substitution produced them (L: ascending columns; U:
//    descending).  The terms inside the chunk are resolved by a 32-step
//    warp loop (cs steps, every group in step): at step t the group's lane
//    t's value is final and is broadcast with a
//    shuffle; lanes whose row uses column c0 + t subtract it.  Together this
//    subtracts every term in exactly the sequential order.
//  - The last warp to leave the kernel resets the claim counter for the
//    next launch.
//  - Every wait is bounded (the caller's budget, 2 s by default, on the
//    GPU's global nanosecond timer); a wait that runs out records an error
//    flag, later waits of the launch give up at once, and the kernel
//    finishes with wrong values instead of hanging.  The solver engine and
//    the apply entry points turn the flag into GK_ERR_TIMEOUT.
// Every subtraction of a product is one fused multiply-add, and U's pivots
// are applied as stored reciprocals (1 / u_ii rounded once, a
// multiplication instead of a division on the in-chunk chain), so that FP64
// results equal the plain substitution with that arithmetic bit for bit.
#pragma once

#include <atomic>
#include <cooperative_groups.h>

#include "gk_internal.cuh"
#include "tma.cuh"

namespace gk {

constexpr int TRSV_CHUNK_MAX = 32;  // rows per warp at most

// Per-direction words (index 0: L, 1: U).
struct TrsvSync {
    unsigned ctr;     // next chunk to claim
    unsigned exited;  // warps that left the current launch
    unsigned err;     // a bounded wait ran out (sticky until cleared)
    unsigned pad;
};

// Device view of one ILU(0) factorisation with values of type T.
template <typename T>
struct IluDev {
    int32_t n = 0, nch = 0;
    int32_t cs = 32;                // rows per chunk (8, 16 or 32)
    int32_t cpw = 1;                // chunks per warp (1 .. 32 / cs)
    const int32_t* rp = nullptr;    // row_ptr[n + 1]
    const int32_t* ci = nullptr;    // col[nnz], strictly ascending per row
    const int32_t* dpos = nullptr;  // position of a_ii in row i
    const T* lu = nullptr;          // factors in CSR order
    const T* rdiag = nullptr;       // 1 / u_ii, rounded once
    const int32_t* ord_l = nullptr;  // chunks in claim order (-1: empty), L
    const int32_t* ord_u = nullptr;  // and U; nord entries each, multiples of 32 / cs
    int32_t nord[2] = {0, 0};
    TrsvSync* sy = nullptr;         // [2]
    int32_t ldiag = 0;              // L scaled by rdiag (0: unit diagonal)
    int32_t udiag = 1;              // U scaled by rdiag (0: unit diagonal)
    unsigned pause_max = 64;        // longest pause between polls (ns)
    unsigned long long wait_ns = WAIT_LIMIT_NS;  // budget of one wait (%globaltimer)
    int32_t warps[2] = {0, 0};      // host: warps per substitution launch
    // level-synchronous mode (lvl != 0, see k_ilu_trsv_cluster): the rows of
    // each triangle sorted by dependency level, and where each level starts
    int32_t lvl = 0;
    const int32_t* lrows[2] = {nullptr, nullptr};   // n rows each (L, U)
    const int32_t* lstart[2] = {nullptr, nullptr};  // nlev + 1 offsets each
    int32_t nlev[2] = {0, 0};
    // window mode (win != 0, see k_ilu_trsv_win): per triangle one record
    // per level-ordered row, and a scratch vector for the level-ordered input
    int32_t win = 0;
    int32_t wdist[2] = {1, 1};           // deepest dependency, in levels
    const void* wrec[2] = {nullptr, nullptr};  // WinRec<T>[n] each
    T* wperm = nullptr;                  // n
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Sentinel of a not-yet-solved slot: a signalling NaN with a fixed payload.
template <typename T> struct Sentinel;
template <> struct Sentinel<double> {
    static constexpr unsigned long long bits = 0x7FF0DEADBEEF1B1BULL;
    __device__ static double value() { return __longlong_as_double((long long)bits); }
    __device__ static bool is(double v) {
        return (unsigned long long)__double_as_longlong(v) == bits;
    }
};
template <> struct Sentinel<float> {
    static constexpr unsigned bits = 0x7F801B1BU;
    __device__ static float value() { return __uint_as_float(bits); }
    __device__ static bool is(float v) { return __float_as_uint(v) == bits; }
};

__device__ __forceinline__ double ld_relaxed_v(const double* p) {
    double v;
    asm volatile("ld.relaxed.gpu.global.f64 %0, [%1];" : "=d"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ float ld_relaxed_v(const float* p) {
    float v;
    asm volatile("ld.relaxed.gpu.global.f32 %0, [%1];" : "=f"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_v(double* p, double v) {
    asm volatile("st.relaxed.gpu.global.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed_v(float* p, float v) {
    asm volatile("st.relaxed.gpu.global.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}

// Spin until *flag == want (acquire), at most limit_ns of %globaltimer; on
// time-out set *err and return false.  Once any wait of the launch has run
// out (*err set), later waits give up at once.  Polls pause 32 to 256 ns.
__device__ __forceinline__ bool wait_flag(const unsigned* flag, unsigned want, unsigned* err,
                                          unsigned long long limit_ns = WAIT_LIMIT_NS) {
    if (ld_acquire_u32(flag) == want) return true;
    const uint64_t t0 = globaltimer_ns();
    unsigned ns = 32;
    for (;;) {
        __nanosleep(ns);
        if (ns < 256) ns <<= 1;
        if (ld_acquire_u32(flag) == want) return true;
        if (ld_relaxed_u32(err) != 0u) return false;
        if (globaltimer_ns() - t0 > limit_ns) {
            atomicExch(err, 1u);
            return false;
        }
    }
}

// The value of slot p once it is no longer the sentinel (v: a first load
// already issued); bounded like wait_flag (limit_ns), pauses 32 to
// pause_max ns.
template <typename T>
__device__ __forceinline__ T wait_value(const T* p, T v, unsigned* err, unsigned pause_max,
                                        unsigned long long limit_ns) {
    if (!Sentinel<T>::is(v)) return v;
    const uint64_t t0 = globaltimer_ns();
    unsigned ns = 32;
    for (;;) {
        __nanosleep(ns);
        if (ns < pause_max) ns <<= 1;
        v = ld_relaxed_v(p);
        if (!Sentinel<T>::is(v)) return v;
        if (ld_relaxed_u32(err) != 0u) return v;
        if (globaltimer_ns() - t0 > limit_ns) {
            atomicExch(err, 1u);
            return v;
        }
    }
}

// a - l * y as one fused multiply-add (rounded once)
__device__ __forceinline__ double sub_mul(double a, double l, double y) {
    return __fma_rn(-l, y, a);
}
__device__ __forceinline__ float sub_mul(float a, float l, float y) {
    return __fmaf_rn(-l, y, a);
}
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }

// ---------------------------------------------------------- sources

template <typename T>
struct IluSrc {  // a plain vector
    const T* p;
    __device__ __forceinline__ const T* ptr() const { return p; }
};

// ---------------------------------------------------------- skips

struct IluSkipNever {
    __device__ __forceinline__ bool skip() const { return false; }
};

// ---------------------------------------------------------- outputs
// dst(): where the unknowns of this substitution are stored (and read back
// by later chunks); extra(i, v): what else row i does with its value.

template <typename T>
struct IluOutStore {
    T* y;
    __device__ __forceinline__ T* dst() const { return y; }
    __device__ __forceinline__ void extra(int64_t, T) const {}
};

// Marks every slot of both substitutions' outputs as unsolved.
template <typename T, class Out, class Skip>
__global__ void __launch_bounds__(256)
k_ilu_mark(int32_t n, T* __restrict__ w, Out out, Skip sk) {
    if (sk.skip()) return;
    T* d = out.dst();
    const T s = Sentinel<T>::value();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        w[i] = s;
        d[i] = s;
    }
}

// One substitution (UP = false: unit-lower L, ascending; UP = true: U with
// its reciprocal pivots, descending).  The last warp of the U launch hands
// the error flags of both directions to on_err (the engine turns a wait
// that ran out into GK_ERR_TIMEOUT and a halt).
template <typename T, bool UP, class Src, class Out, class Skip, class Err>
__global__ void __launch_bounds__(256)
k_ilu_trsv(IluDev<T> f, Src src, Out out, Skip sk, Err on_err) {
    constexpr unsigned FULL = 0xffffffffu;
    constexpr int G = 4;  // out-of-chunk values loaded together
    const int lane = threadIdx.x & 31;
    const int cs = f.cs, cpw = f.cpw;
    const int grp = lane / cs, gl = lane - grp * cs;  // chunk slot, row in the chunk
    TrsvSync* sy = f.sy + (UP ? 1 : 0);
    const int32_t* ord = UP ? f.ord_u : f.ord_l;
    const int nord = f.nord[UP ? 1 : 0];
    const unsigned total = gridDim.x * (blockDim.x >> 5);
    if (!sk.skip()) {
        const T* in = src.ptr();
        T* dst = out.dst();
        for (;;) {
            int c = 0;
            if (lane == 0) c = (int)atomicAdd(&sy->ctr, (unsigned)cpw);
            c = __shfl_sync(FULL, c, 0);
            if (c >= nord) break;
            const int cc = grp < cpw ? ord[c + grp] : -1;  // -1: no chunk for this group
            const int32_t c0 = cc * cs;
            const int32_t c1 = cc >= 0 ? min(c0 + cs, f.n) : c0;
            const int32_t i = c0 + gl;
            const bool has = cc >= 0 && i < f.n;
            T acc = T(0);
            int32_t pin = 0, pend = 0;  // in-chunk entries [pin, pend)
            if (has) {
                acc = mul_rn(in[i], T(1));  // quiets a signalling NaN, else exact
                const int32_t d = f.dpos[i];
                // terms outside the chunk, G at a time, in substitution order
                // (L: ascending from the row start; U: descending from its end)
                int32_t k = UP ? f.rp[i + 1] - 1 : f.rp[i];
                for (;;) {
                    int32_t jj[G];
                    T vv[G], lv[G];
                    int g = 0;
#pragma unroll
                    for (int u = 0; u < G; ++u) {
                        jj[u] = -1;
                        const int32_t ku = UP ? k - u : k + u;
                        if (g == u && (UP ? ku > d : ku < d)) {
                            const int32_t j = f.ci[ku];
                            if (UP ? j >= c1 : j < c0) {
                                jj[u] = j;
                                ++g;
                            }
                        }
                    }
#pragma unroll
                    for (int u = 0; u < G; ++u)
                        if (jj[u] >= 0) {
                            vv[u] = ld_relaxed_v(dst + jj[u]);
                            lv[u] = f.lu[UP ? k - u : k + u];
                        }
#pragma unroll
                    for (int u = 0; u < G; ++u)
                        if (jj[u] >= 0)
                            acc = sub_mul(acc, lv[u],
                                          wait_value(dst + jj[u], vv[u], &sy->err, f.pause_max,
                                                     f.wait_ns));
                    k = UP ? k - g : k + g;
                    if (g < G) break;
                }
                if (!UP) {
                    pin = k;
                    pend = d;
                } else {
                    pin = d + 1;
                    pend = k + 1;
                }
            }
            const int base = grp * cs;  // the group's first lane
            T mine = T(0);
            if (!UP && !f.ldiag) {
                // lane t's value is final at step t; later lanes subtract it
                int32_t col = pin < pend ? f.ci[pin] : INT32_MAX;
                T lv = pin < pend ? f.lu[pin] : T(0);
                for (int t = 0; t < cs; ++t) {
                    const T yt = __shfl_sync(FULL, acc, base + t);
                    if (gl == t) mine = yt;
                    if (col == c0 + t) {  // only lanes > t hold column c0 + t
                        acc = sub_mul(acc, lv, yt);
                        ++pin;
                        col = pin < pend ? f.ci[pin] : INT32_MAX;
                        lv = pin < pend ? f.lu[pin] : T(0);
                    }
                }
            } else if (!UP) {
                // as above, each value scaled by its reciprocal diagonal
                const T rd = has ? f.rdiag[i] : T(1);
                int32_t col = pin < pend ? f.ci[pin] : INT32_MAX;
                T lv = pin < pend ? f.lu[pin] : T(0);
                for (int t = 0; t < cs; ++t) {
                    T v = T(0);
                    if (gl == t) v = mul_rn(acc, rd);
                    const T yt = __shfl_sync(FULL, v, base + t);
                    if (gl == t) mine = yt;
                    if (col == c0 + t) {
                        acc = sub_mul(acc, lv, yt);
                        ++pin;
                        col = pin < pend ? f.ci[pin] : INT32_MAX;
                        lv = pin < pend ? f.lu[pin] : T(0);
                    }
                }
            } else {
                const T rd = has && f.udiag ? f.rdiag[i] : T(1);
                int32_t col = pend > pin ? f.ci[pend - 1] : INT32_MIN;
                T uv = pend > pin ? f.lu[pend - 1] : T(0);
                for (int t = cs - 1; t >= 0; --t) {
                    T v = T(0);
                    if (gl == t) v = mul_rn(acc, rd);
                    const T zt = __shfl_sync(FULL, v, base + t);
                    if (gl == t) mine = zt;
                    if (col == c0 + t) {  // only lanes < t hold column c0 + t
                        acc = sub_mul(acc, uv, zt);
                        --pend;
                        col = pend > pin ? f.ci[pend - 1] : INT32_MIN;
                        uv = pend > pin ? f.lu[pend - 1] : T(0);
                    }
                }
            }
            if (has) {
                st_relaxed_v(dst + i, mine);
                out.extra(i, mine);
            }
        }
    }
    // every warp leaves exactly once; the last one prepares the next launch
    __syncwarp();
    if (lane == 0) {
        const unsigned e = atomicAdd(&sy->exited, 1u);
        if (e == total - 1) {
            if (UP) on_err(ld_acquire_u32(&f.sy[0].err) | ld_acquire_u32(&f.sy[1].err));
            sy->ctr = 0;
            sy->exited = 0;
            __threadfence();
        }
    }
}

struct IluNoErr {
    __device__ __forceinline__ void operator()(unsigned) const {}
};

// ------------------------------------------------ level-synchronous mode
// One thread-block cluster (CLT_BLOCKS blocks of CLT_THREADS) solves a whole
// triangle level by level: the rows of a level are spread over the
// cluster's threads, and a cluster barrier (release/acquire at cluster
// scope) ends the level, so a level's values are visible to the next one
// without polling.  Each row subtracts its terms in the substitution order
// with fused multiply-adds, exactly as the chunked kernel, so the result is
// the same bit for bit.  While a level's barrier completes, each thread
// loads the next level's row data (rows, pivots, the first CLT_TPR terms'
// columns and factors, the input values), which depend on nothing solved;
// only the loads of solved values wait for the barrier.  The unknowns are
// read at GPU scope from L2 (ld.relaxed.gpu): another block of the cluster
// wrote them.  No thread ever waits on another except at the barrier.
constexpr int CLT_BLOCKS = 8;    // a portable cluster size
constexpr int CLT_THREADS = 512;
constexpr int CLT_RPT = 4;       // rows of a level a thread prefetches
constexpr int CLT_TPR = 4;       // terms of a row prefetched

__device__ __forceinline__ void cluster_arrive_release() {
    asm volatile("barrier.cluster.arrive.release;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait_acquire() {
    asm volatile("barrier.cluster.wait.acquire;" ::: "memory");
}

// Arrive on the cluster barrier releasing this block's shared-memory writes
// only (a restricted release fence, then a relaxed arrive; the wait side
// acquires).  For the window mode: blocks exchange values through their
// shared-memory rings alone, and the output vector's stores are read by no
// block of the same launch, so they need not be performed before the
// barrier completes.  A read of another block's ring is ordered before that
// block's later overwrite of the slot by the barrier and by its value being
// used before this block's arrive.
__device__ __forceinline__ void cluster_arrive_release_smem() {
    asm volatile(
        "fence.release.sync_restrict::shared::cta.cluster;\n\t"
        "barrier.cluster.arrive.relaxed;" ::: "memory");
}

template <typename T>
struct CltRow {
    int32_t i;       // row (-1: none)
    int32_t k, ke;   // its terms [k, ke) in substitution order (L ascending, U: k > ke, descending)
    int32_t c[CLT_TPR];
    T v[CLT_TPR];
    T in, rd;
};

template <typename T, bool UP>
__device__ __forceinline__ void clt_load(const IluDev<T>& f, const T* __restrict__ in, int32_t i,
                                         CltRow<T>& R) {
    R.i = i;
    if (i < 0) return;
    const int32_t d = f.dpos[i];
    if (!UP) {
        R.k = f.rp[i];
        R.ke = d;
    } else {
        R.k = f.rp[i + 1] - 1;
        R.ke = d;
    }
#pragma unroll
    for (int t = 0; t < CLT_TPR; ++t) {
        const int32_t kk = UP ? R.k - t : R.k + t;
        const bool ok = UP ? kk > R.ke : kk < R.ke;
        R.c[t] = ok ? f.ci[kk] : -1;
        R.v[t] = ok ? f.lu[kk] : T(0);
    }
    R.in = in[i];
    R.rd = (UP ? f.udiag : f.ldiag) ? f.rdiag[i] : T(1);
}

template <typename T, bool UP>
__device__ __forceinline__ T clt_solve(const IluDev<T>& f, const CltRow<T>& R, const T* dst) {
    T acc = mul_rn(R.in, T(1));  // quiets a signalling NaN, else exact
    T z[CLT_TPR];
#pragma unroll
    for (int t = 0; t < CLT_TPR; ++t) z[t] = R.c[t] >= 0 ? ld_relaxed_v(dst + R.c[t]) : T(0);
#pragma unroll
    for (int t = 0; t < CLT_TPR; ++t)
        if (R.c[t] >= 0) acc = sub_mul(acc, R.v[t], z[t]);
    // terms past the prefetched ones, in the same order
    if (UP) {
        for (int32_t kk = R.k - CLT_TPR; kk > R.ke; --kk)
            acc = sub_mul(acc, f.lu[kk], ld_relaxed_v(dst + f.ci[kk]));
        return mul_rn(acc, R.rd);
    }
    for (int32_t kk = R.k + CLT_TPR; kk < R.ke; ++kk)
        acc = sub_mul(acc, f.lu[kk], ld_relaxed_v(dst + f.ci[kk]));
    return f.ldiag ? mul_rn(acc, R.rd) : acc;
}

template <typename T, bool UP, class Src, class Out, class Skip>
__global__ void __launch_bounds__(CLT_THREADS, 1)
k_ilu_trsv_cluster(IluDev<T> f, Src src, Out out, Skip sk) {
    if (sk.skip()) return;  // read before the launch's first barrier: every block agrees
    const unsigned nblk = gridDim.x;  // one cluster: the grid
    const int32_t nthr = (int32_t)(nblk * CLT_THREADS);
    const int32_t tid = (int32_t)(blockIdx.x * CLT_THREADS + threadIdx.x);
    const int32_t* rows = f.lrows[UP ? 1 : 0];
    const int32_t* start = f.lstart[UP ? 1 : 0];
    const int32_t nlev = f.nlev[UP ? 1 : 0];
    const T* in = src.ptr();
    T* dst = out.dst();
    CltRow<T> R[CLT_RPT];
    auto prefetch = [&](int32_t L) {
        const int32_t b = L < nlev ? start[L] : 0, e = L < nlev ? start[L + 1] : 0;
#pragma unroll
        for (int r = 0; r < CLT_RPT; ++r) {
            const int32_t idx = b + tid + r * nthr;
            clt_load<T, UP>(f, in, idx < e ? rows[idx] : -1, R[r]);
        }
    };
    prefetch(0);
    for (int32_t L = 0; L < nlev; ++L) {
#pragma unroll
        for (int r = 0; r < CLT_RPT; ++r)
            if (R[r].i >= 0) {
                const T v = clt_solve<T, UP>(f, R[r], dst);
                dst[R[r].i] = v;
                out.extra(R[r].i, v);
            }
        // rows of a level wider than CLT_RPT x the cluster's threads
        const int32_t b = start[L], e = start[L + 1];
        for (int32_t idx = b + tid + CLT_RPT * nthr; idx < e; idx += nthr) {
            CltRow<T> X;
            clt_load<T, UP>(f, in, rows[idx], X);
            const T v = clt_solve<T, UP>(f, X, dst);
            dst[X.i] = v;
            out.extra(X.i, v);
        }
        cluster_arrive_release();
        prefetch(L + 1);  // independent of the values being published
        cluster_wait_acquire();
    }
}

// Blocks of 256 threads for a substitution: `warps` warps (a few times the
// widest level), at most the resident ones.
template <typename K>
static unsigned ilu_grid(K kernel, int32_t warps) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, 256, 0) != cudaSuccess || b < 1)
        b = 1;
    const int64_t need = ((int64_t)warps + 7) / 8;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)num_sms() * b));
}

// ------------------------------------------------------------ window mode
// Level-synchronous like k_ilu_trsv_cluster, for matrices whose rows
// depend only on the previous WIN_MAXD levels (stencils in their natural
// order: one level back) with at most WIN_MAXT terms a row per triangle.
// Each of the cluster's blocks owns a contiguous share of every level's
// rows, and keeps the values of its rows of the last D + 1 levels in a
// shared-memory ring; a row reads the values it needs through distributed
// shared memory, so a level's hand-off is a cluster barrier over shared
// memory, without L2 round trips.  Everything else a row needs -- its
// record (the terms' cluster coordinates and factors in substitution
// order, the pivot) and its input, permuted into level order by
// k_perm_gather before the launch -- depends on nothing solved: thread 0
// of a block copies the block's share of a level's records and inputs into
// shared memory with the bulk-copy unit a level ahead, and the threads move
// the next level's into registers while a barrier completes, so no level
// waits on a global load.  The values go to the output vector after the
// arrive, and the arrive releases shared-memory writes only, so the barrier
// never waits for global stores.  The order of subtractions of every row
// is the substitution order, so the result is bit-identical to the other
// modes.
constexpr int WIN_BLOCKS = 16;    // a cluster over the portable 8 blocks
constexpr int WIN_THREADS = 256;
constexpr int WIN_MAXT = 4;       // terms of a row (per triangle)
constexpr int WIN_MAXD = 2;       // deepest dependency, in levels
constexpr int WIN_RPT = 3;        // rows of a level per thread
constexpr int WIN_CAP = WIN_RPT * WIN_THREADS;  // rows of a level per block
// a term's coordinates in the 15 bits of WinRec::co: the index in the
// owner's share, then one bit for the levels back, then the owner's rank
constexpr int WIN_IDX_BITS = WIN_BLOCKS <= 8 ? 11 : 10;
static_assert(WIN_BLOCKS <= (1 << (14 - WIN_IDX_BITS)) && WIN_MAXD <= 2 &&
                  WIN_CAP <= (1 << WIN_IDX_BITS),
              "a term's coordinates must fit the 15 bits of WinRec::co");

// One level-ordered row of a triangle.  co[t]: the block that owns the
// source row in the source's level (the top bits), how many levels back
// that level is, less one (bit WIN_IDX_BITS), and the source's index in
// that block's share (the low WIN_IDX_BITS bits); -1 past the row's terms,
// whose factors are 0.
template <typename T>
struct alignas(16) WinRec {
    T v[WIN_MAXT];          // factors, in substitution order
    T rd;                   // reciprocal pivot
    int16_t co[WIN_MAXT];
};
static_assert(sizeof(WinRec<double>) == 48 && sizeof(WinRec<float>) == 32,
              "records are whole 16-byte chunks");

// dynamic shared memory of k_ilu_trsv_win: two mbarriers, the ring of
// values, two buffers of a level's records as they lie in global memory
// (with 48-byte records a warp's 16-byte reads of them meet no bank
// conflict), then two of inputs (their copy is widened to 16-byte
// boundaries at both ends, so a buffer holds up to 32 bytes more)
template <typename T>
struct WinSmem {
    static constexpr int NC = (int)(sizeof(WinRec<T>) / 16);
    static constexpr int AL = (int)(16 / sizeof(T));  // inputs a 16-byte chunk
    static constexpr int INCAP = WIN_CAP + 2 * AL;
    static constexpr size_t bars = 16;
    static constexpr size_t ring = (size_t)(WIN_MAXD + 1) * WIN_CAP * sizeof(T);
    static constexpr size_t recs = (size_t)2 * WIN_CAP * NC * 16;
    static constexpr size_t ins = (size_t)2 * INCAP * sizeof(T);
    static constexpr size_t bytes = bars + ring + recs + ins;
};
static_assert(WinSmem<double>::bytes <= 227 * 1024, "one block per SM");

// The window mode's wait for a copy: polls the barrier without the
// suspension of mbarrier.try_wait, so a budget shorter than a copy runs out
__device__ __forceinline__ bool win_wait(uint32_t bar, uint32_t parity, uint64_t limit_ns) {
    auto done = [&]() {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n}"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        return ok != 0;
    };
    const uint64_t t0 = globaltimer_ns();
    while (!done())
        if (globaltimer_ns() - t0 >= limit_ns) return false;
    return true;
}

__device__ __forceinline__ void win_slice(const int32_t* start, int32_t L, unsigned rank,
                                          int32_t& a, int32_t& b) {
    const int32_t s0 = start[L], len = start[L + 1] - s0;
    const int32_t per = (len + WIN_BLOCKS - 1) / WIN_BLOCKS;
    a = s0 + min(len, (int32_t)rank * per);
    b = s0 + min(len, (int32_t)(rank + 1) * per);
}

// address of the same shared-memory location in block `rank` of the cluster
__device__ __forceinline__ uint32_t dsmem_map(uint32_t addr, uint32_t rank) {
    uint32_t r;
    asm("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}
__device__ __forceinline__ void dsmem_ld(double& v, uint32_t addr) {
    asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(addr) : "memory");
}
__device__ __forceinline__ void dsmem_ld(float& v, uint32_t addr) {
    asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(addr) : "memory");
}

// the values a row needs, read from the owners' rings: ring1 / ring2 are
// the shared-memory addresses of the slots of the levels one and two back
template <typename T>
__device__ __forceinline__ void win_gather(const WinRec<T>& R, uint32_t ring1, uint32_t ring2,
                                           T (&z)[WIN_MAXT]) {
#pragma unroll
    for (int t = 0; t < WIN_MAXT; ++t) {
        z[t] = T(0);
        const int32_t co = R.co[t];
        if (co >= 0) {
            const uint32_t a = ((co >> WIN_IDX_BITS) & 1 ? ring2 : ring1) +
                               (uint32_t)(co & ((1 << WIN_IDX_BITS) - 1)) * sizeof(T);
            dsmem_ld(z[t], dsmem_map(a, (uint32_t)(co >> (WIN_IDX_BITS + 1))));
        }
    }
}

// in: already multiplied by 1 by k_perm_gather (which quiets a signalling
// NaN, as the other modes do first; exact otherwise)
template <typename T, bool UP>
__device__ __forceinline__ T win_finish(const IluDev<T>& f, const WinRec<T>& R, T in,
                                        const T (&z)[WIN_MAXT]) {
    T acc = in;
#pragma unroll
    for (int t = 0; t < WIN_MAXT; ++t)
        if (R.co[t] >= 0) acc = sub_mul(acc, R.v[t], z[t]);
    if (UP) return mul_rn(acc, f.udiag ? R.rd : T(1));
    return f.ldiag ? mul_rn(acc, R.rd) : acc;
}

template <typename T, bool UP, class Out, class Skip, class Err>
__global__ void __launch_bounds__(WIN_THREADS, 1)
k_ilu_trsv_win(IluDev<T> f, Out out, Skip sk, Err on_err) {
    if (sk.skip()) return;  // read before the first barrier: every block agrees
    using SM = WinSmem<T>;
    extern __shared__ __align__(16) unsigned char wsm[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(wsm);
    T* ring = reinterpret_cast<T*>(wsm + SM::bars);
    WinRec<T>* rbuf = reinterpret_cast<WinRec<T>*>(wsm + SM::bars + SM::ring);
    T* ibuf = reinterpret_cast<T*>(wsm + SM::bars + SM::ring + SM::recs);
    const unsigned rank = blockIdx.x;  // one cluster: the grid
    const int tid = (int)threadIdx.x;
    const int nslot = f.wdist[UP ? 1 : 0] + 1;
    const WinRec<T>* rec = static_cast<const WinRec<T>*>(f.wrec[UP ? 1 : 0]);
    const int32_t* start = f.lstart[UP ? 1 : 0];
    const int32_t* rows = f.lrows[UP ? 1 : 0];
    const int32_t nlev = f.nlev[UP ? 1 : 0];
    const T* inp = f.wperm;
    T* dst = out.dst();
    unsigned* err = &f.sy[UP ? 1 : 0].err;
    // thread 0 copies the block's share of level L's records and inputs into
    // buffer L & 1 with the bulk-copy unit; the buffer's mbarrier completes
    // a phase when the bytes have landed
    auto stage = [&](int32_t L) {
        int32_t a, b;
        win_slice(start, L, rank, a, b);
        const int buf = L & 1;
        const uint32_t bar = smem_addr(bars + buf);
        const int32_t a0 = a & ~(SM::AL - 1), b0 = (b + SM::AL - 1) & ~(SM::AL - 1);
        const uint32_t rb = (uint32_t)(b - a) * (uint32_t)sizeof(WinRec<T>);
        const uint32_t ib = (uint32_t)(b0 - a0) * (uint32_t)sizeof(T);
        mbar_arrive_expect_tx(bar, b > a ? rb + ib : 0u);
        if (b > a) {
            bulk_g2s(smem_addr(rbuf + (size_t)buf * WIN_CAP), rec + a, rb, bar);
            bulk_g2s(smem_addr(ibuf + (size_t)buf * SM::INCAP), inp + a0, ib, bar);
        }
    };
    WinRec<T> R[WIN_RPT];
    T in[WIN_RPT];
    int32_t ii[WIN_RPT];
    bool has[WIN_RPT];
    // level L's rows from its buffer into registers once its copy landed
    // (their row numbers from the level order, needed only after the
    // level's arrive); false if the wait ran out
    auto take = [&](int32_t L) -> bool {
        int32_t a, b;
        win_slice(start, L, rank, a, b);
        const int buf = L & 1;
        const bool ok = win_wait(smem_addr(bars + buf), (uint32_t)(L >> 1) & 1u, f.wait_ns);
        const WinRec<T>* sr = rbuf + (size_t)buf * WIN_CAP;
        const T* si = ibuf + (size_t)buf * SM::INCAP + (a & (SM::AL - 1));
#pragma unroll
        for (int r = 0; r < WIN_RPT; ++r) {
            const int32_t q = tid + r * WIN_THREADS;
            has[r] = ok && a + q < b;
            if (has[r]) {
                R[r] = sr[q];
                in[r] = si[q];
                ii[r] = rows[a + q];
            }
        }
        return ok;
    };
    if (tid == 0) {
        mbar_init(smem_addr(bars), 1);
        mbar_init(smem_addr(bars + 1), 1);
        fence_mbar_init();
    }
    __syncthreads();
    bool live = true;             // every copy issued so far was waited for
    int32_t pend = 0, npend = 0;  // else levels [pend, pend + npend) may be in flight
    if (tid == 0) {
        if (nlev > 0) stage(0);
        if (nlev > 1) stage(1);
    }
    if (nlev > 0) {
        live = __syncthreads_and(take(0)) != 0;
        if (!live) npend = min(nlev, 2);
    }
    const uint32_t ring0 = smem_addr(ring);
    constexpr uint32_t SLOT = WIN_CAP * sizeof(T);
    for (int32_t L = 0; L < nlev; ++L) {
        T* mine = ring + (L % nslot) * WIN_CAP;
        const uint32_t ring1 = ring0 + (uint32_t)((L + 2 * nslot - 1) % nslot) * SLOT;
        const uint32_t ring2 = ring0 + (uint32_t)((L + 2 * nslot - 2) % nslot) * SLOT;
        // every row's reads first, then the arithmetic, then the stores: the
        // compiler cannot tell the rings' slots apart, so a store between
        // two rows would order the next row's reads after it
        T zz[WIN_RPT][WIN_MAXT], zv[WIN_RPT];
#pragma unroll
        for (int r = 0; r < WIN_RPT; ++r)
            if (has[r]) win_gather<T>(R[r], ring1, ring2, zz[r]);
#pragma unroll
        for (int r = 0; r < WIN_RPT; ++r)
            if (has[r]) zv[r] = win_finish<T, UP>(f, R[r], in[r], zz[r]);
#pragma unroll
        for (int r = 0; r < WIN_RPT; ++r)
            if (has[r]) mine[tid + r * WIN_THREADS] = zv[r];
        cluster_arrive_release_smem();
#pragma unroll
        for (int r = 0; r < WIN_RPT; ++r)
            if (has[r]) {
                dst[ii[r]] = zv[r];
                out.extra(ii[r], zv[r]);
            }
        if (L + 1 < nlev) {
            // level L + 1's copy was issued a level ahead; the block barrier
            // also tells that every thread has taken level L's rows out of
            // the buffer that level L + 2 is copied into
            bool ok = live && take(L + 1);
            ok = __syncthreads_and(ok) != 0;
            if (live && !ok) {
                pend = L + 1;
                npend = 1;
            }
            live = ok;
            if (!live)
#pragma unroll
                for (int r = 0; r < WIN_RPT; ++r) has[r] = false;
            if (tid == 0 && live && L + 2 < nlev) {
                fence_proxy_async_smem();
                stage(L + 2);
            }
        }
        cluster_wait_acquire();
    }
    if (npend > 0) {
        // a wait ran out: report it, and keep the shared memory until the
        // copies in flight have landed (with the default limit, not the
        // caller's budget: the block must outlive the copies into it)
        if (tid == 0) {
            atomicExch(err, 1u);
            for (int32_t L = pend; L < pend + npend; ++L)
                mbar_wait_bounded(smem_addr(bars + (L & 1)), (uint32_t)(L >> 1) & 1u);
        }
        __syncthreads();
    }
    if (UP) {
        // the U launch hands both directions' error flags to on_err, after
        // a barrier that orders every block's report before the read
        cluster_arrive_release();
        cluster_wait_acquire();
        if (rank == 0 && tid == 0)
            on_err(ld_acquire_u32(&f.sy[0].err) | ld_acquire_u32(&f.sy[1].err));
    }
}

// out[idx] = src[rows[idx]] * 1: an input in level order, a signalling NaN
// quieted as the substitutions of the other modes do first
template <typename T, class Src, class Skip>
__global__ void __launch_bounds__(256)
k_perm_gather(int32_t n, const int32_t* __restrict__ rows, Src src, T* __restrict__ out, Skip sk) {
    if (sk.skip()) return;
    const T* in = src.ptr();
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
         idx += (int64_t)gridDim.x * blockDim.x)
        out[idx] = mul_rn(in[rows[idx]], T(1));
}

template <typename T, class K>
static gk_status win_attributes(K k) {
    if (WIN_BLOCKS > 8)
        GK_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    GK_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)WinSmem<T>::bytes));
    return GK_OK;
}

template <typename T, bool UP, class Out, class Skip, class Err>
static gk_status launch_win(const IluDev<T>& f, Out out, Skip sk, Err on_err, cudaStream_t s) {
    auto k = k_ilu_trsv_win<T, UP, Out, Skip, Err>;
    // more than the default 48 KB of dynamic shared memory, and a cluster
    // over 8 blocks where WIN_BLOCKS asks for one (attributes of the
    // function, not stream operations: set once, before the first launch)
    static std::atomic<bool> attr{false};
    if (!attr.load(std::memory_order_acquire)) {
        GK_TRY(win_attributes<T>(k));
        attr.store(true, std::memory_order_release);
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(WIN_BLOCKS, 1, 1);
    cfg.blockDim = dim3(WIN_THREADS, 1, 1);
    cfg.dynamicSmemBytes = WinSmem<T>::bytes;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = WIN_BLOCKS;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    GK_CUDA(cudaLaunchKernelEx(&cfg, k, f, out, sk, on_err));
    return GK_OK;
}

template <typename T, class Src, class Skip>
static gk_status perm_gather(const IluDev<T>& f, bool up, Src src, Skip sk, cudaStream_t s) {
    const unsigned g = (unsigned)std::max<int64_t>(
        1, std::min<int64_t>(((int64_t)f.n + 1023) / 1024, (int64_t)num_sms() * 8));
    k_perm_gather<T, Src, Skip><<<g, 256, 0, s>>>(f.n, f.lrows[up ? 1 : 0], src, f.wperm, sk);
    GK_CUDA(cudaGetLastError());
    return GK_OK;
}

// One level-synchronous substitution: a single cluster of CLT_BLOCKS blocks.
template <typename T, bool UP, class Src, class Out, class Skip>
static gk_status launch_clt(const IluDev<T>& f, Src src, Out out, Skip sk, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CLT_BLOCKS, 1, 1);
    cfg.blockDim = dim3(CLT_THREADS, 1, 1);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CLT_BLOCKS;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    GK_CUDA(cudaLaunchKernelEx(&cfg, k_ilu_trsv_cluster<T, UP, Src, Out, Skip>, f, src, out, sk));
    return GK_OK;
}

// z = U^-1 L^-1 src: mark both outputs unsolved, L into w, then U from w
// with the caller's output (level-synchronous mode: two cluster launches,
// nothing to mark, no waits that could run out).
template <typename T, class Src, class Out, class Skip, class Err>
static gk_status ilu_apply(const IluDev<T>& f, Src src, T* w, Out out, Skip sk, Err on_err,
                           cudaStream_t s) {
    if (f.n == 0) return GK_OK;
    if (f.win) {
        GK_TRY((perm_gather<T>(f, false, src, sk, s)));
        GK_TRY((launch_win<T, false>(f, IluOutStore<T>{w}, sk, IluNoErr{}, s)));
        GK_TRY((perm_gather<T>(f, true, IluSrc<T>{w}, sk, s)));
        return launch_win<T, true>(f, out, sk, on_err, s);
    }
    if (f.lvl) {
        GK_TRY((launch_clt<T, false>(f, src, IluOutStore<T>{w}, sk, s)));
        return launch_clt<T, true>(f, IluSrc<T>{w}, out, sk, s);
    }
    auto km = k_ilu_mark<T, Out, Skip>;
    auto kl = k_ilu_trsv<T, false, Src, IluOutStore<T>, Skip, IluNoErr>;
    auto ku = k_ilu_trsv<T, true, IluSrc<T>, Out, Skip, Err>;
    const unsigned mg = (unsigned)std::max<int64_t>(
        1, std::min<int64_t>(((int64_t)f.n + 1023) / 1024, (int64_t)num_sms() * 8));
    km<<<mg, 256, 0, s>>>(f.n, w, out, sk);
    kl<<<ilu_grid(kl, f.warps[0]), 256, 0, s>>>(f, src, IluOutStore<T>{w}, sk, IluNoErr{});
    ku<<<ilu_grid(ku, f.warps[1]), 256, 0, s>>>(f, IluSrc<T>{w}, out, sk, on_err);
    GK_CUDA(cudaGetLastError());
    return GK_OK;
}

// One substitution alone (gk_triangular_solve): mark x unsolved, then the L
// (up = false) or U launch from src into x.
template <typename T>
static gk_status tri_apply(const IluDev<T>& f, bool up, const T* src, T* x, cudaStream_t s) {
    if (f.n == 0) return GK_OK;
    if (f.win) {
        GK_TRY((perm_gather<T>(f, up, IluSrc<T>{src}, IluSkipNever{}, s)));
        if (up) return launch_win<T, true>(f, IluOutStore<T>{x}, IluSkipNever{}, IluNoErr{}, s);
        return launch_win<T, false>(f, IluOutStore<T>{x}, IluSkipNever{}, IluNoErr{}, s);
    }
    if (f.lvl) {
        if (up)
            return launch_clt<T, true>(f, IluSrc<T>{src}, IluOutStore<T>{x}, IluSkipNever{}, s);
        return launch_clt<T, false>(f, IluSrc<T>{src}, IluOutStore<T>{x}, IluSkipNever{}, s);
    }
    auto km = k_ilu_mark<T, IluOutStore<T>, IluSkipNever>;
    const unsigned mg = (unsigned)std::max<int64_t>(
        1, std::min<int64_t>(((int64_t)f.n + 1023) / 1024, (int64_t)num_sms() * 8));
    km<<<mg, 256, 0, s>>>(f.n, x, IluOutStore<T>{x}, IluSkipNever{});
    if (!up) {
        auto kl = k_ilu_trsv<T, false, IluSrc<T>, IluOutStore<T>, IluSkipNever, IluNoErr>;
        kl<<<ilu_grid(kl, f.warps[0]), 256, 0, s>>>(f, IluSrc<T>{src}, IluOutStore<T>{x},
                                                     IluSkipNever{}, IluNoErr{});
    } else {
        auto ku = k_ilu_trsv<T, true, IluSrc<T>, IluOutStore<T>, IluSkipNever, IluNoErr>;
        ku<<<ilu_grid(ku, f.warps[1]), 256, 0, s>>>(f, IluSrc<T>{src}, IluOutStore<T>{x},
                                                     IluSkipNever{}, IluNoErr{});
    }
    GK_CUDA(cudaGetLastError());
    return GK_OK;
}

// Clears the sticky wait-ran-out flags of both directions (before a solve
// or an apply, so that only this run's waits are reported).
template <typename T>
static gk_status ilu_clear_err(const IluDev<T>& f, cudaStream_t s) {
    GK_CUDA(cudaMemsetAsync(&f.sy[0].err, 0, sizeof(unsigned), s));
    GK_CUDA(cudaMemsetAsync(&f.sy[1].err, 0, sizeof(unsigned), s));
    return GK_OK;
}

// host side (ilu.cu): build the factors of A in the vector type on first
// use (GK_ERR_INVALID: columns not strictly ascending; GK_ERR_ZERO_DIAG:
// missing diagonal or zero pivot), and the device view of them.
gk_status ensure_ilu(gk_matrix A, cudaStream_t s);
template <typename T>
IluDev<T> ilu_view(gk_matrix A);

}  // namespace gk
