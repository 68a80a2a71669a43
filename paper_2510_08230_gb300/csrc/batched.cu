// batched.cu - single-block engine: one thread block runs a whole CG or
// BiCGSTAB solve (same algorithm, stopping rule and residual replacement
// as the multi-kernel engine; Section 3.5 Listings 1-2 for the interface).
//
// Used for many small independent systems in one launch (gk_solve_batched)
// and for small single systems (engine 2).  The vector that SpMV gathers
// from (p for CG; phat, then shat for BiCGSTAB) is staged in shared memory;
// the other vectors live in a per-system global workspace that stays in
// L1/L2.  Blocks loop over systems (persistent grid), so the launch is one
// kernel regardless of the number of systems.  Reductions are block-wide,
// fixed order, so a system's result does not depend on the rest of the
// batch or on the grid size.
#include <cstring>
#include <map>
#include <vector>

#include "prims.cuh"

namespace gk {


// SpMV layouts of a system in the batched engine.  Every layout sums a row
// in its CSR order (one fused multiply-add per stored entry, from zero), so
// the layout never changes a result, only the memory access pattern.
enum BatchLayout : int32_t { BL_CSR = 0, BL_ELL = 1, BL_SELLP = 2 };

struct SysDesc {
    int32_t n, fmt;  // fmt: a BatchLayout
    const int32_t* rp;
    const int32_t* ci;
    const void* va;
    const void* b;
    void* x;
    void* work;  // workspace vectors, each `ld` elements
    int64_t ld;
    double tol;  // this system's relative tolerance
    // padded copy (ELL: K columns of pstride rows; SELL-P: slices of S rows
    // with lengths slen[] and offsets sset[] in units of S entries)
    int32_t* pcol;
    void* pval;
    int32_t* slen;
    int32_t* sset;
    int64_t pstride;
    int32_t K, S;
};

struct SysOut {
    int32_t status, iters, restarts, pad;
    double rec, tru;
};

struct BlockOpts {
    double tol;
    int32_t max_iters;
    int32_t prec;
};

// Reductions use VL virtual lanes: row i adds into lane i mod VL, and the
// VL lane partials are summed by warp 0 in a fixed order.  The rounding of
// every dot product is therefore the same for 128, 256 or 512 threads per
// block, so the block size (autotuned) never changes a system's result.
constexpr int VL = 512;

template <int NA>
struct VAcc {
    double v[NA][4];
};

template <int NA>
__device__ __forceinline__ VAcc<NA> vacc() {
    VAcc<NA> a;
#pragma unroll
    for (int k = 0; k < NA; ++k)
#pragma unroll
        for (int s = 0; s < 4; ++s) a.v[k][s] = 0.0;
    return a;
}

// f(i, s) for every row i of this thread; s = (i mod VL) / blockDim.x
template <class F>
__device__ __forceinline__ void for_rows_vl(int32_t n, F&& f) {
    const int ns = VL / (int)blockDim.x;
    for (int32_t i0 = threadIdx.x; i0 < n; i0 += VL) {
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            if (s < ns) {
                const int32_t i = i0 + s * (int32_t)blockDim.x;
                if (i < n) f(i, s);
            }
        }
    }
}

// Sum of the virtual-lane partials, returned to every thread.
template <int NA>
__device__ __forceinline__ void vl_allsum(const VAcc<NA>& acc, double (&out)[NA]) {
    __shared__ double sh[NA][VL];
    __shared__ double tot[NA];
    const int ns = VL / (int)blockDim.x;
#pragma unroll
    for (int a = 0; a < NA; ++a)
#pragma unroll
        for (int s = 0; s < 4; ++s)
            if (s < ns) sh[a][threadIdx.x + s * blockDim.x] = acc.v[a][s];
    __syncthreads();
    if (threadIdx.x < 32) {
#pragma unroll
        for (int a = 0; a < NA; ++a) {
            double t[VL / 32];  // lane l: lanes l, l+32, ... as a pairwise tree
#pragma unroll
            for (int k = 0; k < VL / 32; ++k) t[k] = sh[a][threadIdx.x + 32 * k];
#pragma unroll
            for (int w = VL / 64; w > 0; w >>= 1)
#pragma unroll
                for (int k = 0; k < w; ++k) t[k] += t[k + w];
            const double tt = warp_sum(t[0]);
            if (threadIdx.x == 0) tot[a] = tt;
        }
    }
    __syncthreads();
#pragma unroll
    for (int a = 0; a < NA; ++a) out[a] = tot[a];
    __syncthreads();
}

template <typename V, typename T, typename G>
__device__ __forceinline__ T row_dot(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                     const V* __restrict__ va, const G* __restrict__ g, int32_t i) {
    T s = T(0);
    const int32_t e = rp[i + 1];
    for (int32_t k = rp[i]; k < e; ++k) s = fmadd(cvt<T>(va[k]), (T)g[ci[k]], s);
    return s;
}

// Row i of a system in its layout (see BatchLayout): entries in CSR order,
// padding (column -1) only after a row's last entry.
// L >= 0: every system of the batch has layout L (the branch is resolved at
// compile time); L = -1: the layout is read per system.
template <typename V, typename T, int L, typename G>
__device__ __forceinline__ T sys_row_dot(const SysDesc& d, const G* __restrict__ g, int32_t i) {
    const int fmt = L >= 0 ? L : d.fmt;
    if (fmt == BL_ELL) {
        const int32_t* __restrict__ col = d.pcol;
        const V* __restrict__ val = (const V*)d.pval;
        T s = T(0);
        int64_t p = i;
        for (int32_t k = 0; k < d.K; ++k, p += d.pstride) {
            const int32_t c = col[p];
            if (c < 0) break;
            s = fmadd(cvt<T>(val[p]), (T)g[c], s);
        }
        return s;
    }
    if (fmt == BL_SELLP) {
        const int32_t sl = i / d.S, t = i - sl * d.S;
        const int32_t* __restrict__ col = d.pcol;
        const V* __restrict__ val = (const V*)d.pval;
        const int32_t len = d.slen[sl];
        int64_t p = (int64_t)d.sset[sl] * d.S + t;
        T s = T(0);
        for (int32_t k = 0; k < len; ++k, p += d.S) {
            const int32_t c = col[p];
            if (c < 0) break;
            s = fmadd(cvt<T>(val[p]), (T)g[c], s);
        }
        return s;
    }
    return row_dot<V, T>(d.rp, d.ci, (const V*)d.va, g, i);
}

// Writes the padded copy of every system whose layout is ELL or SELL-P
// (one block per system, grid-stride over systems).  SELL-P: slice lengths
// (longest row of the slice), then their exclusive scan, then the entries.
template <typename V>
__global__ void __launch_bounds__(256) k_batch_pad(SysDesc* __restrict__ sys, int32_t count) {
    for (int32_t sidx = blockIdx.x; sidx < count; sidx += gridDim.x) {
        SysDesc& d = sys[sidx];
        if (d.fmt == BL_CSR) continue;
        const int32_t n = d.n;
        const V* __restrict__ va = (const V*)d.va;
        V* __restrict__ pv = (V*)d.pval;
        if (d.fmt == BL_ELL) {
            for (int64_t i = threadIdx.x; i < d.pstride; i += blockDim.x) {
                const int32_t a = i < n ? d.rp[i] : 0, e = i < n ? d.rp[i + 1] : 0;
                for (int32_t k = 0; k < d.K; ++k) {
                    const int64_t p = (int64_t)k * d.pstride + i;
                    const bool in = a + k < e;
                    d.pcol[p] = in ? d.ci[a + k] : -1;
                    pv[p] = in ? va[a + k] : V(0.0f);
                }
            }
            continue;
        }
        const int32_t S = d.S, ns = (n + S - 1) / S;
        for (int32_t sl = threadIdx.x; sl < ns; sl += blockDim.x) {
            int32_t mx = 0;
            for (int32_t t = 0; t < S; ++t) {
                const int32_t i = sl * S + t;
                if (i < n) mx = max(mx, d.rp[i + 1] - d.rp[i]);
            }
            d.slen[sl] = mx;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int32_t acc = 0;
            for (int32_t sl = 0; sl < ns; ++sl) {
                d.sset[sl] = acc;
                acc += d.slen[sl];
            }
            d.sset[ns] = acc;
        }
        __syncthreads();
        for (int64_t i = threadIdx.x; i < (int64_t)ns * S; i += blockDim.x) {
            const int32_t sl = (int32_t)(i / S), t = (int32_t)(i - (int64_t)sl * S);
            const int32_t a = i < n ? d.rp[i] : 0, e = i < n ? d.rp[i + 1] : 0;
            const int64_t base = (int64_t)d.sset[sl] * S + t;
            for (int32_t k = 0; k < d.slen[sl]; ++k) {
                const int64_t p = base + (int64_t)k * S;
                const bool in = a + k < e;
                d.pcol[p] = in ? d.ci[a + k] : -1;
                pv[p] = in ? va[a + k] : V(0.0f);
            }
        }
        __syncthreads();
    }
}

// Jacobi inverse diagonal of row i; 0 when missing or zero.
template <typename V, typename T>
__device__ __forceinline__ T row_dinv(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                      const V* __restrict__ va, int32_t i) {
    T d = T(0);
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k)
        if (ci[k] == i) d += cvt<T>(va[k]);
    return d == T(0) ? T(0) : T(1) / d;
}

// Prepares a system: Jacobi diagonal (in work slot 0), ||b||, true residual.
// Returns false (and fills o) when the solve is already decided.
template <typename V, typename T, int L>
__device__ bool block_setup(const SysDesc& d, const BlockOpts& opt, T* dinv, T* r, double& bn,
                            double& thr, SysOut& o) {
    const int32_t n = d.n;
    const V* va = (const V*)d.va;
    const T* b = (const T*)d.b;
    T* x = (T*)d.x;
    VAcc<2> acc = vacc<2>();
    for_rows_vl(n, [&](int32_t i, int s) {
        const T bi = b[i];
        acc.v[0][s] = fma((double)bi, (double)bi, acc.v[0][s]);
        if (opt.prec) {
            const T di = row_dinv<V, T>(d.rp, d.ci, va, i);
            dinv[i] = di;
            if (di == T(0)) acc.v[1][s] = 1.0;
        }
    });
    double tot[2];
    vl_allsum<2>(acc, tot);
    o.iters = 0;
    o.restarts = 0;
    o.rec = o.tru = 0.0;
    if (tot[1] != 0.0) {
        o.status = GK_ERR_ZERO_DIAG;
        return false;
    }
    bn = sqrt(tot[0]);
    thr = d.tol * bn;
    if (bn == 0.0) {
        for (int32_t i = threadIdx.x; i < n; i += blockDim.x) x[i] = T(0);
        o.status = GK_OK;
        return false;
    }
    if (!isfinite(bn)) {
        o.status = GK_ERR_NAN;
        return false;
    }
    VAcc<1> rr = vacc<1>();
    for_rows_vl(n, [&](int32_t i, int s) {
        const T ri = b[i] - sys_row_dot<V, T, L>(d, x, i);
        r[i] = ri;
        rr.v[0][s] = fma((double)ri, (double)ri, rr.v[0][s]);
    });
    double t1[1];
    vl_allsum<1>(rr, t1);
    const double rn = sqrt(t1[0]);
    o.rec = o.tru = rn / bn;
    if (!isfinite(rn)) {
        o.status = GK_ERR_NAN;
        return false;
    }
    if (rn <= thr) {
        o.status = GK_OK;
        return false;
    }
    o.status = GK_NOT_CONVERGED;
    return true;
}

// r = b - A x in place; returns ||r||
template <typename V, typename T, int L>
__device__ double block_true_resid(const SysDesc& d, T* r) {
    const V* va = (const V*)d.va;
    const T* b = (const T*)d.b;
    const T* x = (const T*)d.x;
    VAcc<1> tt = vacc<1>();
    for_rows_vl(d.n, [&](int32_t i, int s) {
        const T ri = b[i] - sys_row_dot<V, T, L>(d, x, i);
        r[i] = ri;
        tt.v[0][s] = fma((double)ri, (double)ri, tt.v[0][s]);
    });
    double t[1];
    vl_allsum<1>(tt, t);
    return sqrt(t[0]);
}

// ---------------------------------------------------------------- CG
// work slots: 0 dinv, 1 r, 2 q, 3 scratch (final residual)
constexpr int BLOCK_MAX_THREADS = 512;

template <typename V, typename T, int L>
__global__ void __launch_bounds__(BLOCK_MAX_THREADS, 1) k_block_cg(const SysDesc* __restrict__ sys, SysOut* __restrict__ outs,
                           int32_t count, BlockOpts opt) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* ps = reinterpret_cast<T*>(smem_raw);
    for (int32_t sidx = blockIdx.x; sidx < count; sidx += gridDim.x) {
        const SysDesc d = sys[sidx];
        const int32_t n = d.n;
        const V* va = (const V*)d.va;
        T* x = (T*)d.x;
        T* dinv = (T*)d.work;
        T* r = dinv + d.ld;
        T* q = r + d.ld;
        T* scratch = q + d.ld;
        SysOut o;
        double bn = 0.0, thr = 0.0;
        if (block_setup<V, T, L>(d, opt, dinv, r, bn, thr, o)) {
            double rho = 0.0;
            auto init_dir = [&]() {
                VAcc<1> rz = vacc<1>();
                for_rows_vl(n, [&](int32_t i, int s) {
                    const T ri = r[i];
                    const T zi = opt.prec ? dinv[i] * ri : ri;
                    ps[i] = zi;
                    rz.v[0][s] = fma((double)ri, (double)zi, rz.v[0][s]);
                });
                double t[1];
                vl_allsum<1>(rz, t);
                rho = t[0];
            };
            init_dir();
            int32_t k = 0;
            while (k < opt.max_iters) {
                VAcc<1> pq = vacc<1>();
                for_rows_vl(n, [&](int32_t i, int s) {
                    const T sv = sys_row_dot<V, T, L>(d, ps, i);
                    q[i] = sv;
                    pq.v[0][s] = fma((double)ps[i], (double)sv, pq.v[0][s]);
                });
                double tp[1];
                vl_allsum<1>(pq, tp);
                if (!isfinite(tp[0])) { o.status = GK_ERR_NAN; break; }
                if (tp[0] <= 0.0) { o.status = GK_BREAKDOWN; break; }
                const double alpha = rho / tp[0];
                const T ta = (T)alpha;
                VAcc<2> a2 = vacc<2>();
                for_rows_vl(n, [&](int32_t i, int s) {
                    x[i] = fmadd(ta, ps[i], x[i]);
                    const T ri = fmadd(-ta, q[i], r[i]);
                    r[i] = ri;
                    const T zi = opt.prec ? dinv[i] * ri : ri;
                    a2.v[0][s] = fma((double)ri, (double)zi, a2.v[0][s]);
                    a2.v[1][s] = fma((double)ri, (double)ri, a2.v[1][s]);
                });
                double t2[2];
                vl_allsum<2>(a2, t2);
                ++k;
                const double rn = sqrt(t2[1]);
                o.rec = rn / bn;
                if (!isfinite(rn) || !isfinite(t2[0])) { o.status = GK_ERR_NAN; break; }
                if (rn <= thr) {
                    const double tn = block_true_resid<V, T, L>(d, r);
                    if (tn <= thr) { o.status = GK_OK; break; }
                    o.restarts += 1;  // residual replacement, restart from x
                    init_dir();
                    continue;
                }
                const double beta = t2[0] / rho;
                rho = t2[0];
                const T tb = (T)beta;
                for (int32_t i = threadIdx.x; i < n; i += blockDim.x) {
                    const T zi = opt.prec ? dinv[i] * r[i] : r[i];
                    ps[i] = fmadd(tb, ps[i], zi);
                }
                __syncthreads();
            }
            o.iters = k;
            o.tru = block_true_resid<V, T, L>(d, scratch) / bn;
        }
        if (threadIdx.x == 0) outs[sidx] = o;
        __syncthreads();
    }
}

// ---------------------------------------------------------------- BiCGSTAB
// work slots: 0 dinv, 1 r, 2 rhat, 3 p, 4 phat, 5 v, 6 s, 7 shat, 8 t
template <typename V, typename T, int L>
__global__ void __launch_bounds__(BLOCK_MAX_THREADS, 1) k_block_bicgstab(const SysDesc* __restrict__ sys, SysOut* __restrict__ outs,
                                 int32_t count, BlockOpts opt) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* gs = reinterpret_cast<T*>(smem_raw);  // gathered vector
    for (int32_t sidx = blockIdx.x; sidx < count; sidx += gridDim.x) {
        const SysDesc d = sys[sidx];
        const int32_t n = d.n;
        const V* va = (const V*)d.va;
        T* x = (T*)d.x;
        T* dinv = (T*)d.work;
        T *r = dinv + d.ld, *rh = r + d.ld, *p = rh + d.ld, *ph = p + d.ld, *v = ph + d.ld;
        T *sv = v + d.ld, *sh = sv + d.ld, *t = sh + d.ld;
        SysOut o;
        double bn = 0.0, thr = 0.0;
        if (block_setup<V, T, L>(d, opt, dinv, r, bn, thr, o)) {
            double rho = 1.0, alpha = 1.0, omega = 1.0, rho_new = 0.0;
            auto restart = [&]() {
                VAcc<1> a = vacc<1>();
                for_rows_vl(n, [&](int32_t i, int s) {
                    const T ri = r[i];
                    rh[i] = ri;
                    p[i] = T(0);
                    v[i] = T(0);
                    a.v[0][s] = fma((double)ri, (double)ri, a.v[0][s]);
                });
                double tt[1];
                vl_allsum<1>(a, tt);
                rho = alpha = omega = 1.0;
                rho_new = tt[0];
            };
            restart();
            int32_t k = 0;
            while (k < opt.max_iters) {
                if (!isfinite(rho_new)) { o.status = GK_ERR_NAN; break; }
                if (rho_new == 0.0) { o.status = GK_BREAKDOWN; break; }
                const T beta = (T)((rho_new / rho) * (alpha / omega));
                const T tw = (T)omega;
                for (int32_t i = threadIdx.x; i < n; i += blockDim.x) {
                    const T pi = fmadd(beta, fmadd(-tw, v[i], p[i]), r[i]);
                    p[i] = pi;
                    const T hi = opt.prec ? dinv[i] * pi : pi;
                    ph[i] = hi;
                    gs[i] = hi;
                }
                __syncthreads();
                VAcc<1> rv = vacc<1>();
                for_rows_vl(n, [&](int32_t i, int s) {
                    const T vi = sys_row_dot<V, T, L>(d, gs, i);
                    v[i] = vi;
                    rv.v[0][s] = fma((double)rh[i], (double)vi, rv.v[0][s]);
                });
                double trv[1];
                vl_allsum<1>(rv, trv);
                if (!isfinite(trv[0])) { o.status = GK_ERR_NAN; break; }
                if (trv[0] == 0.0) { o.status = GK_BREAKDOWN; break; }
                alpha = rho_new / trv[0];
                const T ta = (T)alpha;
                VAcc<1> ss = vacc<1>();
                for_rows_vl(n, [&](int32_t i, int s) {
                    const T si = fmadd(-ta, v[i], r[i]);
                    sv[i] = si;
                    ss.v[0][s] = fma((double)si, (double)si, ss.v[0][s]);
                });
                double tss[1];
                vl_allsum<1>(ss, tss);
                ++k;
                const double sn = sqrt(tss[0]);
                if (!isfinite(sn)) { o.status = GK_ERR_NAN; break; }
                if (sn <= thr) {  // half-step exit
                    for (int32_t i = threadIdx.x; i < n; i += blockDim.x) x[i] = fmadd(ta, ph[i], x[i]);
                    o.rec = sn / bn;
                    __syncthreads();
                    const double tn = block_true_resid<V, T, L>(d, r);
                    if (tn <= thr) { o.status = GK_OK; break; }
                    o.restarts += 1;
                    restart();
                    continue;
                }
                for (int32_t i = threadIdx.x; i < n; i += blockDim.x) {
                    const T hi = opt.prec ? dinv[i] * sv[i] : sv[i];
                    sh[i] = hi;
                    gs[i] = hi;
                }
                __syncthreads();
                VAcc<2> a2 = vacc<2>();
                for_rows_vl(n, [&](int32_t i, int s) {
                    const T ti = sys_row_dot<V, T, L>(d, gs, i);
                    t[i] = ti;
                    a2.v[0][s] = fma((double)ti, (double)sv[i], a2.v[0][s]);
                    a2.v[1][s] = fma((double)ti, (double)ti, a2.v[1][s]);
                });
                double t2[2];
                vl_allsum<2>(a2, t2);
                if (!isfinite(t2[0]) || !isfinite(t2[1])) { o.status = GK_ERR_NAN; break; }
                if (t2[1] == 0.0) { o.status = GK_BREAKDOWN; break; }
                omega = t2[0] / t2[1];
                if (omega == 0.0) { o.status = GK_BREAKDOWN; break; }
                const T to = (T)omega;
                VAcc<2> a3 = vacc<2>();
                for_rows_vl(n, [&](int32_t i, int s) {
                    x[i] = fmadd(to, sh[i], fmadd(ta, ph[i], x[i]));
                    const T ri = fmadd(-to, t[i], sv[i]);
                    r[i] = ri;
                    a3.v[0][s] = fma((double)rh[i], (double)ri, a3.v[0][s]);
                    a3.v[1][s] = fma((double)ri, (double)ri, a3.v[1][s]);
                });
                double t3[2];
                vl_allsum<2>(a3, t3);
                rho = rho_new;
                rho_new = t3[0];
                const double rn = sqrt(t3[1]);
                o.rec = rn / bn;
                if (!isfinite(rn)) { o.status = GK_ERR_NAN; break; }
                if (rn <= thr) {
                    const double tn = block_true_resid<V, T, L>(d, r);
                    if (tn <= thr) { o.status = GK_OK; break; }
                    o.restarts += 1;
                    restart();
                }
            }
            o.iters = k;
            o.tru = block_true_resid<V, T, L>(d, t) / bn;
        }
        if (threadIdx.x == 0) outs[sidx] = o;
        __syncthreads();
    }
}

// ---------------------------------------------------------------- host

static int nslots(int method) { return method == GK_CG ? 4 : 9; }

// Layout policy of a batch (picked by the autotuner per batch shape):
// layout BL_CSR runs every system on its CSR arrays; BL_ELL gives each system
// an ELL copy when ELL stores at most 1.2 x its nonzeros, else keeps its
// CSR; BL_SELLP gives each system a SELL-P copy with slices of S rows.
// nt: threads per block.  The untuned default (batches of fewer than
// TUNE_MIN_COUNT systems) is CSR with 256 threads: on lone serving-size systems (n 1,575 to
// 13,689; stencils and banded SPD) CSR took 0.31-0.65x the time of ELL or
// SELL-P(32) in the one-block kernel (e.g. 2D Laplacian n = 13,456: 33.8 ms
// against 56.8 ms with ELL).
constexpr int32_t TUNE_MIN_COUNT = 64;  // smallest batch the autotuner times

struct BatchCfg {
    int nt = 256;
    int layout = BL_CSR;
    int S = 32;
};

struct BatchBufs {
    DevBuf desc, outs, work, pad;
    SysDesc* hdesc = nullptr;
    SysOut* hout = nullptr;
    size_t hcap = 0;
    ~BatchBufs() {
        if (hdesc) cudaFreeHost(hdesc);
        if (hout) cudaFreeHost(hout);
        desc.release();
        outs.release();
        work.release();
        pad.release();
    }
};

// Buffers are pooled: a call takes a free set (or makes one) and returns it,
// so batches launched from different host threads run concurrently.
static std::mutex g_batch_mu;
static std::vector<BatchBufs*> g_batch_pool;

struct BatchLease {
    BatchBufs* b = nullptr;
    BatchLease() {
        std::lock_guard<std::mutex> lk(g_batch_mu);
        if (!g_batch_pool.empty()) {
            b = g_batch_pool.back();
            g_batch_pool.pop_back();
        }
        if (!b) b = new BatchBufs();
    }
    ~BatchLease() {
        std::lock_guard<std::mutex> lk(g_batch_mu);
        g_batch_pool.push_back(b);
    }
};

// The block kernel for a method, value type and batch layout (lay: the one
// layout of every system, or -1 for a mix).
template <typename V, typename T, int L>
static auto block_kernel(int method) {
    return method == GK_CG ? k_block_cg<V, T, L> : k_block_bicgstab<V, T, L>;
}

template <typename V, typename T>
static auto block_kernel(int method, int lay) {
    switch (lay) {
        case BL_CSR: return block_kernel<V, T, BL_CSR>(method);
        case BL_ELL: return block_kernel<V, T, BL_ELL>(method);
        case BL_SELLP: return block_kernel<V, T, BL_SELLP>(method);
        default: return block_kernel<V, T, -1>(method);
    }
}

template <typename V, typename T>
static gk_status launch_block(int method, int lay, const SysDesc* ddesc, SysOut* dout,
                              int32_t count, const BlockOpts& bo, int nt, size_t smem,
                              unsigned grid, cudaStream_t s) {
    auto k = block_kernel<V, T>(method, lay);
    GK_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    k<<<grid, nt, smem, s>>>(ddesc, dout, count, bo);
    GK_CUDA(cudaGetLastError());
    return GK_OK;
}

static size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

// Layout of system A under a policy, and the bytes of its padded copy.
static int sys_layout(const gk_matrix A, const BatchCfg& cfg, size_t* pad_bytes) {
    *pad_bytes = 0;
    if (A->n == 0 || A->nnz == 0 || cfg.layout == BL_CSR) return BL_CSR;
    const size_t sv = value_bytes(A->dtype);
    if (cfg.layout == BL_ELL) {
        const int64_t stride = ((int64_t)A->n + 31) / 32 * 32;
        if ((int64_t)A->max_row * A->n > A->nnz + A->nnz / 5) return BL_CSR;
        *pad_bytes = al256((size_t)A->max_row * stride * 4) + al256((size_t)A->max_row * stride * sv);
        return BL_ELL;
    }
    // SELL-P: at most the longest row in every slice
    const int64_t ns = ((int64_t)A->n + cfg.S - 1) / cfg.S;
    const size_t ent = (size_t)ns * cfg.S * A->max_row;
    *pad_bytes = al256(ent * 4) + al256(ent * sv) + al256(4 * (size_t)ns) + al256(4 * (size_t)(ns + 1));
    return BL_SELLP;
}

// Runs count systems; infos may be null.  All matrices CSR, same dtype.
static gk_status run_batch(int32_t count, const gk_matrix* As, const void* const* bs,
                           void* const* xs, const gk_solve_opts* o, gk_solve_info* infos,
                           cudaStream_t s, const BatchCfg& cfg, float* ms_out) {
    const int nt = cfg.nt;
    const gk_dtype dt = As[0]->dtype;
    const size_t vb = vector_bytes(dt);
    int32_t nmax = 0;
    size_t wbytes = 0, pbytes = 0;
    const int ns = nslots(o->method);
    for (int32_t i = 0; i < count; ++i) {
        nmax = std::max(nmax, As[i]->n);
        const size_t ld = (((size_t)As[i]->n * vb + 255) & ~(size_t)255) / vb;
        wbytes += ld * vb * ns;
        size_t pb = 0;
        sys_layout(As[i], cfg, &pb);
        pbytes += pb;
    }
    const size_t smem = std::max<size_t>((size_t)nmax * vb, 16);
    if (smem > 200 * 1024) return GK_ERR_UNSUPPORTED;
    BatchLease lease;
    BatchBufs& B = *lease.b;
    if (B.hcap < (size_t)count) {
        GateShared gate;
        if (B.hdesc) cudaFreeHost(B.hdesc);
        if (B.hout) cudaFreeHost(B.hout);
        B.hdesc = nullptr;
        B.hout = nullptr;
        GK_CUDA(cudaMallocHost(&B.hdesc, sizeof(SysDesc) * (size_t)count));
        GK_CUDA(cudaMallocHost(&B.hout, sizeof(SysOut) * (size_t)count));
        B.hcap = (size_t)count;
    }
    GK_TRY(B.desc.ensure(sizeof(SysDesc) * (size_t)count));
    GK_TRY(B.outs.ensure(sizeof(SysOut) * (size_t)count));
    GK_TRY(B.work.ensure(wbytes + 256));
    if (pbytes) GK_TRY(B.pad.ensure(pbytes + 256));
    char* w = (char*)B.work.ptr;
    char* pw = (char*)B.pad.ptr;
    bool any_pad = false;
    for (int32_t i = 0; i < count; ++i) {
        gk_matrix A = As[i];
        SysDesc& d = B.hdesc[i];
        std::memset(&d, 0, sizeof(d));
        d.n = A->n;
        size_t pb = 0;
        d.fmt = sys_layout(A, cfg, &pb);
        if (d.fmt == BL_ELL) {
            d.K = A->max_row;
            d.pstride = ((int64_t)A->n + 31) / 32 * 32;
            d.pcol = (int32_t*)pw;
            d.pval = pw + al256((size_t)d.K * d.pstride * 4);
        } else if (d.fmt == BL_SELLP) {
            d.S = cfg.S;
            d.K = A->max_row;
            const int64_t nsl = ((int64_t)A->n + cfg.S - 1) / cfg.S;
            const size_t ent = (size_t)nsl * cfg.S * A->max_row;
            d.pcol = (int32_t*)pw;
            d.pval = pw + al256(ent * 4);
            d.slen = (int32_t*)(pw + al256(ent * 4) + al256(ent * value_bytes(A->dtype)));
            d.sset = d.slen + al256(4 * (size_t)nsl) / 4;
        }
        pw += pb;
        any_pad |= d.fmt != BL_CSR;
        d.rp = A->row_ptr;
        d.ci = A->col;
        d.va = A->val;
        d.b = bs[i];
        d.x = xs[i];
        d.work = w;
        d.ld = (int64_t)((((size_t)A->n * vb + 255) & ~(size_t)255) / vb);
        d.tol = o->batch_tols ? o->batch_tols[i] : o->tol;
        w += (size_t)d.ld * vb * ns;
    }
    GK_CUDA(cudaMemcpyAsync(B.desc.ptr, B.hdesc, sizeof(SysDesc) * (size_t)count,
                            cudaMemcpyHostToDevice, s));
    BlockOpts bo{o->tol, o->max_iters, o->precond == GK_PRECOND_JACOBI};
    int occ = 1;
    const int sms = num_sms();
    cudaEvent_t e0, e1;
    GK_CUDA(cudaEventCreate(&e0));
    GK_CUDA(cudaEventCreate(&e1));
    GK_CUDA(cudaEventRecord(e0, s));
    gk_status st = GK_OK;
    if (any_pad) {  // the padded copies of this batch, one block per system
        const unsigned pg = (unsigned)std::min<int64_t>(count, (int64_t)sms * 8);
        SysDesc* dd = (SysDesc*)B.desc.ptr;
        if (dt == GK_F64) k_batch_pad<double><<<pg, 256, 0, s>>>(dd, count);
        else if (dt == GK_F32) k_batch_pad<float><<<pg, 256, 0, s>>>(dd, count);
        else k_batch_pad<__nv_bfloat16><<<pg, 256, 0, s>>>(dd, count);
        GK_CUDA(cudaGetLastError());
    }
    auto occ_of = [&](auto kern) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        int b = 1;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, nt, smem) != cudaSuccess || b < 1) b = 1;
        return b;
    };
    // one layout for the whole batch: the kernel without the per-row branch
    int lay = count > 0 ? B.hdesc[0].fmt : BL_CSR;
    for (int32_t i = 1; i < count && lay >= 0; ++i)
        if (B.hdesc[i].fmt != lay) lay = -1;
    if (dt == GK_F64) occ = occ_of(block_kernel<double, double>(o->method, lay));
    else if (dt == GK_F32) occ = occ_of(block_kernel<float, float>(o->method, lay));
    else occ = occ_of(block_kernel<__nv_bfloat16, float>(o->method, lay));
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(count, (int64_t)sms * occ));
    const SysDesc* dd = (const SysDesc*)B.desc.ptr;
    SysOut* dout = (SysOut*)B.outs.ptr;
    if (dt == GK_F64)
        st = launch_block<double, double>(o->method, lay, dd, dout, count, bo, nt, smem, grid, s);
    else if (dt == GK_F32)
        st = launch_block<float, float>(o->method, lay, dd, dout, count, bo, nt, smem, grid, s);
    else
        st = launch_block<__nv_bfloat16, float>(o->method, lay, dd, dout, count, bo, nt, smem,
                                                grid, s);
    GK_CUDA(cudaEventRecord(e1, s));
    if (st == GK_OK) {
        GK_CUDA(cudaMemcpyAsync(B.hout, B.outs.ptr, sizeof(SysOut) * (size_t)count,
                                cudaMemcpyDeviceToHost, s));
        GK_CUDA(cudaStreamSynchronize(s));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms_out) *ms_out = ms;
        if (infos)
            for (int32_t i = 0; i < count; ++i) {
                const SysOut& so = B.hout[i];
                infos[i].status = (gk_status)so.status;
                infos[i].iters = so.iters;
                infos[i].restarts = so.restarts;
                infos[i].outer_iters = 0;
                infos[i].rel_res_recurrence = so.rec;
                infos[i].rel_res_true = so.tru;
                infos[i].device_ms = ms;
                infos[i].spmv_format = B.hdesc[i].fmt == BL_ELL     ? GK_ELL
                                       : B.hdesc[i].fmt == BL_SELLP ? GK_SELLP
                                                                    : GK_CSR;
                infos[i].block_threads = nt;
                infos[i].slice_size = B.hdesc[i].fmt == BL_SELLP ? cfg.S : 0;
            }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}


gk_status solve_small(gk_matrix A, const void* b, void* x, const gk_solve_opts* o, cudaStream_t s,
                      SolveOut* out) {
    if (A->fmt != GK_CSR || o->method == GK_GMRES || o->method == GK_CGS || A->dtype == GK_F16 ||
        o->precond >= GK_PRECOND_BLOCK_JACOBI)
        return GK_ERR_UNSUPPORTED;
    gk_solve_info info;
    std::memset(&info, 0, sizeof(info));
    gk_matrix As[1] = {A};
    const void* bs[1] = {b};
    void* xs[1] = {x};
    BatchCfg cfg;
    cfg.nt = BLOCK_MAX_THREADS;
    GK_TRY(run_batch(1, As, bs, xs, o, &info, s, cfg, nullptr));
    out->status = info.status;
    out->iters = info.iters;
    out->restarts = info.restarts;
    out->rec = info.rel_res_recurrence;
    out->tru = info.rel_res_true;
    out->layout = info.spmv_format;
    out->slice = info.slice_size;
    out->threads = info.block_threads;
    return GK_OK;
}

// ------------------------------------------------------------ autotuner
// The configuration of a batch shape -- each system's SpMV layout (policy
// CSR, ELL where its padding is at most 20 %, or SELL-P with slices of
// S = 8, 16 or 32 rows) and the threads per block (128, 256, 512, which set
// how many rows a warp and a thread take per sweep) -- is picked by timing
// every candidate on a run of the batch itself capped at 30 iterations (the
// callers' initial guesses are saved before and restored after the trials)
// and cached per key: value type, method, preconditioner, log2 of the
// largest n and of the system count.  No candidate changes a result: every
// layout sums a row in CSR order and the reductions use fixed virtual lanes.
static std::mutex g_tune_mu;
static std::map<uint64_t, BatchCfg> g_tune;

static uint64_t tune_key(gk_dtype dt, const gk_solve_opts* o, int32_t nmax, int32_t count) {
    auto lg = [](int64_t v) {
        int b = 0;
        while ((1ll << b) < v) ++b;
        return (uint64_t)b;
    };
    return ((uint64_t)dt << 40) | ((uint64_t)o->method << 36) | ((uint64_t)o->precond << 32) |
           (lg(nmax) << 16) | lg(count);
}

static gk_status autotune(int32_t count, const gk_matrix* As, const void* const* bs,
                          void* const* xs, const gk_solve_opts* o, cudaStream_t s,
                          BatchCfg* best) {
    const size_t vb = vector_bytes(As[0]->dtype);
    size_t total = 0;
    for (int32_t i = 0; i < count; ++i) total += (size_t)As[i]->n * vb;
    DevBuf save;
    GK_TRY(save.ensure(total + 256));
    auto copy_all = [&](bool to_save) -> gk_status {
        size_t off = 0;
        for (int32_t i = 0; i < count; ++i) {
            const size_t b = (size_t)As[i]->n * vb;
            char* sp = static_cast<char*>(save.ptr) + off;
            if (b)
                GK_CUDA(cudaMemcpyAsync(to_save ? (void*)sp : xs[i], to_save ? xs[i] : (void*)sp, b,
                                        cudaMemcpyDeviceToDevice, s));
            off += b;
        }
        return GK_OK;
    };
    GK_TRY(copy_all(true));
    gk_solve_opts trial = *o;
    trial.max_iters = std::min(o->max_iters, 30);
    float best_ms = 1e30f;
    *best = BatchCfg();
    const int layouts[5][2] = {{BL_CSR, 0}, {BL_ELL, 0}, {BL_SELLP, 8}, {BL_SELLP, 16}, {BL_SELLP, 32}};
    for (const auto& L : layouts)
        for (int nt : {128, 256, 512}) {
            BatchCfg c;
            c.layout = L[0];
            c.S = L[0] == BL_SELLP ? L[1] : 32;
            c.nt = nt;
            GK_TRY(copy_all(false));
            float ms = 0.f;
            GK_TRY(run_batch(count, As, bs, xs, &trial, nullptr, s, c, &ms));
            if (ms < best_ms) {
                best_ms = ms;
                *best = c;
            }
        }
    GK_TRY(copy_all(false));
    GK_CUDA(cudaStreamSynchronize(s));
    save.release();
    return GK_OK;
}

// GK_BATCH_LAYOUT = csr | ell | sellp8 | sellp16 | sellp32 | sellp64 forces a layout
// policy; GK_BATCH_THREADS = 128 | 256 | 512 forces the block size.
static bool forced_layout(BatchCfg* c) {
    const char* e = getenv("GK_BATCH_LAYOUT");
    if (!e) return false;
    if (!strcmp(e, "csr")) c->layout = BL_CSR;
    else if (!strcmp(e, "ell")) c->layout = BL_ELL;
    else if (!strncmp(e, "sellp", 5)) {
        const int S = atoi(e + 5);
        if (S != 8 && S != 16 && S != 32 && S != 64) return false;
        c->layout = BL_SELLP;
        c->S = S;
    } else {
        return false;
    }
    return true;
}

}  // namespace gk

using namespace gk;

extern "C" gk_status gk_solve_batched(int32_t count, const gk_matrix* As, const void* const* bs,
                                      void* const* xs, const gk_solve_opts* o,
                                      gk_solve_info* infos, void* stream) {
    if (count < 0 || !o || (count > 0 && (!As || !bs || !xs))) return GK_ERR_INVALID;
    if (count == 0) return GK_OK;
    if (o->method == GK_GMRES || o->method == GK_CGS || o->precond >= GK_PRECOND_BLOCK_JACOBI)
        return GK_ERR_UNSUPPORTED;
    if ((o->method != GK_CG && o->method != GK_BICGSTAB) || o->mixed ||
        (o->precond != GK_PRECOND_NONE && o->precond != GK_PRECOND_JACOBI) || !(o->tol >= 0.0) ||
        o->max_iters < 0)
        return GK_ERR_INVALID;
    if (o->batch_tols)
        for (int32_t i = 0; i < count; ++i)
            if (!(o->batch_tols[i] >= 0.0)) return GK_ERR_INVALID;
    int dev = -1;
    cudaGetDevice(&dev);
    for (int32_t i = 0; i < count; ++i) {
        const gk_matrix A = As[i];
        if (A && A->dtype == GK_F16) return GK_ERR_UNSUPPORTED;  // multi-kernel engine only
        if (!A || A->fmt != GK_CSR || A->n != A->ncols || A->dtype != As[0]->dtype ||
            A->n > 16384 || (A->n > 0 && (!bs[i] || !xs[i])))
            return GK_ERR_INVALID;
        if (A->device != dev) return GK_ERR_UNSUPPORTED;
    }
    cudaStream_t s = (cudaStream_t)stream;
    BatchCfg cfg;  // untuned default: CSR, 256 threads
    int nt = 0;
    if (const char* e = getenv("GK_BATCH_THREADS")) nt = atoi(e);
    const bool fnt = nt == 128 || nt == 256 || nt == 512;
    const bool flay = forced_layout(&cfg);
    const char* at = getenv("GK_AUTOTUNE");
    // batches of fewer than TUNE_MIN_COUNT systems run the untuned default:
    // their trial runs cost more than a better layout saves (the serving
    // loop's varying small batches, each a new shape, lost ~20 % of their
    // throughput to them: 81 against 100 solves/s at saturation)
    if (!(fnt && flay) && !(at && at[0] == '0') && count >= TUNE_MIN_COUNT) {
        int32_t nmax = 0;
        for (int32_t i = 0; i < count; ++i) nmax = std::max(nmax, As[i]->n);
        const uint64_t key = tune_key(As[0]->dtype, o, nmax, count);
        bool found = false;
        BatchCfg tuned;
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto it = g_tune.find(key);
            if (it != g_tune.end()) {
                tuned = it->second;
                found = true;
            }
        }
        if (!found) {
            GK_TRY(autotune(count, As, bs, xs, o, s, &tuned));
            std::lock_guard<std::mutex> lk(g_tune_mu);
            g_tune[key] = tuned;
        }
        if (!flay) {
            cfg.layout = tuned.layout;
            cfg.S = tuned.S;
        }
        if (!fnt) cfg.nt = tuned.nt;
    }
    if (fnt) cfg.nt = nt;
    return run_batch(count, As, bs, xs, o, infos, s, cfg, nullptr);
}
