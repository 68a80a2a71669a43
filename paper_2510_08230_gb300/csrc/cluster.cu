// cluster.cu - cluster engine: one thread-block cluster (up to 16 blocks,
// one per SM) runs a whole CG solve of one small system.
//
// CG (optional Jacobi) with the stopping rule and residual replacement of
// the other CG engines (stopping per Listing 2; the true residual confirms
// convergence).  Block r of the cluster owns rows [r*rpb, (r+1)*rpb); each
// thread keeps up to RMAX of those rows' iterates and inverse diagonal in
// registers.  The vector the SpMV gathers from (the direction or u = M^-1 r,
// or x for the true residual) lives in the owners' shared memory and is
// read across the cluster through distributed shared memory.  A reduction
// is a fixed-order block sum, a cluster barrier, and every thread summing
// the C block partials in rank order, so all blocks take identical
// decisions and the result does not depend on timing.  Per CG iteration:
// two cluster barriers with the single-reduction (Chronopoulos-Gear)
// recurrence, the default, or three with Hestenes-Stiefel; no kernel
// launches.  The block's rows are staged in shared memory once per solve
// (see staged_row_dot) when they fit.
#include <cooperative_groups.h>
#include <cstring>
#include <type_traits>

#include "prims.cuh"

namespace cgx = cooperative_groups;

namespace gk {

constexpr int CL_THREADS = 256;
constexpr int CL_RMAX = 4;
constexpr int CL_MAX_BLOCKS = 16;

struct ClusterArgs {
    int32_t n;
    int32_t rpb;  // rows per block
    uint32_t rpb_inv;  // rpb > 1: floor(2^32 / rpb) + 1 (owner = umulhi(col, rpb_inv)); 0: rpb = 1
    const int32_t* rp;
    const int32_t* ci;
    const void* va;
    const void* b;
    void* x;
    double tol;
    int32_t max_iters;
    int32_t prec;
    SolveOut* out;
};

// Sum of NA <= 3 per-thread values over the cluster, identical in all
// threads.  On this part the FP64 pipe is narrow and a dependent FP64
// operation has a long latency, so the tree is shallow and issues few
// FP64 instructions: the threads store their values, warp a (one per SM
// sub-partition) sums value a - 8 per lane added pairwise, then a 5-level
// shuffle tree - and stores the block partial; one cluster barrier; warp a
// loads the C block partials of value a (lane l from block l) and a
// 4-level shuffle tree (C <= 16) finishes.  Every block evaluates the same
// tree over the same values, so all take identical decisions.  fin(tot)
// runs on thread 0 alone before the block barrier that publishes the
// totals: the scalar work on them (divisions, decisions) writes its
// results to shared memory for the block.
// The cluster barrier of this kernel.  Blocks exchange data through
// shared memory only (the gathered vector g_s, the reduction partials red);
// global memory is read at the start and written by each block for its
// own rows at the end.  So the arrive releases this block's shared-memory
// writes only (a restricted release fence, then a relaxed arrive; the wait
// acquires), which keeps the barrier from waiting on the memory system.  A
// remote read of another block's shared memory is ordered before that
// block's later overwrite by the barrier between them and by the read's
// value being stored to this block's shared memory before this block
// arrives.
__device__ __forceinline__ void cluster_sync_smem() {
    asm volatile(
        "fence.release.sync_restrict::shared::cta.cluster;\n\t"
        "barrier.cluster.arrive.relaxed;\n\t"
        "barrier.cluster.wait.acquire;" ::: "memory");
}

struct NoFin {
    __device__ __forceinline__ void operator()(const double*) const {}
};

template <int NA, class Fin = NoFin>
__device__ __forceinline__ void cluster_allsum(cgx::cluster_group& cl, double (&v)[NA],
                                               double (*red)[4], int& tog, Fin fin = Fin()) {
    static_assert(NA >= 1 && NA <= 3 && CL_THREADS == 256, "one warp per value, 8 per lane");
    __shared__ double sh[NA][CL_THREADS];
    __shared__ double tot[4];
    const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
#pragma unroll
    for (int a = 0; a < NA; ++a) sh[a][threadIdx.x] = v[a];
    __syncthreads();
    if (warp < (unsigned)NA) {
        const double* w = sh[warp];
        double t = ((w[lane] + w[lane + 32]) + (w[lane + 64] + w[lane + 96])) +
                   ((w[lane + 128] + w[lane + 160]) + (w[lane + 192] + w[lane + 224]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) red[tog][warp] = t;
    }
    cluster_sync_smem();
    if (warp < (unsigned)NA) {
        double t = 0.0;
        if (lane < cl.num_blocks()) t = cl.map_shared_rank(red, lane)[tog][warp];
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) tot[warp] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) fin(tot);
    __syncthreads();
#pragma unroll
    for (int a = 0; a < NA; ++a) v[a] = tot[a];
    tog ^= 1;
}

template <typename V, typename T>
__device__ __forceinline__ T cluster_row_dot(cgx::cluster_group& cl, const ClusterArgs& A,
                                             const V* __restrict__ va, T* g_s, int32_t i,
                                             unsigned my_rank) {
    T s = T(0);
    const int32_t e = A.rp[i + 1];
    for (int32_t k = A.rp[i]; k < e; ++k) {
        const int32_t c = A.ci[k];
        const unsigned owner = A.rpb_inv ? __umulhi((unsigned)c, A.rpb_inv) : (unsigned)c;  // c / rpb
        const int32_t loc = c - (int32_t)owner * A.rpb;
        const T gv = owner == my_rank ? g_s[loc] : cl.map_shared_rank(g_s, owner)[loc];
        s = fmadd(cvt<T>(va[k]), gv, s);
    }
    return s;
}

// The block's rows staged once per solve (the matrix does not change while
// it runs): value (in the vector type, converted exactly) and source
// (owner rank << 16 | offset in the owner's part) of every entry, in CSR
// order, so that an SpMV issues a row's remote gathers back to back.
template <typename T, int U = 4>
__device__ __forceinline__ T staged_row_dot(cgx::cluster_group& cl, const T* s_val,
                                            const uint32_t* s_src, int32_t a, int32_t e,
                                            T* g_s) {
    T s = T(0);
    for (int32_t k0 = a; k0 < e; k0 += U) {
        T v[U], g[U];
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (k0 + u < e) {
                const uint32_t src = s_src[k0 + u];
                v[u] = s_val[k0 + u];
                g[u] = cl.map_shared_rank(g_s, src >> 16)[src & 0xFFFFu];
            }
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (k0 + u < e) s = fmadd(v[u], g[u], s);
    }
    return s;
}

// SR = false: Hestenes-Stiefel CG, three cluster barriers per iteration
// (publish p; reduce <p, Ap>; reduce <r, z>, ||r||^2).  SR = true: the
// same iterates computed with one reduction per iteration (the
// Chronopoulos-Gear recurrence: s = A p carried by its own update, so
// <r, u>, <A u, u> and ||r||^2 are reduced together after the SpMV of
// u = M^-1 r), two cluster barriers per iteration (publish u; reduce).
template <typename V, typename T, bool STAGED, bool SR>
__global__ void __launch_bounds__(CL_THREADS, 1) k_cluster_cg(ClusterArgs A) {
    cgx::cluster_group cl = cgx::this_cluster();
    const unsigned rank = cl.block_rank();
    __shared__ T g_s[CL_RMAX * CL_THREADS];  // owned part of the gathered vector
    extern __shared__ __align__(16) unsigned char cl_dyn[];  // staged rows (STAGED)
    __shared__ double red[2][4];
    // scalars of the iteration, computed by thread 0 (see cluster_allsum):
    // 0 rho (SR: gamma = <r, u>), 1 alpha, 2 beta, 3 status (0 go on,
    // 1 NaN, 2 breakdown, 3 recurrence residual passed), 4 (SR) kappa =
    // gamma * alpha of the previous iteration
    __shared__ double sc[5];
    int tog = 0;
    const V* va = (const V*)A.va;
    const T* b = (const T*)A.b;
    T* xg = (T*)A.x;
    const int32_t r0 = (int32_t)rank * A.rpb;
    const int32_t nloc = max(0, min(A.rpb, A.n - r0));
    T x[CL_RMAX], r[CL_RMAX], q[CL_RMAX], di[CL_RMAX];
    T p[SR ? CL_RMAX : 1], w[SR ? CL_RMAX : 1];  // SR: p in registers (g_s holds u), q = s
    double acc2[2] = {0.0, 0.0};
    // staged rows: entries [e0, e1) of the CSR belong to this block
    const int32_t e0 = nloc > 0 ? A.rp[r0] : 0, e1 = nloc > 0 ? A.rp[r0 + nloc] : 0;
    T* s_val = reinterpret_cast<T*>(cl_dyn);
    uint32_t* s_src = reinterpret_cast<uint32_t*>(cl_dyn + (((size_t)(e1 - e0) * sizeof(T) + 15) & ~(size_t)15));
    int32_t ra[CL_RMAX], re[CL_RMAX];  // this thread's rows in the staged arrays
    if constexpr (STAGED) {
        for (int32_t k = e0 + (int32_t)threadIdx.x; k < e1; k += CL_THREADS) {
            const int32_t c = A.ci[k];
            const unsigned owner = A.rpb_inv ? __umulhi((unsigned)c, A.rpb_inv) : (unsigned)c;
            s_val[k - e0] = cvt<T>(va[k]);
            s_src[k - e0] = (owner << 16) | (uint32_t)(c - (int32_t)owner * A.rpb);
        }
#pragma unroll
        for (int k = 0; k < CL_RMAX; ++k) {
            const int32_t li = (int32_t)threadIdx.x + k * CL_THREADS;
            ra[k] = li < nloc ? A.rp[r0 + li] - e0 : 0;
            re[k] = li < nloc ? A.rp[r0 + li + 1] - e0 : 0;
        }
    }
    // row i = r0 + li of this block times the gathered vector
    auto row_dot = [&](int k, int32_t li) -> T {
        if constexpr (STAGED) return staged_row_dot<T>(cl, s_val, s_src, ra[k], re[k], g_s);
        else return cluster_row_dot<V, T>(cl, A, va, g_s, r0 + li, rank);
    };
    // x into shared memory (for the initial residual), b norm, Jacobi diagonal
#pragma unroll
    for (int k = 0; k < CL_RMAX; ++k) {
        const int32_t li = (int32_t)threadIdx.x + k * CL_THREADS;
        x[k] = r[k] = q[k] = T(0);
        di[k] = T(1);
        if (li < nloc) {
            const int32_t i = r0 + li;
            x[k] = xg[i];
            g_s[li] = x[k];
            const T bi = b[i];
            acc2[0] = fma((double)bi, (double)bi, acc2[0]);
            if (A.prec) {
                T d = T(0);
                for (int32_t kk = A.rp[i]; kk < A.rp[i + 1]; ++kk)
                    if (A.ci[kk] == i) d += cvt<T>(va[kk]);
                if (d == T(0)) acc2[1] = 1.0;
                di[k] = d == T(0) ? T(0) : T(1) / d;
            }
        }
    }
    cluster_allsum<2>(cl, acc2, red, tog);  // includes the barrier that publishes g_s
    SolveOut o;
    o.status = GK_NOT_CONVERGED;
    const double bn = sqrt(acc2[0]);
    const double thr = A.tol * bn;
    // the iterations test ||r||^2 <= thr^2 (no square root on the critical
    // path); rec2 keeps the last ||r||^2 for the report
    const double thr2 = thr * thr;
    double rec2 = -1.0;
    bool run = true;
    if (acc2[1] != 0.0) {
        o.status = GK_ERR_ZERO_DIAG;
        run = false;
    } else if (bn == 0.0) {
#pragma unroll
        for (int k = 0; k < CL_RMAX; ++k) {
            const int32_t li = (int32_t)threadIdx.x + k * CL_THREADS;
            if (li < nloc) xg[r0 + li] = T(0);
        }
        o.status = GK_OK;
        run = false;
    } else if (!isfinite(bn)) {
        o.status = GK_ERR_NAN;
        run = false;
    }
    // r = b - A x (gathering x)
    auto true_resid = [&](double& nrm) {
        double a[1] = {0.0};
#pragma unroll
        for (int k = 0; k < CL_RMAX; ++k) {
            const int32_t li = (int32_t)threadIdx.x + k * CL_THREADS;
            if (li < nloc) {
                const int32_t i = r0 + li;
                r[k] = b[i] - row_dot(k, li);
                a[0] = fma((double)r[k], (double)r[k], a[0]);
            }
        }
        cluster_allsum<1>(cl, a, red, tog);
        nrm = sqrt(a[0]);
    };
    // p = z = M^-1 r into shared memory; rho = <r, z>
    auto init_dir = [&](double& rho) {
        double a[1] = {0.0};
        cluster_sync_smem();  // every block is done gathering from g_s
#pragma unroll
        for (int k = 0; k < CL_RMAX; ++k) {
            const int32_t li = (int32_t)threadIdx.x + k * CL_THREADS;
            if (li < nloc) {
                const T z = A.prec ? di[k] * r[k] : r[k];
                g_s[li] = z;
                a[0] = fma((double)r[k], (double)z, a[0]);
            }
        }
        cluster_allsum<1>(cl, a, red, tog, [&](const double* t) { sc[0] = t[0]; });
        rho = a[0];  // its barrier published p and sc[0] = rho
    };
    int32_t it = 0;
    double rho = 0.0;
    if (run) {
        double rn = 0.0;
        true_resid(rn);
        o.rec = o.tru = rn / bn;
        if (!isfinite(rn)) {
            o.status = GK_ERR_NAN;
            run = false;
        } else if (rn <= thr) {
            o.status = GK_OK;
            run = false;
        }
    }
    if constexpr (SR) {
        // u = M^-1 r into shared memory, w = A u, p = s = 0; alpha =
        // gamma / delta with gamma = <r, u>, delta = <w, u>, beta = 0
        auto sr_start = [&]() {
            cluster_sync_smem();  // every block is done gathering from g_s
#pragma unroll
            for (int k = 0; k < CL_RMAX; ++k) {
                const int32_t li = (int32_t)threadIdx.x + k * CL_THREADS;
                p[k] = q[k] = T(0);
                if (li < nloc) g_s[li] = A.prec ? di[k] * r[k] : r[k];
            }
            cluster_sync_smem();  // u published
            double a[2] = {0.0, 0.0};
#pragma unroll
            for (int k = 0; k < CL_RMAX; ++k) {
                const int32_t li = (int32_t)threadIdx.x + k * CL_THREADS;
                if (li < nloc) {
                    w[k] = row_dot(k, li);
                    const T u = g_s[li];
                    a[0] = fma((double)r[k], (double)u, a[0]);
                    a[1] = fma((double)w[k], (double)u, a[1]);
                }
            }
            cluster_allsum<2>(cl, a, red, tog, [&](const double* t) {
                sc[3] = !isfinite(t[0]) || !isfinite(t[1]) ? 1.0 : t[1] <= 0.0 ? 2.0 : 0.0;
                sc[0] = t[0];
                sc[1] = t[0] / t[1];
                sc[2] = 0.0;
                sc[4] = t[0] * sc[1];
            });
        };
        if (run) sr_start();
        while (run && it < A.max_iters) {
            if (sc[3] == 1.0) { o.status = GK_ERR_NAN; break; }
            if (sc[3] == 2.0) { o.status = GK_BREAKDOWN; break; }
            const T ta = (T)sc[1], tb = (T)sc[2];
            double a[3] = {0.0, 0.0, 0.0};  // <r, u>, <w, u>, ||r||^2
            // every block finished its gathers of u before the reduction
            // barrier that produced alpha and beta: u may be overwritten
#pragma unroll
            for (int k = 0; k < CL_RMAX; ++k) {
                const int32_t li = (int32_t)threadIdx.x + k * CL_THREADS;
                if (li < nloc) {
                    p[k] = fmadd(tb, p[k], g_s[li]);
                    q[k] = fmadd(tb, q[k], w[k]);  // s = A p
                    x[k] = fmadd(ta, p[k], x[k]);
                    r[k] = fmadd(-ta, q[k], r[k]);
                    const T u = A.prec ? di[k] * r[k] : r[k];
                    g_s[li] = u;
                    a[0] = fma((double)r[k], (double)u, a[0]);
                    a[2] = fma((double)r[k], (double)r[k], a[2]);
                }
            }
            cluster_sync_smem();  // u published
#pragma unroll
            for (int k = 0; k < CL_RMAX; ++k) {
                const int32_t li = (int32_t)threadIdx.x + k * CL_THREADS;
                if (li < nloc) {
                    w[k] = row_dot(k, li);
                    a[1] = fma((double)w[k], (double)g_s[li], a[1]);
                }
            }
            // beta = gamma' / gamma; alpha = gamma' / (delta - beta gamma' /
            // alpha_old) = gamma' kappa / (delta kappa - gamma'^2) with
            // kappa = gamma alpha_old (two independent divisions)
            cluster_allsum<3>(cl, a, red, tog, [&](const double* t) {
                rec2 = t[2];  // thread 0 reports sqrt(rec2) / ||b||
                if (!isfinite(t[2]) || !isfinite(t[0]) || !isfinite(t[1])) {
                    sc[3] = 1.0;
                } else if (t[2] <= thr2) {
                    sc[3] = 3.0;
                } else {
                    const double kap = sc[4];
                    const double den = t[1] * kap - t[0] * t[0];
                    sc[2] = t[0] / sc[0];
                    sc[1] = t[0] * kap / den;
                    sc[3] = den > 0.0 && isfinite(sc[1]) ? 0.0 : 2.0;
                    sc[0] = t[0];
                    sc[4] = t[0] * sc[1];
                }
            });
            ++it;
            if (sc[3] == 3.0) {
                // publish x, recompute the true residual, restart on failure
#pragma unroll
                for (int k = 0; k < CL_RMAX; ++k) {
                    const int32_t li = (int32_t)threadIdx.x + k * CL_THREADS;
                    if (li < nloc) g_s[li] = x[k];
                }
                cluster_sync_smem();
                double tn = 0.0;
                true_resid(tn);
                if (tn <= thr) { o.status = GK_OK; break; }
                o.restarts += 1;
                sr_start();
            }
        }
        run = false;  // the Hestenes-Stiefel loop below does not run
    }
    if (run) init_dir(rho);
    while (run && it < A.max_iters) {
        double pq[1] = {0.0};
#pragma unroll
        for (int k = 0; k < CL_RMAX; ++k) {
            const int32_t li = (int32_t)threadIdx.x + k * CL_THREADS;
            if (li < nloc) {
                q[k] = row_dot(k, li);
                pq[0] = fma((double)g_s[li], (double)q[k], pq[0]);
            }
        }
        cluster_allsum<1>(cl, pq, red, tog, [&](const double* t) {
            sc[3] = !isfinite(t[0]) ? 1.0 : t[0] <= 0.0 ? 2.0 : 0.0;
            sc[1] = sc[0] / t[0];
        });
        if (sc[3] == 1.0) { o.status = GK_ERR_NAN; break; }
        if (sc[3] == 2.0) { o.status = GK_BREAKDOWN; break; }
        const T ta = (T)sc[1];
        double a2[2] = {0.0, 0.0};
#pragma unroll
        for (int k = 0; k < CL_RMAX; ++k) {
            const int32_t li = (int32_t)threadIdx.x + k * CL_THREADS;
            if (li < nloc) {
                x[k] = fmadd(ta, g_s[li], x[k]);
                r[k] = fmadd(-ta, q[k], r[k]);
                const T z = A.prec ? di[k] * r[k] : r[k];
                a2[0] = fma((double)r[k], (double)z, a2[0]);
                a2[1] = fma((double)r[k], (double)r[k], a2[1]);
            }
        }
        cluster_allsum<2>(cl, a2, red, tog, [&](const double* t) {
            rec2 = t[1];  // thread 0 reports sqrt(rec2) / ||b||
            if (!isfinite(t[1]) || !isfinite(t[0])) {
                sc[3] = 1.0;
            } else if (t[1] <= thr2) {
                sc[3] = 3.0;
            } else {
                sc[3] = 0.0;
                sc[2] = t[0] / sc[0];
                sc[0] = t[0];
            }
        });
        ++it;
        if (sc[3] == 1.0) { o.status = GK_ERR_NAN; break; }
        if (sc[3] == 3.0) {
            // publish x, recompute the true residual, replace r on failure
#pragma unroll
            for (int k = 0; k < CL_RMAX; ++k) {
                const int32_t li = (int32_t)threadIdx.x + k * CL_THREADS;
                if (li < nloc) g_s[li] = x[k];
            }
            cluster_sync_smem();
            double tn = 0.0;
            true_resid(tn);
            if (tn <= thr) { o.status = GK_OK; break; }
            o.restarts += 1;
            init_dir(rho);
            continue;
        }
        const T tb = (T)sc[2];
#pragma unroll
        for (int k = 0; k < CL_RMAX; ++k) {
            const int32_t li = (int32_t)threadIdx.x + k * CL_THREADS;
            if (li < nloc) {
                const T z = A.prec ? di[k] * r[k] : r[k];
                g_s[li] = fmadd(tb, g_s[li], z);
            }
        }
        cluster_sync_smem();
    }
    o.iters = it;
    if (rec2 >= 0.0) o.rec = sqrt(rec2) / bn;
    // write x back and recompute the true residual for the report
    if (o.status != GK_ERR_ZERO_DIAG && bn > 0.0) {
        cluster_sync_smem();
#pragma unroll
        for (int k = 0; k < CL_RMAX; ++k) {
            const int32_t li = (int32_t)threadIdx.x + k * CL_THREADS;
            if (li < nloc) {
                xg[r0 + li] = x[k];
                g_s[li] = x[k];
            }
        }
        cluster_sync_smem();
        double tn = 0.0;
        true_resid(tn);
        o.tru = tn / bn;
    }
    cl.sync();  // no block leaves while others may read its shared memory
    if (rank == 0 && threadIdx.x == 0) *A.out = o;
}

// Largest n the cluster engine takes.
int32_t cluster_max_n() { return CL_MAX_BLOCKS * CL_RMAX * CL_THREADS; }

// One CG solve on a cluster of C blocks.  Returns GK_ERR_UNSUPPORTED when
// the system does not fit or the cluster cannot be scheduled.
gk_status solve_cluster(gk_matrix A, const void* b, void* x, const gk_solve_opts* o,
                        cudaStream_t s, SolveOut* out) {
    if (A->fmt != GK_CSR || o->method != GK_CG || A->n > cluster_max_n() || A->dtype == GK_F16 ||
        o->precond >= GK_PRECOND_BLOCK_JACOBI)
        return GK_ERR_UNSUPPORTED;
    int C = 16;
    if (const char* e = getenv("GK_CLUSTER_BLOCKS")) C = atoi(e);
    C = std::max(1, std::min(C, CL_MAX_BLOCKS));
    while (C > 1 && (A->n + C - 1) / C > CL_RMAX * CL_THREADS) ++C;
    const int32_t rpb = (A->n + C - 1) / C;
    if (rpb > CL_RMAX * CL_THREADS || C > CL_MAX_BLOCKS) return GK_ERR_UNSUPPORTED;
    static thread_local DevBuf outbuf;
    static thread_local SolveOut* hout = nullptr;
    GK_TRY(outbuf.ensure(sizeof(SolveOut)));
    if (!hout) {
        GateShared gate;
        GK_CUDA(cudaMallocHost(&hout, sizeof(SolveOut)));
    }
    // col < n <= 16384 and rpb <= 1024, so col * rpb < 2^32 and the
    // multiply-high quotient is exact
    const uint32_t rpb_inv = rpb > 1 ? (uint32_t)((1ull << 32) / (uint64_t)rpb + 1) : 0u;
    ClusterArgs args{A->n, rpb, rpb_inv, A->row_ptr, A->col, A->val, b, x, o->tol, o->max_iters,
                     o->precond == GK_PRECOND_JACOBI, (SolveOut*)outbuf.ptr};
    // stage the rows in shared memory when the largest block's entries fit
    // (bounded by rows per block x longest row)
    const size_t vb = vector_bytes(A->dtype);
    const int64_t ent = (int64_t)rpb * A->max_row;
    const size_t stage_bytes = (((size_t)ent * vb + 15) & ~(size_t)15) + 4 * (size_t)ent;
    const bool staged = stage_bytes <= 160 * 1024;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C, 1, 1);
    cfg.blockDim = dim3(CL_THREADS, 1, 1);
    cfg.dynamicSmemBytes = staged ? stage_bytes : 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    // one reduction per iteration (Chronopoulos-Gear) unless
    // GK_CLUSTER_RECURRENCE=hs asks for the Hestenes-Stiefel recurrence
    bool sr = true;
    if (const char* e = getenv("GK_CLUSTER_RECURRENCE")) sr = strcmp(e, "hs") != 0;
    cudaError_t e;
    auto go = [&](auto kern) -> cudaError_t {
        if (C > 8) {
            cudaError_t a = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
            if (a != cudaSuccess) return a;
        }
        cudaError_t m = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             160 * 1024 + 64);
        if (m != cudaSuccess) return m;
        int nclusters = 0;
        cudaError_t q = cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg);
        if (q != cudaSuccess) return q;
        if (nclusters < 1) return cudaErrorLaunchOutOfResources;
        return cudaLaunchKernelEx(&cfg, kern, args);
    };
    auto pick = [&](auto st, auto srt) -> cudaError_t {
        constexpr bool S = decltype(st)::value, R = decltype(srt)::value;
        if (A->dtype == GK_F64) return go(k_cluster_cg<double, double, S, R>);
        if (A->dtype == GK_F32) return go(k_cluster_cg<float, float, S, R>);
        return go(k_cluster_cg<__nv_bfloat16, float, S, R>);
    };
    using yes = std::true_type;
    using no = std::false_type;
    if (staged) e = sr ? pick(yes{}, yes{}) : pick(yes{}, no{});
    else e = sr ? pick(no{}, yes{}) : pick(no{}, no{});
    if (e != cudaSuccess) {
        cudaGetLastError();
        return GK_ERR_UNSUPPORTED;
    }
    GK_CUDA(cudaMemcpyAsync(hout, outbuf.ptr, sizeof(SolveOut), cudaMemcpyDeviceToHost, s));
    GK_CUDA(cudaStreamSynchronize(s));
    *out = *hout;
    return GK_OK;
}

}  // namespace gk
