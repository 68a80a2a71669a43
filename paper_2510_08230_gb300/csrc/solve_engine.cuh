// solve_engine.cuh - the multi-kernel Krylov engine: device state, the fused
// solver kernels and epilogues, and solve_mk<V, T>, one solve of CG,
// BiCGSTAB, CGS or GMRES(m).  solve_mk is instantiated once per value type
// in its own translation unit (solve_f64.cu, solve_f32.cu, solve_bf16.cu,
// solve_f16.cu) so
// the types compile in parallel; solve.cu holds the host-side helpers and
// the entry points.
//
// solve.cu - Krylov solvers on the device: CG, BiCGSTAB and GMRES(m) with an
// optional Jacobi preconditioner, and FP64 iterative refinement around
// FP32 / BF16-stored inner solves.
//
// The solver LinOp overwrites the initial guess with the solution
// (Section 3.5, Listing 1); stopping is an iteration cap OR
// ||r|| <= tol * ||b|| with the right-hand-side norm as baseline
// (Listing 2).  GMRES keeps the whole least-squares update on the GPU, uses
// Givens rotations and checks the residual estimate after every Hessenberg
// column (Section 6.2.1).
//
// Multi-kernel engine: each iteration is a fixed sequence of fused kernels
// (SpMV + dot, axpys + dots + preconditioner, ...); all scalars (alpha,
// beta, rho, Givens data) live in a device-side state block and are
// produced by the last block of the kernel that finishes each reduction,
// so no host round trip happens inside an iteration.  A chunk of
// iterations is captured once into a CUDA graph and replayed; kernels
// return immediately once the state says "halt".  The host looks at the
// state only between chunks.
#pragma once

#include <cstring>
#include <unordered_map>
#include <vector>

#include "ilu.cuh"
#include "spmv.cuh"

namespace gk {

constexpr int MAXM = 64;

struct KState {
    double thr;        // tol * ||b||
    double bnorm;
    double rho, alpha, beta, omega;
    double rnorm;      // last recurrence residual (or Givens estimate)
    double tnorm;      // last true residual norm
    double snorm;
    int32_t iter, max_iters;
    int32_t halt;      // 0 run; 1 recurrence passed (host checks true residual); 2 stop
    int32_t status;
    int32_t half;      // BiCGSTAB: stopped at the half step
    int32_t fresh;     // CGS: the next step is the first after a (re)start
    int32_t restarts;
    // GMRES
    int32_t k, m, cycle_end, v0_pending;
    double beta0, inv_h;
    double stag;       // GMRES: stop when a cycle's residual > stag * the previous (0: off)
    double prev_beta0;
    double best_rn;    // CG/BiCGSTAB/CGS inner solves: best residual so far ...
    int32_t best_iter; // ... and its iteration
    int32_t stall;     // stop after this many iterations without a 10 % gain (0: off)
    // the solver loop on the device (see k_ctl_*): the requested reduction,
    // the loop's control words and its bounds
    double tol;
    int32_t inner;      // a refinement inner solve (stops after two replacements)
    int32_t done;       // the loop ends after this pass
    int32_t nocheck;    // 0: this pass confirms a passed recurrence by the true residual
    int32_t noreplace;  // 0: this pass restarts from x with r = b - A x
    int32_t nofinal;    // 0: the exit computes the true residual
    int32_t nozero;     // 0: b = 0, the exit zeroes x
    int32_t loops, max_loops, checks_left;
    double H[(MAXM + 1) * MAXM];
    double cs[MAXM], sn[MAXM], g[MAXM + 1], y[MAXM];
    double h1[MAXM + 1], h2[MAXM + 1];
};

__device__ __forceinline__ bool halted(const KState* st) {
    return *reinterpret_cast<const volatile int32_t*>(&st->halt) != 0;
}

// Inner solves of iterative refinement: a solve whose residual has not
// dropped below 0.9x its best for `stall` iterations stops (CGS and
// BiCGSTAB can stagnate or wander in FP32); the refinement step continues
// from the iterate it reached.  Run by the last block's fin.
__device__ __forceinline__ bool stalled(KState* st, double rn) {
    if (st->stall <= 0) return false;
    if (!(st->best_rn > 0.0) || rn < 0.9 * st->best_rn) {
        st->best_rn = rn;
        st->best_iter = st->iter;
        return false;
    }
    return st->iter - st->best_iter >= st->stall;
}

// ------------------------------------------------------------ grids

static unsigned ew_grid(int64_t n) {
    int64_t b = (n + 1023) / 1024;
    int64_t cap = (int64_t)num_sms() * 8;
    return (unsigned)std::max<int64_t>(1, std::min(b, cap));
}

// Grid of a grid-stride element-wise kernel (256 threads): at most one wave
// of the blocks the kernel can keep resident (its register count decides:
// 4 to 8 per SM), so no ragged second wave; at least ~4 elements a thread.
template <typename K>
static unsigned ewg(K kernel, int64_t n) {
    static std::mutex mu;
    static std::unordered_map<const void*, int> occ;
    int b = 0;
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = occ.find((const void*)kernel);
        if (it == occ.end()) {
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, 256, 0) != cudaSuccess ||
                b < 1)
                b = 1;
            b = std::min(b, 8);
            occ[(const void*)kernel] = b;
        } else {
            b = it->second;
        }
    }
    const int64_t need = (n + 1023) / 1024;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)num_sms() * b));
}

// ------------------------------------------------------------ fins
// (run by thread 0 of the last block with the grid totals)

struct FinNorm {  // ||v|| -> field
    KState* st;
    int which;  // 0 bnorm, 1 tnorm
    __device__ void operator()(double* t) const {
        double v = sqrt(t[0]);
        if (which == 0) st->bnorm = v;
        else st->tnorm = v;
    }
};

// ------------------------------------------------------------ epilogues

// r_i = b_i - s ; acc += r_i^2  (true residual)
template <typename T, class Fin>
struct EpiResid {
    T* __restrict__ r;
    const T* __restrict__ b;
    const int32_t* halt;
    double* partials;
    unsigned* ticket;
    Fin fin;
    static constexpr int NA = 1;
    using acc_t = T;  // per-thread partial sums in the vector type
    __device__ __forceinline__ bool skip() const {
        return halt && *reinterpret_cast<const volatile int32_t*>(halt) != 0;
    }
    __device__ __forceinline__ void row(int64_t i, T s, T* acc) const {
        T v = b[i] - s;
        r[i] = v;
        acc[0] = fmadd(v, v, acc[0]);
    }
    __device__ __forceinline__ void finish(T* acc) const {
        double a[1] = {(double)acc[0]};
        grid_reduce_finish<1>(a, partials, ticket, fin);
    }
    __device__ __forceinline__ void timed_out() const {}
};

// y_i = s ; acc += w_i * s
template <typename T, class Fin>
struct EpiDot {
    T* __restrict__ y;
    const T* __restrict__ w;
    const int32_t* halt;
    double* partials;
    unsigned* ticket;
    Fin fin;
    static constexpr int NA = 1;
    using acc_t = T;  // per-thread partial sums in the vector type
    __device__ __forceinline__ bool skip() const {
        return halt && *reinterpret_cast<const volatile int32_t*>(halt) != 0;
    }
    __device__ __forceinline__ void row(int64_t i, T s, T* acc) const {
        y[i] = s;
        acc[0] = fmadd(w[i], s, acc[0]);
    }
    __device__ __forceinline__ void finish(T* acc) const {
        double a[1] = {(double)acc[0]};
        grid_reduce_finish<1>(a, partials, ticket, fin);
    }
    __device__ __forceinline__ void timed_out() const {}
};

// y_i = s ; acc0 += s * u_i ; acc1 += s * s
template <typename T, class Fin>
struct EpiDot2 {
    T* __restrict__ y;
    const T* __restrict__ u;
    const int32_t* halt;
    double* partials;
    unsigned* ticket;
    Fin fin;
    static constexpr int NA = 2;
    using acc_t = T;
    __device__ __forceinline__ bool skip() const {
        return halt && *reinterpret_cast<const volatile int32_t*>(halt) != 0;
    }
    __device__ __forceinline__ void row(int64_t i, T s, T* acc) const {
        y[i] = s;
        acc[0] = fmadd(s, u[i], acc[0]);
        acc[1] = fmadd(s, s, acc[1]);
    }
    __device__ __forceinline__ void finish(T* acc) const {
        double a[2] = {(double)acc[0], (double)acc[1]};
        grid_reduce_finish<2>(a, partials, ticket, fin);
    }
    __device__ __forceinline__ void timed_out() const {}
};

// plain store with a halt check (GMRES w = A z)
template <typename T>
struct EpiStoreHalt {
    T* __restrict__ y;
    const int32_t* halt;
    static constexpr int NA = 0;
    using acc_t = T;
    __device__ __forceinline__ bool skip() const {
        return halt && *reinterpret_cast<const volatile int32_t*>(halt) != 0;
    }
    __device__ __forceinline__ void row(int64_t i, T s, T*) const { y[i] = s; }
    __device__ __forceinline__ void finish(T*) const {}
    __device__ __forceinline__ void timed_out() const {}
};

// ------------------------------------------------------------ elementwise

// per-thread partial sums in T, promoted to double for the grid reduction
template <int NA, typename T, class Fin>
__device__ __forceinline__ void finish_ew(T (&a)[NA], double* partials, unsigned* ticket,
                                          const Fin& fin) {
    double d[NA];
#pragma unroll
    for (int k = 0; k < NA; ++k) d[k] = (double)a[k];
    grid_reduce_finish<NA>(d, partials, ticket, fin);
}

// Element-wise kernels run 256 threads per block (ewg sizes their grids).
#define EW_BOUNDS __launch_bounds__(256)

#define GRID_LOOP(i, n)                                                             \
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); \
         i += (int64_t)gridDim.x * blockDim.x)

// 16-byte packs (2 doubles or 4 floats) for the streaming solver kernels.
// A thread visits packs j = tid, tid + G, ...; pack j holds elements
// [jN, jN + N).  When every pointer is 16-byte aligned a full pack moves as
// one 16-byte access, else element by element; the elements a thread sees
// and their order are the same either way, so no result depends on the
// alignment of the caller's vectors.  Twice (FP64) or four times (FP32) the
// bytes in flight per load instruction compared with scalar accesses.
template <typename T>
struct alignas(16) Pack {
    static constexpr int N = 16 / (int)sizeof(T);
    T v[N];
};

__device__ __forceinline__ bool al16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

template <typename T>
__device__ __forceinline__ Pack<T> pld(const T* __restrict__ p, int64_t j, int32_t n, bool vec) {
    constexpr int N = Pack<T>::N;
    const int64_t i0 = j * N;
    Pack<T> r;
    if (vec && i0 + N <= n) {
        r = *reinterpret_cast<const Pack<T>*>(p + i0);
    } else {
#pragma unroll
        for (int c = 0; c < N; ++c) r.v[c] = i0 + c < n ? p[i0 + c] : T(0);
    }
    return r;
}

template <typename T>
__device__ __forceinline__ void pst(T* __restrict__ p, int64_t j, int32_t n, bool vec,
                                    const Pack<T>& r) {
    constexpr int N = Pack<T>::N;
    const int64_t i0 = j * N;
    if (vec && i0 + N <= n) {
        *reinterpret_cast<Pack<T>*>(p + i0) = r;
    } else {
#pragma unroll
        for (int c = 0; c < N; ++c)
            if (i0 + c < n) p[i0 + c] = r.v[c];
    }
}

#define PACK_LOOP(j, n, T)                                                                 \
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x,                       \
                 j##_end = ((int64_t)(n) + Pack<T>::N - 1) / Pack<T>::N;                    \
         j < j##_end; j += (int64_t)gridDim.x * blockDim.x)

template <typename T, class Fin>
__global__ void EW_BOUNDS k_norm2(int32_t n, const T* __restrict__ v, double* partials, unsigned* ticket,
                        Fin fin) {
    constexpr int N = Pack<T>::N;
    const bool vec = al16(v);
    T a[1] = {T(0)};
    PACK_LOOP(j, n, T) {
        const Pack<T> V = pld(v, j, n, vec);
#pragma unroll
        for (int c = 0; c < N; ++c) a[0] = fmadd(V.v[c], V.v[c], a[0]);  // padding adds 0
    }
    finish_ew<1>(a, partials, ticket, fin);
}

template <typename T>
__global__ void EW_BOUNDS k_zero(int32_t n, T* __restrict__ v, const int32_t* gate = nullptr) {
    if (gate && *reinterpret_cast<const volatile int32_t*>(gate) != 0) return;
    GRID_LOOP(i, n) v[i] = T(0);
}

template <typename T>
__global__ void EW_BOUNDS k_copy(int32_t n, const T* __restrict__ a, T* __restrict__ b,
                                 const int32_t* gate = nullptr) {
    if (gate && *reinterpret_cast<const volatile int32_t*>(gate) != 0) return;
    GRID_LOOP(i, n) b[i] = a[i];
}

// Jacobi: dinv_i = 1 / a_ii (sum of stored diagonal entries); a missing or
// zero diagonal sets *bad.
template <typename V, typename T>
__global__ void k_jacobi_gen(int32_t n, const int32_t* __restrict__ rp,
                             const int32_t* __restrict__ ci, const V* __restrict__ va,
                             T* __restrict__ dinv, int32_t* bad) {
    GRID_LOOP(i, n) {
        T d = T(0);
        bool found = false;
        for (int32_t k = rp[i]; k < rp[i + 1]; ++k)
            if (ci[k] == i) {
                d += cvt<T>(va[k]);
                found = true;
            }
        if (!found || d == T(0)) {
            atomicOr(bad, 1);
            dinv[i] = T(0);
        } else {
            dinv[i] = T(1) / d;
        }
    }
}

// ---------------------------------------------------------------- CG
// Hestenes-Stiefel with left preconditioner M = D (Jacobi) or I.

struct CgAlphaFin {
    KState* st;
    __device__ void operator()(double* t) const {
        const double pq = t[0];
        if (!isfinite(pq)) {
            st->status = GK_ERR_NAN;
            st->halt = 2;
        } else if (pq <= 0.0) {
            st->status = GK_BREAKDOWN;
            st->halt = 2;
        } else {
            st->alpha = st->rho / pq;
        }
    }
};

struct CgUpdFin {
    KState* st;
    int prec;
    __device__ void operator()(double* t) const {
        st->iter += 1;
        const double rn = sqrt(t[1]);
        st->rnorm = rn;
        if (!isfinite(rn) || !isfinite(t[0])) {
            st->status = GK_ERR_NAN;
            st->halt = 2;
            return;
        }
        if (rn <= st->thr) {
            st->halt = 1;
            return;
        }
        if (st->iter >= st->max_iters || stalled(st, rn)) {
            st->status = GK_NOT_CONVERGED;
            st->halt = 2;
            return;
        }
        if (prec >= 2) return;  // block-Jacobi / ILU: the fin after z = M^-1 r takes <r, z>
        const double rz = prec ? t[0] : t[1];
        st->beta = rz / st->rho;
        st->rho = rz;
    }
};

// block-Jacobi / ILU CG: beta from <r, z> with z = M^-1 r (k_bj_apply, k_dot_fin)
struct CgBetaFin {
    KState* st;
    __device__ void operator()(double* t) const {
        const double rz = t[0];
        if (!isfinite(rz)) {
            st->status = GK_ERR_NAN;
            st->halt = 2;
            return;
        }
        st->beta = rz / st->rho;
        st->rho = rz;
    }
};

// x += alpha p ; r -= alpha q ; z = D^-1 r ; <r,z>, <r,r>
template <typename T>
__device__ __forceinline__ void cg_update_pack(int64_t j, int32_t n, bool vec, T alpha, T* x, T* r,
                                               T* z, const T* p, const T* q, const T* dinv,
                                               T (&a)[2]) {
    constexpr int N = Pack<T>::N;
    const Pack<T> P = pld(p, j, n, vec), Q = pld(q, j, n, vec);
    Pack<T> X = pld(x, j, n, vec), R = pld(r, j, n, vec);
    Pack<T> Z = dinv ? pld(dinv, j, n, vec) : Pack<T>{};
#pragma unroll
    for (int c = 0; c < N; ++c) {  // padding lanes are 0 and add 0
        X.v[c] = fmadd(alpha, P.v[c], X.v[c]);
        R.v[c] = fmadd(-alpha, Q.v[c], R.v[c]);
        if (dinv) {
            Z.v[c] = Z.v[c] * R.v[c];
            a[0] = fmadd(R.v[c], Z.v[c], a[0]);
        }
        a[1] = fmadd(R.v[c], R.v[c], a[1]);
    }
    pst(x, j, n, vec, X);
    pst(r, j, n, vec, R);
    if (dinv) pst(z, j, n, vec, Z);
}

// A thread visits packs j, j + G, j + 2G, ... in that order.  FP32 takes
// two of them per step (16-byte accesses only, while both are whole and
// every pointer is aligned) so that twice the bytes are in flight; the
// order of the additions is the same as one pack per step.
template <typename T>
__global__ void EW_BOUNDS k_cg_update(int32_t n, T* __restrict__ x, T* __restrict__ r, T* __restrict__ z,
                            const T* __restrict__ p, const T* __restrict__ q,
                            const T* __restrict__ dinv, KState* st, double* partials,
                            unsigned* ticket, int pkind) {
    if (halted(st)) return;
    constexpr int N = Pack<T>::N;
    const T alpha = (T)st->alpha;
    const bool vec = al16(x) && al16(r) && al16(z) && al16(p) && al16(q) && al16(dinv);
    T a[2] = {T(0), T(0)};
    const int64_t G = (int64_t)gridDim.x * blockDim.x;
    const int64_t np = ((int64_t)n + N - 1) / N;
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if constexpr (sizeof(T) == 4) {
        if (vec) {
            const int64_t whole = (int64_t)n / N;  // packs with N elements
            using P4 = Pack<T>;
            for (; j + G < whole; j += 2 * G) {
                const int64_t j1 = j + G;
                const P4 P0 = reinterpret_cast<const P4*>(p)[j], P1 = reinterpret_cast<const P4*>(p)[j1];
                const P4 Q0 = reinterpret_cast<const P4*>(q)[j], Q1 = reinterpret_cast<const P4*>(q)[j1];
                P4 X0 = reinterpret_cast<P4*>(x)[j], X1 = reinterpret_cast<P4*>(x)[j1];
                P4 R0 = reinterpret_cast<P4*>(r)[j], R1 = reinterpret_cast<P4*>(r)[j1];
                P4 Z0{}, Z1{};
                if (dinv) {
                    Z0 = reinterpret_cast<const P4*>(dinv)[j];
                    Z1 = reinterpret_cast<const P4*>(dinv)[j1];
                }
#pragma unroll
                for (int c = 0; c < N; ++c) {
                    X0.v[c] = fmadd(alpha, P0.v[c], X0.v[c]);
                    R0.v[c] = fmadd(-alpha, Q0.v[c], R0.v[c]);
                    if (dinv) {
                        Z0.v[c] = Z0.v[c] * R0.v[c];
                        a[0] = fmadd(R0.v[c], Z0.v[c], a[0]);
                    }
                    a[1] = fmadd(R0.v[c], R0.v[c], a[1]);
                }
#pragma unroll
                for (int c = 0; c < N; ++c) {
                    X1.v[c] = fmadd(alpha, P1.v[c], X1.v[c]);
                    R1.v[c] = fmadd(-alpha, Q1.v[c], R1.v[c]);
                    if (dinv) {
                        Z1.v[c] = Z1.v[c] * R1.v[c];
                        a[0] = fmadd(R1.v[c], Z1.v[c], a[0]);
                    }
                    a[1] = fmadd(R1.v[c], R1.v[c], a[1]);
                }
                reinterpret_cast<P4*>(x)[j] = X0;
                reinterpret_cast<P4*>(x)[j1] = X1;
                reinterpret_cast<P4*>(r)[j] = R0;
                reinterpret_cast<P4*>(r)[j1] = R1;
                if (dinv) {
                    reinterpret_cast<P4*>(z)[j] = Z0;
                    reinterpret_cast<P4*>(z)[j1] = Z1;
                }
            }
        }
    }
    if constexpr (sizeof(T) == 8) {
        // FP64: the next pack's loads are issued before this pack's FMAs, so
        // that the narrow FP64 pipe works while the loads are in flight
        // (the same packs in the same order, so the same sums)
        if (vec && j < np) {
            Pack<T> P = pld(p, j, n, true), Q = pld(q, j, n, true);
            Pack<T> X = pld(x, j, n, true), R = pld(r, j, n, true);
            Pack<T> Z = dinv ? pld(dinv, j, n, true) : Pack<T>{};
            for (;;) {
                const int64_t jn = j + G;
                const bool more = jn < np;
                Pack<T> Pn{}, Qn{}, Xn{}, Rn{}, Zn{};
                if (more) {
                    Pn = pld(p, jn, n, true);
                    Qn = pld(q, jn, n, true);
                    Xn = pld(x, jn, n, true);
                    Rn = pld(r, jn, n, true);
                    if (dinv) Zn = pld(dinv, jn, n, true);
                }
#pragma unroll
                for (int c = 0; c < N; ++c) {  // as cg_update_pack
                    X.v[c] = fmadd(alpha, P.v[c], X.v[c]);
                    R.v[c] = fmadd(-alpha, Q.v[c], R.v[c]);
                    if (dinv) {
                        Z.v[c] = Z.v[c] * R.v[c];
                        a[0] = fmadd(R.v[c], Z.v[c], a[0]);
                    }
                    a[1] = fmadd(R.v[c], R.v[c], a[1]);
                }
                pst(x, j, n, true, X);
                pst(r, j, n, true, R);
                if (dinv) pst(z, j, n, true, Z);
                if (!more) break;
                P = Pn;
                Q = Qn;
                X = Xn;
                R = Rn;
                Z = Zn;
                j = jn;
            }
            j = np;
        }
    }
    for (; j < np; j += G) cg_update_pack(j, n, vec, alpha, x, r, z, p, q, dinv, a);
    finish_ew<2>(a, partials, ticket, CgUpdFin{st, pkind});
}

// p = z + beta p (FP32: two packs per step, as in k_cg_update)
template <typename T>
__global__ void EW_BOUNDS k_cg_p(int32_t n, T* __restrict__ p, const T* __restrict__ z, const KState* st) {
    if (halted(st)) return;
    constexpr int N = Pack<T>::N;
    const T beta = (T)st->beta;
    const bool vec = al16(p) && al16(z);
    const int64_t G = (int64_t)gridDim.x * blockDim.x;
    const int64_t np = ((int64_t)n + N - 1) / N;
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if constexpr (sizeof(T) == 4) {
        if (vec) {
            const int64_t whole = (int64_t)n / N;
            using P4 = Pack<T>;
            for (; j + G < whole; j += 2 * G) {
                P4 P0 = reinterpret_cast<P4*>(p)[j], P1 = reinterpret_cast<P4*>(p)[j + G];
                const P4 Z0 = reinterpret_cast<const P4*>(z)[j], Z1 = reinterpret_cast<const P4*>(z)[j + G];
#pragma unroll
                for (int c = 0; c < N; ++c) {
                    P0.v[c] = fmadd(beta, P0.v[c], Z0.v[c]);
                    P1.v[c] = fmadd(beta, P1.v[c], Z1.v[c]);
                }
                reinterpret_cast<P4*>(p)[j] = P0;
                reinterpret_cast<P4*>(p)[j + G] = P1;
            }
        }
    }
    for (; j < np; j += G) {
        Pack<T> P = pld(p, j, n, vec);
        const Pack<T> Z = pld(z, j, n, vec);
#pragma unroll
        for (int c = 0; c < N; ++c) P.v[c] = fmadd(beta, P.v[c], Z.v[c]);
        pst(p, j, n, vec, P);
    }
}

struct CgInitFin {
    KState* st;
    __device__ void operator()(double* t) const { st->rho = t[0]; }
};

// z = D^-1 r ; p = z ; rho = <r, z>
template <typename T>
__global__ void EW_BOUNDS k_cg_init(int32_t n, const T* __restrict__ r, T* __restrict__ z, T* __restrict__ p,
                          const T* __restrict__ dinv, KState* st, double* partials,
                          unsigned* ticket, const int32_t* gate = nullptr) {
    if (gate && *reinterpret_cast<const volatile int32_t*>(gate) != 0) return;
    T a[1] = {T(0)};
    GRID_LOOP(i, n) {
        const T ri = r[i];
        const T zi = dinv ? dinv[i] * ri : ri;
        if (dinv) z[i] = zi;
        p[i] = zi;
        a[0] = fmadd(ri, zi, a[0]);
    }
    finish_ew<1>(a, partials, ticket, CgInitFin{st});
}

// ---------------------------------------------------------------- BiCGSTAB
// van der Vorst, right preconditioning (phat = M^-1 p, shat = M^-1 s).

struct BiAlphaFin {
    KState* st;
    __device__ void operator()(double* t) const {
        const double rv = t[0];
        if (!isfinite(rv)) {
            st->status = GK_ERR_NAN;
            st->halt = 2;
        } else if (rv == 0.0) {
            st->status = GK_BREAKDOWN;
            st->halt = 2;
        } else {
            st->alpha = st->rho / rv;  // rho holds rho' of this iteration
        }
    }
};

// beta = (rho'/rho_old)(alpha/omega) is prepared by the previous update's fin
// p = r + beta (p - omega v) ; phat = M^-1 p
template <typename T>
__global__ void EW_BOUNDS k_bi_p(int32_t n, T* __restrict__ p, T* __restrict__ ph, const T* __restrict__ r,
                       const T* __restrict__ v, const T* __restrict__ dinv, const KState* st) {
    if (halted(st)) return;
    constexpr int N = Pack<T>::N;
    const T beta = (T)st->beta, omega = (T)st->omega;
    const bool vec = al16(p) && al16(ph) && al16(r) && al16(v) && al16(dinv);
    PACK_LOOP(j, n, T) {
        Pack<T> P = pld(p, j, n, vec);
        const Pack<T> Vv = pld(v, j, n, vec), R = pld(r, j, n, vec);
        Pack<T> D = dinv ? pld(dinv, j, n, vec) : Pack<T>{};
#pragma unroll
        for (int c = 0; c < N; ++c) {
            P.v[c] = fmadd(beta, fmadd(-omega, Vv.v[c], P.v[c]), R.v[c]);
            D.v[c] = D.v[c] * P.v[c];
        }
        pst(p, j, n, vec, P);
        if (dinv) pst(ph, j, n, vec, D);
    }
}

struct BiSFin {
    KState* st;
    __device__ void operator()(double* t) const {
        st->iter += 1;
        const double sn = sqrt(t[0]);
        st->snorm = sn;
        if (!isfinite(sn)) {
            st->status = GK_ERR_NAN;
            st->halt = 2;
        } else if (sn <= st->thr) {
            st->half = 1;  // half-step exit: x += alpha phat in the next kernel
            st->rnorm = sn;
        }
    }
};

// s = r - alpha v ; shat = M^-1 s ; ||s||^2
template <typename T>
__global__ void EW_BOUNDS k_bi_s(int32_t n, T* __restrict__ s, T* __restrict__ sh, const T* __restrict__ r,
                       const T* __restrict__ v, const T* __restrict__ dinv, KState* st,
                       double* partials, unsigned* ticket) {
    if (halted(st)) return;
    constexpr int N = Pack<T>::N;
    const T alpha = (T)st->alpha;
    const bool vec = al16(s) && al16(sh) && al16(r) && al16(v) && al16(dinv);
    T a[1] = {T(0)};
    PACK_LOOP(j, n, T) {
        const Pack<T> Vv = pld(v, j, n, vec);
        Pack<T> S = pld(r, j, n, vec);
        Pack<T> D = dinv ? pld(dinv, j, n, vec) : Pack<T>{};
#pragma unroll
        for (int c = 0; c < N; ++c) {
            S.v[c] = fmadd(-alpha, Vv.v[c], S.v[c]);
            D.v[c] = D.v[c] * S.v[c];
            a[0] = fmadd(S.v[c], S.v[c], a[0]);
        }
        pst(s, j, n, vec, S);
        if (dinv) pst(sh, j, n, vec, D);
    }
    finish_ew<1>(a, partials, ticket, BiSFin{st});
}

struct BiOmegaFin {
    KState* st;
    __device__ void operator()(double* t) const {
        const double ts = t[0], tt = t[1];
        if (!isfinite(ts) || !isfinite(tt)) {
            st->status = GK_ERR_NAN;
            st->halt = 2;
        } else if (tt == 0.0) {
            st->status = GK_BREAKDOWN;
            st->halt = 2;
        } else {
            st->omega = ts / tt;
            if (st->omega == 0.0) {
                st->status = GK_BREAKDOWN;
                st->halt = 2;
            }
        }
    }
};

struct BiUpdFin {
    KState* st;
    __device__ void operator()(double* t) const {
        if (st->half) {  // x was updated with alpha phat only
            st->half = 0;
            st->halt = 1;
            return;
        }
        const double rho_new = t[0];
        const double rn = sqrt(t[1]);
        st->rnorm = rn;
        if (!isfinite(rn) || !isfinite(rho_new)) {
            st->status = GK_ERR_NAN;
            st->halt = 2;
            return;
        }
        if (rn <= st->thr) {
            st->halt = 1;
            return;
        }
        if (st->iter >= st->max_iters || stalled(st, rn)) {
            st->status = GK_NOT_CONVERGED;
            st->halt = 2;
            return;
        }
        if (rho_new == 0.0) {
            st->status = GK_BREAKDOWN;
            st->halt = 2;
            return;
        }
        st->beta = (rho_new / st->rho) * (st->alpha / st->omega);
        st->rho = rho_new;
    }
};

// full step: x += alpha phat + omega shat ; r = s - omega t ; <rhat, r>, <r, r>
// half step (st->half): x += alpha phat only.
template <typename T>
__global__ void EW_BOUNDS k_bi_update(int32_t n, T* __restrict__ x, T* __restrict__ r,
                            const T* __restrict__ ph, const T* __restrict__ sh,
                            const T* __restrict__ s, const T* __restrict__ t,
                            const T* __restrict__ rh, KState* st, double* partials,
                            unsigned* ticket) {
    if (halted(st)) return;
    const bool half = st->half != 0;
    constexpr int N = Pack<T>::N;
    const T alpha = (T)st->alpha, omega = (T)st->omega;
    const bool vec = al16(x) && al16(r) && al16(ph) && al16(sh) && al16(s) && al16(t) && al16(rh);
    T a[2] = {T(0), T(0)};
    if (half) {
        PACK_LOOP(j, n, T) {
            Pack<T> X = pld(x, j, n, vec);
            const Pack<T> PH = pld(ph, j, n, vec);
#pragma unroll
            for (int c = 0; c < N; ++c) X.v[c] = fmadd(alpha, PH.v[c], X.v[c]);
            pst(x, j, n, vec, X);
        }
    } else {
        PACK_LOOP(j, n, T) {
            Pack<T> X = pld(x, j, n, vec);
            const Pack<T> PH = pld(ph, j, n, vec), SH = pld(sh, j, n, vec);
            const Pack<T> Tt = pld(t, j, n, vec), RH = pld(rh, j, n, vec);
            Pack<T> R = pld(s, j, n, vec);
#pragma unroll
            for (int c = 0; c < N; ++c) {
                X.v[c] = fmadd(omega, SH.v[c], fmadd(alpha, PH.v[c], X.v[c]));
                R.v[c] = fmadd(-omega, Tt.v[c], R.v[c]);
                a[0] = fmadd(RH.v[c], R.v[c], a[0]);
                a[1] = fmadd(R.v[c], R.v[c], a[1]);
            }
            pst(x, j, n, vec, X);
            pst(r, j, n, vec, R);
        }
    }
    finish_ew<2>(a, partials, ticket, BiUpdFin{st});
}

struct BiInitFin {
    KState* st;
    __device__ void operator()(double* t) const {
        const double rho = t[0];
        st->rho = rho;
        st->alpha = 1.0;
        st->omega = 1.0;
        // first iteration: beta = (rho'/1)(1/1) with rho' = <rhat, r>
        st->beta = 0.0;  // p = r exactly (p and v are zero)
        if (rho == 0.0) {
            st->status = GK_BREAKDOWN;
            st->halt = 2;
        }
    }
};

// rhat = r ; p = v = 0 ; rho = <rhat, r>
template <typename T>
__global__ void EW_BOUNDS k_bi_init(int32_t n, const T* __restrict__ r, T* __restrict__ rh, T* __restrict__ p,
                          T* __restrict__ v, KState* st, double* partials, unsigned* ticket,
                          const int32_t* gate = nullptr) {
    if (gate && *reinterpret_cast<const volatile int32_t*>(gate) != 0) return;
    T a[1] = {T(0)};
    GRID_LOOP(i, n) {
        const T ri = r[i];
        rh[i] = ri;
        p[i] = T(0);
        v[i] = T(0);
        a[0] = fmadd(ri, ri, a[0]);
    }
    finish_ew<1>(a, partials, ticket, BiInitFin{st});
}

// ---------------------------------------------------------------- CGS
// Sonneveld's conjugate gradient squared with M^-1 on the search
// directions; shadow residual rt = r_0.  One iteration, four kernels:
//   k_cgs_p : u = r + beta q ; p = u + beta (q + beta p) ; ph = M^-1 p
//             (first step after a (re)start: u = p = r)
//   SpMV    : vh = A ph ; <rt, vh> -> alpha = rho / <rt, vh>
//   k_cgs_q : q = u - alpha vh ; uh = M^-1 (u + q) ; x += alpha uh
//   SpMV    : r -= alpha A uh ; <rt, r>, ||r||^2 -> stopping test, beta, rho

// rt = r ; rho = <rt, r>
struct CgsInitFin {
    KState* st;
    __device__ void operator()(double* t) const {
        st->rho = t[0];
        st->fresh = 1;
        if (!isfinite(t[0])) {
            st->status = GK_ERR_NAN;
            st->halt = 2;
        } else if (t[0] == 0.0) {
            st->status = GK_BREAKDOWN;
            st->halt = 2;
        }
    }
};

template <typename T>
__global__ void EW_BOUNDS k_cgs_init(int32_t n, const T* __restrict__ r, T* __restrict__ rt,
                                     KState* st, double* partials, unsigned* ticket,
                                     const int32_t* gate = nullptr) {
    if (gate && *reinterpret_cast<const volatile int32_t*>(gate) != 0) return;
    constexpr int N = Pack<T>::N;
    const bool vec = al16(r) && al16(rt);
    T a[1] = {T(0)};
    PACK_LOOP(j, n, T) {
        const Pack<T> R = pld(r, j, n, vec);
        pst(rt, j, n, vec, R);
#pragma unroll
        for (int c = 0; c < N; ++c) a[0] = fmadd(R.v[c], R.v[c], a[0]);  // padding adds 0
    }
    finish_ew<1>(a, partials, ticket, CgsInitFin{st});
}

template <typename T>
__global__ void EW_BOUNDS k_cgs_p(int32_t n, T* __restrict__ u, T* __restrict__ p,
                                  T* __restrict__ ph, const T* __restrict__ r,
                                  const T* __restrict__ q, const T* __restrict__ dinv,
                                  const KState* st) {
    if (halted(st)) return;
    constexpr int N = Pack<T>::N;
    const bool first = st->fresh != 0;
    const T beta = first ? T(0) : (T)st->beta;
    const bool vec = al16(u) && al16(p) && al16(ph) && al16(r) && al16(q) && al16(dinv);
    PACK_LOOP(j, n, T) {
        Pack<T> U = pld(r, j, n, vec);
        Pack<T> P{};
        if (!first) {
            const Pack<T> Q = pld(q, j, n, vec);
            P = pld(p, j, n, vec);
#pragma unroll
            for (int c = 0; c < N; ++c) {
                U.v[c] = fmadd(beta, Q.v[c], U.v[c]);
                P.v[c] = fmadd(beta, fmadd(beta, P.v[c], Q.v[c]), U.v[c]);
            }
        } else {
            P = U;
        }
        pst(u, j, n, vec, U);
        pst(p, j, n, vec, P);
        if (dinv) {
            Pack<T> D = pld(dinv, j, n, vec);
#pragma unroll
            for (int c = 0; c < N; ++c) D.v[c] = D.v[c] * P.v[c];
            pst(ph, j, n, vec, D);
        }
    }
}

// alpha = rho / <rt, vh>
struct CgsAlphaFin {
    KState* st;
    __device__ void operator()(double* t) const {
        const double sg = t[0];
        st->fresh = 0;
        if (!isfinite(sg)) {
            st->status = GK_ERR_NAN;
            st->halt = 2;
        } else if (sg == 0.0) {
            st->status = GK_BREAKDOWN;
            st->halt = 2;
        } else {
            st->alpha = st->rho / sg;
        }
    }
};

template <typename T>
__global__ void EW_BOUNDS k_cgs_q(int32_t n, T* __restrict__ q, T* __restrict__ uh,
                                  T* __restrict__ x, const T* __restrict__ u,
                                  const T* __restrict__ vh, const T* __restrict__ dinv,
                                  const KState* st, T* __restrict__ tout) {
    if (halted(st)) return;
    constexpr int N = Pack<T>::N;
    const T alpha = (T)st->alpha;
    const bool vec = al16(q) && al16(uh) && al16(x) && al16(u) && al16(vh) && al16(dinv);
    PACK_LOOP(j, n, T) {
        const Pack<T> U = pld(u, j, n, vec), VH = pld(vh, j, n, vec);
        if (tout) {  // block-Jacobi: t = u + q here, uh = B t and x += alpha uh in k_bj_apply
            Pack<T> Q, Tt;
#pragma unroll
            for (int c = 0; c < N; ++c) {
                Q.v[c] = fmadd(-alpha, VH.v[c], U.v[c]);
                Tt.v[c] = U.v[c] + Q.v[c];
            }
            pst(q, j, n, vec, Q);
            pst(tout, j, n, vec && al16(tout), Tt);
            continue;
        }
        Pack<T> X = pld(x, j, n, vec);
        Pack<T> Q, UH = dinv ? pld(dinv, j, n, vec) : Pack<T>{};
#pragma unroll
        for (int c = 0; c < N; ++c) {
            Q.v[c] = fmadd(-alpha, VH.v[c], U.v[c]);
            const T tc = U.v[c] + Q.v[c];
            UH.v[c] = dinv ? UH.v[c] * tc : tc;
            X.v[c] = fmadd(alpha, UH.v[c], X.v[c]);
        }
        pst(q, j, n, vec, Q);
        pst(uh, j, n, vec, UH);
        pst(x, j, n, vec, X);
    }
}

// r -= alpha s (s = (A uh)_i) ; <rt, r>, <r, r>
struct CgsRFin {
    KState* st;
    __device__ void operator()(double* t) const {
        st->iter += 1;
        const double rn = sqrt(t[1]);
        st->rnorm = rn;
        if (!isfinite(rn) || !isfinite(t[0])) {
            st->status = GK_ERR_NAN;
            st->halt = 2;
            return;
        }
        if (rn <= st->thr) {
            st->halt = 1;
            return;
        }
        if (st->iter >= st->max_iters || stalled(st, rn)) {
            st->status = GK_NOT_CONVERGED;
            st->halt = 2;
            return;
        }
        if (t[0] == 0.0) {
            st->status = GK_BREAKDOWN;
            st->halt = 2;
            return;
        }
        st->beta = t[0] / st->rho;
        st->rho = t[0];
    }
};

template <typename T>
struct EpiCgsR {
    T* __restrict__ r;
    const T* __restrict__ rt;
    const KState* st;
    double* partials;
    unsigned* ticket;
    static constexpr int NA = 2;
    using acc_t = T;
    __device__ __forceinline__ bool skip() const { return halted(st); }
    __device__ __forceinline__ void row(int64_t i, T s, T* acc) const {
        const T v = fmadd(-(T)st->alpha, s, r[i]);
        r[i] = v;
        acc[0] = fmadd(rt[i], v, acc[0]);
        acc[1] = fmadd(v, v, acc[1]);
    }
    __device__ __forceinline__ void finish(T* acc) const {
        double a[2] = {(double)acc[0], (double)acc[1]};
        grid_reduce_finish<2>(a, partials, ticket, CgsRFin{const_cast<KState*>(st)});
    }
    __device__ __forceinline__ void timed_out() const {}
};

// ---------------------------------------------------------------- GMRES
// V: n x (m+1), column j at V + j*ldv (ldv spans a multiple of 256 bytes).
// CGS2 orthogonalisation, three passes over the basis per Arnoldi step:
//   h1 = V^T w ;  w -= V h1, h2 = V^T w (one kernel: a block subtracts on its
//   row chunk, then takes the dots from the chunk it just wrote) ;
//   w -= V h2, ||w|| and the Givens step.
// A pass over V is FP64-FMA-bound on this part (one FMA per 8 bytes), so the
// kernels keep every lane busy and many independent loads in flight.

constexpr int MD_ROWS = 2048;   // rows per block in the multi-dot kernels
constexpr int MD_THREADS = 256;
constexpr int MD_UNROLL = 4;    // independent pack loads per lane per step

// Stages w's row chunk into shared memory, zero-padded to whole packs.
template <typename T>
__device__ __forceinline__ void stage_chunk(const T* __restrict__ w, int64_t r0, int32_t rows,
                                            T* s_w) {
    constexpr int N = Pack<T>::N;
    const int32_t padded = (rows + N - 1) / N * N;
    for (int i = threadIdx.x; i < padded; i += blockDim.x) s_w[i] = i < rows ? w[r0 + i] : T(0);
}

// Dot products of the staged chunk s_w with columns 0..kk of V, added to
// the block's running column sums s_colsum.  Work items are (column, row
// segment): with few columns a column is split into segments so that all 8
// warps work; a warp's lanes step over 16-byte packs of the segment,
// MD_UNROLL independent loads at a time.  Segment sums are added per column
// in segment order.
template <typename T>
__device__ void multidot_chunk(int64_t ldv, const T* __restrict__ V, const T* s_w, int64_t r0,
                               int32_t rows, int32_t kk, bool vec, double* s_colsum) {
    constexpr int N = Pack<T>::N;
    __shared__ double s_part[(MAXM + 1) * 8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int np = (rows + N - 1) / N;
    const int ncol = kk + 1;
    int S = 1;  // segments per column (power of two, ncol * S >= nw when possible)
    while (S < 8 && ncol * S * 2 <= nw) S *= 2;
    const int seg = (np + S - 1) / S;
    for (int it = warp; it < ncol * S; it += nw) {
        const int j = it / S, sgi = it - j * S;
        const T* col = V + (int64_t)j * ldv + r0;
        const int p0 = sgi * seg, p1 = min(np, p0 + seg);
        T acc[MD_UNROLL][N];
#pragma unroll
        for (int u = 0; u < MD_UNROLL; ++u)
#pragma unroll
            for (int c = 0; c < N; ++c) acc[u][c] = T(0);
        for (int pb = p0 + lane; pb < p1; pb += 32 * MD_UNROLL) {
            Pack<T> cp[MD_UNROLL], wp[MD_UNROLL];
#pragma unroll
            for (int u = 0; u < MD_UNROLL; ++u) {
                const int p = pb + 32 * u;
                if (p < p1) {
                    cp[u] = pld(col, p, rows, vec);
                    wp[u] = *reinterpret_cast<const Pack<T>*>(s_w + p * N);
                } else {
#pragma unroll
                    for (int c = 0; c < N; ++c) cp[u].v[c] = wp[u].v[c] = T(0);
                }
            }
#pragma unroll
            for (int u = 0; u < MD_UNROLL; ++u)
#pragma unroll
                for (int c = 0; c < N; ++c) acc[u][c] = fmadd(cp[u].v[c], wp[u].v[c], acc[u][c]);
        }
        T a = T(0);
#pragma unroll
        for (int u = 0; u < MD_UNROLL; ++u)
#pragma unroll
            for (int c = 0; c < N; ++c) a += acc[u][c];
        const double d = warp_sum((double)a);
        if (lane == 0) s_part[it] = d;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < ncol; j += blockDim.x) {
        double t = s_colsum[j];
        for (int q = 0; q < S; ++q) t += s_part[j * S + q];
        s_colsum[j] = t;
    }
    __syncthreads();
}

// Rows of this block: an equal share of whole 8-row groups, so that every
// block of a one-wave grid does the same work; processed in chunks of at
// most MD_ROWS rows.
__device__ __forceinline__ void md_block_rows(int32_t n, int64_t& beg, int64_t& end) {
    const int64_t R = (((int64_t)n + gridDim.x - 1) / gridDim.x + 7) / 8 * 8;
    beg = min((int64_t)n, (int64_t)blockIdx.x * R);
    end = min((int64_t)n, beg + R);
}

// Last block: h[j] = sum over blocks of partials[j][*] for j < ncol.
static __device__ bool multidot_finish(int32_t ncol, double* partials, unsigned* ticket, double* h) {
    __shared__ bool am_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        am_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!am_last) return false;
    __threadfence();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int j = warp; j < ncol; j += nw) {
        double s = 0.0;
        for (unsigned b = lane; b < gridDim.x; b += 32) s += __ldcg(partials + (size_t)j * gridDim.x + b);
        s = warp_sum(s);
        if (lane == 0) h[j] = s;
    }
    __syncthreads();
    return true;
}

// w -= V h on a row chunk (h negated in s_nh), thread per 16-byte pack of
// rows, the chunk's packs of a thread (MD_ROWS / 256 / N of them) updated
// together so their loads of each column are in flight at once.  Returns
// the thread's sum of squares of the new w when want_norm.
template <typename T, int CU = 1>
__device__ __forceinline__ T subtract_chunk(const T* __restrict__ V, int64_t ldv, T* __restrict__ wc,
                                            int64_t r0, int32_t rows, int32_t kk, const T* s_nh,
                                            bool vec, T* s_w) {
    constexpr int N = Pack<T>::N;
    constexpr int PP = MD_ROWS / MD_THREADS / N;  // packs per thread
    const int np = (rows + N - 1) / N;
    Pack<T> W[PP];
#pragma unroll
    for (int q = 0; q < PP; ++q) {
        const int p = threadIdx.x + q * MD_THREADS;
        if (p < np) W[q] = pld(wc, p, rows, vec);
    }
    // CU > 1: CU columns' loads issued before their FMAs (more bytes in
    // flight); every element still takes its FMAs in column order
    int j = 0;
    if constexpr (CU > 1) {
        for (; j + CU <= kk + 1; j += CU) {
            Pack<T> Vj[CU][PP];
#pragma unroll
            for (int u = 0; u < CU; ++u) {
                const T* col = V + (int64_t)(j + u) * ldv + r0;
#pragma unroll
                for (int q = 0; q < PP; ++q) {
                    const int p = threadIdx.x + q * MD_THREADS;
                    if (p < np) Vj[u][q] = pld(col, p, rows, vec);
                }
            }
#pragma unroll
            for (int u = 0; u < CU; ++u) {
                const T hj = s_nh[j + u];
#pragma unroll
                for (int q = 0; q < PP; ++q) {
                    const int p = threadIdx.x + q * MD_THREADS;
                    if (p < np) {
#pragma unroll
                        for (int c = 0; c < N; ++c) W[q].v[c] = fmadd(hj, Vj[u][q].v[c], W[q].v[c]);
                    }
                }
            }
        }
    }
    for (; j <= kk; ++j) {
        const T* col = V + (int64_t)j * ldv + r0;
        const T hj = s_nh[j];
#pragma unroll
        for (int q = 0; q < PP; ++q) {
            const int p = threadIdx.x + q * MD_THREADS;
            if (p < np) {
                const Pack<T> Vj = pld(col, p, rows, vec);
#pragma unroll
                for (int c = 0; c < N; ++c) W[q].v[c] = fmadd(hj, Vj.v[c], W[q].v[c]);
            }
        }
    }
    T a = T(0);
#pragma unroll
    for (int q = 0; q < PP; ++q) {
        const int p = threadIdx.x + q * MD_THREADS;
        if (p < np) {
            pst(wc, p, rows, vec, W[q]);
            if (s_w) *reinterpret_cast<Pack<T>*>(s_w + p * N) = W[q];
#pragma unroll
            for (int c = 0; c < N; ++c) a = fmadd(W[q].v[c], W[q].v[c], a);  // padding adds 0
        }
    }
    return a;
}

// h1 = V^T w  (columns 0..k)
template <typename T>
__global__ void __launch_bounds__(MD_THREADS, 4)
k_gm_dot1(int32_t n, int64_t ldv, const T* __restrict__ V, const T* __restrict__ w, KState* st,
          double* partials, unsigned* ticket) {
    if (halted(st)) return;
    __shared__ __align__(16) T s_w[MD_ROWS];
    __shared__ double s_colsum[MAXM + 1];
    const int32_t kk = st->k;
    for (int j = threadIdx.x; j <= kk; j += blockDim.x) s_colsum[j] = 0.0;
    int64_t beg, end;
    md_block_rows(n, beg, end);
    for (int64_t r0 = beg; r0 < end; r0 += MD_ROWS) {
        const int32_t rows = (int32_t)min((int64_t)MD_ROWS, end - r0);
        __syncthreads();
        stage_chunk(w, r0, rows, s_w);
        __syncthreads();
        multidot_chunk(ldv, V, s_w, r0, rows, kk, al16(V), s_colsum);
    }
    __syncthreads();
    for (int j = threadIdx.x; j <= kk; j += blockDim.x)
        partials[(size_t)j * gridDim.x + blockIdx.x] = s_colsum[j];
    if (multidot_finish(kk + 1, partials, ticket, st->h1) && threadIdx.x == 0) *ticket = 0u;
}

// w -= V h1 ; h2 = V^T w
template <typename T>
__global__ void __launch_bounds__(MD_THREADS, 4)
k_gm_dot2(int32_t n, int64_t ldv, const T* __restrict__ V, T* __restrict__ w, KState* st,
          double* partials, unsigned* ticket) {
    if (halted(st)) return;
    __shared__ __align__(16) T s_w[MD_ROWS];  // the updated chunk (padding lanes stay 0)
    __shared__ T s_nh[MAXM + 1];
    __shared__ double s_colsum[MAXM + 1];
    const int32_t kk = st->k;
    for (int j = threadIdx.x; j <= kk; j += blockDim.x) {
        s_nh[j] = -(T)st->h1[j];
        s_colsum[j] = 0.0;
    }
    const bool vec = al16(V) && al16(w);
    int64_t beg, end;
    md_block_rows(n, beg, end);
    for (int64_t r0 = beg; r0 < end; r0 += MD_ROWS) {
        const int32_t rows = (int32_t)min((int64_t)MD_ROWS, end - r0);
        __syncthreads();
        subtract_chunk(V, ldv, w + r0, r0, rows, kk, s_nh, vec, s_w);
        __syncthreads();
        multidot_chunk(ldv, V, s_w, r0, rows, kk, vec, s_colsum);
    }
    __syncthreads();
    for (int j = threadIdx.x; j <= kk; j += blockDim.x)
        partials[(size_t)j * gridDim.x + blockIdx.x] = s_colsum[j];
    if (multidot_finish(kk + 1, partials, ticket, st->h2) && threadIdx.x == 0) *ticket = 0u;
}

// Givens step on column k, residual estimate, cycle decision and, at the
// end of a cycle, the back substitution H y = g.
struct GmGivensFin {
    KState* st;
    __device__ void operator()(double* t) const {
        const int k = st->k, m = st->m;
        double* H = st->H;
        const double hk1 = sqrt(t[0]);
        for (int j = 0; j <= k; ++j) H[j * m + k] = st->h1[j] + st->h2[j];
        H[(k + 1) * m + k] = hk1;
        for (int j = 0; j < k; ++j) {
            const double a = H[j * m + k], b = H[(j + 1) * m + k];
            H[j * m + k] = st->cs[j] * a + st->sn[j] * b;
            H[(j + 1) * m + k] = -st->sn[j] * a + st->cs[j] * b;
        }
        const double a = H[k * m + k], b = H[(k + 1) * m + k];
        const double d = hypot(a, b);
        if (!isfinite(d)) {
            st->status = GK_ERR_NAN;
            st->halt = 2;
            return;
        }
        if (d == 0.0) {
            st->status = GK_BREAKDOWN;
            st->halt = 2;
            return;
        }
        st->v0_pending = 0;
        st->cs[k] = a / d;
        st->sn[k] = b / d;
        H[k * m + k] = d;
        H[(k + 1) * m + k] = 0.0;
        st->g[k + 1] = -st->sn[k] * st->g[k];
        st->g[k] = st->cs[k] * st->g[k];
        st->iter += 1;
        st->k = k + 1;
        const double est = fabs(st->g[k + 1]);
        st->rnorm = est;
        if (!isfinite(est)) {
            st->status = GK_ERR_NAN;
            st->halt = 2;
            return;
        }
        if (hk1 == 0.0 || est <= st->thr || k + 1 == m || st->iter >= st->max_iters) {
            st->cycle_end = 1;
            const int kk = k + 1;
            for (int i = kk - 1; i >= 0; --i) {
                double s = st->g[i];
                for (int j = i + 1; j < kk; ++j) s -= H[i * m + j] * st->y[j];
                st->y[i] = s / H[i * m + i];
            }
        } else {
            st->cycle_end = 0;
            st->inv_h = 1.0 / hk1;
        }
    }
};

// w -= V h2 ; ||w||^2 -> Givens fin
template <typename T>
__global__ void __launch_bounds__(MD_THREADS)
k_gm_orth(int32_t n, int64_t ldv, const T* __restrict__ V, T* __restrict__ w, KState* st,
          double* partials, unsigned* ticket) {
    if (halted(st)) return;
    __shared__ T s_nh[MAXM + 1];
    const int32_t kk = st->k;
    for (int j = threadIdx.x; j <= kk; j += blockDim.x) s_nh[j] = -(T)st->h2[j];
    __syncthreads();
    const bool vec = al16(V) && al16(w);
    int64_t beg, end;
    md_block_rows(n, beg, end);
    T a[1] = {T(0)};
    for (int64_t r0 = beg; r0 < end; r0 += MD_ROWS) {
        const int32_t rows = (int32_t)min((int64_t)MD_ROWS, end - r0);
        // 4-byte types are bound by the loads in flight, FP64 by its FMA pipe
        a[0] += subtract_chunk<T, sizeof(T) == 4 ? 4 : 1>(V, ldv, w + r0, r0, rows, kk, s_nh, vec,
                                                          (T*)nullptr);
    }
    finish_ew<1>(a, partials, ticket, GmGivensFin{st});
}

// not at the end of a cycle: v_{k} = w / h ; z = M^-1 v_k
// at the end of a cycle:     x += M^-1 (V y)
template <typename T>
__global__ void EW_BOUNDS k_gm_next(int32_t n, int64_t ldv, T* __restrict__ V, const T* __restrict__ w,
                          T* __restrict__ z, T* __restrict__ x, const T* __restrict__ dinv,
                          const KState* st, T* __restrict__ ubuf) {
    if (halted(st)) return;
    const int32_t k = st->k;
    constexpr int N = Pack<T>::N;
    // ldv spans a multiple of 256 bytes, so every basis vector shares V's alignment
    const bool vec = al16(V) && al16(w) && al16(z) && al16(x) && al16(dinv);
    if (!st->cycle_end) {
        const T ih = (T)st->inv_h;
        T* vk = V + (int64_t)k * ldv;
        PACK_LOOP(j, n, T) {
            Pack<T> Vk = pld(w, j, n, vec);
            Pack<T> Z = dinv ? pld(dinv, j, n, vec) : Pack<T>{};
#pragma unroll
            for (int c = 0; c < N; ++c) {
                Vk.v[c] = Vk.v[c] * ih;
                Z.v[c] = dinv ? Z.v[c] * Vk.v[c] : Vk.v[c];
            }
            pst(vk, j, n, vec, Vk);
            pst(z, j, n, vec, Z);
        }
    } else {
        __shared__ T s_y[MAXM];
        for (int j = threadIdx.x; j < k; j += blockDim.x) s_y[j] = (T)st->y[j];
        __syncthreads();
        PACK_LOOP(j, n, T) {
            Pack<T> U{};
            for (int l = 0; l < k; ++l) {
                const Pack<T> Vl = pld(V + (int64_t)l * ldv, j, n, vec);
#pragma unroll
                for (int c = 0; c < N; ++c) U.v[c] = fmadd(Vl.v[c], s_y[l], U.v[c]);
            }
            if (ubuf) {  // block-Jacobi: k_bj_gm adds B (V y) to x
                pst(ubuf, j, n, vec && al16(ubuf), U);
                continue;
            }
            Pack<T> X = pld(x, j, n, vec);
            const Pack<T> D = dinv ? pld(dinv, j, n, vec) : Pack<T>{};
#pragma unroll
            for (int c = 0; c < N; ++c) X.v[c] = fmadd(dinv ? D.v[c] : T(1), U.v[c], X.v[c]);
            pst(x, j, n, vec, X);
        }
    }
}

// Cycle start (fin of the true residual r = b - A x): converged, out of
// steps, or v_0 = r / beta0 and g = beta0 e_1.
struct GmRestartFin {
    KState* st;
    __device__ void operator()(double* t) const {
        const double b0 = sqrt(t[0]);
        st->tnorm = b0;
        st->beta0 = b0;
        if (!isfinite(b0)) {
            st->status = GK_ERR_NAN;
            st->halt = 2;
            return;
        }
        if (b0 <= st->thr) {
            st->status = GK_OK;
            st->halt = 2;
            return;
        }
        if (st->iter >= st->max_iters) {
            st->status = GK_NOT_CONVERGED;
            st->halt = 2;
            return;
        }
        if (st->stag > 0.0 && st->prev_beta0 > 0.0 && b0 > st->stag * st->prev_beta0) {
            st->status = GK_NOT_CONVERGED;  // stagnating inner solve: hand back
            st->halt = 2;
            return;
        }
        st->prev_beta0 = b0;
        if (st->cycle_end) st->restarts += 1;  // a cycle ended and a new one starts
        for (int j = 0; j <= st->m; ++j) st->g[j] = 0.0;
        st->g[0] = b0;
        st->k = 0;
        st->cycle_end = 0;
        st->inv_h = 1.0 / b0;
        st->v0_pending = 1;
    }
};

// true residual at cycle end (skipped inside a cycle)
template <typename T>
struct EpiGmResid {
    T* __restrict__ r;
    const T* __restrict__ b;
    const KState* st;
    double* partials;
    unsigned* ticket;
    GmRestartFin fin;
    static constexpr int NA = 1;
    using acc_t = T;  // per-thread partial sums in the vector type
    __device__ __forceinline__ bool skip() const {
        return halted(st) || !*reinterpret_cast<const volatile int32_t*>(&st->cycle_end);
    }
    __device__ __forceinline__ void row(int64_t i, T s, T* acc) const {
        const T v = b[i] - s;
        r[i] = v;
        acc[0] = fmadd(v, v, acc[0]);
    }
    __device__ __forceinline__ void finish(T* acc) const {
        double a[1] = {(double)acc[0]};
        grid_reduce_finish<1>(a, partials, ticket, fin);
    }
    __device__ __forceinline__ void timed_out() const {}
};

// v_0 = r / beta0 ; z = M^-1 v_0 (after a restart decided to continue)
template <typename T>
__global__ void EW_BOUNDS k_gm_v0(int32_t n, T* __restrict__ V, const T* __restrict__ r, T* __restrict__ z,
                        const T* __restrict__ dinv, const KState* st) {
    if (halted(st) || !st->v0_pending) return;
    constexpr int N = Pack<T>::N;
    const T ib = (T)st->inv_h;
    const bool vec = al16(V) && al16(r) && al16(z) && al16(dinv);
    PACK_LOOP(j, n, T) {
        Pack<T> V0 = pld(r, j, n, vec);
        Pack<T> Z = dinv ? pld(dinv, j, n, vec) : Pack<T>{};
#pragma unroll
        for (int c = 0; c < N; ++c) {
            V0.v[c] = V0.v[c] * ib;
            Z.v[c] = dinv ? Z.v[c] * V0.v[c] : V0.v[c];
        }
        pst(V, j, n, vec, V0);
        pst(z, j, n, vec, Z);
    }
}


// Jacobi diagonal of ELL / SELL-P matrices (first stored entry with col == i)
template <typename V, typename T>
__global__ void k_jacobi_gen_padded(int32_t n, int fmt, int64_t stride, int32_t K, int32_t S,
                                    const int32_t* __restrict__ slen,
                                    const int64_t* __restrict__ sset,
                                    const int32_t* __restrict__ pc, const V* __restrict__ pv,
                                    T* __restrict__ dinv, int32_t* bad) {
    GRID_LOOP(i, n) {
        T d = T(0);
        bool found = false;
        if (fmt == GK_ELL) {
            for (int32_t j = 0; j < K; ++j) {
                const int64_t at = (int64_t)j * stride + i;
                if (pc[at] == i) { d += cvt<T>(pv[at]); found = true; }
            }
        } else {
            const int64_t sl = i / S, t = i - sl * S;
            for (int32_t j = 0; j < slen[sl]; ++j) {
                const int64_t at = (sset[sl] + j) * S + t;
                if (pc[at] == i) { d += cvt<T>(pv[at]); found = true; }
            }
        }
        if (!found || d == T(0)) {
            atomicOr(bad, 1);
            dinv[i] = T(0);
        } else {
            dinv[i] = T(1) / d;
        }
    }
}

// Setup fins: ||b|| -> thr; initial true residual
struct FinBnorm {
    KState* st;
    double tol;  // < 0: the state's tol
    __device__ void operator()(double* t) const {
        const double bn = sqrt(t[0]);
        st->bnorm = bn;
        st->thr = (tol < 0.0 ? st->tol : tol) * bn;
        if (!isfinite(bn)) {
            st->status = GK_ERR_NAN;
            st->halt = 2;
        } else if (bn == 0.0) {
            st->status = GK_OK;
            st->halt = 2;
        }
    }
};

struct FinTrue {  // true residual norm; mode 0: initial check, 1: recheck
    KState* st;
    int mode;
    __device__ void operator()(double* t) const {
        const double tn = sqrt(t[0]);
        st->tnorm = tn;
        if (mode == 0) st->rnorm = tn;
        if (!isfinite(tn)) {
            st->status = GK_ERR_NAN;
            st->halt = 2;
        } else if (tn <= st->thr) {
            st->status = GK_OK;
            st->halt = 2;
        }
    }
};

// EpiTResid: true residual with a fin but no halt check
template <typename T, class Fin>
using EpiRes = EpiResid<T, Fin>;

// BiCGSTAB t = A shat, skipped at a half-step exit
template <typename T>
struct EpiBiT {
    T* __restrict__ y;
    const T* __restrict__ u;
    const KState* st;
    double* partials;
    unsigned* ticket;
    BiOmegaFin fin;
    static constexpr int NA = 2;
    using acc_t = T;
    __device__ __forceinline__ bool skip() const {
        return halted(st) || *reinterpret_cast<const volatile int32_t*>(&st->half) != 0;
    }
    __device__ __forceinline__ void row(int64_t i, T s, T* acc) const {
        y[i] = s;
        acc[0] = fmadd(s, u[i], acc[0]);
        acc[1] = fmadd(s, s, acc[1]);
    }
    __device__ __forceinline__ void finish(T* acc) const {
        double a[2] = {(double)acc[0], (double)acc[1]};
        grid_reduce_finish<2>(a, partials, ticket, fin);
    }
    __device__ __forceinline__ void timed_out() const {}
};

template <typename T>
__global__ void EW_BOUNDS k_cast_add(int32_t n, double* __restrict__ x, const T* __restrict__ d) {
    GRID_LOOP(i, n) x[i] += (double)d[i];
}
template <typename T>
__global__ void EW_BOUNDS k_cast_to(int32_t n, const double* __restrict__ r, T* __restrict__ o) {
    GRID_LOOP(i, n) o[i] = (T)r[i];
}

// ---------------------------------------------------------------- block-Jacobi
// Diagonal blocks of bs consecutive rows (the last may be shorter), inverted
// once per matrix (k_bj_gen) and applied as z = B r (k_bj_apply, k_bj_gm).
// The inverses are stored per block column-major in the vector type T:
// entry (i, j) of block kb at binvT[kb*bs*bs + j*bs + i], so that the rows
// of a block read consecutive addresses for each j.

constexpr int BJ_MAX = 32;  // largest block size

// One warp per block: gather A's block from CSR (lane i sums row i's
// entries in CSR order), Gauss-Jordan on [A | I] in double with partial
// pivoting (largest |a|, the first on ties), lanes over the columns.  A block
// with no nonzero pivot left sets *bad (singular: the zero-diagonal error).
template <typename V, typename T>
__global__ void __launch_bounds__(32)
k_bj_gen(int32_t n, int32_t bs, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
         const V* __restrict__ va, T* __restrict__ binvT, int32_t* bad) {
    __shared__ double aug[BJ_MAX][2 * BJ_MAX + 1];
    const int lane = threadIdx.x;
    const int64_t kb = blockIdx.x;
    const int32_t r0 = (int32_t)(kb * bs);
    const int m = min(bs, n - r0);
    for (int i = 0; i < m; ++i)
        for (int c = lane; c < 2 * m; c += 32) aug[i][c] = (c - m == i) ? 1.0 : 0.0;
    __syncwarp();
    if (lane < m) {
        const int i = lane;
        for (int32_t k = rp[r0 + i]; k < rp[r0 + i + 1]; ++k) {
            const int32_t j = ci[k] - r0;
            if (j >= 0 && j < m) aug[i][j] += cvt<double>(va[k]);
        }
    }
    __syncwarp();
    for (int c = 0; c < m; ++c) {
        // pivot: largest |a_rc| over r >= c, the smallest r on ties
        double best = -1.0;
        int piv = c;
        if (lane >= c && lane < m) {
            best = fabs(aug[lane][c]);
            piv = lane;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double ob = __shfl_down_sync(0xffffffffu, best, o);
            const int op = __shfl_down_sync(0xffffffffu, piv, o);
            if (ob > best || (ob == best && op < piv)) {
                best = ob;
                piv = op;
            }
        }
        piv = __shfl_sync(0xffffffffu, piv, 0);
        if (aug[piv][c] == 0.0) {
            if (lane == 0) atomicExch(bad, 1);
            return;
        }
        if (piv != c)
            for (int col = lane; col < 2 * m; col += 32) {
                const double t = aug[c][col];
                aug[c][col] = aug[piv][col];
                aug[piv][col] = t;
            }
        __syncwarp();
        const double d = aug[c][c];
        __syncwarp();
        for (int col = lane; col < 2 * m; col += 32) aug[c][col] = aug[c][col] / d;
        __syncwarp();
        for (int r = 0; r < m; ++r) {
            if (r == c) continue;
            const double f = aug[r][c];
            __syncwarp();
            if (f != 0.0)
                for (int col = lane; col < 2 * m; col += 32)
                    aug[r][col] = aug[r][col] - f * aug[c][col];
            __syncwarp();
        }
    }
    T* out = binvT + (size_t)kb * bs * bs;
    for (int e = lane; e < bs * bs; e += 32) {
        const int j = e / bs, i = e - j * bs;
        out[e] = (i < m && j < m) ? cvt<T>(aug[i][m + j]) : T(0);
    }
}

// z_i = sum_j B[i][j] r[r0 + j] per row, handed to an epilogue (store,
// store + dot with a fin, store + x update); exits at once when halted.
template <typename T, class Epi>
__global__ void EW_BOUNDS k_bj_apply(int32_t n, int32_t bs, const T* __restrict__ binvT,
                                     const T* __restrict__ r, Epi epi) {
    if (epi.skip()) return;
    typename Epi::acc_t acc[Epi::NA > 0 ? Epi::NA : 1] = {};
    GRID_LOOP(i, n) {
        const int32_t kb = (int32_t)(i / bs), li = (int32_t)(i - (int64_t)kb * bs);
        const int64_t r0 = (int64_t)kb * bs;
        const int m = (int)min((int64_t)bs, (int64_t)n - r0);
        const T* col = binvT + (size_t)kb * bs * bs + li;
        T s = T(0);
        for (int j = 0; j < m; ++j) s = fmadd(col[(size_t)j * bs], r[r0 + j], s);
        epi.row(i, s, acc);
    }
    epi.finish(acc);
}

// y_i = s ; x_i += alpha s  (CGS: uh = B (u + q), x += alpha uh)
template <typename T>
struct EpiBjX {
    T* __restrict__ y;
    T* __restrict__ x;
    const KState* st;
    static constexpr int NA = 0;
    using acc_t = T;
    __device__ __forceinline__ bool skip() const { return halted(st); }
    __device__ __forceinline__ void row(int64_t i, T s, T*) const {
        y[i] = s;
        x[i] = fmadd((T)st->alpha, s, x[i]);
    }
    __device__ __forceinline__ void finish(T*) const {}
    __device__ __forceinline__ void timed_out() const {}
};

// GMRES v_0 step: z = B v_0, only when a restart decided to continue
template <typename T>
struct EpiBjV0 {
    T* __restrict__ y;
    const KState* st;
    static constexpr int NA = 0;
    using acc_t = T;
    __device__ __forceinline__ bool skip() const { return halted(st) || !st->v0_pending; }
    __device__ __forceinline__ void row(int64_t i, T s, T*) const { y[i] = s; }
    __device__ __forceinline__ void finish(T*) const {}
    __device__ __forceinline__ void timed_out() const {}
};

// GMRES after k_gm_next: inside a cycle z = B v_k; at the end of a cycle
// x += B (V y) (V y left in ubuf by k_gm_next).
template <typename T>
__global__ void EW_BOUNDS k_bj_gm(int32_t n, int32_t bs, const T* __restrict__ binvT,
                                  const T* __restrict__ V, int64_t ldv,
                                  const T* __restrict__ ubuf, T* __restrict__ z,
                                  T* __restrict__ x, const KState* st) {
    if (halted(st)) return;
    const bool ce = st->cycle_end != 0;
    const T* src = ce ? ubuf : V + (int64_t)st->k * ldv;
    GRID_LOOP(i, n) {
        const int32_t kb = (int32_t)(i / bs), li = (int32_t)(i - (int64_t)kb * bs);
        const int64_t r0 = (int64_t)kb * bs;
        const int m = (int)min((int64_t)bs, (int64_t)n - r0);
        const T* col = binvT + (size_t)kb * bs * bs + li;
        T s = T(0);
        for (int j = 0; j < m; ++j) s = fmadd(col[(size_t)j * bs], src[r0 + j], s);
        if (ce) x[i] += s;
        else z[i] = s;
    }
}

// ---------------------------------------------------------------- ILU(0)
// The engine applies ILU(0) where it applies block-Jacobi (the substitution
// kernels of ilu.cuh), with these sources, skips and outputs.

// GMRES after k_gm_next: V y (ubuf) at a cycle end, else the new v_k
template <typename T>
struct IluSrcGm {
    const T* V;
    int64_t ldv;
    const T* ubuf;
    const KState* st;
    __device__ __forceinline__ const T* ptr() const {
        return st->cycle_end ? ubuf : V + (int64_t)st->k * ldv;
    }
};

struct IluSkipHalt {
    const KState* st;
    __device__ __forceinline__ bool skip() const { return halted(st); }
};

// runs only while *gate is 0 (a gated step of the device solver loop)
struct IluSkipGate {
    const int32_t* gate;
    __device__ __forceinline__ bool skip() const {
        return *reinterpret_cast<const volatile int32_t*>(gate) != 0;
    }
};

// GMRES v_0 step: only when a restart decided to continue
struct IluSkipV0 {
    const KState* st;
    __device__ __forceinline__ bool skip() const { return halted(st) || !st->v0_pending; }
};

// y = s ; x += alpha s  (CGS: uh = M^-1 (u + q), x += alpha uh)
template <typename T>
struct IluOutX {
    T* y;
    T* x;
    const KState* st;
    __device__ __forceinline__ T* dst() const { return y; }
    __device__ __forceinline__ void extra(int64_t i, T v) const {
        x[i] = fmadd((T)st->alpha, v, x[i]);
    }
};

// GMRES: inside a cycle z = M^-1 v_k; at a cycle end x += M^-1 (V y), the
// substitution's unknowns kept in a scratch vector
template <typename T>
struct IluOutGm {
    T* z;
    T* scratch;
    T* x;
    const KState* st;
    __device__ __forceinline__ T* dst() const { return st->cycle_end ? scratch : z; }
    __device__ __forceinline__ void extra(int64_t i, T v) const {
        if (st->cycle_end) x[i] += v;
    }
};

// a substitution wait that ran out stops the solve with GK_ERR_TIMEOUT
struct IluErrSt {
    KState* st;
    __device__ __forceinline__ void operator()(unsigned e) const {
        if (e) {
            st->status = GK_ERR_TIMEOUT;
            st->halt = 2;
        }
    }
};

// <a, b> handed to a fin (CG with ILU: rho = <r, z> after z = M^-1 r)
template <typename T, class Fin>
__global__ void EW_BOUNDS k_dot_fin(int32_t n, const T* __restrict__ a, const T* __restrict__ b,
                                    const int32_t* halt, double* partials, unsigned* ticket,
                                    Fin fin) {
    if (halt && *reinterpret_cast<const volatile int32_t*>(halt) != 0) return;
    constexpr int N = Pack<T>::N;
    const bool vec = al16(a) && al16(b);
    T acc[1] = {T(0)};
    PACK_LOOP(j, n, T) {
        const Pack<T> A_ = pld(a, j, n, vec), B_ = pld(b, j, n, vec);
#pragma unroll
        for (int c = 0; c < N; ++c) acc[0] = fmadd(A_.v[c], B_.v[c], acc[0]);
    }
    finish_ew<1>(acc, partials, ticket, fin);
}

// ------------------------------------------------------------ host side

constexpr size_t HDR = offsetof(KState, H);

// ------------------------------------------------------------ device solver loop
// The Krylov loop of the multi-kernel engine runs inside one CUDA graph: a
// conditional WHILE node repeats a body made of a chunk of iterations and
// the one-thread control steps below; cudaGraphSetConditional ends it.  The
// control is the stopping rule: a recurrence residual that passes is
// confirmed by the true residual b - A x; if that fails, the recurrence
// restarts from x with r = b - A x (residual replacement), at most
// checks_left times, and an inner solve of refinement stops after two
// replacements.  max_loops bounds the passes whatever happens, so the loop
// always ends.  The steps that run only on some passes (the confirmation,
// the replacement, the exit's true residual) are kernels that return at once
// unless their gate word in the state is 0.

// A solve's state header: zero, then its parameters (on the caller's stream,
// before the graph).
static __global__ void k_state_init(KState* st, double tol, int32_t max_iters, int32_t m, double stag,
                             int32_t stall, int32_t inner, int32_t max_loops, int32_t max_checks) {
    unsigned long long* w = reinterpret_cast<unsigned long long*>(st);
    for (size_t k = 0; k < HDR / sizeof(unsigned long long); ++k) w[k] = 0ull;
    st->tol = tol;
    st->max_iters = max_iters;
    st->m = m;
    st->stag = stag;
    st->stall = stall;
    st->inner = inner;
    st->max_loops = max_loops;
    st->checks_left = max_checks;
    st->nocheck = st->noreplace = st->nofinal = st->nozero = 1;
}

// after a chunk (CG, BiCGSTAB, CGS): stop, or confirm a passed recurrence
static __global__ void k_ctl_check(KState* st) {
    st->loops += 1;
    st->nocheck = 1;
    st->noreplace = 1;
    if (st->halt == 2) {
        st->done = 1;
        return;
    }
    if (st->loops > st->max_loops) {
        st->status = GK_ERR_TIMEOUT;
        st->halt = 2;
        st->done = 1;
        return;
    }
    if (st->halt == 1) {
        if (st->inner && st->restarts >= 2) {  // the outer FP64 residual decides
            st->done = 1;
            return;
        }
        if (--st->checks_left < 0) {
            st->status = GK_ERR_TIMEOUT;
            st->halt = 2;
            st->done = 1;
            return;
        }
        st->halt = 0;
        st->nocheck = 0;  // the true residual runs next
    }
}

// after the true residual: converged (its fin set halt = 2), out of
// iterations, or replace r and restart
static __global__ void k_ctl_replace(KState* st) {
    if (st->nocheck) return;
    st->nocheck = 1;
    if (st->halt == 2) {
        st->done = 1;
        return;
    }
    if (st->iter >= st->max_iters) {
        st->status = GK_NOT_CONVERGED;
        st->halt = 2;
        st->done = 1;
        return;
    }
    st->noreplace = 0;  // r = b - A x and the method's restart run next
}

// end of a pass: count a replacement, and loop again unless done (cond = 0:
// an unrolled graph without the loop node, see capture_solve)
static __global__ void k_ctl_next(KState* st, cudaGraphConditionalHandle h, int cond) {
    if (!st->noreplace) {
        st->restarts += 1;
        st->noreplace = 1;
    }
    if (cond) cudaGraphSetConditional(h, st->done ? 0u : 1u);
}

// end of a GMRES pass: loop until halted (restarts are decided inside)
static __global__ void k_ctl_gmres(KState* st, cudaGraphConditionalHandle h, int cond) {
    st->loops += 1;
    if (st->halt == 0 && st->loops > st->max_loops) {
        st->status = GK_ERR_TIMEOUT;
        st->halt = 2;
    }
    if (cond) cudaGraphSetConditional(h, st->halt ? 0u : 1u);
}

// after the loop: whether the exit computes the true residual (not for an
// inner solve that stopped on its recurrence) or zeroes x (b = 0)
static __global__ void k_ctl_exit(KState* st) {
    const bool inner_pass = st->inner && st->halt == 1;
    st->nofinal = (st->bnorm > 0.0 && !inner_pass) ? 0 : 1;
    st->nozero = st->bnorm == 0.0 ? 0 : 1;
}

// The outcome of a solve from its state (the rules of gk_solve): written
// to info (host or device memory) by write_info / k_write_info.
__host__ __device__ inline void solve_outcome(const KState* st, bool rowtile_err, int32_t layout,
                                              int32_t slice, gk_solve_info* o) {
    int status = st->status;
    const bool inner_pass = st->inner && st->halt == 1;
    const double bn = st->bnorm;
    o->iters = st->iter;
    o->restarts = st->restarts;
    o->outer_iters = 0;
    o->rel_res_recurrence = bn > 0.0 ? st->rnorm / bn : 0.0;
    o->rel_res_true = inner_pass ? o->rel_res_recurrence : (bn > 0.0 ? st->tnorm / bn : 0.0);
    if (inner_pass) status = GK_OK;
    if (bn == 0.0) {
        status = GK_OK;
        o->iters = 0;
        o->rel_res_recurrence = o->rel_res_true = 0.0;
    }
    if (rowtile_err) status = GK_ERR_TIMEOUT;
    o->status = (gk_status)status;
    o->device_ms = 0.f;
    o->spmv_format = layout;
    o->slice_size = slice;
    o->block_threads = 0;
}

static __global__ void k_write_info(const KState* st, gk_solve_info* info, const int32_t* rowtile_err,
                             int32_t layout, int32_t slice) {
    gk_solve_info o;
    solve_outcome(st, rowtile_err && *rowtile_err != 0, layout, slice, &o);
    *info = o;
}

struct SolverCache {
    DevBuf vecs, partials, ticket, state;
    KState* hst = nullptr;  // pinned mirror of the state header
    int32_t* hzero = nullptr;
    cudaGraphExec_t exec = nullptr;
    // host-driven loop: the passes and the exit as graphs of their own, and
    // two pinned header slots with their events (pass k writes slot k % 2)
    cudaGraphExec_t exec_body = nullptr, exec_post = nullptr;
    KState* hring = nullptr;
    cudaEvent_t evr[2] = {nullptr, nullptr};
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // key of the captured graph
    void* kv = nullptr;
    int kmethod = -1, kprec = -1, km = -1, kchunk = 0, khost = -1;
    uint64_t kwait = 0;  // wait budget the graph's kernels were captured with
    ~SolverCache() {
        if (exec) cudaGraphExecDestroy(exec);
        if (exec_body) cudaGraphExecDestroy(exec_body);
        if (exec_post) cudaGraphExecDestroy(exec_post);
        if (hring) cudaFreeHost(hring);
        for (cudaEvent_t e : evr)
            if (e) cudaEventDestroy(e);
        if (hst) cudaFreeHost(hst);
        if (hzero) cudaFreeHost(hzero);
        if (ev0) cudaEventDestroy(ev0);
        if (ev1) cudaEventDestroy(ev1);
        vecs.release();
        partials.release();
        ticket.release();
        state.release();
    }
};

// host-side helpers (solve.cu)
gk_status get_cache(gk_matrix A, SolverCache** out);
gk_status side_stream(gk_matrix A);
gk_status read_hdr(SolverCache* C, cudaStream_t s);
gk_status clear_halt(SolverCache* C, cudaStream_t s);
gk_status ensure_block_jacobi(gk_matrix A, int32_t bs, cudaStream_t s);

template <typename T>
static T* vec_at(SolverCache* C, int64_t n, int idx) {
    const size_t stride = ((size_t)n * sizeof(T) + 255) & ~(size_t)255;
    return reinterpret_cast<T*>(static_cast<char*>(C->vecs.ptr) + stride * (size_t)idx);
}

template <typename T>
static gk_status ensure_vecs(SolverCache* C, int64_t n, int count) {
    const size_t stride = ((size_t)n * sizeof(T) + 255) & ~(size_t)255;
    return C->vecs.ensure(stride * (size_t)count + 256);
}

// Captures a whole solve into C->exec: pre(stream), then a conditional
// WHILE node whose body is body(stream, handle, 1) (it must end with a
// kernel that sets the handle), then post(stream).  The body is captured on
// the handle's second library stream into the node's child graph.
// GK_SOLVE_UNROLLED=k (k > 0) instead repeats body(stream, 0, 0) k times
// with no loop node: the solve runs at most k passes, and every kernel of
// it can be profiled (profilers do not see into graphs with conditional
// nodes); for measurement only.
// host_loop: three graphs instead -- C->exec = pre, C->exec_body = one
// pass, body(stream, 0, 0), and C->exec_post = post -- which run_host_loop
// launches, the passes from the host.
template <class F>
static gk_status capture_one(cudaStream_t cs, F&& f, cudaGraphExec_t* out) {
    cudaGraph_t g = nullptr;
    GK_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    gk_status st = f(cs);
    cudaError_t e = cudaStreamEndCapture(cs, &g);
    if (st != GK_OK || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return st != GK_OK ? st : GK_ERR_CUDA;
    }
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    GK_CUDA(e);
    return GK_OK;
}

template <class Pre, class Body, class Post>
static gk_status capture_solve(gk_matrix A, SolverCache* C, Pre&& pre, Body&& body, Post&& post,
                               bool host_loop) {
    GateCapture gate;  // one capture at a time, no device-wide call meanwhile
    GK_TRY(side_stream(A));
    for (cudaGraphExec_t* x : {&C->exec, &C->exec_body, &C->exec_post})
        if (*x) {
            cudaGraphExecDestroy(*x);
            *x = nullptr;
        }
    if (host_loop) {
        if (!C->hring) GK_CUDA(cudaMallocHost(&C->hring, 2 * HDR));
        for (cudaEvent_t& e : C->evr)
            if (!e) GK_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        GK_TRY(capture_one(A->side, pre, &C->exec));
        GK_TRY(capture_one(A->side, [&](cudaStream_t cs) { return body(cs, 0, 0); },
                           &C->exec_body));
        return capture_one(A->side, post, &C->exec_post);
    }
    int unrolled = 0;
    if (const char* e = getenv("GK_SOLVE_UNROLLED")) unrolled = std::max(0, atoi(e));
    cudaGraph_t g = nullptr;
    GK_CUDA(cudaStreamBeginCapture(A->side, cudaStreamCaptureModeThreadLocal));
    gk_status st = pre(A->side);
    for (int k = 0; k < unrolled && st == GK_OK; ++k) st = body(A->side, 0, 0);
    if (st == GK_OK && !unrolled) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        cudaGraph_t cg = nullptr;
        const cudaGraphNode_t* deps = nullptr;
        size_t ndeps = 0;
        cudaGraphConditionalHandle hc = 0;
        cudaGraphNodeParams cp = {};
        cudaGraphNode_t node = nullptr;
        if (cudaStreamGetCaptureInfo(A->side, &cs, nullptr, &cg, &deps, nullptr, &ndeps) !=
                cudaSuccess ||
            cs != cudaStreamCaptureStatusActive ||
            cudaGraphConditionalHandleCreate(&hc, cg, 1, cudaGraphCondAssignDefault) != cudaSuccess) {
            st = GK_ERR_CUDA;
        } else {
            cp.type = cudaGraphNodeTypeConditional;
            cp.conditional.handle = hc;
            cp.conditional.type = cudaGraphCondTypeWhile;
            cp.conditional.size = 1;
            if (cudaGraphAddNode(&node, cg, deps, nullptr, ndeps, &cp) != cudaSuccess ||
                cudaStreamUpdateCaptureDependencies(A->side, &node, nullptr, 1,
                                                    cudaStreamSetCaptureDependencies) != cudaSuccess)
                st = GK_ERR_CUDA;
        }
        if (st == GK_OK) {
            if (cudaStreamBeginCaptureToGraph(A->side2, cp.conditional.phGraph_out[0], nullptr,
                                              nullptr, 0, cudaStreamCaptureModeThreadLocal) !=
                cudaSuccess) {
                st = GK_ERR_CUDA;
            } else {
                st = body(A->side2, hc, 1);
                cudaGraph_t bg = nullptr;
                if (cudaStreamEndCapture(A->side2, &bg) != cudaSuccess && st == GK_OK)
                    st = GK_ERR_CUDA;
            }
        }
    }
    if (st == GK_OK) st = post(A->side);
    cudaError_t e = cudaStreamEndCapture(A->side, &g);
    if (st != GK_OK) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return st;
    }
    GK_CUDA(e);
    e = cudaGraphInstantiate(&C->exec, g, 0);
    cudaGraphDestroy(g);
    GK_CUDA(e);
    return GK_OK;
}

inline int chunk_for(int64_t n) { return n < 200000 ? 32 : 8; }

// Where the Krylov loop runs: on the device (one graph with a conditional
// WHILE node, the default) or, with GK_SOLVE_LOOP=host, from the host:
// one graph per pass, launched while the previous pass runs.
inline bool solve_loop_on_host() {
    const char* e = getenv("GK_SOLVE_LOOP");
    return e && strcmp(e, "host") == 0;
}

// A captured host-driven solve: pre, then passes until the state says the
// loop is over (done; GMRES: halt) with two passes in flight, then post.
// Each pass copies the state header into its pinned slot (pass k: slot
// k % 2) and records that slot's event.  The pass issued after the last one
// needed finds the solve halted and every kernel of it returns at once, so
// the result is the device loop's, bit for bit.
static gk_status run_host_loop(SolverCache* C, cudaStream_t s, bool gmres, int32_t max_loops) {
    GK_CUDA(cudaGraphLaunch(C->exec, s));
    char* ring = reinterpret_cast<char*>(C->hring);
    auto issue = [&](int k) -> gk_status {
        GK_CUDA(cudaGraphLaunch(C->exec_body, s));
        GK_CUDA(cudaMemcpyAsync(ring + (size_t)(k & 1) * HDR, C->state.ptr, HDR,
                                cudaMemcpyDeviceToHost, s));
        GK_CUDA(cudaEventRecord(C->evr[k & 1], s));
        return GK_OK;
    };
    int issued = 0;
    GK_TRY(issue(issued++));
    GK_TRY(issue(issued++));
    for (int k = 0;; ++k) {
        GK_CUDA(cudaEventSynchronize(C->evr[k & 1]));
        const KState* h = reinterpret_cast<const KState*>(ring + (size_t)(k & 1) * HDR);
        const bool over = gmres ? h->halt != 0 : h->done != 0;
        if (over || k > max_loops + 2) break;  // the device bounds the passes too
        GK_TRY(issue(issued++));
    }
    GK_CUDA(cudaGraphLaunch(C->exec_post, s));
    return GK_OK;
}


// Runs one Krylov solve on the multi-kernel engine.  b, x: device vectors
// of type T.  Result status and counters in *out.
// inner = true: a refinement inner solve.  It confirms a passed recurrence
// residual with the true residual like any solve, but after two residual
// replacements it stops anyway: the outer FP64 residual decides
// convergence, and an FP32 solve can stall above a tight inner tolerance.
template <typename V, typename T>
gk_status solve_mk(gk_matrix A, const T* b, T* x, int method, int pkind, int32_t bs, double tol,
                   int32_t max_iters, int32_t m, cudaStream_t s, SolveOut* out, bool inner,
                   gk_solve_info* info_dev = nullptr) {
    const int32_t n = A->n;
    SolverCache* C = nullptr;
    GK_TRY(get_cache(A, &C));
    // a row-tile SpMV whose wait ran past the budget sets the matrix's error
    // word: cleared here, turned into GK_ERR_TIMEOUT at the end
    const bool rowtile = A->fmt == GK_CSR && (A->plan.kind == 1 || A->plan.kind == 3) && A->plan.err;
    if (rowtile) GK_CUDA(cudaMemsetAsync(A->plan.err, 0, sizeof(int32_t), s));
    auto rowtile_timeout = [&]() -> bool {
        if (!rowtile) return false;
        int32_t e = 0;
        if (cudaMemcpyAsync(&e, A->plan.err, sizeof(e), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return true;
        return e != 0;
    };
    // preconditioner: pkind 0 none, 1 Jacobi (fused into the update kernels
    // as dinv), 2 block-Jacobi of bs rows (separate k_bj_* kernels; the
    // update kernels then run unpreconditioned into the vectors B is
    // applied to), 3 ILU(0) (the two substitution kernels where
    // block-Jacobi runs k_bj_*)
    const bool prec = pkind != 0;
    const bool block = pkind == 2;
    const bool ilu = pkind == 3;
    const bool sep = block || ilu;  // preconditioner applied by its own kernels
    const T* dinv = nullptr;
    const T* binv = nullptr;
    IluDev<T> ild;
    if (pkind == 1) {
        GK_TRY(ensure_jacobi(A, s));
        dinv = (const T*)A->dinv;
    } else if (block) {
        GK_TRY(ensure_block_jacobi(A, bs, s));
        binv = (const T*)A->binv;
    } else if (ilu) {
        GK_TRY(ensure_ilu(A, s));
        ild = ilu_view<T>(A);
        ild.wait_ns = A->wait_ns;
        GK_TRY(ilu_clear_err(ild, s));
    }
    const int nvec0 = method == GK_CG ? 5 : (method == GK_BICGSTAB || method == GK_CGS) ? 10 : m + 5;
    // ILU: two more vectors, the L substitution's output and GMRES's scratch
    const int nvec = nvec0 + (ilu ? 2 : 0);
    GK_TRY(ensure_vecs<T>(C, n, nvec + 2));  // + the solve's copies of b and x
    T* ilu_w = ilu ? vec_at<T>(C, n, nvec0) : nullptr;
    T* ilu_s = ilu ? vec_at<T>(C, n, nvec0 + 1) : nullptr;
    // multi-dot kernels: one wave of resident blocks sharing the rows equally
    const int64_t md_need = std::max<int64_t>(1, ((int64_t)n + MD_ROWS - 1) / MD_ROWS);
    auto md_grid_of = [&](auto kern) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, MD_THREADS, 0) != cudaSuccess || b < 1)
            b = 1;
        return (unsigned)std::min<int64_t>(md_need, (int64_t)num_sms() * std::min(b, 8));
    };
    const unsigned md_grid = (unsigned)std::min<int64_t>(md_need, (int64_t)num_sms() * 8);
    const size_t pcount = (size_t)std::max<unsigned>(num_sms() * 8, md_grid) * (size_t)(MAXM + 2);
    GK_TRY(C->partials.ensure(pcount * sizeof(double)));
    double* part = (double*)C->partials.ptr;
    unsigned* tk = (unsigned*)C->ticket.ptr;
    KState* st = (KState*)C->state.ptr;
    const int32_t* halt = &st->halt;

    // The solve reads and writes the handle's own copies of b and x, so the
    // cached graph serves every right-hand side and initial guess.
    T* bi = vec_at<T>(C, n, nvec);
    T* xi = vec_at<T>(C, n, nvec + 1);
    GK_CUDA(cudaMemcpyAsync(bi, b, sizeof(T) * (size_t)n, cudaMemcpyDeviceToDevice, s));
    GK_CUDA(cudaMemcpyAsync(xi, x, sizeof(T) * (size_t)n, cudaMemcpyDeviceToDevice, s));
    const int chunk = chunk_for(n);
    const int32_t max_checks = max_iters + 4;
    const int32_t max_loops = method == GK_GMRES ? max_iters / chunk + 8
                                                 : max_iters / chunk + max_checks + 8;
    k_state_init<<<1, 1, 0, s>>>(st, tol, max_iters, m, inner ? 0.95 : 0.0, inner ? 200 : 0,
                                 inner ? 1 : 0, max_loops, max_checks);
    GK_CUDA(cudaGetLastError());
    const int pkey = pkind * 64 + (block ? bs : 0);
    T* r = vec_at<T>(C, n, 0);
    T* tmp = vec_at<T>(C, n, 1);
    // exit: the true residual (unless an inner solve stopped on its
    // recurrence) or x = 0 for b = 0
    auto post = [&](cudaStream_t cs) -> gk_status {
        k_ctl_exit<<<1, 1, 0, cs>>>(st);
        EpiResid<T, FinNorm> ef{tmp, bi, &st->nofinal, part, tk, FinNorm{st, 1}};
        GK_TRY((launch_spmv_rows<V, T>(A, xi, ef, cs)));
        k_zero<T><<<ewg(k_zero<T>, n), 256, 0, cs>>>(n, xi, &st->nozero);
        GK_CUDA(cudaGetLastError());
        return GK_OK;
    };
    const bool host_loop = !info_dev && solve_loop_on_host();
    const bool stale = !C->exec || C->kmethod != method || C->kprec != pkey || C->km != m ||
                       C->kchunk != chunk || C->kv != (void*)C->vecs.ptr ||
                       C->kwait != A->wait_ns || C->khost != (int)host_loop;
    if (method == GK_GMRES && stale) {
        T* Vm = vec_at<T>(C, n, 3);
        T *w = vec_at<T>(C, n, 1), *z = vec_at<T>(C, n, 2);
        const int64_t ldv = (int64_t)(((size_t)n * sizeof(T) + 255) & ~(size_t)255) / sizeof(T);
        T* ubuf = vec_at<T>(C, n, m + 4);  // V y at a cycle end (block-Jacobi / ILU only)
        auto pre = [&](cudaStream_t cs) -> gk_status {
            k_norm2<T, FinBnorm><<<ewg(k_norm2<T, FinBnorm>, n), 256, 0, cs>>>(
                n, bi, part, tk, FinBnorm{st, -1.0});
            // cycle start: r = b - A x, restart fin sets g, k; v0 = r / beta0
            EpiResid<T, GmRestartFin> e0{r, bi, halt, part, tk, GmRestartFin{st}};
            GK_TRY((launch_spmv_rows<V, T>(A, xi, e0, cs)));
            k_gm_v0<T><<<ewg(k_gm_v0<T>, n), 256, 0, cs>>>(n, Vm, r, z, dinv, st);
            if (block)
                k_bj_apply<T, EpiBjV0<T>><<<ewg(k_bj_apply<T, EpiBjV0<T>>, n), 256, 0, cs>>>(
                    n, bs, binv, Vm, EpiBjV0<T>{z, st});
            if (ilu)
                GK_TRY(ilu_apply<T>(ild, IluSrc<T>{Vm}, ilu_w, IluOutStore<T>{z}, IluSkipV0{st},
                                    IluErrSt{st}, cs));
            GK_CUDA(cudaGetLastError());
            return GK_OK;
        };
        auto body = [&](cudaStream_t cs, cudaGraphConditionalHandle hc, int cond) -> gk_status {
            for (int c = 0; c < chunk; ++c) {
                EpiStoreHalt<T> e1{w, halt};
                GK_TRY((launch_spmv_rows<V, T>(A, z, e1, cs)));
                k_gm_dot1<T><<<md_grid_of(k_gm_dot1<T>), MD_THREADS, 0, cs>>>(n, ldv, Vm, w, st,
                                                                               part, tk);
                k_gm_dot2<T><<<md_grid_of(k_gm_dot2<T>), MD_THREADS, 0, cs>>>(n, ldv, Vm, w, st,
                                                                               part, tk);
                k_gm_orth<T><<<md_grid_of(k_gm_orth<T>), MD_THREADS, 0, cs>>>(n, ldv, Vm, w, st,
                                                                               part, tk);
                k_gm_next<T><<<ewg(k_gm_next<T>, n), 256, 0, cs>>>(n, ldv, Vm, w, z, xi, dinv, st,
                                                                   sep ? ubuf : nullptr);
                if (block)
                    k_bj_gm<T><<<ewg(k_bj_gm<T>, n), 256, 0, cs>>>(n, bs, binv, Vm, ldv, ubuf, z,
                                                                   xi, st);
                if (ilu)
                    GK_TRY(ilu_apply<T>(ild, IluSrcGm<T>{Vm, ldv, ubuf, st}, ilu_w,
                                        IluOutGm<T>{z, ilu_s, xi, st}, IluSkipHalt{st},
                                        IluErrSt{st}, cs));
                EpiGmResid<T> e2{r, bi, st, part, tk, GmRestartFin{st}};
                GK_TRY((launch_spmv_rows<V, T>(A, xi, e2, cs)));
                k_gm_v0<T><<<ewg(k_gm_v0<T>, n), 256, 0, cs>>>(n, Vm, r, z, dinv, st);
                if (block)
                    k_bj_apply<T, EpiBjV0<T>><<<ewg(k_bj_apply<T, EpiBjV0<T>>, n), 256, 0, cs>>>(
                        n, bs, binv, Vm, EpiBjV0<T>{z, st});
                if (ilu)
                    GK_TRY(ilu_apply<T>(ild, IluSrc<T>{Vm}, ilu_w, IluOutStore<T>{z},
                                        IluSkipV0{st}, IluErrSt{st}, cs));
            }
            k_ctl_gmres<<<1, 1, 0, cs>>>(st, hc, cond);
            GK_CUDA(cudaGetLastError());
            return GK_OK;
        };
        GK_TRY(capture_solve(A, C, pre, body, post, host_loop));
    } else if (stale) {
        // (re)start of the recurrence from r: gated by *gate when given
        auto init = [&](cudaStream_t q, const int32_t* gate) -> gk_status {
            if (method == GK_CG && block) {  // z = B r, rho = <r, z> ; p = z
                T *zb = vec_at<T>(C, n, 4), *pb = vec_at<T>(C, n, 3);
                using E0 = EpiDot<T, CgInitFin>;
                k_bj_apply<T, E0><<<ewg(k_bj_apply<T, E0>, n), 256, 0, q>>>(
                    n, bs, binv, r, E0{zb, r, gate, part, tk, CgInitFin{st}});
                k_copy<T><<<ewg(k_copy<T>, n), 256, 0, q>>>(n, zb, pb, gate);
            } else if (method == GK_CG && ilu) {  // z = M^-1 r, rho = <r, z> ; p = z
                T *zb = vec_at<T>(C, n, 4), *pb = vec_at<T>(C, n, 3);
                if (gate)
                    GK_TRY(ilu_apply<T>(ild, IluSrc<T>{r}, ilu_w, IluOutStore<T>{zb},
                                        IluSkipGate{gate}, IluErrSt{st}, q));
                else
                    GK_TRY(ilu_apply<T>(ild, IluSrc<T>{r}, ilu_w, IluOutStore<T>{zb},
                                        IluSkipNever{}, IluErrSt{st}, q));
                k_dot_fin<T, CgInitFin><<<ewg(k_dot_fin<T, CgInitFin>, n), 256, 0, q>>>(
                    n, r, zb, gate, part, tk, CgInitFin{st});
                k_copy<T><<<ewg(k_copy<T>, n), 256, 0, q>>>(n, zb, pb, gate);
            } else if (method == GK_CG)  // slots: 0 r, 1 tmp, 2 q, 3 p, 4 z
                k_cg_init<T><<<ewg(k_cg_init<T>, n), 256, 0, q>>>(
                    n, r, vec_at<T>(C, n, 4), vec_at<T>(C, n, 3), dinv, st, part, tk, gate);
            else if (method == GK_CGS)
                // slots: 0 r, 1 tmp, 2 rt, 3 u, 4 p, 5 q, 6 ph, 7 vh, 8 uh
                k_cgs_init<T><<<ewg(k_cgs_init<T>, n), 256, 0, q>>>(n, r, vec_at<T>(C, n, 2), st,
                                                                    part, tk, gate);
            else
                // slots: 0 r, 1 tmp, 2 rhat, 3 p, 4 phat, 5 s, 6 v, 7 shat, 8 t
                k_bi_init<T><<<ewg(k_bi_init<T>, n), 256, 0, q>>>(
                    n, r, vec_at<T>(C, n, 2), vec_at<T>(C, n, 3), vec_at<T>(C, n, 6), st, part,
                    tk, gate);
            GK_CUDA(cudaGetLastError());
            return GK_OK;
        };
        auto pre = [&](cudaStream_t cs) -> gk_status {
            k_norm2<T, FinBnorm><<<ewg(k_norm2<T, FinBnorm>, n), 256, 0, cs>>>(
                n, bi, part, tk, FinBnorm{st, -1.0});
            // initial true residual r = b - A x (stops at once when it passes)
            EpiResid<T, FinTrue> e0{r, bi, halt, part, tk, FinTrue{st, 0}};
            GK_TRY((launch_spmv_rows<V, T>(A, xi, e0, cs)));
            return init(cs, nullptr);
        };
        auto step = [&](cudaStream_t cs) -> gk_status {
            if (method == GK_CG) {
                T *z = prec ? vec_at<T>(C, n, 4) : r, *p = vec_at<T>(C, n, 3),
                  *q = vec_at<T>(C, n, 2);
                EpiDot<T, CgAlphaFin> e1{q, p, halt, part, tk, CgAlphaFin{st}};
                GK_TRY((launch_spmv_rows<V, T>(A, p, e1, cs)));
                k_cg_update<T><<<ewg(k_cg_update<T>, n), 256, 0, cs>>>(n, xi, r, z, p, q, dinv, st,
                                                                       part, tk, pkind);
                if (block) {  // z = B r ; beta = <r, z> / rho
                    using E1 = EpiDot<T, CgBetaFin>;
                    k_bj_apply<T, E1><<<ewg(k_bj_apply<T, E1>, n), 256, 0, cs>>>(
                        n, bs, binv, r, E1{z, r, halt, part, tk, CgBetaFin{st}});
                }
                if (ilu) {  // z = M^-1 r ; beta = <r, z> / rho
                    GK_TRY(ilu_apply<T>(ild, IluSrc<T>{r}, ilu_w, IluOutStore<T>{z},
                                        IluSkipHalt{st}, IluErrSt{st}, cs));
                    k_dot_fin<T, CgBetaFin><<<ewg(k_dot_fin<T, CgBetaFin>, n), 256, 0, cs>>>(
                        n, r, z, halt, part, tk, CgBetaFin{st});
                }
                k_cg_p<T><<<ewg(k_cg_p<T>, n), 256, 0, cs>>>(n, p, z, st);
            } else if (method == GK_CGS) {
                T *rt = vec_at<T>(C, n, 2), *u = vec_at<T>(C, n, 3), *p = vec_at<T>(C, n, 4);
                T *q = vec_at<T>(C, n, 5), *ph = vec_at<T>(C, n, 6), *vh = vec_at<T>(C, n, 7);
                T *uh = vec_at<T>(C, n, 8), *tb = vec_at<T>(C, n, 9);
                const T* phs = prec ? ph : p;
                k_cgs_p<T><<<ewg(k_cgs_p<T>, n), 256, 0, cs>>>(n, u, p, ph, r, q, dinv, st);
                if (block)
                    k_bj_apply<T, EpiStoreHalt<T>><<<ewg(k_bj_apply<T, EpiStoreHalt<T>>, n), 256, 0, cs>>>(
                        n, bs, binv, p, EpiStoreHalt<T>{ph, halt});
                if (ilu)
                    GK_TRY(ilu_apply<T>(ild, IluSrc<T>{p}, ilu_w, IluOutStore<T>{ph},
                                        IluSkipHalt{st}, IluErrSt{st}, cs));
                EpiDot<T, CgsAlphaFin> e1{vh, rt, halt, part, tk, CgsAlphaFin{st}};
                GK_TRY((launch_spmv_rows<V, T>(A, phs, e1, cs)));
                k_cgs_q<T><<<ewg(k_cgs_q<T>, n), 256, 0, cs>>>(n, q, uh, xi, u, vh, dinv, st,
                                                               sep ? tb : nullptr);
                if (block)
                    k_bj_apply<T, EpiBjX<T>><<<ewg(k_bj_apply<T, EpiBjX<T>>, n), 256, 0, cs>>>(
                        n, bs, binv, tb, EpiBjX<T>{uh, xi, st});
                if (ilu)
                    GK_TRY(ilu_apply<T>(ild, IluSrc<T>{tb}, ilu_w, IluOutX<T>{uh, xi, st},
                                        IluSkipHalt{st}, IluErrSt{st}, cs));
                EpiCgsR<T> e2{r, rt, st, part, tk};
                GK_TRY((launch_spmv_rows<V, T>(A, uh, e2, cs)));
            } else {
                T *rh = vec_at<T>(C, n, 2), *p = vec_at<T>(C, n, 3), *ph = vec_at<T>(C, n, 4);
                T *v = vec_at<T>(C, n, 6), *sv = vec_at<T>(C, n, 5), *sh = vec_at<T>(C, n, 7);
                T* t = vec_at<T>(C, n, 8);
                const T* phs = prec ? ph : p;
                const T* shs = prec ? sh : sv;
                k_bi_p<T><<<ewg(k_bi_p<T>, n), 256, 0, cs>>>(n, p, ph, r, v, dinv, st);
                if (block)
                    k_bj_apply<T, EpiStoreHalt<T>><<<ewg(k_bj_apply<T, EpiStoreHalt<T>>, n), 256, 0, cs>>>(
                        n, bs, binv, p, EpiStoreHalt<T>{ph, halt});
                if (ilu)
                    GK_TRY(ilu_apply<T>(ild, IluSrc<T>{p}, ilu_w, IluOutStore<T>{ph},
                                        IluSkipHalt{st}, IluErrSt{st}, cs));
                EpiDot<T, BiAlphaFin> e1{v, rh, halt, part, tk, BiAlphaFin{st}};
                GK_TRY((launch_spmv_rows<V, T>(A, phs, e1, cs)));
                k_bi_s<T><<<ewg(k_bi_s<T>, n), 256, 0, cs>>>(n, sv, sh, r, v, dinv, st, part, tk);
                if (block)
                    k_bj_apply<T, EpiStoreHalt<T>><<<ewg(k_bj_apply<T, EpiStoreHalt<T>>, n), 256, 0, cs>>>(
                        n, bs, binv, sv, EpiStoreHalt<T>{sh, halt});
                if (ilu)
                    GK_TRY(ilu_apply<T>(ild, IluSrc<T>{sv}, ilu_w, IluOutStore<T>{sh},
                                        IluSkipHalt{st}, IluErrSt{st}, cs));
                EpiBiT<T> e2{t, sv, st, part, tk, BiOmegaFin{st}};
                GK_TRY((launch_spmv_rows<V, T>(A, shs, e2, cs)));
                k_bi_update<T><<<ewg(k_bi_update<T>, n), 256, 0, cs>>>(n, xi, r, phs, shs, sv, t,
                                                                       rh, st, part, tk);
            }
            GK_CUDA(cudaGetLastError());
            return GK_OK;
        };
        auto body = [&](cudaStream_t cs, cudaGraphConditionalHandle hc, int cond) -> gk_status {
            for (int c = 0; c < chunk; ++c) GK_TRY(step(cs));
            k_ctl_check<<<1, 1, 0, cs>>>(st);
            // a passed recurrence: the true residual decides (tmp = b - A x)
            EpiResid<T, FinTrue> et{tmp, bi, &st->nocheck, part, tk, FinTrue{st, 1}};
            GK_TRY((launch_spmv_rows<V, T>(A, xi, et, cs)));
            k_ctl_replace<<<1, 1, 0, cs>>>(st);
            // residual replacement: r = tmp and the method restarts from x
            k_copy<T><<<ewg(k_copy<T>, n), 256, 0, cs>>>(n, tmp, r, &st->noreplace);
            GK_TRY(init(cs, &st->noreplace));
            k_ctl_next<<<1, 1, 0, cs>>>(st, hc, cond);
            GK_CUDA(cudaGetLastError());
            return GK_OK;
        };
        GK_TRY(capture_solve(A, C, pre, body, post, host_loop));
    }
    if (stale) {
        C->kmethod = method;
        C->kprec = pkey;
        C->km = m;
        C->kchunk = chunk;
        C->kv = C->vecs.ptr;
        C->kwait = A->wait_ns;
        C->khost = (int)host_loop;
    }
    if (host_loop)
        GK_TRY(run_host_loop(C, s, method == GK_GMRES, max_loops));
    else
        GK_CUDA(cudaGraphLaunch(C->exec, s));
    GK_CUDA(cudaMemcpyAsync(x, xi, sizeof(T) * (size_t)n, cudaMemcpyDeviceToDevice, s));
    if (info_dev) {  // asynchronous: the outcome goes to device memory
        k_write_info<<<1, 1, 0, s>>>(st, info_dev, rowtile ? A->plan.err : nullptr, A->fmt,
                                     A->fmt == GK_SELLP ? A->S : 0);
        GK_CUDA(cudaGetLastError());
        return GK_OK;
    }
    GK_TRY(read_hdr(C, s));
    gk_solve_info o;
    solve_outcome(C->hst, rowtile_timeout(), A->fmt, A->fmt == GK_SELLP ? A->S : 0, &o);
    out->status = o.status;
    out->iters = o.iters;
    out->restarts = o.restarts;
    out->rec = o.rel_res_recurrence;
    out->tru = o.rel_res_true;
    return GK_OK;
}


// one solve on the multi-kernel engine (instantiated per value type);
// info_dev != nullptr: enqueue only, the outcome is written there
template <typename V, typename T>
gk_status solve_mk(gk_matrix A, const T* b, T* x, int method, int pkind, int32_t bs, double tol,
                   int32_t max_iters, int32_t m, cudaStream_t s, SolveOut* out, bool inner,
                   gk_solve_info* info_dev);

extern template gk_status solve_mk<double, double>(gk_matrix, const double*, double*, int, int, int32_t,
                                                   double, int32_t, int32_t, cudaStream_t,
                                                   SolveOut*, bool, gk_solve_info*);
extern template gk_status solve_mk<float, float>(gk_matrix, const float*, float*, int, int, int32_t,
                                                 double, int32_t, int32_t, cudaStream_t, SolveOut*,
                                                 bool, gk_solve_info*);
extern template gk_status solve_mk<__nv_bfloat16, float>(gk_matrix, const float*, float*, int,
                                                         int, int32_t, double, int32_t, int32_t,
                                                         cudaStream_t, SolveOut*, bool,
                                                         gk_solve_info*);
extern template gk_status solve_mk<__half, float>(gk_matrix, const float*, float*, int, int, int32_t,
                                                  double, int32_t, int32_t, cudaStream_t,
                                                  SolveOut*, bool, gk_solve_info*);

}  // namespace gk
