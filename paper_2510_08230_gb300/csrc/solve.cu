// solve.cu - Krylov solver entry points: gk_solve (engine choice, solver
// SpMV layout, FP64 iterative refinement around FP32 / BF16-stored inner
// solves) and the host-side helpers of the multi-kernel engine
// (solve_engine.cuh).
#include "solve_engine.cuh"

namespace gk {

void free_solver_cache(gk_matrix A) {
    GateShared gate;
    delete A->solver;
    A->solver = nullptr;
}

gk_status get_cache(gk_matrix A, SolverCache** out) {
    if (!A->solver) {
        GateShared gate;
        SolverCache* C = new (std::nothrow) SolverCache();
        if (!C) return GK_ERR_OOM;
        A->solver = C;
        GK_CUDA(cudaMallocHost(&C->hst, sizeof(KState)));
        GK_CUDA(cudaMallocHost(&C->hzero, 64));
        std::memset(C->hzero, 0, 64);
        GK_TRY(C->ticket.ensure(256));
        GK_CUDA(cudaMemset(C->ticket.ptr, 0, 256));
        GK_TRY(C->state.ensure(sizeof(KState)));
        GK_CUDA(cudaEventCreate(&C->ev0));
        GK_CUDA(cudaEventCreate(&C->ev1));
    }
    *out = A->solver;
    return GK_OK;
}

gk_status ensure_jacobi(gk_matrix A, cudaStream_t s) {
    if (A->dinv_state == 1) return GK_OK;
    if (A->dinv_state == -1) return GK_ERR_ZERO_DIAG;
    const size_t vb = vector_bytes(A->dtype);
    GK_CUDA(dmalloc(&A->dinv, vb * (size_t)std::max(A->n, 1)));
    DevBuf bad;
    GK_TRY(bad.ensure(16));
    GK_CUDA(cudaMemsetAsync(bad.ptr, 0, 16, s));
    const unsigned g = ew_grid(A->n);
    auto go = [&](auto vt, auto tt) {
        using V = decltype(vt);
        using T = decltype(tt);
        if (A->fmt == GK_CSR)
            k_jacobi_gen<V, T><<<g, 256, 0, s>>>(A->n, A->row_ptr, A->col, (const V*)A->val,
                                                 (T*)A->dinv, (int32_t*)bad.ptr);
        else
            k_jacobi_gen_padded<V, T><<<g, 256, 0, s>>>(A->n, A->fmt, A->stride, A->K, A->S,
                                                        A->slice_len, A->slice_set, A->col,
                                                        (const V*)A->val, (T*)A->dinv,
                                                        (int32_t*)bad.ptr);
    };
    if (A->n > 0) {
        if (A->dtype == GK_F64) go(double(), double());
        else if (A->dtype == GK_F32) go(float(), float());
        else if (A->dtype == GK_F16) go(__half(), float());
        else go(__nv_bfloat16(), float());
    }
    GK_CUDA(cudaGetLastError());
    int32_t h = 0;
    GK_CUDA(cudaMemcpyAsync(&h, bad.ptr, 4, cudaMemcpyDeviceToHost, s));
    GK_CUDA(cudaStreamSynchronize(s));
    if (h) {
        A->dinv_state = -1;
        return GK_ERR_ZERO_DIAG;
    }
    A->dinv_state = 1;
    return GK_OK;
}

// Block-Jacobi inverses of A's diagonal blocks of bs rows (k_bj_gen), built
// once per (matrix, block size) from the CSR arrays (a padded matrix goes
// through a temporary CSR copy), stored in the vector type.
gk_status ensure_block_jacobi(gk_matrix A, int32_t bs, cudaStream_t s) {
    if (A->binv_bs == bs && A->binv) return GK_OK;
    if (A->binv_bs == -bs) return GK_ERR_ZERO_DIAG;  // known singular
    dfree(A->binv);
    A->binv = nullptr;
    A->binv_bs = 0;
    gk_matrix C = A, tmp = nullptr;
    if (A->fmt != GK_CSR) {
        GK_TRY(gk_matrix_convert(A, GK_CSR, A->dtype, 0, 0, s, &tmp));
        C = tmp;
    }
    const int64_t nb = ((int64_t)A->n + bs - 1) / bs;
    const size_t vb = vector_bytes(A->dtype);
    DevBuf bad;
    gk_status st = GK_OK;
    if (dmalloc(&A->binv, vb * (size_t)std::max<int64_t>(nb, 1) * bs * bs) != cudaSuccess) st = GK_ERR_OOM;
    if (st == GK_OK) st = bad.ensure(16);
    if (st == GK_OK && cudaMemsetAsync(bad.ptr, 0, 16, s) != cudaSuccess) st = GK_ERR_CUDA;
    if (st == GK_OK && nb > 0) {
        auto go = [&](auto vt, auto tt) {
            using V = decltype(vt);
            using T = decltype(tt);
            k_bj_gen<V, T><<<(unsigned)nb, 32, 0, s>>>(C->n, bs, C->row_ptr, C->col,
                                                       (const V*)C->val, (T*)A->binv,
                                                       (int32_t*)bad.ptr);
        };
        if (A->dtype == GK_F64) go(double(), double());
        else if (A->dtype == GK_F32) go(float(), float());
        else if (A->dtype == GK_F16) go(__half(), float());
        else go(__nv_bfloat16(), float());
        if (cudaGetLastError() != cudaSuccess) st = GK_ERR_CUDA;
    }
    int32_t h = 0;
    if (st == GK_OK && (cudaMemcpyAsync(&h, bad.ptr, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                        cudaStreamSynchronize(s) != cudaSuccess))
        st = GK_ERR_CUDA;
    if (tmp) gk_matrix_destroy(tmp);
    if (st != GK_OK) return st;
    if (h) {
        A->binv_bs = -bs;
        return GK_ERR_ZERO_DIAG;
    }
    A->binv_bs = bs;
    return GK_OK;
}

gk_status get_lowp(gk_matrix A, gk_dtype d, cudaStream_t s, gk_matrix* out) {
    if (A->dtype == d) {
        *out = A;
        return GK_OK;
    }
    if (!A->lowp[d]) {
        gk_matrix B = nullptr;
        GK_TRY(gk_matrix_convert(A, A->fmt, d, A->S, A->f, s, &B));
        A->lowp[d] = B;
    }
    *out = A->lowp[d];
    return GK_OK;
}

// SpMV layout for solves on a CSR matrix (solver format selection).  The
// padded layouts stream their column/value arrays with paired, fully
// coalesced loads and no row-pointer indirection, so when padding costs
// little they beat the CSR row-tile and merge kernels.  The CSR warp-tile
// kernel (short rows of near-uniform length) comes within a few per cent of
// ELL on large matrices (GB300, 3D 7-point 256^3: 262 against 255 us in
// FP64, 166 against 163 us in FP32), so those solve on their own CSR arrays
// and keep no padded copy, which would cost gigabytes.  On smaller ones the
// warp-tile launch's ramp (a full wave of blocks staging tiles into shared
// memory) costs more than ELL's padding, and its shared memory keeps
// concurrent solves from overlapping: six mid-size serving solves (n 70K to
// 430K) took 225 ms one after another and 131 ms at once on the CSR, 193 and
// 97 ms with the ELL copy.  Default rule, decided on the first solve and
// kept: the CSR itself when its plan is the warp-tile kernel and it holds at
// least SOLVE_CSR_MIN_NNZ entries, else ELL when its stored entries are at most 1.2 x nnz,
// else SELL-P(32) when its stored entries are at most 1.2 x nnz, else the CSR
// itself.  The rule depends only on the sparsity pattern, so every handle of
// a matrix solves with the same summation order (bit-identical results).
// GK_SOLVE_FORMAT=csr|ell|sellp forces a layout; GK_SOLVE_FORMAT=timed times
// three SpMVs of each admissible layout and keeps the fastest.  The copy holds
// the same values bit for bit, so the choice changes the order of the row
// sums, not the matrix.
constexpr int64_t SOLVE_CSR_MIN_NNZ = int64_t(1) << 24;

static gk_status solve_matrix(gk_matrix A, cudaStream_t s, gk_matrix* out) {
    *out = A;
    if (A->fmt != GK_CSR || A->n == 0) return GK_OK;
    if (A->solve_fmt_tuned) {
        *out = A->solve_fmt ? A->solve_fmt : A;
        return GK_OK;
    }
    const char* env = getenv("GK_SOLVE_FORMAT");
    const bool timed = env && !strcmp(env, "timed");
    const bool force = env && !timed && strcmp(env, "auto") != 0;
    if (!force && !timed && A->plan.kind == 3 && A->nnz >= SOLVE_CSR_MIN_NNZ) {
        A->solve_fmt = nullptr;
        A->solve_fmt_tuned = 1;
        return GK_OK;
    }
    const bool want_ell = !force || !strcmp(env, "ell");
    const bool want_sellp = !force || !strcmp(env, "sellp");
    auto padding_ok = [&](int64_t stored) { return force || stored <= A->nnz + A->nnz / 5; };
    std::vector<gk_matrix> cand;
    if (want_ell && padding_ok((int64_t)A->max_row * A->n)) {
        gk_matrix E = nullptr;
        GK_TRY(gk_matrix_convert(A, GK_ELL, A->dtype, 0, 0, s, &E));
        cand.push_back(E);
    }
    if (want_sellp && (timed || cand.empty())) {
        gk_matrix P = nullptr;
        GK_TRY(gk_matrix_convert(A, GK_SELLP, A->dtype, 32, 1, s, &P));
        if (padding_ok(P->stored)) cand.push_back(P);
        else gk_matrix_destroy(P);
    }
    gk_matrix best = cand.empty() ? A : cand.front();
    if (timed && !cand.empty()) {
        const size_t vb = vector_bytes(A->dtype);
        DevBuf xv, yv;
        GK_TRY(xv.ensure(vb * (size_t)A->ncols));
        GK_TRY(yv.ensure(vb * (size_t)A->n));
        GK_CUDA(cudaMemsetAsync(xv.ptr, 0, vb * (size_t)A->ncols, s));
        cudaEvent_t e0, e1;
        GK_CUDA(cudaEventCreate(&e0));
        GK_CUDA(cudaEventCreate(&e1));
        float best_ms = 1e30f;
        std::vector<gk_matrix> all = cand;
        all.insert(all.begin(), A);
        for (gk_matrix M : all) {
            GK_TRY(spmv_dispatch(M, 1.0, xv.ptr, 0.0, yv.ptr, s));  // warm-up
            GK_CUDA(cudaEventRecord(e0, s));
            for (int r = 0; r < 3; ++r) GK_TRY(spmv_dispatch(M, 1.0, xv.ptr, 0.0, yv.ptr, s));
            GK_CUDA(cudaEventRecord(e1, s));
            GK_CUDA(cudaEventSynchronize(e1));
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best_ms) {
                best_ms = ms;
                best = M;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    for (gk_matrix M : cand)
        if (M != best) gk_matrix_destroy(M);
    A->solve_fmt = best == A ? nullptr : best;
    A->solve_fmt_tuned = 1;
    *out = best;
    return GK_OK;
}

gk_status side_stream(gk_matrix A) {
    if (!A->side) GK_CUDA(cudaStreamCreateWithFlags(&A->side, cudaStreamNonBlocking));
    if (!A->side2) GK_CUDA(cudaStreamCreateWithFlags(&A->side2, cudaStreamNonBlocking));
    return GK_OK;
}

gk_status read_hdr(SolverCache* C, cudaStream_t s) {
    GK_CUDA(cudaMemcpyAsync(C->hst, C->state.ptr, HDR, cudaMemcpyDeviceToHost, s));
    GK_CUDA(cudaStreamSynchronize(s));
    return GK_OK;
}

gk_status clear_halt(SolverCache* C, cudaStream_t s) {
    KState* st = (KState*)C->state.ptr;
    GK_CUDA(cudaMemcpyAsync(&st->halt, C->hzero, sizeof(int32_t), cudaMemcpyHostToDevice, s));
    return GK_OK;
}

}  // namespace gk

// ---------------------------------------------------------------- entry points
namespace gk {

static gk_status check_opts(gk_matrix A, const gk_solve_opts* o) {
    if (!o) return GK_ERR_INVALID;
    if (o->method != GK_CG && o->method != GK_BICGSTAB && o->method != GK_GMRES &&
        o->method != GK_CGS)
        return GK_ERR_INVALID;
    if (o->precond != GK_PRECOND_NONE && o->precond != GK_PRECOND_JACOBI &&
        o->precond != GK_PRECOND_BLOCK_JACOBI && o->precond != GK_PRECOND_ILU)
        return GK_ERR_INVALID;
    if (o->precond == GK_PRECOND_BLOCK_JACOBI && (o->block_size < 1 || o->block_size > BJ_MAX))
        return GK_ERR_INVALID;
    if (!(o->tol >= 0.0) || o->max_iters < 0) return GK_ERR_INVALID;
    if (o->krylov_dim < 0 || o->krylov_dim > MAXM) return GK_ERR_INVALID;
    if (o->mixed < 0 || o->mixed > 3) return GK_ERR_INVALID;
    if (o->mixed && A->dtype != GK_F64) return GK_ERR_INVALID;
    if (o->engine < 0 || o->engine > 3) return GK_ERR_INVALID;
    if (o->wait_budget_ns < 0) return GK_ERR_INVALID;
    if (A->n != A->ncols) return GK_ERR_INVALID;
    return GK_OK;
}

// The wait budget of a solve reaches every handle whose kernels the solve
// launches (A, its solver layout copy, its low-precision copies); after the
// solve they return to the default.
static void reset_wait(gk_matrix A) {
    A->wait_ns = WAIT_LIMIT_NS;
    if (A->solve_fmt) A->solve_fmt->wait_ns = WAIT_LIMIT_NS;
    for (gk_matrix L : A->lowp)
        if (L) {
            L->wait_ns = WAIT_LIMIT_NS;
            if (L->solve_fmt) L->solve_fmt->wait_ns = WAIT_LIMIT_NS;
        }
}

template <typename V, typename T>
static gk_status solve_plain(gk_matrix A, const void* b, void* x, const gk_solve_opts* o,
                             cudaStream_t s, SolveOut* out) {
    const int m = o->method == GK_GMRES ? (o->krylov_dim ? o->krylov_dim : 30) : 0;
    gk_matrix M = nullptr;
    GK_TRY(solve_matrix(A, s, &M));
    M->wait_ns = A->wait_ns;
    GK_TRY((solve_mk<V, T>(M, (const T*)b, (T*)x, o->method, (int)o->precond, o->block_size,
                           o->tol, o->max_iters, m, s, out, false)));
    out->layout = M->fmt;
    out->slice = M->fmt == GK_SELLP ? M->S : 0;
    return GK_OK;
}

// FP64 iterative refinement: r = b - A x in FP64; inner solve of
// A_low d = r (FP32, BF16- or FP16-stored values, FP32 vectors) to inner_tol;
// x += d in FP64; until ||b - A x|| <= tol ||b||.
static gk_status solve_ir(gk_matrix A, const double* b, double* x, const gk_solve_opts* o,
                          cudaStream_t s, SolveOut* out, int32_t* outer) {
    const int32_t n = A->n;
    gk_matrix L = nullptr;
    GK_TRY(get_lowp(A, o->mixed == 2 ? GK_BF16 : o->mixed == 3 ? GK_F16 : GK_F32, s, &L));
    GK_TRY(solve_matrix(L, s, &L));  // layout of the inner SpMV
    gk_matrix A64 = nullptr;
    GK_TRY(solve_matrix(A, s, &A64));  // layout of the outer FP64 residual
    L->wait_ns = A64->wait_ns = A->wait_ns;
    SolverCache* C = nullptr;
    GK_TRY(get_cache(A, &C));
    // FP64 workspace: r64 ; FP32: r32, d32 (in the low-precision handle's cache
    // the inner solver keeps its own vectors)
    const size_t s64 = ((size_t)n * 8 + 255) & ~(size_t)255;
    const size_t s32 = ((size_t)n * 4 + 255) & ~(size_t)255;
    GK_TRY(C->vecs.ensure(2 * s64 + 2 * s32 + 256));
    double* r64 = (double*)C->vecs.ptr;
    float* r32 = (float*)((char*)C->vecs.ptr + s64);
    float* d32 = (float*)((char*)C->vecs.ptr + s64 + s32);
    double* xb = (double*)((char*)C->vecs.ptr + s64 + 2 * s32);  // the best iterate so far
    const size_t pcount = (size_t)num_sms() * 8 * 4;
    GK_TRY(C->partials.ensure(pcount * sizeof(double)));
    double* part = (double*)C->partials.ptr;
    unsigned* tk = (unsigned*)C->ticket.ptr;
    KState* st = (KState*)C->state.ptr;
    KState* h = C->hst;
    std::memset(h, 0, HDR);
    GK_CUDA(cudaMemcpyAsync(st, h, HDR, cudaMemcpyHostToDevice, s));
    k_norm2<double, FinBnorm><<<ewg(k_norm2<double, FinBnorm>, n), 256, 0, s>>>(n, b, part, tk, FinBnorm{st, o->tol});
    GK_TRY(read_hdr(C, s));
    const double bnorm = C->hst->bnorm, thr = C->hst->thr;
    if (!(bnorm > 0.0)) {
        if (bnorm == 0.0) {
            k_zero<double><<<ewg(k_zero<double>, n), 256, 0, s>>>(n, x);
            GK_CUDA(cudaGetLastError());
            out->status = GK_OK;
            return GK_OK;
        }
        out->status = GK_ERR_NAN;
        return GK_OK;
    }
    const int max_outer = o->max_outer > 0 ? o->max_outer : 50;
    // default inner reduction (see the header): 1e-2 where the inner system is
    // itself accurate to about that (BF16 / FP16 values) or where the inner
    // method restarts anyway (GMRES(m)); else 1e-5
    const double inner_tol = o->inner_tol > 0 ? o->inner_tol
                             : (o->mixed >= 2 || o->method == GK_GMRES) ? 1e-2 : 1e-5;
    const int m = o->method == GK_GMRES ? (o->krylov_dim ? o->krylov_dim : 30) : 0;
    int32_t total_inner = 0, restarts = 0;
    double tn = 0.0, last_rec = 0.0;
    gk_status status = GK_NOT_CONVERGED;
    // Safeguard: the iterate with the smallest true residual is kept.  A
    // step whose true residual exceeds 4x that smallest one (an inner solve
    // in low precision that wandered on an ill-conditioned system), is not
    // finite, or whose inner solve broke down or met a NaN, ends the
    // refinement: x returns to the best iterate and the solve finishes in
    // FP64 from there.  Smaller rises are let through: refinement with a
    // loose inner tolerance is not monotone and recovers from them.  So does
    // stagnation: three outer steps that together cut the smallest residual
    // by less than 2x (inner solves that stop early on a system the low
    // precision cannot resolve).
    constexpr double GROWTH = 4.0;
    constexpr int STAG_STEPS = 3;
    bool finish64 = false;
    double best_tn = INFINITY;
    std::vector<double> best_hist;  // best_tn before each outer step
    int k = 0;
    for (;; ++k) {
        // r = b - A x in FP64 (and its norm)
        std::memset(h, 0, HDR);
        h->thr = thr;
        h->bnorm = bnorm;
        GK_CUDA(cudaMemcpyAsync(st, h, HDR, cudaMemcpyHostToDevice, s));
        EpiResid<double, FinNorm> er{r64, b, nullptr, part, tk, FinNorm{st, 1}};
        GK_TRY((launch_spmv_rows<double, double>(A64, x, er, s)));
        GK_TRY(read_hdr(C, s));
        tn = C->hst->tnorm;
        if (k > 0 && !(tn <= GROWTH * best_tn)) {
            GK_CUDA(cudaMemcpyAsync(x, xb, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, s));
            tn = best_tn;
            finish64 = true;
            break;
        }
        if (k >= STAG_STEPS && tn > thr &&
            std::min(tn, best_tn) > 0.5 * best_hist[(size_t)(k - STAG_STEPS)]) {
            if (tn > best_tn) {
                GK_CUDA(cudaMemcpyAsync(x, xb, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, s));
                tn = best_tn;
            }
            finish64 = true;
            break;
        }
        if (!std::isfinite(tn)) {
            status = GK_ERR_NAN;
            break;
        }
        if (tn <= thr) {
            status = GK_OK;
            break;
        }
        if (k >= max_outer || total_inner >= o->max_iters) break;
        best_hist.push_back(std::min(tn, best_tn));
        k_cast_to<float><<<ewg(k_cast_to<float>, n), 256, 0, s>>>(n, r64, r32);
        k_zero<float><<<ewg(k_zero<float>, n), 256, 0, s>>>(n, d32);
        GK_CUDA(cudaGetLastError());
        SolveOut io;
        const int pk = (int)o->precond;
        const int32_t bsz = o->block_size;
        const int32_t left = o->max_iters - total_inner;
        if (L->dtype == GK_F32)
            GK_TRY((solve_mk<float, float>(L, r32, d32, o->method, pk, bsz, inner_tol, left, m, s,
                                           &io, true)));
        else if (L->dtype == GK_F16)
            GK_TRY((solve_mk<__half, float>(L, r32, d32, o->method, pk, bsz, inner_tol, left, m, s,
                                            &io, true)));
        else
            GK_TRY((solve_mk<__nv_bfloat16, float>(L, r32, d32, o->method, pk, bsz, inner_tol, left,
                                                   m, s, &io, true)));
        total_inner += io.iters;
        restarts += io.restarts;
        last_rec = io.rec;
        if (tn < best_tn) {  // x (not yet corrected) is the best iterate
            GK_CUDA(cudaMemcpyAsync(xb, x, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, s));
            best_tn = tn;
        }
        if (io.status == GK_BREAKDOWN || io.status == GK_ERR_NAN) {
            if (tn > best_tn) {
                GK_CUDA(cudaMemcpyAsync(x, xb, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, s));
                tn = best_tn;
            }
            finish64 = true;
            break;
        }
        if (io.status < 0) {  // an error other than NaN (a timed-out wait, CUDA): d is invalid
            status = io.status;
            break;
        }
        k_cast_add<float><<<ewg(k_cast_add<float>, n), 256, 0, s>>>(n, x, d32);
        GK_CUDA(cudaGetLastError());
    }
    if (finish64) {
        gk_solve_opts o64 = *o;
        o64.mixed = 0;
        o64.max_iters = std::max(0, o->max_iters - total_inner);
        SolveOut fo;
        GK_TRY((solve_plain<double, double>(A, b, x, &o64, s, &fo)));
        status = fo.status;
        total_inner += fo.iters;
        restarts += fo.restarts + 1;
        last_rec = fo.rec;
        tn = fo.tru * bnorm;
    }
    out->status = status;
    out->iters = total_inner;
    out->restarts = restarts;
    out->rec = last_rec;
    out->tru = tn / bnorm;
    out->layout = A64->fmt;
    out->slice = A64->fmt == GK_SELLP ? A64->S : 0;
    *outer = k;
    return GK_OK;
}

gk_status solve_small(gk_matrix A, const void* b, void* x, const gk_solve_opts* o, cudaStream_t s,
                      SolveOut* out);
gk_status solve_cluster(gk_matrix A, const void* b, void* x, const gk_solve_opts* o,
                        cudaStream_t s, SolveOut* out);
int32_t cluster_max_n();

}  // namespace gk

using namespace gk;

namespace gk {
// info of a solve decided before any iteration (n = 0), in device memory
__global__ void k_info_trivial(gk_solve_info* info, int32_t layout) {
    gk_solve_info o = {};
    o.status = GK_OK;
    o.spmv_format = layout;
    *info = o;
}
}  // namespace gk

extern "C" gk_status gk_solve_async(gk_matrix A, const void* b, void* x,
                                    const gk_solve_opts* opts, gk_solve_info* info,
                                    void* stream) {
    if (!A || !opts || !info) return GK_ERR_INVALID;
    if (A->n > 0 && (!b || !x)) return GK_ERR_INVALID;
    GK_TRY(check_opts(A, opts));
    if (opts->mixed) return GK_ERR_UNSUPPORTED;  // refinement's outer loop runs on the host
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != A->device) return GK_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(A->mu);
    A->wait_ns = opts->wait_budget_ns > 0 ? (uint64_t)opts->wait_budget_ns : WAIT_LIMIT_NS;
    struct ResetWait {
        gk_matrix A;
        ~ResetWait() { reset_wait(A); }
    } reset_on_exit{A};
    if (A->n == 0) {
        k_info_trivial<<<1, 1, 0, s>>>(info, A->fmt);
        GK_CUDA(cudaGetLastError());
        return GK_OK;
    }
    gk_matrix M = nullptr;
    GK_TRY(solve_matrix(A, s, &M));
    M->wait_ns = A->wait_ns;
    const int m = opts->method == GK_GMRES ? (opts->krylov_dim ? opts->krylov_dim : 30) : 0;
    SolveOut out;
    const int pk = (int)opts->precond;
    switch (A->dtype) {
        case GK_F64:
            return solve_mk<double, double>(M, (const double*)b, (double*)x, opts->method, pk,
                                            opts->block_size, opts->tol, opts->max_iters, m, s,
                                            &out, false, info);
        case GK_F32:
            return solve_mk<float, float>(M, (const float*)b, (float*)x, opts->method, pk,
                                          opts->block_size, opts->tol, opts->max_iters, m, s, &out,
                                          false, info);
        case GK_F16:
            return solve_mk<__half, float>(M, (const float*)b, (float*)x, opts->method, pk,
                                           opts->block_size, opts->tol, opts->max_iters, m, s, &out,
                                           false, info);
        default:
            return solve_mk<__nv_bfloat16, float>(M, (const float*)b, (float*)x, opts->method, pk,
                                                  opts->block_size, opts->tol, opts->max_iters, m, s,
                                                  &out, false, info);
    }
}

extern "C" gk_status gk_solve(gk_matrix A, const void* b, void* x, const gk_solve_opts* opts,
                              gk_solve_info* info, void* stream) {
    if (!A || !opts) return GK_ERR_INVALID;
    if (A->n > 0 && (!b || !x)) return GK_ERR_INVALID;
    GK_TRY(check_opts(A, opts));
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != A->device) return GK_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(A->mu);
    SolveOut out;
    int32_t outer = 0;
    SolverCache* C = nullptr;
    GK_TRY(get_cache(A, &C));
    A->wait_ns = opts->wait_budget_ns > 0 ? (uint64_t)opts->wait_budget_ns : WAIT_LIMIT_NS;
    struct ResetWait {
        gk_matrix A;
        ~ResetWait() { reset_wait(A); }
    } reset_on_exit{A};
    GK_CUDA(cudaEventRecord(C->ev0, s));
    gk_status st = GK_OK;
    if (A->n == 0) {
        out.status = GK_OK;
    } else if (opts->mixed) {
        st = solve_ir(A, (const double*)b, (double*)x, opts, s, &out, &outer);
    } else {
        int engine = opts->engine;
        if (engine == 0 && A->fmt == GK_CSR && opts->method == GK_CG && A->n <= cluster_max_n())
            engine = 3;
        if (engine == 3) {
            st = solve_cluster(A, b, x, opts, s, &out);
            if (st == GK_ERR_UNSUPPORTED && opts->engine == 0) engine = 1;  // cannot schedule
        }
        if (engine == 2) {
            st = solve_small(A, b, x, opts, s, &out);
        } else if (engine == 3) {
        } else if (A->dtype == GK_F64) {
            st = solve_plain<double, double>(A, b, x, opts, s, &out);
        } else if (A->dtype == GK_F32) {
            st = solve_plain<float, float>(A, b, x, opts, s, &out);
        } else if (A->dtype == GK_F16) {
            st = solve_plain<__half, float>(A, b, x, opts, s, &out);
        } else {
            st = solve_plain<__nv_bfloat16, float>(A, b, x, opts, s, &out);
        }
    }
    GK_CUDA(cudaEventRecord(C->ev1, s));
    GK_CUDA(cudaEventSynchronize(C->ev1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, C->ev0, C->ev1);
    if (st != GK_OK) {
        if (info) info->status = st;
        return st;
    }
    if (info) {
        info->status = out.status;
        info->iters = out.iters;
        info->restarts = out.restarts;
        info->outer_iters = outer;
        info->rel_res_recurrence = out.rec;
        info->rel_res_true = out.tru;
        info->device_ms = ms;
        info->spmv_format = out.layout;
        info->slice_size = out.slice;
        info->block_threads = out.threads;
    }
    return out.status;
}
