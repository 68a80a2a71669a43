// apply.cu - gk_apply / gk_apply_adv: x = alpha A b + beta x on any format
// (the LinOp apply of Section 4.2; the paper's SpMV benchmark, Section 6.1).
#include "spmv.cuh"

namespace gk {

static bool is_device_ptr(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// One merge-path instance (E path items per thread; block or warp units).
template <int E, typename V, typename T>
static gk_status launch_merge(gk_matrix A, const T* b, const EpiStore<T>& epi, int32_t* crow,
                              T* cval, cudaStream_t s) {
    if (A->plan.merge_warp == 2) {
        constexpr size_t smem = MergeRegShape<E>::BYTES;
        const int64_t units = A->plan.merge_blocks;
        k_csr_merge_reg<E, V, T><<<(unsigned)((units + 7) / 8), 256, smem, s>>>(
            A->n, A->nnz, A->row_ptr, A->col, (const V*)A->val, b, epi, A->plan.block_row, units,
            crow, cval);
        return GK_OK;
    }
    if (A->plan.merge_warp) {
        constexpr size_t smem = MergeWarpShape<E, V, T>::BYTES;
        static bool attr = false;
        if (!attr) {
            GK_CUDA(cudaFuncSetAttribute(k_csr_merge_warp<E, V, T>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            attr = true;
        }
        const int64_t units = A->plan.merge_blocks;
        k_csr_merge_warp<E, V, T><<<(unsigned)((units + 7) / 8), 256, smem, s>>>(
            A->n, A->nnz, A->row_ptr, A->col, (const V*)A->val, b, epi, A->plan.block_row, units,
            crow, cval);
        return GK_OK;
    }
    constexpr size_t smem = merge_smem_bytes<E, V, T>();
    static bool attr = false;
    if (!attr) {
        GK_CUDA(cudaFuncSetAttribute(k_csr_merge<E, V, T>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr = true;
    }
    k_csr_merge<E, V, T><<<(unsigned)A->plan.merge_blocks, 256, smem, s>>>(
        A->n, A->nnz, A->row_ptr, A->col, (const V*)A->val, b, epi, A->plan.block_row, crow, cval);
    return GK_OK;
}

template <typename V, typename T>
static gk_status spmv_typed(gk_matrix A, double alpha, const void* b, double beta, void* x,
                            cudaStream_t s) {
    const int mode = (beta == 0.0) ? (alpha == 1.0 ? 0 : 1) : 2;
    EpiStore<T> epi{static_cast<T*>(x), (T)alpha, (T)beta, mode};
    if (A->n == 0) return GK_OK;
    if (A->coo) {
        const int E = A->coo_e;
        const int64_t units = (A->nnz + 32 * E - 1) / (32 * E);
        if (units > 0) {
            GK_TRY(A->carry.ensure((size_t)units * (sizeof(int32_t) + sizeof(T)) + 16));
            int32_t* crow = static_cast<int32_t*>(A->carry.ptr);
            T* cval = reinterpret_cast<T*>(static_cast<char*>(A->carry.ptr) +
                                           (((size_t)units * sizeof(int32_t) + 15) & ~(size_t)15));
            const unsigned g = (unsigned)((units + 7) / 8);
            const int32_t* rw = A->coo_row;
            const V* vals = (const V*)A->val;
            const T* bt = static_cast<const T*>(b);
            switch (E) {
                case 8: k_coo_warp<2, V, T><<<g, 256, 0, s>>>(A->n, A->nnz, rw, A->col, vals, bt, epi, units, crow, cval); break;
                case 12: k_coo_warp<3, V, T><<<g, 256, 0, s>>>(A->n, A->nnz, rw, A->col, vals, bt, epi, units, crow, cval); break;
                case 16: k_coo_warp<4, V, T><<<g, 256, 0, s>>>(A->n, A->nnz, rw, A->col, vals, bt, epi, units, crow, cval); break;
                default: k_coo_warp<1, V, T><<<g, 256, 0, s>>>(A->n, A->nnz, rw, A->col, vals, bt, epi, units, crow, cval); break;
            }
            const unsigned fg =
                (unsigned)std::max<int64_t>(1, std::min<int64_t>((units + 255) / 256, 4096));
            k_csr_merge_fixup<T><<<fg, 256, 0, s>>>((int32_t)units, crow, cval, static_cast<T*>(x),
                                                    (T)alpha, mode);
        }
        if (A->n_empty) {
            const unsigned eg = (unsigned)std::max<int64_t>(
                1, std::min<int64_t>((A->n_empty + 255) / 256, (int64_t)num_sms() * 8));
            k_coo_empty<T><<<eg, 256, 0, s>>>(A->n_empty, A->empty_rows, epi);
        }
        GK_CUDA(cudaGetLastError());
        return GK_OK;
    }
    if (A->fmt == GK_CSR && A->plan.kind == 2) {
        const int64_t nb = A->plan.merge_blocks;
        GK_TRY(A->carry.ensure((size_t)nb * (sizeof(int32_t) + sizeof(T)) + 16));
        int32_t* crow = static_cast<int32_t*>(A->carry.ptr);
        T* cval = reinterpret_cast<T*>(static_cast<char*>(A->carry.ptr) +
                                       (((size_t)nb * sizeof(int32_t) + 15) & ~(size_t)15));
        const T* bt = static_cast<const T*>(b);
        switch (A->plan.merge_e) {
            case 4: GK_TRY((launch_merge<4, V, T>(A, bt, epi, crow, cval, s))); break;
            case 6: GK_TRY((launch_merge<6, V, T>(A, bt, epi, crow, cval, s))); break;
            default: GK_TRY((launch_merge<8, V, T>(A, bt, epi, crow, cval, s))); break;
        }
        const unsigned fg = (unsigned)std::max<int64_t>(1, std::min<int64_t>((nb + 255) / 256, 4096));
        k_csr_merge_fixup<T><<<fg, 256, 0, s>>>((int32_t)nb, crow, cval, static_cast<T*>(x),
                                                (T)alpha, mode);
        GK_CUDA(cudaGetLastError());
        return GK_OK;
    }
    return launch_spmv_rows<V, T>(A, static_cast<const T*>(b), epi, s);
}

gk_status spmv_dispatch(gk_matrix A, double alpha, const void* b, double beta, void* x,
                        cudaStream_t s) {
    switch (A->dtype) {
        case GK_F64: return spmv_typed<double, double>(A, alpha, b, beta, x, s);
        case GK_F32: return spmv_typed<float, float>(A, alpha, b, beta, x, s);
        case GK_BF16: return spmv_typed<__nv_bfloat16, float>(A, alpha, b, beta, x, s);
        case GK_F16: return spmv_typed<__half, float>(A, alpha, b, beta, x, s);
    }
    return GK_ERR_INVALID;
}

static gk_status apply_common(gk_matrix A, double alpha, const void* b, double beta, void* x,
                              void* stream) {
    if (!A || (!b && A->ncols > 0) || (!x && A->n > 0)) return GK_ERR_INVALID;
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != A->device) return GK_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    if (A->n == 0) return GK_OK;
    const bool db = A->ncols == 0 || is_device_ptr(b);
    const bool dx = is_device_ptr(x);
    if (db && dx) return spmv_dispatch(A, alpha, b, beta, x, s);
    if (db != dx && A->ncols > 0) return GK_ERR_INVALID;  // mixed host/device vectors
    // host vectors: stage through device buffers owned by the handle
    std::lock_guard<std::mutex> lk(A->mu);
    const size_t vb = vector_bytes(A->dtype);
    GK_TRY(A->stage_in.ensure(vb * (size_t)std::max(A->ncols, 1)));
    GK_TRY(A->stage_out.ensure(vb * (size_t)A->n));
    if (A->ncols > 0)
        GK_CUDA(cudaMemcpyAsync(A->stage_in.ptr, b, vb * (size_t)A->ncols, cudaMemcpyHostToDevice, s));
    if (beta != 0.0)
        GK_CUDA(cudaMemcpyAsync(A->stage_out.ptr, x, vb * (size_t)A->n, cudaMemcpyHostToDevice, s));
    GK_TRY(spmv_dispatch(A, alpha, A->stage_in.ptr, beta, A->stage_out.ptr, s));
    GK_CUDA(cudaMemcpyAsync(x, A->stage_out.ptr, vb * (size_t)A->n, cudaMemcpyDeviceToHost, s));
    GK_CUDA(cudaStreamSynchronize(s));
    return GK_OK;
}

}  // namespace gk

extern "C" {

gk_status gk_apply(gk_matrix A, const void* b, void* x, void* stream) {
    return gk::apply_common(A, 1.0, b, 0.0, x, stream);
}

gk_status gk_apply_adv(gk_matrix A, double alpha, const void* b, double beta, void* x,
                       void* stream) {
    return gk::apply_common(A, alpha, b, beta, x, stream);
}

}  // extern "C"
