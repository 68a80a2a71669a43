// noalloc.cu - FP64 CSR SpMV for callers that cannot allocate device
// memory.  The paper has no counterpart; this is an addition of this
// library.
//
// Some callers cannot call cudaMalloc: their device memory belongs to a
// framework's pool allocator that must not see foreign allocations, or
// they run in a loop where an allocation (which can synchronise the
// device) is not allowed.  gk_spmv_csr_f64_noalloc serves them: it runs the
// same merge-path kernels as gk_apply, with the per-block carry scratch
// held in the file-scope device array below instead of a cudaMalloc'd
// buffer.  Every GPU that loads this library holds the array (768 KB)
// until the process exits.
#include "spmv.cuh"

namespace gk {

constexpr int NA_ITEMS_PER_THREAD = 8;  // merge items per thread (FP64 kernel)
constexpr int64_t NA_MAX_BLOCKS = GK_NOALLOC_MAX_ITEMS / (256 * NA_ITEMS_PER_THREAD);
static_assert(NA_MAX_BLOCKS * 256 * NA_ITEMS_PER_THREAD == GK_NOALLOC_MAX_ITEMS,
              "limit must be a whole number of merge blocks");

// carry_row[NA_MAX_BLOCKS] (int32) followed by carry_val[NA_MAX_BLOCKS] (double)
static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_MAX_BLOCKS * (4 + 8)];

constexpr int NA_MAX_DEVICES = 64;
static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[NA_MAX_DEVICES] = {};

// Device address of the scratch array on the current device.  Looked up once
// per device (host code must not use the symbol itself as an address).
static gk_status noalloc_scratch(void** out) {
    int dev = -1;
    GK_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NA_MAX_DEVICES) return GK_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        GK_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        GK_CUDA(cudaFuncSetAttribute(k_csr_merge<NA_ITEMS_PER_THREAD, double, double>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)merge_smem_bytes<NA_ITEMS_PER_THREAD, double, double>()));
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return GK_OK;
}

}  // namespace gk

using namespace gk;

extern "C" gk_status gk_spmv_csr_f64_noalloc(int32_t n, int32_t ncols, int64_t nnz,
                                             const int32_t* row_ptr, const int32_t* col_idx,
                                             const double* values, double alpha, const double* b,
                                             double beta, double* x, void* stream) {
    if (n < 0 || ncols < 0 || nnz < 0) return GK_ERR_INVALID;
    if ((int64_t)n + nnz > GK_NOALLOC_MAX_ITEMS) return GK_ERR_INVALID;
    if (n == 0) return GK_OK;
    if (!row_ptr || !x || (nnz > 0 && (!col_idx || !values || !b))) return GK_ERR_INVALID;
    void* scratch = nullptr;
    GK_TRY(noalloc_scratch(&scratch));
    cudaStream_t s = (cudaStream_t)stream;
    const int mode = (beta == 0.0) ? (alpha == 1.0 ? 0 : 1) : 2;
    EpiStore<double> epi{x, alpha, beta, mode};
    constexpr int E = NA_ITEMS_PER_THREAD;
    const int64_t nb = ((int64_t)n + nnz + 256 * E - 1) / (256 * E);
    // every block writes its carry slot before the fix-up reads it, so the
    // scratch needs no clearing between calls
    int32_t* crow = static_cast<int32_t*>(scratch);
    double* cval = reinterpret_cast<double*>(static_cast<char*>(scratch) + NA_MAX_BLOCKS * 4);
    constexpr size_t smem = merge_smem_bytes<E, double, double>();
    k_csr_merge<E, double, double><<<(unsigned)nb, 256, smem, s>>>(
        n, nnz, row_ptr, col_idx, values, b, epi, nullptr, crow, cval);
    const unsigned fg = (unsigned)std::max<int64_t>(1, std::min<int64_t>((nb + 255) / 256, 4096));
    k_csr_merge_fixup<double><<<fg, 256, 0, s>>>((int32_t)nb, crow, cval, x, alpha, mode);
    GK_CUDA(cudaGetLastError());
    return GK_OK;
}
