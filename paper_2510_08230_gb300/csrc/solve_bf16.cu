// solve_bf16.cu - the multi-kernel Krylov engine for __nv_bfloat16 values (float vectors).
#include "solve_engine.cuh"

namespace gk {
template gk_status solve_mk<__nv_bfloat16, float>(gk_matrix, const float*, float*, int, int, int32_t, double, int32_t,
                                      int32_t, cudaStream_t, SolveOut*, bool, gk_solve_info*);
}  // namespace gk
