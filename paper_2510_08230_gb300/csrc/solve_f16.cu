// solve_f16.cu - the multi-kernel Krylov engine for IEEE half values (float vectors).
#include "solve_engine.cuh"

namespace gk {
template gk_status solve_mk<__half, float>(gk_matrix, const float*, float*, int, int, int32_t, double,
                                           int32_t, int32_t, cudaStream_t, SolveOut*, bool, gk_solve_info*);
}  // namespace gk
