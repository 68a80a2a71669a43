// solve_f32.cu - the multi-kernel Krylov engine for float values (float vectors).
#include "solve_engine.cuh"

namespace gk {
template gk_status solve_mk<float, float>(gk_matrix, const float*, float*, int, int, int32_t, double, int32_t,
                                      int32_t, cudaStream_t, SolveOut*, bool, gk_solve_info*);
}  // namespace gk
