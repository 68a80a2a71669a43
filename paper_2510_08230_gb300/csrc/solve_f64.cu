// solve_f64.cu - the multi-kernel Krylov engine for double values (double vectors).
#include "solve_engine.cuh"

namespace gk {
template gk_status solve_mk<double, double>(gk_matrix, const double*, double*, int, int, int32_t, double, int32_t,
                                      int32_t, cudaStream_t, SolveOut*, bool, gk_solve_info*);
}  // namespace gk
