// Solver kernels and graph construction for BF16 iteration vectors
// (one translation unit per storage type, compiled in parallel).
#include "solver.cuh"

namespace gb {
template int solve_launch<__nv_bfloat16>(const SolveCall &, bool, cudaStream_t);
template int solve_profiled<__nv_bfloat16>(const SolveCall &, bool, gbpcg_result *, cudaStream_t);
}  // namespace gb
