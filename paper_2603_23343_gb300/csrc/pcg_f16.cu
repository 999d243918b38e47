// Solver kernels and graph construction for FP16 iteration vectors
// (one translation unit per storage type, compiled in parallel).
#include "solver.cuh"

namespace gb {
template int solve_launch<__half>(const SolveCall &, bool, cudaStream_t);
template int solve_profiled<__half>(const SolveCall &, bool, gbpcg_result *, cudaStream_t);
}  // namespace gb
